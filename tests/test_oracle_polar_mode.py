"""Pins for the oracle's polar-rotation mode (R_k = rotation factor of F_k, the
co-rotational FEM energy of the standard FEM model §4 compares against): the
gradient at fixed R is the true gradient of the FEM energy (finite
differences), the FEM energy in singular values, rest and rigid closed forms,
and the minimality of each mode's solution in its own energy."""
import numpy as np
import pytest

from oracle import diag, element, solve as S
from synth import bar_mesh, bar_twist_config, figure_config, identity_pose, rigid_pose, rodrigues


def _fem_energy(st, y, model):
    R = diag.polar(element.deformation_gradient(y, st.T, st.G))[0]
    return element.element_energy(y, st.T, st.G, st.vol, R, model, st.mu, st.lam).sum()


@pytest.mark.parametrize("model", ["arap", "corot", "snh"])
def test_gradient_at_polar_rotation_is_the_true_gradient(model, rng):
    X, T = bar_mesh(2, 2, 3)
    st = S.Setup(X, T, [[1.0, 1.0, 0.0]], [-1], 1.3, 2.1, cluster_rule="joint", pin_verts=[0],
                 pin_handle=[0])
    y = X + 0.15 * rng.normal(size=X.shape)
    R = diag.polar(element.deformation_gradient(y, st.T, st.G))[0]
    g = element.gradient(y, st.T, st.G, st.vol, R, model, st.mu, st.lam)
    h = 1e-6
    for v, i in [(0, 0), (5, 1), (11, 2), (17, 0), (len(X) - 1, 2)]:
        yp, ym = y.copy(), y.copy()
        yp[v, i] += h
        ym[v, i] -= h
        fd = (_fem_energy(st, yp, model) - _fem_energy(st, ym, model)) / (2 * h)
        assert abs(fd - g[v, i]) <= 1e-6 * (1 + abs(g[v, i])), (v, i, fd, g[v, i])


def test_arap_fem_energy_in_signed_singular_values(rng):
    X, T = bar_mesh(2, 1, 2)
    st = S.Setup(X, T, [[0.0, 0.0, 0.0]], [-1], 0.7, 0.0, cluster_rule="joint", pin_verts=[0],
                 pin_handle=[0])
    y = X + 0.6 * rng.normal(size=X.shape)
    F = element.deformation_gradient(y, st.T, st.G)
    sv = np.linalg.svd(F, compute_uv=False)
    sv[:, 2] *= np.sign(np.linalg.det(F))       # inverted tets: the least stretch is negative
    want = np.sum(st.vol * 0.7 * np.sum((sv - 1.0) ** 2, axis=1))
    assert np.any(np.linalg.det(F) < 0)
    assert _fem_energy(st, y, "arap") == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("model", ["corot", "snh"])
def test_rest_and_rigid_poses_in_polar_mode(model):
    cfg = figure_config(3000, seeds=[], model=model)
    st = S.Setup.from_config(cfg)
    H = len(cfg["joints"])
    # the start is the solution: the gradient is rounding noise, a few steps keep it
    x, info = S.solve(st, identity_pose(H), model, rotation="polar", newton_tol=1e-12, newton_max=2)
    assert np.abs(x - cfg["X"]).max() <= 1e-12 * st.bbox_diag
    Q = rodrigues([0.3, -1.0, 0.5], 1.1)
    t = np.array([0.1, 0.2, -0.3])
    x, info = S.solve(st, rigid_pose(H, Q, t), model, rotation="polar", newton_tol=1e-12, newton_max=2)
    assert np.abs(x - (cfg["X"] @ Q.T + t)).max() <= 1e-12 * st.bbox_diag


@pytest.mark.parametrize("model", ["arap", "snh"])
def test_each_mode_minimises_its_own_energy(model):
    cfg = dict(bar_twist_config(3, 3, 8), model=model, mu=1.0, lam=3.0 if model == "snh" else 0.0)
    st = S.Setup.from_config(cfg)
    xf = cfg["xfs"][0]
    x_fem, info = S.solve(st, xf, model, rotation="polar", newton_tol=1e-11, newton_max=100)
    assert info["converged"]
    x_rig, _ = S.solve(st, xf, model, newton_tol=1e-12)

    def energy(x, rotation):
        return S.solve(st, xf, model, init=x, newton_max=0, rotation=rotation)[1]["final_energy"]

    assert energy(x_fem, "polar") < energy(x_rig, "polar")
    assert energy(x_rig, "rig") < energy(x_fem, "rig")
    assert np.abs(x_fem - x_rig).max() / st.bbox_diag > 1e-3
    # the FEM solution is stationary: its energy does not fall along random moves
    rng = np.random.default_rng(3)
    free = np.setdiff1d(np.arange(st.n), st.pin_verts)
    e0 = energy(x_fem, "polar")
    for _ in range(3):
        d = np.zeros_like(x_fem)
        d[free] = rng.normal(size=(len(free), 3)) * 1e-4
        assert energy(x_fem + d, "polar") >= e0 - 1e-12 * abs(e0)
