"""Pins for oracle.solve: rest and rigid closed forms, patch and uniaxial tests,
brute-force minimisation, force balance, scale invariances, penalty limit,
and agreement of the two linear solvers."""
import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import element, rig, solve as S
from synth import (bar_mesh, bar_twist_config, figure_config, identity_pose, rigid_pose,
                   rodrigues, kuhn_voxel_mesh)

MODELS = ["arap", "corot", "snh"]


@pytest.fixture(scope="module")
def fig():
    return figure_config(3000, seeds=range(2))


@pytest.mark.parametrize("model", MODELS)
def test_rest_pose_returns_rest_shape(model, fig):
    st = S.Setup.from_config(fig)
    xf = identity_pose(len(fig["joints"]))
    x, info = S.solve(st, xf, model, init="rest", newton_tol=1e-12, newton_max=3)
    # F(X) = I up to rounding, so the rest gradient is rounding noise
    assert info["gnorm"][0] <= 1e-12 * st.mu.max() * st.vol.sum() / st.bbox_diag
    assert np.abs(x - st.X).max() <= 1e-13 * st.bbox_diag
    assert abs(info["final_energy"]) <= 1e-14 * st.mu.max() * st.vol.sum()


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("init", ["rest", "rigid"])
def test_common_rigid_motion_is_reproduced(model, init, fig):
    """ARAP/corot have one minimiser (E = 0 at the rigid motion) from any start.
    SNH is not convex in S: from the rest shape Newton may end in another
    equilibrium, so for SNH only the rigid start is a closed form."""
    if model == "snh" and init == "rest":
        pytest.skip("SNH from the rest shape need not reach the rigid minimiser")
    st = S.Setup.from_config(fig)
    Q = rodrigues([0.3, -1.0, 0.5], 1.1)
    t = np.array([0.2, -0.4, 0.7])
    x, info = S.solve(st, rigid_pose(len(fig["joints"]), Q, t), model, init=init,
                      newton_tol=1e-13, newton_max=60)
    assert np.abs(x - (st.X @ Q.T + t)).max() <= 1e-9 * st.bbox_diag
    assert abs(info["final_energy"]) <= 1e-12 * np.sum(st.vol) * st.mu.max()


def _single_handle_setup(X, T, pin_verts, mu, lam):
    return S.Setup(X, T, joints=np.zeros((1, 3)), parent=[-1], mu=mu, lam=lam,
                   cluster_rule="joint", pin_verts=pin_verts,
                   pin_handle=np.zeros(len(pin_verts), dtype=np.int64))


@pytest.mark.parametrize("model", MODELS)
def test_patch_test_affine_boundary_gives_affine_interior(model):
    """Boundary pinned to x = A X + c with one rig rotation Q for every tet: the
    affine field has constant stress, so the interior must be exactly affine."""
    X, T = kuhn_voxel_mesh(np.ones((3, 3, 3), bool))
    bnd = np.nonzero(np.any((X == 0) | (X == 3), axis=1))[0]
    Q = rodrigues([1.0, 2.0, 0.5], 0.7)
    U = np.array([[1.05, 0.02, -0.03], [0.02, 0.97, 0.01], [-0.03, 0.01, 1.02]])
    A = Q @ U
    c = np.array([0.3, 0.1, -0.2])
    st = _single_handle_setup(X, T, bnd, 1.3, 4.0)
    x = _solve_with_targets(st, Q, X[bnd] @ A.T + c, model)
    assert np.abs(x - (X @ A.T + c)).max() <= 1e-10


def _solve_with_targets(st, Q, targets, model):
    """Newton with the oracle's pieces but explicit pin targets (a pin-target
    map that is not a rigid handle transform)."""
    R = np.broadcast_to(Q, (st.m, 3, 3))
    x = st.X.copy()
    x[st.pin_verts] = targets
    free = np.ones((st.n, 3), bool)
    free[st.pin_verts] = False
    fidx = np.nonzero(free.reshape(-1))[0]
    args = (st.T, st.G, st.vol, R, model, st.mu, st.lam)
    import scipy.sparse.linalg as spla
    for _ in range(30):
        g = element.gradient(x, *args).reshape(-1)[fidx]
        if np.linalg.norm(g) < 1e-13:
            break
        K = element.assemble(element.element_hessians(x, *args), st.T, st.n)[fidx][:, fidx]
        d = np.zeros(3 * st.n)
        d[fidx] = spla.spsolve(K.tocsc(), -g)
        x = x + d.reshape(st.n, 3)
    return x


@pytest.mark.parametrize("model", ["arap", "corot"])
def test_uniaxial_stretch_without_poisson_effect(model):
    """nu = 0 (lam = 0): a bar with its end faces pulled to diag(1,1,1+e) stays
    exactly diag(1,1,1+e) X (lateral faces carry no traction)."""
    X, T = bar_mesh(2, 2, 6)
    ends = np.nonzero((X[:, 2] == 0) | (X[:, 2] == 6))[0]
    st = _single_handle_setup(X, T, ends, 2.0, 0.0)
    D = np.diag([1.0, 1.0, 1.07])
    x = _solve_with_targets(st, np.eye(3), X[ends] @ D.T, model)
    assert np.abs(x - X @ D.T).max() <= 1e-11


@pytest.mark.parametrize("model", MODELS)
def test_newton_matches_brute_force_minimisation(model, rng):
    """One cube (8 verts), 4 pinned: minimise E over the 12 free coordinates
    with derivative-free-gradient BFGS on the energy alone."""
    X, T = bar_mesh(1, 1, 1)
    joints = np.array([[0.5, 0.5, 0.0], [0.5, 0.5, 1.0]])
    pins = np.array([0, 1, 6, 7])     # corners (0,0,0),(0,0,1),(1,1,0),(1,1,1)
    st = S.Setup(X, T, joints, [-1, -1], 1.0, 3.0, cluster_rule="joint",
                 pin_verts=pins, pin_handle=(X[pins, 2] > 0.5).astype(int))
    xf = np.stack([np.concatenate([rodrigues([0, 0, 1], 0.0), np.zeros((3, 1))], 1).reshape(12),
                   np.concatenate([rodrigues([1, 1, 0], 0.4), np.array([[0.1], [0.0], [0.2]])], 1).reshape(12)])
    x_n, info = S.solve(st, xf, model, init="rest", newton_tol=1e-14, newton_max=60)
    Q, t = rig.unpack_pose(xf)
    R = Q[st.cluster]
    xp = rig.pin_targets(X, pins, st.pin_handle, Q, t)
    free = np.setdiff1d(np.arange(8), pins)

    def E(z):
        x = X.copy()
        x[pins] = xp
        x[free] = z.reshape(-1, 3)
        return element.element_energy(x, T, st.G, st.vol, R, model, st.mu, st.lam).sum()

    res = minimize(E, X[free].reshape(-1), method="BFGS", options=dict(gtol=1e-10, maxiter=5000))
    assert np.abs(res.x.reshape(-1, 3) - x_n[free]).max() < 2e-5
    assert info["final_energy"] <= res.fun + 1e-12


def test_direct_and_cg_solvers_agree():
    cfg = bar_twist_config()
    st = S.Setup.from_config(cfg)
    x1, i1 = S.solve(st, cfg["xfs"][0], "arap", newton_max=20, newton_tol=0.0)
    x2, i2 = S.solve(st, cfg["xfs"][0], "arap", newton_max=20, newton_tol=0.0,
                     linear="cg", cg_tol=1e-13)
    assert np.abs(x1 - x2).max() <= 1e-10 * st.bbox_diag
    # ARAP with rig rotations is quadratic: one solve reaches the minimiser, the
    # other 19 iterations only see rounding-level gradients
    assert i1["gnorm"][1] <= 1e-12 * i1["gnorm"][0]
    assert max(i1["gnorm"][1:]) <= 1e-12 * i1["gnorm"][0]


@pytest.mark.parametrize("model", MODELS)
def test_force_balance_of_multipliers(model, fig):
    """At x*, sum_k W_k B_k^T lambda_k vanishes on free vertices (Eq. 6
    stationarity in x), with lambda_k from element_outputs."""
    st = S.Setup.from_config(fig)
    xf = fig["xfs"][0]
    x, info = S.solve(st, xf, model, newton_tol=1e-11, newton_max=80)
    assert info["converged"]
    s, lam = S.element_outputs(st, xf, model, x)
    f = st.vol[:, None, None] * np.einsum("kij,kaj->kai", lam.reshape(-1, 3, 3), st.G)
    r = np.zeros((st.n, 3))
    np.add.at(r, st.T.reshape(-1), f.reshape(-1, 3))
    free = np.ones(st.n, bool)
    free[st.pin_verts] = False
    scale = np.abs(f).max()
    assert np.abs(r[free]).max() <= 1e-9 * scale
    assert np.abs(r[~free]).max() > 1e-6 * scale          # pins carry the reactions


def test_scale_invariance_in_elimination_mode(fig):
    st1 = S.Setup.from_config(fig)
    st2 = S.Setup.from_config(fig, mu=fig["mu"] * 7.0, lam=fig["lam"] * 7.0)
    for model in MODELS:
        x1, _ = S.solve(st1, fig["xfs"][1], model, newton_tol=1e-12, newton_max=80)
        x2, _ = S.solve(st2, fig["xfs"][1], model, newton_tol=1e-12, newton_max=80)
        assert np.abs(x1 - x2).max() <= 1e-9 * st1.bbox_diag
    # ARAP does not depend on mu at all, even when mu varies per tet
    st3 = S.Setup.from_config(fig, mu=np.random.default_rng(3).uniform(0.1, 10, st1.m))
    x1, _ = S.solve(st1, fig["xfs"][1], "arap", newton_tol=1e-12)
    x3, _ = S.solve(st3, fig["xfs"][1], "arap", newton_tol=1e-12)
    assert np.abs(x1 - x3).max() > 1e-6 * st1.bbox_diag   # heterogeneous mu changes x*
    st4 = S.Setup.from_config(fig, mu=3.3)
    x4, _ = S.solve(st4, fig["xfs"][1], "arap", newton_tol=1e-12)
    assert np.abs(x1 - x4).max() <= 1e-9 * st1.bbox_diag


def test_penalty_converges_to_elimination(fig):
    st = S.Setup.from_config(fig)
    xf = fig["xfs"][0]
    x_inf, _ = S.solve(st, xf, "corot", newton_tol=1e-12)
    errs = []
    for ks in [1e6, 1e7, 1e8]:
        x, _ = S.solve(st, xf, "corot", constraint="penalty", ks=ks, newton_tol=1e-12)
        errs.append(np.abs(x - x_inf).max())
    assert errs[0] > errs[1] > errs[2]
    assert 5.0 < errs[0] / errs[1] < 20.0 and 5.0 < errs[1] / errs[2] < 20.0   # O(1/k_s)


def test_bar_twist_matches_stored_oracle_solution():
    """Regression pin: tests/golden/bar_twist_solution.txt was written by
    tests/golden/make_bar_golden.py from the oracle."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "bar_twist_solution.txt")
    ref = np.loadtxt(path)
    cfg = bar_twist_config()
    st = S.Setup.from_config(cfg)
    x, _ = S.solve(st, cfg["xfs"][0], "arap", newton_max=20, newton_tol=0.0)
    v = ref[:, 0].astype(int)
    assert np.abs(x[v] - ref[:, 1:]).max() <= 1e-12 * st.bbox_diag
    # the twisted end really turned: its pinned face follows handle 1
    assert np.allclose(x[st.pin_verts[st.pin_handle == 1]][:, 2], 16.5)
