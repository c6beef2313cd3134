"""GPU parity of the polar-rotation mode (R_k = rotation factor of F_k: the
co-rotational FEM energy of the standard FEM model §4 compares against) with
the oracle: solutions for every model and precision, closed forms, and element
outputs at a state with inverted tets."""
import numpy as np
import pytest

from oracle import solve as S
from synth import bar_mesh, bar_twist_config, figure_config, identity_pose, rigid_pose, rodrigues

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-9
TOL_MIXED = 1e-5


@pytest.fixture(scope="module")
def mfem():
    from paper_2408_04066_gb300 import build, mfem as m
    build.build()
    m.load()
    return m


@pytest.fixture(scope="module")
def fig3k():
    return figure_config(3000, seeds=range(3))


@pytest.mark.parametrize("model", ["arap", "corot", "snh"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_figure_polar_mode_parity(mfem, fig3k, model, precision):
    cfg = dict(fig3k, model=model)
    so = S.Setup.from_config(cfg)
    opts = dict(newton_tol=1e-11, cg_tol=1e-9) if precision == "fp64" else dict(newton_tol=1e-9, cg_tol=1e-3)
    ctx = mfem.Context.from_config(cfg, precision=precision, rotation="polar", newton_max=200, **opts)
    for seed in (0, 1):
        ctx.set_pose(cfg["xfs"][seed])
        x, st = ctx.solve()
        xo, info = S.solve(so, cfg["xfs"][seed], model, rotation="polar", newton_tol=1e-12, newton_max=200)
        assert info["converged"] and st["converged"] == 1, st
        e = np.abs(x - xo).max() / so.bbox_diag
        assert e <= (TOL_FP64 if precision == "fp64" else TOL_MIXED), (seed, e, st)
        if precision == "fp64":
            assert abs(st["energy"] - info["final_energy"]) <= 1e-9 * abs(info["final_energy"])
    xr, _ = S.solve(so, cfg["xfs"][0], model, newton_tol=1e-12)
    ctx.set_pose(cfg["xfs"][0])
    x, _ = ctx.solve()
    assert np.abs(x - xr).max() / so.bbox_diag > 1e-4       # not the rig-rotation solution


def test_bar_twist_polar_mode_fp64(mfem):
    cfg = bar_twist_config()
    so = S.Setup.from_config(cfg)
    ctx = mfem.Context.from_config(cfg, precision="fp64", rotation="polar", newton_tol=1e-11, cg_tol=1e-10,
                                   newton_max=200)
    ctx.set_pose(cfg["xfs"][0])
    x, st = ctx.solve()
    xo, info = S.solve(so, cfg["xfs"][0], "arap", rotation="polar", newton_tol=1e-12, newton_max=200)
    assert st["converged"] == 1 and info["converged"]
    assert np.abs(x - xo).max() / so.bbox_diag <= TOL_FP64


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_polar_mode_rest_and_rigid(mfem, fig3k, precision):
    cfg = dict(fig3k, model="snh")
    H = len(cfg["joints"])
    bbox = np.linalg.norm(cfg["X"].max(0) - cfg["X"].min(0))
    ctx = mfem.Context.from_config(cfg, precision=precision, rotation="polar", newton_tol=1e-10, newton_max=3)
    ctx.set_pose(identity_pose(H))
    x, _ = ctx.solve()
    assert np.abs(x - cfg["X"]).max() <= 1e-12 * bbox
    Q = rodrigues([0.3, -1.0, 0.5], 1.1)
    t = np.array([0.1, 0.2, -0.3])
    ctx.set_pose(rigid_pose(H, Q, t))
    x, _ = ctx.solve()
    assert np.abs(x - (cfg["X"] @ Q.T + t)).max() <= 1e-12 * bbox


def test_polar_element_outputs_with_inverted_tets(mfem, rng):
    X, T = bar_mesh(3, 3, 4)
    cfg = dict(X=X, T=T, joints=np.array([[1.5, 1.5, 0.0]]), parent=np.array([-1]), model="snh", mu=1.0,
               lam=4.0, cluster_rule="joint", pin_verts=np.array([0], dtype=np.int32),
               pin_handle=np.array([0], dtype=np.int32), pin_radius=0.0)
    y = X + 0.45 * rng.normal(size=X.shape)
    so = S.Setup.from_config(cfg)
    from oracle import element
    detF = np.linalg.det(element.deformation_gradient(y, so.T, so.G))
    assert np.sum(detF < 0) >= 5
    ctx = mfem.Context.from_config(cfg, precision="fp64", rotation="polar")
    ctx.set_pose(identity_pose(1))
    ctx.set_state(y)
    s, lam = ctx.get_elem()
    s_o, lam_o = S.element_outputs(so, identity_pose(1), "snh", y, rotation="polar")
    plain = s_o.copy()
    plain[:, 3:] /= np.sqrt(2.0)
    ok = np.abs(detF) > 1e-6                      # away from singular F
    assert np.abs(s - plain)[ok].max() <= 1e-11 * np.abs(plain).max()
    assert np.abs(lam - lam_o)[ok].max() <= 1e-9 * np.abs(lam_o).max()
