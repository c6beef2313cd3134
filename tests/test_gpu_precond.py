"""The two-level preconditioner (block Jacobi plus a coarse correction on the
rigid modes of vertex aggregates, rest-shape coarse matrix turned with the rig):
same solutions as block Jacobi and the oracle, fewer PCG iterations, and every
combination of model, precision, constraint and rotation mode still converges."""
import numpy as np
import pytest

from oracle import solve as S
from synth import figure_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mfem():
    from paper_2408_04066_gb300 import build, mfem as m
    build.build()
    m.load()
    return m


@pytest.fixture(scope="module")
def fig10k():
    return figure_config(10000, seeds=range(4), model="snh")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_two_level_matches_block_jacobi_and_oracle(mfem, fig10k, precision):
    so = S.Setup.from_config(fig10k)
    tight = dict(newton_tol=1e-11, cg_tol=1e-9) if precision == "fp64" else dict(newton_tol=1e-9, cg_tol=1e-3)
    tol = 1e-9 if precision == "fp64" else 1e-5
    tl = mfem.Context.from_config(fig10k, precision=precision, max_batch=4, newton_max=80, **tight)
    bj = mfem.Context.from_config(fig10k, precision=precision, max_batch=4, newton_max=80, precond="block_jacobi",
                                  **tight)
    xt, st_t = tl.solve_batch(fig10k["xfs"])
    pt = tl.profile()
    xb, st_b = bj.solve_batch(fig10k["xfs"])
    pb = bj.profile()
    assert pt["coarse_dof"] > 0 and pb["coarse_dof"] == 0 and pt["coarse_launches"] > 0
    for b in range(4):
        assert st_t[b]["converged"] == 1 and st_b[b]["converged"] == 1
        xo, _ = S.solve(so, fig10k["xfs"][b], "snh", newton_tol=1e-12, newton_max=80)
        assert np.abs(xt[b] - xo).max() / so.bbox_diag <= tol
        assert np.abs(xb[b] - xo).max() / so.bbox_diag <= tol


def test_two_level_cuts_pcg_iterations_at_default_tolerances(mfem):
    cfg = figure_config(50000, seeds=range(4), model="snh")
    tl = mfem.Context.from_config(cfg, precision="mixed", max_batch=4)
    bj = mfem.Context.from_config(cfg, precision="mixed", max_batch=4, precond="block_jacobi")
    _, st_t = tl.solve_batch(cfg["xfs"])
    _, st_b = bj.solve_batch(cfg["xfs"])
    it_t = sum(s["pcg_iters"] for s in st_t)
    it_b = sum(s["pcg_iters"] for s in st_b)
    assert all(s["converged"] for s in st_t + st_b)
    assert it_t < 0.7 * it_b, (it_t, it_b)


@pytest.mark.parametrize("model", ["arap", "corot"])
@pytest.mark.parametrize("rotation", ["rig", "polar"])
def test_two_level_other_models_and_rotation_modes(mfem, fig10k, model, rotation):
    cfg = dict(fig10k, model=model)
    so = S.Setup.from_config(cfg)
    ctx = mfem.Context.from_config(cfg, precision="fp64", rotation=rotation, newton_tol=1e-11, cg_tol=1e-9,
                                   newton_max=200)
    ctx.set_pose(cfg["xfs"][1])
    x, st = ctx.solve()
    xo, _ = S.solve(so, cfg["xfs"][1], model, rotation=rotation, newton_tol=1e-12, newton_max=200)
    assert st["converged"] == 1
    assert np.abs(x - xo).max() / so.bbox_diag <= 1e-9


def test_two_level_penalty_mode(mfem, fig10k):
    ks = 1.0e5
    so = S.Setup.from_config(fig10k)
    ctx = mfem.Context.from_config(fig10k, precision="fp64", constraint="penalty", k_s=ks, newton_tol=1e-11,
                                   cg_tol=1e-9, newton_max=80)
    ctx.set_pose(fig10k["xfs"][2])
    x, st = ctx.solve()
    xo, _ = S.solve(so, fig10k["xfs"][2], "snh", constraint="penalty", ks=ks, newton_tol=1e-12, newton_max=80)
    assert st["converged"] == 1
    assert np.abs(x - xo).max() / so.bbox_diag <= 1e-9


def test_graph_replay_equals_direct_launches(mfem, fig10k):
    """PCG chunks replayed from captured CUDA graphs give the same bits as
    launching every kernel."""
    g = mfem.Context.from_config(fig10k, precision="mixed", max_batch=4, launch="graph")
    d = mfem.Context.from_config(fig10k, precision="mixed", max_batch=4, launch="direct")
    for _ in range(2):   # the second solve replays cached graphs
        xg, sg = g.solve_batch(fig10k["xfs"])
        xd, sd = d.solve_batch(fig10k["xfs"])
        assert np.array_equal(xg, xd)
        assert [s["pcg_iters"] for s in sg] == [s["pcg_iters"] for s in sd]
