"""GPU parity for external vertex forces (§4, "Collision response") and for the
vertex energy terms (force work, penalty pins) in the reported energy."""
import numpy as np
import pytest

from oracle import solve as S
from synth import bar_pull_config, figure_config

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
    return figure_config(3000, seeds=range(4), model="snh")


def _poke(cfg, st, per_vertex=30.0, k=9):
    """A push on the k free vertices nearest a point on the chest (a flour-sack
    style local load), and a second field on the back."""
    X = cfg["X"]
    free = np.setdiff1d(np.arange(len(X)), st.pin_verts)
    out = []
    for y, sgn in ((X[:, 1].max(), -1.0), (X[:, 1].min(), 1.0)):
        c = np.array([0.0, y, 0.6])
        sel = free[np.argsort(np.linalg.norm(X[free] - c, axis=1))[:k]]
        f = np.zeros_like(X)
        f[sel] = [0.0, sgn * per_vertex, 0.0]
        out.append(f)
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pulled_bar_closed_form(mfem, precision):
    cfg = bar_pull_config(traction=0.05, mu=1.3)
    opts = dict(newton_tol=1e-12, cg_tol=1e-11, newton_max=10) if precision == "fp64" else \
        dict(newton_tol=1e-9, cg_tol=1e-4, newton_max=20)
    ctx = mfem.Context.from_config(cfg, precision=precision, **opts)
    ctx.set_forces(cfg["f_ext"])
    ctx.set_pose(cfg["xfs"][0])
    x, st = ctx.solve()
    X = cfg["X"]
    want = X + np.outer(X[:, 2] * cfg["traction"] / (2 * cfg["mu"]), [0, 0, 1])
    bbox = np.linalg.norm(X.max(0) - X.min(0))
    assert np.abs(x - want).max() / bbox <= (TOL_FP64 if precision == "fp64" else TOL_MIXED)
    ctx.set_forces(None)                        # removing the force restores the rest shape
    x0, _ = ctx.solve()
    assert np.abs(x0 - X).max() <= 1e-12 * bbox


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_figure_snh_with_local_force(mfem, fig3k, precision):
    so = S.Setup.from_config(fig3k)
    f, _ = _poke(fig3k, so)
    opts = dict(newton_tol=1e-11, cg_tol=1e-9) if precision == "fp64" else dict(newton_tol=1e-9, cg_tol=1e-3)
    ctx = mfem.Context.from_config(fig3k, precision=precision, newton_max=80, **opts)
    ctx.set_forces(f)
    ctx.set_pose(fig3k["xfs"][0])
    x, st = ctx.solve()
    xo, info = S.solve(so, fig3k["xfs"][0], "snh", newton_tol=1e-12, newton_max=80, f_ext=f)
    assert st["converged"] == 1
    e = np.abs(x - xo).max() / so.bbox_diag
    assert e <= (TOL_FP64 if precision == "fp64" else TOL_MIXED), e
    assert abs(st["energy"] - info["final_energy"]) <= 1e-9 * abs(info["final_energy"])
    x_free, _ = S.solve(so, fig3k["xfs"][0], "snh", newton_tol=1e-12)
    assert np.abs(xo - x_free).max() / so.bbox_diag > 1e-3     # the load visibly moves the figure


def test_batch_force_fields(mfem, fig3k):
    so = S.Setup.from_config(fig3k)
    f0, f1 = _poke(fig3k, so)
    fields = np.stack([f0, f1, 0 * f0])
    ctx = mfem.Context.from_config(fig3k, precision="fp64", newton_tol=1e-11, cg_tol=1e-9, max_batch=3)
    ctx.set_forces(fields)
    xb, stb = ctx.solve_batch(fig3k["xfs"][:3])
    for b in range(3):
        xo, _ = S.solve(so, fig3k["xfs"][b], "snh", newton_tol=1e-12, f_ext=fields[b])
        assert np.abs(xb[b] - xo).max() / so.bbox_diag <= TOL_FP64, b
    with pytest.raises(mfem.MfemError) as e:
        ctx.solve_batch(fig3k["xfs"][:4])              # more poses than fields
    assert e.value.status == mfem.MFEM_EINVAL
    ctx.set_forces(f1)                                 # one field shared by every pose
    xs, _ = ctx.solve_batch(fig3k["xfs"][:2])
    xo, _ = S.solve(so, fig3k["xfs"][0], "snh", newton_tol=1e-12, f_ext=f1)
    assert np.abs(xs[0] - xo).max() / so.bbox_diag <= TOL_FP64
    bad = f1.copy()
    bad[3, 1] = np.nan
    with pytest.raises(mfem.MfemError) as e:
        ctx.set_forces(bad)
    assert e.value.status == mfem.MFEM_EINVAL


def test_penalty_energy_and_line_search(mfem, fig3k):
    """SNH under the penalty form: the energy the line search tests includes
    k_s/2 |x_v - x_p|^2, so steps, iterates and the final energy follow the
    oracle's."""
    ks = 1.0e5
    so = S.Setup.from_config(fig3k)
    ctx = mfem.Context.from_config(fig3k, precision="fp64", constraint="penalty", k_s=ks, newton_tol=1e-11,
                                   cg_tol=1e-9, newton_max=80)
    ctx.set_pose(fig3k["xfs"][1])
    x, st = ctx.solve()
    xo, info = S.solve(so, fig3k["xfs"][1], "snh", constraint="penalty", ks=ks, newton_tol=1e-12,
                       newton_max=80)
    assert st["converged"] == 1
    assert np.abs(x - xo).max() / so.bbox_diag <= TOL_FP64
    assert abs(st["energy"] - info["final_energy"]) <= 1e-9 * abs(info["final_energy"])
