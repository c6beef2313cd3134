"""Several meshes in one solve (mfem_solve_multi) and warm-started animation
streams: results equal each pose solved alone, and warm starts reach the
oracle's solution of every frame."""
import numpy as np
import pytest

from oracle import solve as S
from synth import bar_twist_config, figure_animation, figure_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mfem():
    from paper_2408_04066_gb300 import build, mfem as m
    build.build()
    m.load()
    return m


@pytest.fixture(scope="module")
def meshes():
    return [dict(figure_config(3000, seeds=range(3)), model="snh"),
            dict(figure_config(10000, seeds=range(3, 5), scale=0.5), model="corot")]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_multi_equals_alone(mfem, meshes, precision):
    # the SpMV shape is fixed: contexts that autotune it separately may pick
    # different splits of a row's sum, which round differently
    ctxs = [mfem.Context.from_config(c, precision=precision, max_batch=3, tile_rows=128, spmv_split=1)
            for c in meshes]
    outs, stats = mfem.solve_multi(ctxs, [c["xfs"] for c in meshes])
    for i, cfg in enumerate(meshes):
        alone = mfem.Context.from_config(cfg, precision=precision, max_batch=3, tile_rows=128, spmv_split=1)
        for b in range(len(cfg["xfs"])):
            x, st = alone.solve_batch(cfg["xfs"][b:b + 1])
            assert np.array_equal(x[0], outs[i][b]), (i, b)
            assert st[0]["newton_iters"] == stats[i][b]["newton_iters"]
            assert st[0]["pcg_iters"] == stats[i][b]["pcg_iters"]
        alone.close()
    # device buffers give the same answers
    import torch
    outs_d, _ = mfem.solve_multi(ctxs, [torch.tensor(c["xfs"], device="cuda") for c in meshes])
    for i in range(2):
        assert np.array_equal(outs_d[i].cpu().numpy(), outs[i])
    with pytest.raises(mfem.MfemError):
        mfem.solve_multi([ctxs[0], ctxs[0]], [meshes[0]["xfs"], meshes[0]["xfs"]])


def test_warm_started_animation_reaches_each_frame(mfem, meshes):
    cfg = meshes[0]
    so = S.Setup.from_config(cfg)
    anim = np.stack([figure_animation(cfg["joints"], cfg["parent"], s, 5) for s in (7, 8)], axis=1)
    tight = dict(precision="fp64", max_batch=2, newton_tol=1e-10, cg_tol=1e-8)
    warm = mfem.Context.from_config(cfg, init="warm", **tight)
    cold = mfem.Context.from_config(cfg, init="corot", **tight)
    other = mfem.Context.from_config(meshes[1], precision="fp64", max_batch=2, newton_tol=1e-10, cg_tol=1e-8)
    for f in range(3):
        (xw, _), (sw, _) = mfem.solve_multi([warm, other], [anim[f], meshes[1]["xfs"]])
        if f == 0:        # no previous solve in the slots: the COROT start
            xc, sc = cold.solve_batch(anim[f])
            assert np.array_equal(xw, xc)
            assert [s["newton_iters"] for s in sw] == [s["newton_iters"] for s in sc]
        for b in range(2):
            xo, _ = S.solve(so, anim[f][b], "snh", newton_tol=1e-12)
            assert np.abs(xw[b] - xo).max() / so.bbox_diag <= 1e-8, (f, b)
    # at the solver's default tolerances the carried correction saves Newton steps
    warm_d = mfem.Context.from_config(cfg, init="warm", precision="mixed", max_batch=2)
    cold_d = mfem.Context.from_config(cfg, init="corot", precision="mixed", max_batch=2)
    iw, ic = [], []
    for f in range(5):
        _, sw = warm_d.solve_batch(anim[f])
        _, sc = cold_d.solve_batch(anim[f])
        assert all(s["converged"] for s in sw + sc)
        if f > 0:
            iw += [s["newton_iters"] for s in sw]
            ic += [s["newton_iters"] for s in sc]
    assert sum(iw) < sum(ic), (iw, ic)
    # a caller's state is used as it is
    warm.set_state(cfg["X"])
    x, st = warm.solve_batch(anim[4][:1])
    xo, _ = S.solve(so, anim[4][0], "snh", newton_tol=1e-12)
    assert np.abs(x[0] - xo).max() / so.bbox_diag <= 1e-8
    for c in (warm, cold, other, warm_d, cold_d):
        c.close()
