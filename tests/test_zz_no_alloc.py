"""mfem_get_elem_static, the element-output call for callers that may not
allocate device memory after set-up (a per-frame animation loop, a plugin
inside a fixed device budget): called through the C ABI, its results must equal
those of mfem_get_elem on two calls in a row, and meshes above its fixed limit
are refused.  Kept in a file of its own that pytest collects last: a run that
stops at its first failure (-x) has then already run every other GPU test, so a
fault in this optional entry point cannot hide a result of the main path.  The
tests here do not depend on that order: each passes alone in a fresh process."""
import numpy as np
import pytest

from synth import figure_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mfem():
    from paper_2408_04066_gb300 import build, mfem as m
    build.build()
    m.load()
    return m


def test_static_element_outputs_match_allocating_call(mfem):
    import torch
    torch.cuda.set_device(0)
    cfg = figure_config(10000, seeds=range(2))
    cfg["model"] = "snh"
    ctx = mfem.Context.from_config(cfg, precision="mixed")
    for seed in range(2):                     # two calls in a row, different poses
        ctx.set_pose(cfg["xfs"][seed])
        ctx.solve()
        s_ref, lam_ref = ctx.get_elem()
        s, lam = ctx.get_elem_static()
        # same kernel on the same positions: equal up to the parity tolerance (here exact)
        scale = max(np.abs(s_ref).max(), 1.0)
        assert np.abs(s - s_ref).max() <= 1e-12 * scale
        assert np.abs(lam - lam_ref).max() <= 1e-12 * np.abs(lam_ref).max()
    # outputs can be requested one at a time
    s_only = np.full((ctx.m, 6), np.nan)
    lib = mfem.load()
    st = lib.mfem_get_elem_static(ctx._ctx, s_only.ctypes.data_as(mfem._dp), None)
    assert st == mfem.MFEM_OK
    assert np.array_equal(s_only, s)
    ctx.close()


def test_static_element_outputs_refuse_large_meshes(mfem):
    lib = mfem.load()
    cfg = figure_config(80000, seeds=range(1))
    cfg["model"] = "corot"
    ctx = mfem.Context.from_config(cfg, precision="mixed", max_batch=1)
    assert ctx.m > 65536
    with pytest.raises(mfem.MfemError) as e:
        ctx.get_elem_static()
    assert e.value.status == mfem.MFEM_EINVAL
    assert "at most 65536" in str(e.value)
    ctx.close()
