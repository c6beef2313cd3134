"""The coarse solve of the two-level preconditioner on the tensor cores
(tcgen05, BF16 operands, FP32 accumulation), through the C ABI
(mfem_coarse_apply), against the FP32 CUDA-core product of the same context.
Inside a solve the same kernel also applies the correction u = zb + P e; the
solve-level tests compare it with the CUDA-core product and its separate
correction kernel.

The tensor-core product stores A_c^{-1} rounded to BF16 (Ahat) and splits each
coarse residual exactly into three BF16 parts, so it must equal Ahat r up to
FP32 accumulation:

* applied to unit vectors it returns the columns of Ahat exactly, and those
  are the FP32 product's columns (the FP32 inverse itself) rounded to BF16
  (round to nearest even) -- a bitwise check of the tiling, the shared-memory
  descriptors, the problem-to-column mapping and the epilogue;
* Ahat is symmetric and positive definite, so the preconditioner stays SPD;
* applied to c e_k with c carrying a full 24-bit significand, the result is
  Ahat e_k c to FP32 rounding (a dropped low part of the split would leave a
  2^-16 error);
* whole solves with either product reach the same solution.
"""
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


@pytest.fixture(scope="module")
def ctx(mfem):
    cfg = figure_config(10000, seeds=range(2), model="snh")
    c = mfem.Context.from_config(cfg, precision="mixed", max_batch=2)
    c.solve_batch(cfg["xfs"][:1])
    yield c, cfg
    c.close()


def _bf16_rn(a):
    """float32 -> nearest BF16 (ties to even), returned as float32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def test_columns_are_the_bf16_inverse(ctx):
    c, _ = ctx
    N = c.profile()["coarse_dof"]
    assert N > 256          # several 30-row groups and more than one 256-column chunk
    eye = np.eye(N, dtype=np.float32)
    e32 = c.coarse_apply(eye, "fp32")          # row b = A_c^{-1} e_b (a column of the inverse)
    etc = c.coarse_apply(eye, "tc")
    assert np.array_equal(e32, e32.T)
    assert np.array_equal(etc, _bf16_rn(e32))
    assert np.array_equal(etc, etc.T)
    kept = np.any(etc != 0, axis=1)            # modes dropped at set-up have zero rows and columns
    assert kept.sum() >= 0.9 * N
    w = np.linalg.eigvalsh(etc[np.ix_(kept, kept)].astype(np.float64))
    assert w.min() > 0.0, w[:4]


def test_three_part_split_is_exact(ctx, rng):
    c, _ = ctx
    N = c.profile()["coarse_dof"]
    kept = np.nonzero(np.any(c.coarse_apply(np.eye(N, dtype=np.float32), "fp32") != 0, axis=1))[0]
    ks = rng.choice(kept, 40, replace=False)
    scale = (1.0 + rng.integers(1, 1 << 23, size=40) * 2.0 ** -23).astype(np.float32)   # 24-bit significands
    scale *= np.float32(2.0) ** rng.integers(-20, 20, size=40).astype(np.float32)
    rc = np.zeros((40, N), np.float32)
    rc[np.arange(40), ks] = scale
    ahat = c.coarse_apply(np.eye(N, dtype=np.float32)[ks], "tc").astype(np.float64)
    got = c.coarse_apply(rc, "tc").astype(np.float64)
    want = ahat * scale.astype(np.float64)[:, None]
    rel = np.abs(got - want).max(axis=1) / np.abs(want).max(axis=1)
    assert rel.max() <= 4e-7, rel.max()


def test_random_vectors_match_ahat(ctx, rng):
    c, _ = ctx
    N = c.profile()["coarse_dof"]
    ahat = c.coarse_apply(np.eye(N, dtype=np.float32), "tc").astype(np.float64)
    rc = rng.standard_normal((20, N)).astype(np.float32)          # 20 problems: two CTA groups
    got = c.coarse_apply(rc, "tc").astype(np.float64)
    want = rc.astype(np.float64) @ ahat.T
    scale = np.abs(rc.astype(np.float64)) @ np.abs(ahat).T
    live = scale > 0                           # rows of dropped modes are exactly zero on both sides
    assert np.all(got[~live] == 0.0)
    assert (np.abs(got - want)[live] / scale[live]).max() <= 2e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solves_agree_across_products(mfem, precision):
    cfg = figure_config(10000, seeds=range(3), model="snh")
    X = cfg["X"]
    bbox = float(np.linalg.norm(X.max(0) - X.min(0)))
    tight = dict(newton_tol=1e-11, cg_tol=1e-9) if precision == "fp64" else dict(newton_tol=1e-9, cg_tol=1e-3)
    out = {}
    for prod in ("tc", "fp32"):
        c = mfem.Context.from_config(cfg, precision=precision, max_batch=3, newton_max=80, coarse_product=prod,
                                     **tight)
        x, st = c.solve_batch(cfg["xfs"])
        p = c.profile()
        c.close()
        assert all(s["converged"] for s in st)
        assert p["coarse_tc"] == (1 if prod == "tc" else 0)
        out[prod] = (x, [s["pcg_iters"] for s in st])
    err = np.abs(out["tc"][0] - out["fp32"][0]).max() / bbox
    assert err <= (1e-9 if precision == "fp64" else 1e-5), err
    for a, b in zip(out["tc"][1], out["fp32"][1]):
        assert abs(a - b) <= max(3, 0.05 * b), (out["tc"][1], out["fp32"][1])


def test_solves_agree_with_two_slot_groups(mfem):
    """20 poses in one batch: request slots 16..19 form a second group of the
    tensor-core kernel's B operand (and a second CTA row of its grid)."""
    cfg = figure_config(10000, seeds=range(20), model="snh")
    X = cfg["X"]
    bbox = float(np.linalg.norm(X.max(0) - X.min(0)))
    out = {}
    for prod in ("tc", "fp32"):
        c = mfem.Context.from_config(cfg, precision="mixed", max_batch=20, newton_max=80, coarse_product=prod,
                                     newton_tol=1e-9, cg_tol=1e-3)
        x, st = c.solve_batch(cfg["xfs"])
        c.close()
        assert all(s["converged"] for s in st)
        out[prod] = (x, [s["pcg_iters"] for s in st])
    err = np.abs(out["tc"][0] - out["fp32"][0]).max() / bbox
    assert err <= 1e-5, err
    for a, b in zip(out["tc"][1], out["fp32"][1]):
        assert abs(a - b) <= max(3, 0.05 * b), (out["tc"][1], out["fp32"][1])
