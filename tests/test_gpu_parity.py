"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (positions, max |x_gpu - x_oracle| / bbox diagonal): 1e-9 for the
FP64 path and 1e-5 for the mixed FP32/FP64 path.  Both sides solve to tight
gradient tolerances so the comparison measures the arithmetic, not the stop
rule.
"""
import numpy as np
import pytest

from oracle import solve as S, diag
from synth import bar_twist_config, character_config, figure_config, identity_pose, rigid_pose, rodrigues, bar_mesh

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
def fig10k():
    return figure_config(10000, seeds=range(4))


@pytest.fixture(scope="module")
def fig3k():
    return figure_config(3000, seeds=range(6))


def _err(x, ref, st):
    return np.abs(x - ref).max() / st.bbox_diag


def test_bar_twist_fp64(mfem):
    cfg = bar_twist_config()
    ctx = mfem.Context.from_config(cfg, precision="fp64", newton_tol=0.0, newton_max=20, cg_tol=1e-10)
    ctx.set_pose(cfg["xfs"][0])
    x, st = ctx.solve()
    so = S.Setup.from_config(cfg)
    xo, info = S.solve(so, cfg["xfs"][0], "arap", newton_max=20, newton_tol=0.0)
    assert _err(x, xo, so) <= TOL_FP64
    gold = np.loadtxt(__file__.replace("test_gpu_parity.py", "golden/bar_twist_solution.txt"))
    assert np.abs(x[gold[:, 0].astype(int)] - gold[:, 1:]).max() / so.bbox_diag <= TOL_FP64
    assert st["newton_iters"] == 20
    assert st["rel_grad"] <= 1e-9          # one solve reaches the minimiser
    assert st["status"] == mfem.MFEM_ENOTCONV or st["status"] == mfem.MFEM_OK


def test_bar_twist_mixed(mfem):
    cfg = bar_twist_config()
    ctx = mfem.Context.from_config(cfg, precision="mixed", newton_tol=1e-9, newton_max=40, cg_tol=1e-3)
    ctx.set_pose(cfg["xfs"][0])
    x, st = ctx.solve()
    so = S.Setup.from_config(cfg)
    xo, _ = S.solve(so, cfg["xfs"][0], "arap", newton_max=20, newton_tol=0.0)
    assert st["converged"] == 1
    assert _err(x, xo, so) <= TOL_MIXED


@pytest.mark.parametrize("model", ["arap", "corot", "snh"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_figure_parity(mfem, fig10k, model, precision):
    cfg = dict(fig10k, model=model)
    so = S.Setup.from_config(cfg)
    opts = dict(precision=precision, newton_max=80)
    if precision == "fp64":
        opts.update(newton_tol=1e-11, cg_tol=1e-9)
    else:
        opts.update(newton_tol=1e-9, cg_tol=1e-3)
    ctx = mfem.Context.from_config(cfg, **opts)
    for seed in (0, 1):
        ctx.set_pose(cfg["xfs"][seed])
        x, st = ctx.solve()
        xo, info = S.solve(so, cfg["xfs"][seed], model, newton_tol=1e-12, newton_max=80)
        assert st["converged"] == 1, st
        e = _err(x, xo, so)
        assert e <= (TOL_FP64 if precision == "fp64" else TOL_MIXED), (seed, e, st)


def test_element_outputs(mfem, fig10k):
    cfg = dict(fig10k, model="snh")
    ctx = mfem.Context.from_config(cfg, precision="fp64", newton_tol=1e-10, cg_tol=1e-8)
    ctx.set_pose(cfg["xfs"][2])
    x, _ = ctx.solve()
    s, lam = ctx.get_elem()
    so = S.Setup.from_config(cfg)
    s_o, lam_o = S.element_outputs(so, cfg["xfs"][2], "snh", x)
    # oracle s is Mandel; the ABI returns plain components (S00,S11,S22,S12,S02,S01)
    plain = s_o.copy()
    plain[:, 3:] /= np.sqrt(2.0)
    assert np.abs(s - plain).max() <= 1e-12 * np.abs(plain).max()
    assert np.abs(lam - lam_o).max() <= 1e-10 * np.abs(lam_o).max()


def test_diagnostics(mfem, fig10k):
    cfg = dict(fig10k, model="corot")
    ctx = mfem.Context.from_config(cfg, precision="mixed", diagnostics=1)
    ctx.set_pose(cfg["xfs"][1])
    x, st = ctx.solve()
    so = S.Setup.from_config(cfg)
    d = diag.diagnostics(so, cfg["xfs"][1], x)
    assert st["inverted"] == d["inverted"]
    assert abs(st["max_rel_skew"] - d["max_rel_skew"]) <= 1e-5
    if d["inverted"] == 0:
        assert abs(st["max_angle"] - d["max_angle"]) <= 1e-4


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_alone(mfem, fig3k, precision):
    cfg = dict(fig3k, model="snh")
    xfs = cfg["xfs"][:4]
    ctx = mfem.Context.from_config(cfg, precision=precision, max_batch=4)
    xb, stb = ctx.solve_batch(xfs)
    for b in range(4):
        xa, sta = ctx.solve_batch(xfs[b:b + 1])
        assert np.array_equal(xa[0], xb[b])
        assert sta[0]["newton_iters"] == stb[b]["newton_iters"]
        assert sta[0]["pcg_iters"] == stb[b]["pcg_iters"]


def test_batch_host_and_device_memory_agree(mfem, fig3k):
    import torch
    cfg = dict(fig3k, model="corot")
    ctx = mfem.Context.from_config(cfg, precision="mixed", max_batch=6)
    xh, _ = ctx.solve_batch(cfg["xfs"])
    xd, _ = ctx.solve_batch(torch.tensor(cfg["xfs"], device="cuda"))
    assert np.array_equal(xh, xd.cpu().numpy())


def test_penalty_mode(mfem):
    cfg = bar_twist_config()
    ks = 1.0e3
    ctx = mfem.Context.from_config(cfg, precision="fp64", constraint="penalty", k_s=ks, newton_tol=1e-12,
                                   cg_tol=1e-11, newton_max=10)
    ctx.set_pose(cfg["xfs"][0])
    x, st = ctx.solve()
    so = S.Setup.from_config(cfg)
    xo, _ = S.solve(so, cfg["xfs"][0], "arap", constraint="penalty", ks=ks, newton_tol=1e-13)
    assert _err(x, xo, so) <= TOL_FP64
    # penalty pins are soft: the twisted face is near, not at, its target
    xe, _ = S.solve(so, cfg["xfs"][0], "arap", newton_tol=1e-13)
    assert 1e-6 < _err(x, xe, so) < 1e-1


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_rest_and_rigid_closed_forms(mfem, fig3k, precision):
    cfg = dict(fig3k, model="snh")
    H = len(cfg["joints"])
    ctx = mfem.Context.from_config(cfg, precision=precision, newton_tol=1e-10)
    ctx.set_pose(identity_pose(H))
    x, st = ctx.solve()
    bbox = np.linalg.norm(cfg["X"].max(0) - cfg["X"].min(0))
    assert np.abs(x - cfg["X"]).max() <= 1e-12 * bbox
    Q = rodrigues([0.2, 1.0, -0.4], 0.9)
    t = np.array([0.3, -0.2, 0.1])
    ctx.set_pose(rigid_pose(H, Q, t))
    x, st = ctx.solve()
    assert np.abs(x - (cfg["X"] @ Q.T + t)).max() <= 1e-12 * bbox


def test_tiny_and_ragged_meshes(mfem):
    """A single tet (4 verts, 3 pinned) and a 3x1x1 bar (ragged slices and tiles)."""
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    T = np.array([[0, 1, 2, 3]])
    joints = np.array([[0.3, 0.3, 0.0], [0.0, 0.0, 1.0]])
    pins = np.array([0, 1, 2])
    cfg = dict(X=X, T=T, joints=joints, parent=np.array([-1, -1]), model="corot", mu=1.0, lam=2.0,
               cluster_rule="joint", pin_verts=pins, pin_handle=np.array([0, 0, 0]), pin_radius=0.0)
    xf = np.stack([np.concatenate([rodrigues([0, 0, 1], 0.3), [[0.1], [0], [0]]], 1).reshape(12),
                   np.concatenate([rodrigues([1, 0, 0], -0.5), [[0], [0.2], [0]]], 1).reshape(12)])
    for prec, tol in (("fp64", TOL_FP64), ("mixed", TOL_MIXED)):
        ctx = mfem.Context.from_config(cfg, precision=prec, newton_tol=1e-12, cg_tol=1e-10)
        ctx.set_pose(xf)
        x, st = ctx.solve()
        so = S.Setup.from_config(cfg)
        xo, _ = S.solve(so, xf, "corot", newton_tol=1e-13)
        assert _err(x, xo, so) <= tol
    X, T = bar_mesh(3, 1, 1)
    joints = np.array([[0.5, 0.5, 0.0], [0.5, 0.5, 1.0]])
    ends = np.nonzero((X[:, 2] == 0) | (X[:, 2] == 1))[0][:6]
    cfg = dict(X=X, T=T, joints=joints, parent=np.array([-1, 0]), model="snh", mu=3.0, lam=10.0,
               cluster_rule="bone", pin_verts=ends, pin_handle=(X[ends, 2] > 0.5).astype(int), pin_radius=0)
    xf = np.stack([np.concatenate([np.eye(3), np.zeros((3, 1))], 1).reshape(12),
                   np.concatenate([rodrigues([0, 1, 0], 0.2), [[0.05], [0], [0.05]]], 1).reshape(12)])
    ctx = mfem.Context.from_config(cfg, precision="fp64", newton_tol=1e-12, cg_tol=1e-10)
    ctx.set_pose(xf)
    x, _ = ctx.solve()
    so = S.Setup.from_config(cfg)
    xo, _ = S.solve(so, xf, "snh", newton_tol=1e-13)
    assert _err(x, xo, so) <= TOL_FP64


def test_error_codes(mfem, fig3k):
    cfg = dict(fig3k, model="snh")
    ctx = mfem.Context.from_config(cfg, precision="mixed")
    bad = cfg["xfs"][0].copy()
    bad[3, 0] *= 1.01                                   # not a rotation
    with pytest.raises(mfem.MfemError) as e:
        ctx.set_pose(bad)
    assert e.value.status == mfem.MFEM_EINVAL
    bad = cfg["xfs"][0].copy()
    bad[0, 5] = np.inf
    with pytest.raises(mfem.MfemError):
        ctx.solve_batch(bad[None])
    with pytest.raises(mfem.MfemError) as e:
        ctx.solve()                                     # no pose set yet
    # iteration cap: ENOTCONV still returns the best x
    ctx2 = mfem.Context.from_config(cfg, precision="mixed", newton_max=1, newton_tol=1e-12)
    ctx2.set_pose(cfg["xfs"][0])
    x, st = ctx2.solve()
    assert st["status"] == mfem.MFEM_ENOTCONV and st["newton_iters"] == 1
    assert np.all(np.isfinite(x))
    with pytest.raises(mfem.MfemError) as e:
        T = cfg["T"].copy()
        T[7, [1, 2]] = T[7, [2, 1]]
        mfem.Context(cfg["X"], T, cfg["joints"], cfg["parent"], pin_radius=cfg["pin_radius"])
    assert e.value.status == mfem.MFEM_EDEGEN


def test_warm_state_roundtrip(mfem, fig3k):
    cfg = dict(fig3k, model="corot")
    ctx = mfem.Context.from_config(cfg, precision="fp64", init="warm", newton_tol=1e-10, cg_tol=1e-8)
    ctx.set_pose(cfg["xfs"][0])
    x0, st0 = ctx.solve()
    assert np.array_equal(ctx.get_state(), x0)
    x1, st1 = ctx.solve()                         # warm start at the solution: no step needed
    assert st1["newton_iters"] == 0 or st1["rel_grad"] <= 1e-10
    ctx.set_state(cfg["X"])
    x2, _ = ctx.solve()
    bbox = np.linalg.norm(cfg["X"].max(0) - cfg["X"].min(0))
    assert np.abs(x2 - x0).max() <= 1e-8 * bbox  # unique minimiser from any start


def test_full_size_figure_property_check(mfem):
    """200k tets, the bench's launch configuration (mixed, batch): the FP64
    free gradient recomputed by the oracle at the GPU solution meets the
    1e-6 relative tolerance, and sampled element outputs match the oracle."""
    cfg = figure_config(200000, seeds=(0, 5))
    cfg["model"] = "snh"
    ctx = mfem.Context.from_config(cfg, precision="mixed", max_batch=2)
    xb, stb = ctx.solve_batch(cfg["xfs"])
    so = S.Setup.from_config(cfg)
    from oracle import element, rig
    for b in range(2):
        assert stb[b]["converged"] == 1
        Q, t = rig.unpack_pose(cfg["xfs"][b])
        R = Q[so.cluster]
        args = (so.T, so.G, so.vol, R, "snh", so.mu, so.lam)
        g = element.gradient(xb[b], *args)
        g[so.pin_verts] = 0.0
        x0 = S.initial_guess(so, Q, t, "rigid")
        x0[so.pin_verts] = rig.pin_targets(so.X, so.pin_verts, so.pin_handle, Q, t)
        g0 = element.gradient(x0, *args)
        g0[so.pin_verts] = 0.0
        rel = np.linalg.norm(g) / np.linalg.norm(g0)
        assert rel <= 1.5e-6, rel
        assert abs(stb[b]["rel_grad"] - rel) <= 1e-3 * rel + 1e-9
        # pins sit exactly on their targets
        xp = rig.pin_targets(so.X, so.pin_verts, so.pin_handle, Q, t)
        assert np.abs(xb[b][so.pin_verts] - xp).max() <= 1e-12 * so.bbox_diag


def test_rig_above_the_staged_handle_limit(mfem):
    """Rigs above the element kernels' staged-handle limit (64) read the pose
    rotations from global memory: an 80-handle character on the 10k-tet
    capsule mesh, FP64 solved tightly against the oracle, and mixed (the
    float-float element pass) at the default tolerance by the oracle's FP64
    gradient and energy at its solutions."""
    from oracle import element, rig
    cfg = character_config(10000, n_handles=80, seeds=range(2), max_angle_deg=15.0)
    assert len(cfg["joints"]) == 80
    so = S.Setup.from_config(cfg)
    ctx = mfem.Context.from_config(cfg, precision="fp64", newton_tol=1e-11, cg_tol=1e-9, newton_max=80)
    ctx.set_pose(cfg["xfs"][0])
    x, st = ctx.solve()
    xo, info = S.solve(so, cfg["xfs"][0], "snh", newton_tol=1e-12, newton_max=80)
    assert st["converged"] == 1, st
    assert _err(x, xo, so) <= TOL_FP64
    ctx = mfem.Context.from_config(cfg, precision="mixed", max_batch=2)
    xb, stb = ctx.solve_batch(cfg["xfs"])
    for b in range(2):
        assert stb[b]["converged"] == 1
        Q, t = rig.unpack_pose(cfg["xfs"][b])
        args = (so.T, so.G, so.vol, Q[so.cluster], "snh", so.mu, so.lam)
        g = element.gradient(xb[b], *args)
        g[so.pin_verts] = 0.0
        x0 = S.initial_guess(so, Q, t, "rigid")
        x0[so.pin_verts] = rig.pin_targets(so.X, so.pin_verts, so.pin_handle, Q, t)
        g0 = element.gradient(x0, *args)
        g0[so.pin_verts] = 0.0
        assert np.linalg.norm(g) / np.linalg.norm(g0) <= 1.5e-6
        en = float(np.sum(element.element_energy(xb[b], *args)))
        assert abs(stb[b]["energy"] - en) <= 1e-10 * abs(en)
