"""Serving on the GPU: continuous batching over resident meshes.  Every request's
result equals the same pose solved alone (same kernels, per-problem
deterministic reductions)."""
import numpy as np
import pytest

from synth import bar_twist_config, figure_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mfem():
    from paper_2408_04066_gb300 import build, mfem as m
    build.build()
    m.load()
    return m


def test_served_results_equal_alone(mfem):
    figA = dict(figure_config(3000, seeds=range(5)), model="snh")
    figB = dict(figure_config(10000, seeds=range(5, 10)), model="corot")
    opts = dict(precision="mixed", tile_rows=128)
    alone = {}
    for name, cfg in (("A", figA), ("B", figB)):
        ctx = mfem.Context.from_config(cfg, **opts)
        for i, xf in enumerate(cfg["xfs"]):
            x, st = ctx.solve_batch(xf[None])
            alone[(name, i)] = (x[0], st[0])
        ctx.close()
    srv = mfem.Server(device_mem_budget=0, max_slots=4)
    ids = {"A": srv.add(mfem.Context.from_config(figA, **opts)),
           "B": srv.add(mfem.Context.from_config(figB, **opts))}
    tickets = []
    for i in range(5):   # interleave meshes; more requests than slots
        for name, cfg in (("A", figA), ("B", figB)):
            tickets.append(((name, i), srv.submit(ids[name], cfg["xfs"][i])))
    for key, t in tickets:
        out, st, lat = srv.wait(t, timeout_ms=120000)
        xa, sa = alone[key]
        assert np.array_equal(out, xa), key
        assert st["newton_iters"] == sa["newton_iters"]
        assert lat > 0
    c = srv.counters()
    assert c["completed"] == 10 and c["peak_slots"] <= 4
    srv.close()


def test_server_rejects_bad_requests(mfem):
    cfg = bar_twist_config()
    srv = mfem.Server(max_slots=2)
    mid = srv.add(mfem.Context.from_config(cfg, precision="mixed"))
    bad = cfg["xfs"][0].copy()
    bad[1, 0] = 2.0
    with pytest.raises(mfem.MfemError):
        srv.submit(mid, bad)
    with pytest.raises(mfem.MfemError):
        srv.submit(mid + 5, cfg["xfs"][0])
    t = srv.submit(mid, cfg["xfs"][0])
    res = srv.wait(t, timeout_ms=60000)
    assert res is not None and res[1]["converged"] == 1
    srv.close()


def test_server_budget_refuses_too_large_mesh(mfem):
    cfg = figure_config(3000, seeds=[])
    cfg["model"] = "corot"
    srv = mfem.Server(device_mem_budget=1 << 16, max_slots=2)   # 64 KiB: no slot fits
    with pytest.raises(mfem.MfemError) as e:
        srv.add(mfem.Context.from_config(cfg, precision="mixed"))
    assert e.value.status == mfem.MFEM_ENOMEM
    srv.close()


def test_served_animation_continues_from_the_latest_frame(mfem):
    """WARM meshes keep their latest solution resident: frames of one animation
    submitted one after another reach the oracle's solutions, and after the
    first frame take fewer Newton steps than frames started cold."""
    from oracle import solve as S
    from synth import figure_animation
    cfg = dict(figure_config(3000, seeds=[]), model="snh")
    anim = figure_animation(cfg["joints"], cfg["parent"], 21, 6)
    so = S.Setup.from_config(cfg)
    srv = mfem.Server(max_slots=4)
    mid = srv.add(mfem.Context.from_config(cfg, precision="fp64", init="warm", newton_tol=1e-10, cg_tol=1e-8))
    cold = mfem.Context.from_config(cfg, precision="fp64", newton_tol=1e-10, cg_tol=1e-8)
    warm_it, cold_it = [], []
    for f in range(6):
        out, st, _ = srv.wait(srv.submit(mid, anim[f]), timeout_ms=120000)
        xo, _ = S.solve(so, anim[f], "snh", newton_tol=1e-12)
        assert st["converged"] == 1
        assert np.abs(out - xo).max() / so.bbox_diag <= 1e-8, f
        cold.set_pose(anim[f])
        _, sc = cold.solve()
        if f > 0:
            warm_it.append(st["newton_iters"])
            cold_it.append(sc["newton_iters"])
    assert sum(warm_it) < sum(cold_it), (warm_it, cold_it)
    srv.close()


def test_admission_by_device_memory_grows_and_releases_slot_pools(mfem):
    """A mesh starts with one pool of 8 request slots; a burst of requests gets
    further pools (sharing the mesh's device data) while the budget has room,
    the rest wait in the queue; every result equals the pose solved alone; pools
    idle for two seconds are released and their memory returns to the budget."""
    import time
    cfg = dict(figure_config(3000, seeds=range(20)), model="snh")
    opts = dict(precision="mixed", tile_rows=128)
    alone = mfem.Context.from_config(cfg, **opts)
    ref = [alone.solve_batch(cfg["xfs"][i:i + 1])[0][0] for i in range(20)]
    probe = mfem.Server(max_slots=64)
    probe.add(mfem.Context.from_config(cfg, **opts))
    one_pool = probe.counters()["device_bytes"]           # the first pool: 8 slots
    probe.close()
    budget = int(2.6 * one_pool)                           # room for two more pools of 8 slots at most
    srv = mfem.Server(device_mem_budget=budget, max_slots=64)
    mid = srv.add(mfem.Context.from_config(cfg, **opts))
    tickets = [srv.submit(mid, cfg["xfs"][i]) for i in range(20)]
    for i, t in enumerate(tickets):
        out, st, _ = srv.wait(t, timeout_ms=120000)
        assert st["converged"] == 1
        assert np.array_equal(out, ref[i]), i
    c = srv.counters()
    assert c["completed"] == 20 and c["pools_added"] >= 1
    assert 8 < c["peak_slots"] <= 24 and c["device_bytes"] <= budget
    time.sleep(2.3)
    out, st, _ = srv.wait(srv.submit(mid, cfg["xfs"][3]), timeout_ms=120000)   # wakes the worker: idle pools go
    assert np.array_equal(out, ref[3])
    c2 = srv.counters()
    assert c2["pools_released"] >= 1 and c2["device_bytes"] < c["device_bytes"]
    srv.close()
    alone.close()
