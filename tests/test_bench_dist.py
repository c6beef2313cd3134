"""bench.py's replica aggregation across ranks (the N-GPU path is replicas only:
no collective on the data path, only the timing max and pose counts), run as
two gloo processes on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    d = bench.Dist()
    try:
        assert d.world == world and d.rank == rank
        d.barrier()
        t_max = d.max(10.0 + rank)            # per-rank step time in ms
        poses = d.sum(16)                     # poses each replica solved
        out[rank] = (t_max, poses, 1e3 * poses / t_max)
    finally:
        d.close()


def test_two_replicas_aggregate_with_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    t_max, poses, value = res[0]
    assert t_max == 11.0 and poses == 32
    assert value == pytest.approx(32 / 0.011)     # whole-job throughput over the slowest rank


def test_single_process_needs_no_process_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    import bench
    d = bench.Dist()
    assert d.world == 1 and d.pg is None
    assert d.max(3.0) == 3.0 and d.sum(5) == 5


def _json_lines(text):
    import json
    return [json.loads(l) for l in text.splitlines() if l.startswith("{")]


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the oracle arm) on a small figure: one JSON
    line with the contract's keys; its e2e moves no bytes (host program)."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--tets", "3000"], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    for k in ("metric", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "scaling", "dtype", "data", "config"):
        assert k in d, k
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_under_torchrun_prints_on_rank_zero_only():
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0", "--tets", "3000"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2


def test_oracle_on_all_cores_runs_one_pose_per_process():
    """The all-core CPU baseline: spawned oracle processes time one full frame
    each, started together; a failing process is reported, not waited on."""
    import bench
    times = bench.oracle_concurrent_frame_times(3000, "snh", 2)
    assert len(times) == 2 and all(isinstance(t, float) and t > 0 for t in times)
    with pytest.raises(RuntimeError):
        bench.oracle_concurrent_frame_times(3000, "no-such-model", 2)


def test_single_thread_baseline_times_five_frames():
    """cpu_baseline: the median of 5 full oracle frames after a warm-up frame."""
    import argparse
    import bench
    d = bench.cpu_baseline(argparse.Namespace(tets=3000, model="snh"))
    assert d["kind"] == "oracle" and d["cores"] == 1 and d["value"] > 0
    assert d["sample"].startswith("median of 5 frames")
    assert d["sample"].count(",") >= 4          # five frame times listed


def test_roofline_arithmetic():
    """`roofline` of the JSON line: achieved = algorithmic bytes / PCG time,
    frac = achieved / peak, traffic = (the ncu record's row-kernel bytes per
    pose-iteration x pose-iterations + its coarse-product bytes per launch x
    coarse launches) per launch pair (or None without a record for the current
    kernel source)."""
    import bench
    profs = [dict(pcg_ms=2.0, pcg_bytes=8e9, pcg_launches=40, pcg_iters=100, coarse_launches=15),
             dict(pcg_ms=3.0, pcg_bytes=12e9, pcg_launches=60, pcg_iters=140, coarse_launches=25)]
    r = bench._roofline(profs, total_ms=10.0, mesh=(198474, 40103))
    peak, kind = bench.hbm_peak()
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == peak
    assert r["achieved"] == pytest.approx(20e9 / 5e-3 / 1e9)           # 4000 GB/s
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["launch_pairs"] == 50 and r["pose_iterations_per_pair"] == pytest.approx(240 / 50)
    assert r["share_of_step"] == pytest.approx(0.5)
    rec = bench.pcg_traffic_record((198474, 40103))
    assert bench._roofline(profs, total_ms=10.0, mesh=(10, 20))["traffic"] is None   # another mesh: no record
    if rec is None:
        assert r["traffic"] is None
    else:
        assert r["traffic"] == pytest.approx((rec["row_dram_bytes_per_pose_iteration"] * 240
                                              + rec["coarse_dram_bytes_per_launch"] * 40) / 50)
    fake = {"row_dram_bytes_per_pose_iteration": 3.0, "coarse_dram_bytes_per_launch": 100.0}
    assert bench.pcg_traffic(fake, 10, 2, 4) == pytest.approx((30 + 200) / 4)
    assert bench.pcg_traffic(None, 10, 2, 4) is None
