"""Oracle solves of many poses in parallel, for the GPU parity tests.

The pool uses the spawn start method (a process forked after the first CUDA
call can hang), one oracle solve per task, single-threaded BLAS in each worker.
"""
import concurrent.futures as cf
import multiprocessing as mp
import os


def _solve(cfg, xf, model, kw):
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    from oracle import solve as S
    st = S.Setup.from_config(cfg)
    x, info = S.solve(st, xf, model, **kw)
    return x, info


def solve_many(cfg, xfs, model, workers=None, **kw):
    """Oracle solutions of every pose in xfs (list of (x, info))."""
    n = len(xfs)
    workers = workers or max(1, min(n, (os.cpu_count() or 2) - 1))
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(_solve, cfg, xf, model, kw) for xf in xfs]
        return [f.result() for f in futs]


def solve_jobs(jobs, workers=None):
    """jobs: list of (cfg, xf, model, kw); returns their (x, info) in order."""
    workers = workers or max(1, min(len(jobs), (os.cpu_count() or 2) - 1))
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(_solve, *j) for j in jobs]
        return [f.result() for f in futs]
