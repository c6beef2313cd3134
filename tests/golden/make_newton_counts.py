"""Write figure200k_newton_steps.txt: Newton steps the oracle takes per pose on
the 200k-tet stick figure (stable neo-Hookean, E = 1e5, nu = 0.45), seeds
0..15, stop at |g_free| <= 1e-6 |g_free(x_ref)|, inexact Newton with the
oracle's Jacobi-PCG at relative tolerance 1e-2.

Calls only the oracle and the seeded input generators; the CPU baseline of
bench.py times single Newton steps and converts them to frames/s with these
counts.  Run from the repo root (several minutes):
    python tests/golden/make_newton_counts.py
"""
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)


def _one(seed):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import solve as S
    from synth import figure_config
    cfg = figure_config(200000, seeds=[seed])
    st = S.Setup.from_config(cfg)
    _, info = S.solve(st, cfg["xfs"][0], "snh", newton_max=100, newton_tol=1e-6, linear="cg", cg_tol=1e-2)
    return seed, info["newton_iters"], int(info["converged"])


if __name__ == "__main__":
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        rows = sorted(pool.map(_one, range(16)))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "figure200k_newton_steps.txt")
    with open(out, "w") as f:
        f.write("# oracle Newton steps per pose: 200k-tet figure, SNH, newton_tol 1e-6, CG 1e-2\n")
        f.write("# written by tests/golden/make_newton_counts.py; columns: seed steps converged\n")
        for s, k, c in rows:
            f.write(f"{s} {k} {c}\n")
    print(open(out).read())
