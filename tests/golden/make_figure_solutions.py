"""Write figure200k_snh_solutions.npz: the oracle's solutions of two poses of
the ~200k-tet stick figure (stable neo-Hookean, E = 1e5, nu = 0.45, seeds 0
and 1), solved with sparse direct Newton steps to |g_free| <= 1e-11
|g_free(x_ref)| (paper §3 Eq. 12, Algorithm 1), sampled at 4096 seeded
vertices.  The GPU parity test of the benchmark's own settings compares
against these; a direct solve of that mesh takes the oracle minutes per pose,
so the values are stored rather than recomputed on the GPU machine.

Calls only the oracle and the seeded input generators.  The file also holds a
checksum of the mesh, so a test notices if the generators drift.  Run from the
repo root (about five minutes, two processes):
    python tests/golden/make_figure_solutions.py
"""
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

SEEDS = (0, 1)
TETS = 200000
N_SAMPLE = 4096


def _one(seed):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import solve as S
    from synth import figure_config
    cfg = figure_config(TETS, seeds=[seed])
    st = S.Setup.from_config(cfg)
    x, info = S.solve(st, cfg["xfs"][0], "snh", newton_max=40, newton_tol=1e-11)
    return seed, x, info["final_rel_grad"], info["newton_iters"], info["g0"]


if __name__ == "__main__":
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    from synth import figure_config
    from golden_util import mesh_checksum
    cfg = figure_config(TETS, seeds=[])
    X, T = cfg["X"], cfg["T"]
    idx = np.sort(np.random.default_rng(7).choice(len(X), N_SAMPLE, replace=False))
    with mp.get_context("spawn").Pool(len(SEEDS)) as pool:
        res = sorted(pool.map(_one, SEEDS), key=lambda r: r[0])
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "figure200k_snh_solutions.npz")
    np.savez_compressed(out, seeds=np.array(SEEDS), idx=idx, x=np.stack([r[1][idx] for r in res]),
                        rel_grad=np.array([r[2] for r in res]), newton_iters=np.array([r[3] for r in res]),
                        g0=np.array([r[4] for r in res]), mesh_checksum=mesh_checksum(X, T),
                        bbox_diag=float(np.linalg.norm(X.max(0) - X.min(0))))
    for r in res:
        print(f"seed {r[0]}: newton {r[3]}, final rel grad {r[2]:.2e}")
    print("wrote", out)
