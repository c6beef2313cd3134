"""FP64 CPU oracle for the mixed-FEM skinning pose solve.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its cpu_baseline
and reference legs) may import this package.  The product library never calls
it and shares no code with it: no kernels, headers, helpers, tables or pre- and
post-processing.  It is plain numpy/scipy in float64, written for a reader to
check against the paper by eye, not for speed.

What it computes (paper §3, Eq. 5-6 and Eq. 10-12, Algorithm 1):
  per tet k:  F_k = B_k x (Eq. 4 text), S_k = sym(R_k^T F_k) -- the least-squares
  solution of F_k = R_k S_k, i.e. the batched pseudo-inverse of [R] (Eq. 12 text),
  with R_k the rotation of the rig handle of the tet's rotation cluster (§3.1);
  E(x) = sum_k W_k Psi(S_k) (+ the pin penalty C(x) of Eq. 6 in penalty mode);
  pinned vertices follow x_p = H x_hat_p (§3.2, "Initial shape preservation");
  x* minimises E; Newton on E with the condensed SPD Hessian of Eq. 12.

Modules: ``mandel`` (6-vector form of symmetric S), ``material`` (Psi and its
derivatives), ``element`` (F, S, energy, gradient, Hessian), ``rig``
(clusters, pins, pose targets), ``solve`` (Newton driver), ``diag`` (polar
decomposition and per-element diagnostics).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, finite differences, brute-force minimisation, library
least squares, or invariants; none is "parity unpinned".
"""
from . import mandel, material, element, rig, solve, diag  # noqa: F401
