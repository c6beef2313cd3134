"""Write bar_twist_solution.txt: the oracle's solution of the 4x4x16 bar twist
(ARAP, 20 Newton iterations, direct solves) at every 17th vertex.

Calls only the oracle and the seeded input generators.  Run from the repo root:
    python tests/golden/make_bar_golden.py
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle import solve as S  # noqa: E402
from synth import bar_twist_config  # noqa: E402

cfg = bar_twist_config()
st = S.Setup.from_config(cfg)
x, info = S.solve(st, cfg["xfs"][0], "arap", newton_max=20, newton_tol=0.0)
out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bar_twist_solution.txt")
with open(out, "w") as f:
    f.write("# oracle solution of the 4x4x16 bar twist (ARAP, 20 Newton iterations)\n")
    f.write("# written by tests/golden/make_bar_golden.py; columns: vertex x y z\n")
    for v in range(0, st.n, 17):
        f.write(f"{v} {x[v, 0]:.17g} {x[v, 1]:.17g} {x[v, 2]:.17g}\n")
print("wrote", out)
