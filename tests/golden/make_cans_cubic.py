"""Writes cans_cubic.txt: the minimax odd cubic p(x) = c1 x + c3 x^3 for 1 - p on [a, b]
(the degree-3 CANS step, Appendix A.4 / B.8), computed without the closed form that the
oracle uses: a linear program over a dense grid of [a, b],

    minimize t  subject to  -t <= 1 - c1 x_i - c3 x_i^3 <= t  for every grid point x_i,

solved by scipy's HiGHS.  The degenerate interval a = b = 1 has no unique minimax cubic;
its row is the classical Newton-Schulz step X (3 I - X^T X) / 2 of Section 3, the limit the
CANS steps reach once the interval has collapsed.

    python tests/golden/make_cans_cubic.py
"""
import os

import numpy as np
from scipy.optimize import linprog

HERE = os.path.dirname(os.path.abspath(__file__))
INTERVALS = [(0.1, 1.0), (0.01, 1.99)]


def minimax_cubic(a: float, b: float, points: int = 20001):
    x = np.linspace(a, b, points)
    # variables (c1, c3, t); rows: 1 - c1 x - c3 x^3 <= t  and  -(1 - c1 x - c3 x^3) <= t
    ones = np.ones_like(x)
    a_ub = np.vstack([np.column_stack([-x, -x ** 3, -ones]), np.column_stack([x, x ** 3, -ones])])
    b_ub = np.concatenate([-ones, ones])
    res = linprog(c=[0.0, 0.0, 1.0], A_ub=a_ub, b_ub=b_ub, bounds=[(None, None)] * 3, method="highs")
    if not res.success:
        raise RuntimeError(res.message)
    return res.x


def main():
    lines = ["# Minimax odd cubic p(x) = c1 x + c3 x^3 for 1 - p on [a, b] (degree-3 CANS step,",
             "# Appendix A.4 / B.8), written by tests/golden/make_cans_cubic.py: a linear program on a",
             "# 20001-point grid of [a, b] (no closed form); E is the minimax error.  The a = b = 1 row",
             "# is the classical Newton-Schulz step of Section 3.",
             "# columns: a b c1 c3 E"]
    for a, b in INTERVALS:
        c1, c3, e = minimax_cubic(a, b)
        lines.append(f"{a:<5g} {b:<5g} {c1:.6f}  {c3:.6f}  {e:.6f}")
    lines.append(f"{1.0:<5g} {1.0:<5g} {1.5:.6f}  {-0.5:.6f}  {0.0:.6f}")
    with open(os.path.join(HERE, "cans_cubic.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
