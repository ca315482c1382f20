"""Write ``tiny_exact.txt``: exact-rational expected values on a tiny grid.

The expected values come only from ``oracle/bruteforce.py`` (exact rational
evaluation of the interpolation definition); nothing from the CUDA path.  The
grid has two Q subgrids (3 + 4 knots, threshold duplicated), 5 x knots ending
at x = 1, three flavours, and queries inside the grid, on knots, on the
threshold and in all four extrapolation regions.

Run:  python tests/golden/make_golden.py
"""
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.bruteforce import ExactGrid, exact_alphas  # noqa: E402

X = [3e-5, 2e-4, 4e-3, 0.07, 1.0]
NQ = [3, 4]
Q = [1.1, 1.6, 2.5, 2.5, 7.0, 30.0, 200.0]
PIDS = [-2, 0, 3]


def value(r, k, a):
    # a fixed, irregular table (no formula needed: any numbers will do)
    return round(math.sin(1.7 * r + 0.9 * k + 2.3 * a) * 2.0 + 0.25 * a, 6)


def main():
    rows = len(Q)
    V = [[[value(r, k, a) for a in range(len(PIDS))] for k in range(len(X))] for r in range(rows)]
    V[3] = [row[:] for row in V[2]]                  # duplicated threshold row
    AS = [round(0.45 - 0.02 * r, 6) for r in range(rows)]
    AS[3] = AS[2]
    U = [math.log(x) for x in X]
    W = [math.log(q * q) for q in Q]
    Wsub = [W[0:3], W[3:7]]
    queries = [(1e-4, 3.0), (3e-5, 1.21), (0.07, 6.25), (1.0, 40000.0), (0.5, 2.0),
               (2e-3, 6.25), (2e-3, 6.2499), (1e-6, 4.0), (1e-6, 0.5), (0.3, 1e6),
               (0.01, 1.0), (0.9, 900.0), (5e-5, 50000.0), (0.2, 1.3), (1e-3, 20.0)]
    lines = ["# exact-rational expected values, written by make_golden.py from oracle/bruteforce.py",
             "x_knots " + " ".join(repr(v) for v in X),
             "n_q " + " ".join(str(v) for v in NQ),
             "q_knots " + " ".join(repr(v) for v in Q),
             "pids " + " ".join(str(v) for v in PIDS),
             "alphas " + " ".join(repr(v) for v in AS)]
    for r in range(rows):
        for k in range(len(X)):
            lines.append(f"value {r} {k} " + " ".join(repr(v) for v in V[r][k]))
    for x, q2 in queries:
        u, w = math.log(x), math.log(q2)
        outs = []
        for a in range(len(PIDS)):
            Vsub = [[[V[r][k][a] for k in range(len(X))] for r in range(0, 3)],
                    [[V[r][k][a] for k in range(len(X))] for r in range(3, 7)]]
            outs.append(float(ExactGrid(U, Wsub, Vsub).eval(u, w)[0]))
        al = float(exact_alphas(Wsub, [AS[0:3], AS[3:7]], w))
        lines.append(f"query {x!r} {q2!r} " + " ".join(repr(v) for v in outs) + f" alphas {al!r}")
    with open(os.path.join(HERE, "tiny_exact.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
