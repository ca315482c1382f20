"""Reader for ``tests/golden/tiny_exact.txt``."""
import os

import numpy as np

from paper_2012_08221_gb300 import synth

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tiny_exact.txt")


def load():
    head, vals, queries = {}, {}, []
    with open(PATH) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            if tok[0] == "value":
                vals[(int(tok[1]), int(tok[2]))] = [float(t) for t in tok[3:]]
            elif tok[0] == "query":
                i = tok.index("alphas")
                queries.append((float(tok[1]), float(tok[2]),
                                [float(t) for t in tok[3:i]], float(tok[i + 1])))
            else:
                head[tok[0]] = tok[1:]
    x = np.array([float(t) for t in head["x_knots"]])
    nq = np.array([int(t) for t in head["n_q"]], dtype=np.int32)
    q = np.array([float(t) for t in head["q_knots"]])
    pids = np.array([int(t) for t in head["pids"]], dtype=np.int32)
    al = np.array([float(t) for t in head["alphas"]])
    v = np.zeros((1, q.size, x.size, pids.size))
    for (r, k), row in vals.items():
        v[0, r, k] = row
    grid = synth.Grid(x, nq, q, pids, v, al, "golden-tiny")
    qx = np.array([t[0] for t in queries])
    qq = np.array([t[1] for t in queries])
    exp = np.array([t[2] for t in queries])
    exp_as = np.array([t[3] for t in queries])
    return grid, qx, qq, exp, exp_as
