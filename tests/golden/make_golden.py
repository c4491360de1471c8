"""Write the stored PageRank vectors under tests/golden/ from the FP64 oracle.

Each fixture is the solution of Eq. 2 of the paper, (I - cP')pi = (1-c)p with
P' = P + p d^T (Sec. 2.1), computed by the oracle's Gaussian elimination
(oracle.dense_solve) on a small seeded graph from graphgen, and cross-checked
here against the oracle's Power iteration (Eq. 1) to 1e-13 before it is
written.  Only oracle/ and graphgen/ are used.

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402

CASES = [
    # name, graph factory, c, personalization (None = uniform, else {vertex: weight})
    ("small40_s3_c085", lambda: gg.random_small(40, 3.0, 0.2, 0.1, seed=3), 0.85, None),
    ("small40_s3_c050_ppr", lambda: gg.random_small(40, 3.0, 0.2, 0.1, seed=3), 0.50, {0: 1.0, 7: 3.0}),
    ("small25_s8_loops_c099", lambda: gg.random_small(25, 2.0, 0.1, 0.2, seed=8, loops=True), 0.99, None),
    ("instar9_c085", lambda: gg.in_star(9), 0.85, None),
    ("chain6_c085_ppr", lambda: gg.chain(6), 0.85, {2: 1.0}),
]


def p_of(n, spec):
    if spec is None:
        return gg.p_uniform(n)
    p = np.zeros(n)
    for v, w in spec.items():
        p[v] = w
    return p / p.sum()


def main():
    for name, make, c, spec in CASES:
        g = make()
        p = p_of(g.n, spec)
        pi = oracle.dense_solve(g, c, p)
        pw = oracle.power(g, c, p, tol=1e-15)[0]
        assert np.abs(pi - pw).sum() < 1e-13, name
        off, dst = g.csr32()
        with open(os.path.join(HERE, name + ".txt"), "w") as f:
            f.write(f"# {name}: PageRank of Eq. 2 (Sec. 2.1), c = {c!r}, p = {spec or 'uniform'}\n")
            f.write("# written by tests/golden/make_golden.py (oracle.dense_solve, checked against oracle.power)\n")
            f.write(f"n {g.n} m {g.m} c {c!r}\n")
            f.write("p " + " ".join(repr(float(v)) for v in p) + "\n")
            f.write("out_off " + " ".join(str(int(v)) for v in off) + "\n")
            f.write("out_dst " + " ".join(str(int(v)) for v in dst) + "\n")
            f.write("pi " + " ".join(repr(float(v)) for v in pi) + "\n")


if __name__ == "__main__":
    main()
