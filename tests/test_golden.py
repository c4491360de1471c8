"""Stored PageRank vectors (tests/golden/*.txt, written by make_golden.py from
the oracle's Gaussian elimination of Eq. 2).  On the CPU they pin the oracle
against regressions and the in-star fixture against its closed form; on the
GPU every algorithm and precision must reproduce them within its certified
bound."""
import glob
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FILES = sorted(glob.glob(os.path.join(HERE, "*.txt")))


def load(path):
    d = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        key, *vals = line.split()
        if key == "n":  # "n <n> m <m> c <c>"
            words = [key] + vals
            for k in range(0, len(words), 2):
                d[words[k]] = [words[k + 1]]
        else:
            d[key] = vals
    n = int(d["n"][0])
    c = float(d["c"][0])
    off = np.array(d["out_off"], dtype=np.int32)
    dst = np.array(d.get("out_dst", []), dtype=np.int32)
    src = np.repeat(np.arange(n, dtype=np.int32), np.diff(off))
    g = gg.from_edges(n, src, dst)
    return g, c, np.array(d["p"], dtype=np.float64), np.array(d["pi"], dtype=np.float64)


def test_fixtures_present():
    assert len(FILES) >= 5


@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(f) for f in FILES])
def test_oracle_reproduces_golden(path):
    g, c, p, pi = load(path)
    assert abs(pi.sum() - 1.0) < 1e-14
    assert np.abs(oracle.dense_solve(g, c, p) - pi).sum() < 1e-14
    assert np.abs(oracle.power(g, c, p, tol=1e-15)[0] - pi).sum() < 1e-13


def test_instar_golden_closed_form():
    g, c, p, pi = load(os.path.join(HERE, "instar9_c085.txt"))
    n = g.n
    y = np.full(n, 1.0 / n)  # Eq. 4: the mass pushed along P; leaves push once into the centre
    y[0] = 1.0 / n + c * (n - 1) / n
    assert np.abs(y / y.sum() - pi).max() < 1e-15


@pytest.mark.gpu
@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(f) for f in FILES])
def test_gpu_reproduces_golden(path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_03245_gb300 as pr
    pr.build()
    g, c, p, pi = load(path)
    with pr.Graph(g.n, g.m, *g.csr32()) as h:
        for algo in (pr.PR_IFP1, pr.PR_IFP2, pr.PR_POWER):
            for prec in (pr.PR_DF64, pr.PR_FP64, pr.PR_FP32):
                # FP32 Power stops on ||delta||_1, whose FP32 rounding floor is near 1e-7
                eps = (1e-6 if algo == pr.PR_POWER else 1e-7) if prec == pr.PR_FP32 else 1e-12
                out, st, s = h.solve(c, eps, algo, prec, p=p)
                assert s == pr.PR_OK
                tol = st["err_bound"] + (2e-6 if prec == pr.PR_FP32 else 1e-13)
                assert np.abs(out - pi).sum() <= tol, (algo, prec)
