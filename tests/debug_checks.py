"""Payload of tests/test_gpu_debug.py, run in its own process with
PR_LIBRARY=debug so that the binding loads libpr_debug.so (index checks on
every graph-array load, invariant checks after every round).  Prints one JSON
line with what it saw; exits non-zero on the first failed expectation."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402
import paper_2302_03245_gb300 as pr  # noqa: E402

C = 0.85
DBG_IN_SRC, DBG_OUT_DST, DBG_BIN, DBG_PERM, DBG_MASS, DBG_IDENTITY = 1, 2, 3, 4, 16, 17
DBG_SORT_WAIT = 6


def l1(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).sum())


def main():
    assert pr.DEBUG, "PR_LIBRARY=debug was not set"
    pr.build()
    import torch
    torch.cuda.set_device(0)
    assert pr.pr_is_debug_build()
    pr.pr_debug_report_get(reset=True)
    out = {"solves": 0}
    graphs = [gg.cycle(17), gg.chain(30), gg.in_star(20), gg.random_small(150, 3.0, 0.2, 0.1, seed=5),
              gg.rmat(11, 8, dangling=0.15, unref=0.10, seed=7), gg.er(3000, 6.0, dangling=0.2, unref=0.1, seed=8)]
    for g in graphs:
        truth = oracle.power(g, C, gg.p_uniform(g.n), tol=1e-15)[0]
        with pr.Graph(g.n, g.m, *g.csr32()) as G:
            for algo in (pr.PR_IFP1, pr.PR_IFP2, pr.PR_POWER):
                for prec, eps in ((pr.PR_FP64, 1e-11), (pr.PR_DF64, 1e-11), (pr.PR_FP32, 1e-7)):
                    if algo == pr.PR_POWER and prec == pr.PR_FP32:
                        eps = 1e-6  # FP32 Power's ||delta||_1 floors near 1e-7
                    modes = (pr.PR_MODE_AUTO,) if algo == pr.PR_POWER else \
                        (pr.PR_MODE_AUTO, pr.PR_MODE_PUSH, pr.PR_MODE_PULL, pr.PR_MODE_ASYNC) + \
                        ((pr.PR_MODE_APULL,) if prec != pr.PR_FP32 else ())
                    for mode in modes:
                        res, st, status = G.solve(C, eps, algo, prec, opts=dict(mode=mode))
                        assert status == pr.PR_OK, (g.n, algo, prec, mode, status)
                        tol = 1e-9 if prec != pr.PR_FP32 else (1e-5 if algo == pr.PR_POWER else 1e-6)
                        assert l1(res, truth) <= tol, (g.n, algo, prec, mode, l1(res, truth))
                        out["solves"] += 1
    rep = pr.pr_debug_report_get(reset=True)
    assert rep["fails"] == 0, rep
    assert rep["checks"] > 500, rep  # invariant checks ran after the rounds
    out["clean"] = rep
    # a batch runs with its index checks too
    hs = [pr.Graph(g.n, g.m, *g.csr32()) for g in graphs[3:]]
    outs, sts, status = pr.pr_solve_batch(hs, C, 1e-10, pr.PR_IFP2, pr.PR_FP32)
    assert status == pr.PR_OK
    for g, o in zip(graphs[3:], outs):
        assert l1(o, oracle.power(g, C, gg.p_uniform(g.n), tol=1e-15)[0]) <= 1e-6
    for h in hs:
        h.close()
    assert pr.pr_debug_report_get(reset=True)["fails"] == 0
    # the net itself: each forced site turns the solve into PR_ECHECK, with no invalid access
    g = graphs[4]
    forced = {}
    with pr.Graph(g.n, g.m, *g.csr32()) as G:
        for site, mode in ((DBG_IN_SRC, pr.PR_MODE_PULL), (DBG_OUT_DST, pr.PR_MODE_PUSH), (DBG_BIN, pr.PR_MODE_PUSH),
                           (DBG_PERM, pr.PR_MODE_AUTO), (DBG_MASS, pr.PR_MODE_AUTO),
                           (DBG_IDENTITY, pr.PR_MODE_AUTO)):
            pr.pr_debug_inject(site)
            try:
                G.solve(C, 1e-10, pr.PR_IFP1, pr.PR_FP64, opts=dict(mode=mode))
                raise AssertionError(f"site {site}: the forced check did not fail the solve")
            except pr.PrError as e:
                assert e.status == pr.PR_ECHECK, (site, e)
            rep = pr.pr_debug_report_get(reset=True)
            assert rep["fails"] > 0 and rep["first_site"] == site, (site, rep)
            forced[site] = rep["fails"]
        pr.pr_debug_inject(0)
        res, st, status = G.solve(C, 1e-10, pr.PR_IFP1, pr.PR_FP64)
        assert status == pr.PR_OK
        assert pr.pr_debug_report_get(reset=True)["fails"] == 0
    out["forced"] = forced
    # graph creation's radix sort: every bounded wait gives up at once, the
    # creation fails cleanly with PR_ECUDA, and the next creation works
    pr.pr_debug_inject(DBG_SORT_WAIT)
    try:
        pr.pr_graph_create(g.n, g.m, *g.csr32())
        raise AssertionError("the forced sort wait did not fail the creation")
    except pr.PrError as e:
        assert e.status == pr.PR_ECUDA and "gave up" in str(e), e
    pr.pr_debug_inject(0)
    with pr.Graph(g.n, g.m, *g.csr32()) as G:
        res, st, status = G.solve(C, 1e-10, pr.PR_IFP2, pr.PR_FP64)
        assert status == pr.PR_OK
        assert l1(res, oracle.power(g, C, gg.p_uniform(g.n), tol=1e-15)[0]) <= 1e-9
    assert pr.pr_debug_report_get(reset=True)["fails"] == 0
    out["sort_wait"] = True
    print(json.dumps(out))


if __name__ == "__main__":
    main()
