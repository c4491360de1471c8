"""Launch parameters (pull bins, block budget, push/pull switch) and the
autotuner: they change how rounds map onto the GPU, never what a solve
computes, so every tuning must give the oracle's PageRank within the
certified bound and the same round counts."""
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_03245_gb300 as pr  # noqa: E402

C = 0.85


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pr.build()


@pytest.fixture(scope="module")
def graph():
    g = gg.rmat(14, 12, dangling=0.2, unref=0.1, seed=21)
    h = pr.Graph(g.n, g.m, *g.csr32())
    truth = oracle.power(g, C, gg.p_uniform(g.n), tol=1e-15)[0]
    yield g, h, truth
    h.close()


def l1(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).sum())


def test_default_tuning_describes_the_bins(graph):
    g, h, _ = graph
    t = h.tuning()
    assert t["pull_thr"] == [4096, 64, 32, 16, 8, 4]
    assert sum(t["bin_rows"]) == h.info["n_nd"]
    assert all(r >= 0 for r in t["bin_rows"])
    assert 0 < t["pull_ratio"] < 1 and t["pull_blocks"] >= 1
    # the bins really partition by in-degree: rows of bin 0 have in-degree > thr[0], ...
    indeg = np.sort(np.diff(g.in_off)[np.diff(g.out_off) > 0])[::-1]
    n_ref = h.info["n_ref"]
    assert np.count_nonzero(indeg[:n_ref] > t["pull_thr"][1]) == t["bin_rows"][0] + t["bin_rows"][1]


@pytest.mark.parametrize("thr,budget", [([1024, 64, 32, 16, 8, 4], 152 * 8), ([16384, 16, 8, 4, 2, 1], 152 * 32),
                                        ([0, 0, 0, 0, 0, 0], 152), ([1 << 30] * 6, 1000)])
def test_any_tuning_gives_the_same_pagerank(graph, thr, budget):
    g, h, truth = graph
    ref, st0, _ = h.solve(C, 1e-11, pr.PR_IFP2, pr.PR_DF64, opts=dict(mode=pr.PR_MODE_PULL))
    old = h.tuning()
    try:
        h.set_tuning(pull_thr=thr, block_budget=budget)
        for prec in (pr.PR_DF64, pr.PR_FP64):
            for mode in (pr.PR_MODE_PULL, pr.PR_MODE_AUTO):
                out, st, s = h.solve(C, 1e-11, pr.PR_IFP2, prec, opts=dict(mode=mode))
                assert s == pr.PR_OK
                assert l1(out, truth) <= st["err_bound"] + 1e-12
                if mode == pr.PR_MODE_PULL:
                    assert abs(st["rounds"] - st0["rounds"]) <= 1
                    assert l1(out, ref) <= 1e-12
        out, st, s = h.solve(C, 1e-11, pr.PR_POWER, pr.PR_DF64)
        assert l1(out, truth) <= st["err_bound"] + 1e-12
    finally:
        h.set_tuning(pull_thr=old["pull_thr"], block_budget=old["block_budget"])


def test_retuning_reaches_graph_launched_rounds(graph):
    """The rounds run inside a captured CUDA graph whose launches carry the
    plans: after a retune, a graph-launched solve must run the new plans, i.e.
    match the host-driven rounds bit for bit (the pull order is fixed by the
    plan, and different plans sum in different orders)."""
    g, h, _ = graph
    old = h.tuning()
    try:
        h.solve(C, 1e-11, pr.PR_IFP2, pr.PR_DF64, opts=dict(mode=pr.PR_MODE_PULL))  # captures the rounds
        outs = []
        for thr, budget in (([0] * 6, 152), ([1 << 30] * 6, 1000)):
            h.set_tuning(pull_thr=thr, block_budget=budget)
            a, _, _ = h.solve(C, 1e-11, pr.PR_IFP2, pr.PR_DF64, opts=dict(mode=pr.PR_MODE_PULL))
            b, _, _ = h.solve(C, 1e-11, pr.PR_IFP2, pr.PR_DF64, opts=dict(mode=pr.PR_MODE_PULL, use_graph=-1))
            assert np.array_equal(a, b)
            outs.append(a)
        assert not np.array_equal(outs[0], outs[1])  # the two plans really sum differently
    finally:
        h.set_tuning(pull_thr=old["pull_thr"], block_budget=old["block_budget"])


def test_invalid_tuning_is_refused_and_keeps_the_graph(graph):
    g, h, _ = graph
    old = h.tuning()
    for thr, budget in (([32, 64, 16, 8, 4, 2], 100), ([4096, 32, 16, 8, 4, -1], 100), ([4096, 32, 16, 8, 4, 2], 0),
                        ([4096, 32, 16, 8, 4, 2], 1 << 20)):
        with pytest.raises(pr.PrError) as e:
            h.set_tuning(pull_thr=thr, block_budget=budget)
        assert e.value.status == pr.PR_EINVAL
        assert h.tuning() == old


def test_autotune_and_cache(graph, tmp_path):
    g, h, truth = graph
    old = h.tuning()
    try:
        t, rep = h.autotune(pr.PR_DF64, max_ms=400.0)
        assert "chosen" in rep and t == h.tuning()
        assert sum(t["bin_rows"]) == h.info["n_nd"]
        assert 0 < t["pull_ratio"] <= 1
        out, st, s = h.solve(C, 1e-11, pr.PR_IFP2, pr.PR_DF64)
        assert s == pr.PR_OK and l1(out, truth) <= st["err_bound"] + 1e-12
        path = os.path.join(tmp_path, "tune.json")
        t1, rep1 = h.autotune(pr.PR_DF64, max_ms=200.0, cache_path=path)
        assert rep1 != "from cache" and len(json.load(open(path))) == 1
        h.set_tuning(pull_thr=old["pull_thr"], block_budget=old["block_budget"], pull_ratio=old["pull_ratio"])
        t2, rep2 = h.autotune(pr.PR_DF64, cache_path=path)
        assert rep2 == "from cache"
        assert (t2["pull_thr"], t2["block_budget"], t2["pull_ratio"]) == (t1["pull_thr"], t1["block_budget"],
                                                                           t1["pull_ratio"])
    finally:
        h.set_tuning(pull_thr=old["pull_thr"], block_budget=old["block_budget"], pull_ratio=old["pull_ratio"])
