"""The data-parallel generator (graphgen.torchgen) makes exactly the graphs of
the C generator (graphgen) from the same arguments, so benchmarks may build
their inputs on the device while tests and the oracle use the host copy."""
import numpy as np
import pytest

import graphgen as gg

torch = pytest.importorskip("torch")
from graphgen import torchgen as tg  # noqa: E402


def same(a, b):
    return a.n == b.n and all(np.array_equal(x, y.cpu().numpy()) for x, y in (
        (a.out_off, b.out_off), (a.out_dst, b.out_dst), (a.in_off, b.in_off), (a.in_src, b.in_src)))


@pytest.mark.parametrize("kw", [dict(scale=10), dict(scale=12, dag_frac=0.7, dangling=0.25),
                                dict(scale=11, nverts=1500, edge_factor=12), dict(scale=9, permute=False),
                                dict(scale=8, edge_factor=4, dangling=0.0, unref=0.0, seed=7),
                                dict(scale=10, undirected=True, dangling=0.1, unref=0.0)])
def test_rmat_same_graph(kw, monkeypatch):
    monkeypatch.setattr(tg, "CHUNK", 1000)  # several passes with a ragged last one
    assert same(gg.rmat(**kw), tg.rmat(device="cpu", **kw))


@pytest.mark.parametrize("permute", [False, True])
def test_er_same_graph(permute):
    kw = dict(n=3000, avg_deg=6.0, dangling=0.2, unref=0.1, seed=2, permute=permute)
    assert same(gg.er(**kw), tg.er(device="cpu", **kw))


def test_draws_and_permutation():
    idx = torch.arange(1000)
    u = tg.draw_u01(5, 600, idx).numpy()
    assert np.array_equal(u, np.array([gg._L().gg_u01(5, 600, i) for i in range(1000)]))
    perm = tg.permutation(5000, 3, 1, "cpu").numpy()
    assert np.array_equal(np.sort(perm), np.arange(5000))


def test_stats_and_host_copy():
    b = tg.rmat(10, device="cpu")
    a = gg.rmat(10)
    assert b.stats() == a.stats()
    assert same(a, b.to_host().__class__(b.n, *[torch.from_numpy(x) for x in (
        b.to_host().out_off, b.to_host().out_dst, b.to_host().in_off, b.to_host().in_src)]))


def test_undirected_rmat_is_symmetric():
    """Without deletions every edge comes with its reverse; no vertex is
    dangling or unreferenced unless it is isolated."""
    g = gg.rmat(11, 8, dangling=0.0, unref=0.0, undirected=True, seed=3)
    src = np.repeat(np.arange(g.n), np.diff(g.out_off))
    fwd = set(zip(src.tolist(), g.out_dst.tolist()))
    assert fwd == {(d, s) for s, d in fwd}
    outdeg, indeg = np.diff(g.out_off), np.diff(g.in_off)
    assert np.array_equal(outdeg, indeg)
