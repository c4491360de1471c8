"""The gather tiles of the IEEE FP64 kernels (short rows staged in shared
memory) against the oracle, on graphs built to hit their edges: tiles full of
rows whose in-lists hold only unreferenced sources (no tile entries, the most
rows per tile), rows at the 64-entry cap, and a spread of lengths so that tile
ends fall on every kind of row.  The double-float kernels keep the per-row
lane bins, so the two precisions also check each other."""
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


def l1(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).sum())


def unref_fed(n_src, n_dst, fan, seed):
    """n_src sources without in-edges, each pointing to `fan` of n_dst targets.
    The even targets point to a dangling sink only, so their in-lists hold
    unreferenced sources alone (empty tile rows: the most rows per tile); the
    odd ones also form a cycle, so they have one referenced source each."""
    rng = np.random.default_rng(seed)
    src, dst = [], []
    sink = n_src + n_dst
    for s in range(n_src):
        t = rng.choice(n_dst, size=fan, replace=False) + n_src
        src += [s] * fan
        dst += list(t)
    odd = [n_src + k for k in range(1, n_dst, 2)]
    for k in range(n_dst):
        v = n_src + k
        src.append(v)
        dst.append(sink)
        if k % 2:
            src.append(v)
            dst.append(odd[(odd.index(v) + 1) % len(odd)])
    return gg.from_edges(n_src + n_dst + 1, np.array(src), np.array(dst))


def capped_rows(n_rows, seed):
    """Rows with 64 (the tile cap), 63, 2 and 1 referenced sources, some of
    them also fed by unreferenced sources (which pushes them past the cap into
    the warp bin), plus dangling vertices."""
    rng = np.random.default_rng(seed)
    n = n_rows + 200
    src, dst = [], []
    for j in range(n_rows):
        d = (64, 63, 1, 2)[j % 4]
        s = rng.choice(np.setdiff1d(np.arange(n_rows), [j]), size=d, replace=False)
        src += list(s)
        dst += [j] * d
    for k in range(200):  # 100 unreferenced sources, 100 dangling sinks
        if k < 100:
            src += [n_rows + k] * 3
            dst += list(rng.choice(n_rows, size=3, replace=False))
        else:
            src.append(int(rng.integers(n_rows)))
            dst.append(n_rows + k)
    return gg.from_edges(n, np.array(src), np.array(dst))


GRAPHS = [
    ("unref_fed", lambda: unref_fed(40, 3000, 25, 1)),
    ("capped_rows", lambda: capped_rows(2400, 2)),
    ("rmat13", lambda: gg.rmat(13, 8, dangling=0.15, unref=0.10, seed=4)),
    ("spread", lambda: gg.random_small(6000, 9.0, 0.2, 0.1, seed=5)),
]


@pytest.mark.parametrize("gcase", GRAPHS, ids=lambda c: c[0])
@pytest.mark.parametrize("algo", (pr.PR_IFP1, pr.PR_IFP2))
def test_tiled_rounds_match_oracle(gcase, algo):
    g = gcase[1]()
    ref = oracle.ifp_rounds(algo, g, C, 1e-10, gg.p_uniform(g.n), xi_act=1e-300)
    assert ref["status"] == 0
    with pr.Graph(g.n, g.m, *g.csr32()) as G:
        assert G.tuning()["pull_thr"][1] <= 64  # the short rows go to tiles
        out, st, s = G.solve(C, 1e-10, algo, pr.PR_FP64,
                             opts=dict(xi_act=1e-300, mode=pr.PR_MODE_PULL, trace_cap=ref["rounds"] + 5))
        assert s == pr.PR_OK and st["rounds"] == ref["rounds"]
        k = ref["rounds"]
        assert np.array_equal(st["trace"]["F"][:k], ref["F"])
        assert np.array_equal(st["trace"]["E"][:k], ref["E"])
        assert np.allclose(st["trace"]["R"][:k + 1], ref["R"], rtol=1e-11, atol=1e-300)
        assert l1(out, ref["pi"]) <= 1e-12
        df, _, _ = G.solve(C, 1e-10, algo, pr.PR_DF64, opts=dict(xi_act=1e-300, mode=pr.PR_MODE_PULL))
        assert l1(out, df) <= 1e-12  # lane bins (double-float) and tiles (FP64) agree


@pytest.mark.parametrize("gcase", GRAPHS, ids=lambda c: c[0])
def test_tiled_sweeps(gcase):
    """Power, IFP2 (with its phase 2) and IFP1 in AUTO mode through the tiled
    FP64 kernels."""
    g = gcase[1]()
    truth = oracle.power(g, C, gg.p_uniform(g.n), tol=1e-15)[0]
    with pr.Graph(g.n, g.m, *g.csr32()) as G:
        out, st, s = G.solve(C, 1e-13, pr.PR_POWER, pr.PR_FP64)
        assert s == pr.PR_OK and l1(out, truth) <= st["err_bound"] + 1e-12
        out, st, s = G.solve(C, 1e-11, pr.PR_IFP2, pr.PR_FP64)
        assert s == pr.PR_OK and l1(out, truth) <= st["err_bound"] + 1e-13
        out, st, s = G.solve(C, 1e-11, pr.PR_IFP1, pr.PR_FP64, opts=dict(mode=pr.PR_MODE_AUTO))
        assert s == pr.PR_OK and l1(out, truth) <= st["err_bound"] + 1e-13


def test_tiles_follow_a_retune():
    """A retune recuts the tiles (thresholds move rows between tiles and warps)."""
    g = gg.rmat(12, 10, dangling=0.2, unref=0.1, seed=8)
    truth = oracle.power(g, C, gg.p_uniform(g.n), tol=1e-15)[0]
    with pr.Graph(g.n, g.m, *g.csr32()) as G:
        for thr in ([4096, 64, 32, 16, 8, 4], [4096, 16, 8, 4, 2, 1], [4096, 1, 1, 1, 1, 1],
                    [4096, 128, 64, 32, 16, 8]):  # the last one: no tiles (above the cap)
            G.set_tuning(pull_thr=thr, block_budget=1000)
            out, st, s = G.solve(C, 1e-11, pr.PR_IFP2, pr.PR_FP64)
            assert s == pr.PR_OK and l1(out, truth) <= st["err_bound"] + 1e-13, thr
