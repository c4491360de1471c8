"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Two kinds of check.  (1) The same algorithm: the GPU's synchronous rounds
against the oracle's (frontier sizes and edge counts exact, residuals to
rounding), and the GPU result against the oracle's result at the same eps.
(2) The exact PageRank (Eq. 2; the oracle's Power method run to 1e-13 or
1e-15, or a closed form): every solve lies within its certified bound, and
at the stopping thresholds the benchmark uses (IFP2 eps 5e-10 for FP64 and
double-float, 5e-7 for the FP32 form) FP64 solves are within L1 1e-9 and
FP32-form solves within L1 1e-6.  With xi_act ~ 0 every vertex with a
nonzero residual is active, so the per-round frontier sizes and edge counts
are integers the GPU must reproduce exactly.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import IFP1, IFP2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_03245_gb300 as pr  # noqa: E402

C = 0.85
ALGOS = (pr.PR_IFP1, pr.PR_IFP2, pr.PR_POWER)
MODES = (pr.PR_MODE_AUTO, pr.PR_MODE_PUSH, pr.PR_MODE_PULL)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pr.build()


def l1(a, b):
    return float(np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)).sum())


def gpu_graph(g):
    return pr.Graph(g.n, g.m, *g.csr32())


# ------------------------------------------------------------ closed forms
def closed_forms():
    out = []
    n = 9
    out.append(("cycle", gg.cycle(n), None, np.full(n, 1.0 / n)))
    p = np.zeros(n)
    p[3] = 1.0
    k = (np.arange(n) - 3) % n
    out.append(("cycle_ppr", gg.cycle(n), p, (1 - C) * C ** k / (1 - C ** n)))
    n = 40
    y = (1 - C ** (np.arange(n) + 1)) / (n * (1 - C))
    out.append(("chain", gg.chain(n), None, y / y.sum()))
    n = 33
    y = np.full(n, 1.0 / n + C / (n * (n - 1)))
    y[0] = 1.0 / n
    out.append(("out_star", gg.out_star(n), None, y / y.sum()))
    y = np.full(n, 1.0 / n)
    y[0] = 1.0 / n + C * (n - 1) / n
    out.append(("in_star", gg.in_star(n), None, y / y.sum()))
    pe = gg.p_random(13, 5)
    pe /= pe.sum()
    out.append(("empty", gg.empty(13), pe, pe))
    out.append(("single", gg.empty(1), None, np.ones(1)))
    y0, y1 = 1 / 3, 1 / 3 + C / 6
    y2 = 1 / 3 + C / 6 + C * y1
    out.append(("tri", gg.from_edges(3, [0, 0, 1], [1, 2, 2]), None, np.array([y0, y1, y2]) / (y0 + y1 + y2)))
    return out


@pytest.mark.parametrize("case", closed_forms(), ids=lambda c: c[0])
@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("prec", (pr.PR_FP64, pr.PR_FP32, pr.PR_DF64))
@pytest.mark.parametrize("mode", MODES)
def test_closed_forms(case, algo, prec, mode):
    name, g, p, truth = case
    with gpu_graph(g) as G:
        fp32_power = algo == pr.PR_POWER and prec == pr.PR_FP32
        # Power stops on ||delta||_1, whose rounding floor is set by the gathered
        # values: FP32 in the FP32 form (near 1e-7), double-float pairs (48-bit)
        # in DF64 and FP64 (near 1e-14 on these graphs); the certified error is
        # c * delta / (1 - c)
        eps = 1e-13 if algo != pr.PR_POWER else {pr.PR_FP64: 1e-13, pr.PR_DF64: 1e-13, pr.PR_FP32: 1e-6}[prec]
        out, st, status = G.solve(C, eps, algo, prec, p=p, opts=dict(mode=mode))
        assert status == pr.PR_OK, st
        tol = 1e-12 if prec != pr.PR_FP32 else (C * eps / (1 - C) + 1e-6 if fp32_power else 2e-7)
        assert l1(out, truth) <= tol, (name, l1(out, truth), st)
        assert abs(out.sum() - 1.0) < 1e-12


def test_cycle_round_count_and_trace():
    """No dangling vertex: R_t = c^t, rounds = ceil(ln eps / ln c) (Sec. 3.3.1)."""
    g = gg.cycle(11)
    with gpu_graph(g) as G:
        for use_graph in (0, -1):
            out, st, status = G.solve(C, 1e-10, pr.PR_IFP1, opts=dict(trace_cap=200, use_graph=use_graph))
            assert status == pr.PR_OK and st["rounds"] == 142
            R = st["trace"]["R"][:143]
            assert np.allclose(R, C ** np.arange(143), rtol=1e-12, atol=0)
            assert np.all(st["trace"]["F"][:142] == 11)


@pytest.mark.parametrize("algo", (pr.PR_IFP1, pr.PR_IFP2))
def test_chain_drains_exactly(algo):
    g = gg.chain(40)
    with gpu_graph(g) as G:
        out, st, status = G.solve(C, 1e-300, algo, opts=dict(xi_act=1e-300))
        assert status == pr.PR_OK and st["rounds"] == 39 and st["resid_l1"] == 0.0


# ------------------------------------------------------------ round parity
def hub_graph(n, seed):
    """ER edges plus a vertex pointing to everyone and one everyone points to:
    rows above the warp and CTA thresholds in both directions."""
    base = gg.random_small(n, avg_deg=4.0, dangling=0.2, unref=0.1, seed=seed)
    src = list(np.repeat(np.arange(n), base.outdeg))
    dst = list(base.out_dst)
    od = base.outdeg
    hub_out = int(np.argmax(od))  # a non-dangling vertex
    nd = np.nonzero(od > 0)[0]
    hub_in = int(nd[1])
    others = np.arange(n)
    src += [hub_out] * n + list(nd)
    dst += list(others) + [hub_in] * len(nd)
    return gg.from_edges(n, np.array(src), np.array(dst), drop_loops=True)


ROUND_GRAPHS = [
    ("small200", lambda: gg.random_small(200, 4.0, 0.2, 0.1, seed=1)),
    ("small3000", lambda: gg.random_small(3000, 6.0, 0.25, 0.1, seed=2)),
    ("rmat13", lambda: gg.rmat(13, 8, dangling=0.15, unref=0.10, seed=4)),
    ("hub20k", lambda: hub_graph(20000, 3)),
    # the paper's losing case: every edge also taken reversed (no dangling or
    # unreferenced vertices but the isolated ones)
    ("undirected12", lambda: gg.rmat(12, 8, dangling=0.0, unref=0.0, undirected=True, seed=5)),
]


@pytest.mark.parametrize("gcase", ROUND_GRAPHS, ids=lambda c: c[0])
@pytest.mark.parametrize("algo", (IFP1, IFP2))
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("prec", (pr.PR_FP64, pr.PR_DF64))
def test_rounds_match_oracle_exactly(gcase, algo, mode, prec):
    g = gcase[1]()
    p = gg.p_uniform(g.n)
    eps = 1e-10
    ref = oracle.ifp_rounds(algo, g, C, eps, p, xi_act=1e-300)
    assert ref["status"] == 0
    # the stop decision compares R_t with eps: keep away from exact ties
    assert np.all(np.abs(ref["R"] / eps - 1) > 1e-6)
    with gpu_graph(g) as G:
        out, st, status = G.solve(C, eps, algo, prec,
                                  opts=dict(xi_act=1e-300, mode=mode, trace_cap=ref["rounds"] + 5))
        assert status == pr.PR_OK
        k = ref["rounds"]
        assert st["rounds"] == k
        tr = st["trace"]
        assert np.array_equal(tr["F"][:k], ref["F"])
        assert np.array_equal(tr["E"][:k], ref["E"])
        assert np.allclose(tr["R"][:k + 1], ref["R"], rtol=1e-11, atol=1e-300)
        assert l1(out, ref["pi"]) <= 1e-12
        saved = g.stats()["m_d"] if algo == IFP2 else 0
        assert st["edges_pushed"] == ref["E"].sum() + saved
        assert st["pushes"] == ref["F"].sum()
        if mode == pr.PR_MODE_PUSH:
            assert st["rounds_pull"] == 0
        if mode == pr.PR_MODE_PULL:
            assert st["rounds_push"] == 0


# ------------------------------------------------------------ vs exact PageRank
@pytest.mark.parametrize("seed", (1, 2, 3))
def test_rmat_scale14_all_algorithms(seed):
    """R-MAT (0.57,0.19,0.19,0.05), 2^14 vertices, 131072 sampled edges, 15% dangling,
    10% unreferenced, c = 0.85, stop at residual L1 <= 1e-10."""
    g = gg.rmat(14, 8, dangling=0.15, unref=0.10, seed=seed)
    truth = oracle.power(g, C, gg.p_uniform(g.n), tol=1e-15)[0]
    with gpu_graph(g) as G:
        for algo in ALGOS:
            for prec in (pr.PR_FP64, pr.PR_DF64):
                out, st, status = G.solve(C, 1e-10, algo, prec)
                err = l1(out, truth)
                assert status == pr.PR_OK and err <= 1e-9, (algo, prec, err)
                assert err <= st["err_bound"] + 1e-13
        for algo in (pr.PR_IFP1, pr.PR_IFP2):
            out, st, status = G.solve(C, 1e-7, algo, pr.PR_FP32)
            err = l1(out, truth)
            assert status == pr.PR_OK and err <= 1e-6, (algo, err)
        out, st, status = G.solve(C, 1e-8, pr.PR_POWER, pr.PR_FP32)
        assert status == pr.PR_OK and l1(out, truth) <= 1e-6


def test_undirected_rmat_every_form():
    """The undirected stress graph (R-MAT scale 13, every sampled edge also
    taken reversed): IFP1 and IFP2 in every delivery mode and precision, and
    Power, against the exact PageRank, within the certified bound."""
    g = gg.rmat(13, 8, dangling=0.0, unref=0.0, undirected=True, seed=6)
    assert np.array_equal(np.sort(g.out_dst), np.sort(g.in_src))  # symmetric: in-lists = out-lists
    truth = oracle.power(g, C, gg.p_uniform(g.n), tol=1e-15)[0]
    modes = (pr.PR_MODE_AUTO, pr.PR_MODE_PUSH, pr.PR_MODE_PULL, pr.PR_MODE_ASYNC, pr.PR_MODE_APULL)
    with gpu_graph(g) as G:
        for algo in (pr.PR_IFP1, pr.PR_IFP2):
            for prec in (pr.PR_FP64, pr.PR_DF64):
                for mode in modes:
                    out, st, status = G.solve(C, 1e-10, algo, prec, opts=dict(mode=mode))
                    err = l1(out, truth)
                    assert status == pr.PR_OK and err <= 1e-9, (algo, prec, mode, err)
                    assert err <= st["err_bound"] + 1e-13
            out, st, status = G.solve(C, 1e-7, algo, pr.PR_FP32)
            assert status == pr.PR_OK and l1(out, truth) <= 1e-6
        for prec in (pr.PR_FP64, pr.PR_DF64):
            out, st, status = G.solve(C, 1e-11, pr.PR_POWER, prec)
            assert status == pr.PR_OK and l1(out, truth) <= st["err_bound"] + 1e-13 and l1(out, truth) <= 1e-10


def test_ifp1_ifp2_agree_and_ifp2_pushes_less():
    g = gg.rmat(13, 8, dangling=0.25, unref=0.10, seed=9)
    with gpu_graph(g) as G:
        a, sa, _ = G.solve(C, 1e-12, pr.PR_IFP1)
        b, sb, _ = G.solve(C, 1e-12, pr.PR_IFP2)
        assert l1(a, b) < 1e-10
        assert sb["edges_pushed"] < sa["edges_pushed"]


# ------------------------------------------------------------ personalization
@pytest.mark.parametrize("k", (1, 5, 64))
@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("prec", (pr.PR_FP64, pr.PR_DF64))
def test_ppr_sparse_seeds(k, algo, prec):
    g = gg.rmat(13, 8, dangling=0.15, unref=0.10, seed=5)
    idx, val = gg.p_seeds(g.n, k, seed=k)
    p = gg.dense_from_sparse(g.n, idx, val)
    truth = oracle.power(g, C, p, tol=1e-15)[0]
    with gpu_graph(g) as G:
        out, st, status = G.solve(C, 1e-11, algo, prec, p=val, p_idx=idx)
        assert status == pr.PR_OK and l1(out, truth) <= 1e-9
        # device-resident sparse p
        out2, st2, _ = G.solve(C, 1e-11, algo, prec, p=torch.tensor(val, device="cuda"),
                               p_idx=torch.tensor(idx, device="cuda"), p_is_device=True)
        assert l1(out2, truth) <= 1e-9


def test_ppr_dense_unnormalised_p():
    g = gg.rmat(12, 8, dangling=0.2, unref=0.1, seed=6)
    p = gg.p_random(g.n, 3, zero_frac=0.5) * 7.0
    truth = oracle.power(g, C, p / p.sum(), tol=1e-15)[0]
    with gpu_graph(g) as G:
        for algo in ALGOS:
            for prec in (pr.PR_FP64, pr.PR_DF64):
                out, st, status = G.solve(C, 1e-11, algo, prec, p=p)
                assert status == pr.PR_OK and l1(out, truth) <= 1e-9
                assert abs(st["p_scale"] - 1.0 / p.sum()) < 1e-15
            out, st, status = G.solve(C, 1e-7 if algo != pr.PR_POWER else 1e-6, algo, pr.PR_FP32, p=p)
            assert status == pr.PR_OK and l1(out, truth) <= 1e-5


# ------------------------------------------------------------ ABI behaviour
def test_device_arrays_and_device_output():
    g = gg.rmat(12, 8, dangling=0.15, unref=0.1, seed=7)
    truth = oracle.power(g, C, gg.p_uniform(g.n), tol=1e-15)[0]
    off, dst = g.csr32()
    ioff, isrc = g.csc32()
    d = [torch.tensor(a, device="cuda") for a in (off, dst, ioff, isrc)]
    with pr.Graph(g.n, g.m, *d, mem_is_device=True, stream=torch.cuda.current_stream()) as G:
        assert G.info["m"] == g.m and G.info["n_d"] == g.stats()["n_d"] and G.info["m_d"] == g.stats()["m_d"]
        out = torch.empty(g.n, dtype=torch.float64, device="cuda")
        _, st, status = G.solve(C, 1e-11, pr.PR_IFP2, out=out)
        torch.cuda.synchronize()
        assert status == pr.PR_OK and l1(out.cpu().numpy(), truth) <= 1e-9


def test_output_placements_and_host_created_graphs():
    """The same graph created from host arrays (copied, then checked on the
    device) and from device arrays gives the same solve, bit for bit,
    and every output placement receives it: a numpy array, a pinned CPU
    tensor and an unpinned CPU tensor (host copies), and a CUDA tensor."""
    g = gg.rmat(12, 8, dangling=0.15, unref=0.1, seed=9)
    off, dst = g.csr32()
    outs = []
    with pr.Graph(g.n, g.m, off, dst) as H, \
            pr.Graph(g.n, g.m, *[torch.tensor(a, device="cuda") for a in (off, dst)], mem_is_device=True,
                     stream=torch.cuda.current_stream()) as D:
        for G in (H, D):
            for out in (np.empty(g.n), torch.empty(g.n, dtype=torch.float64).pin_memory(),
                        torch.empty(g.n, dtype=torch.float64), torch.empty(g.n, dtype=torch.float64, device="cuda")):
                res, st, status = G.solve(C, 1e-11, pr.PR_IFP2, pr.PR_DF64, out=out)
                torch.cuda.synchronize()
                assert status == pr.PR_OK and res is out
                outs.append(out.cpu().numpy() if isinstance(out, torch.Tensor) else out)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    with pr.Graph(g.n, g.m, off, dst) as H:
        with pytest.raises(TypeError):
            H.solve(C, 1e-11, pr.PR_IFP2, out=torch.empty(g.n, dtype=torch.float32, device="cuda"))


def test_invalid_host_sizes_rejected_before_any_copy():
    """m that disagrees with out_off[n] is refused before the m entries are read."""
    g = gg.random_small(50, 3.0, 0.2, 0.1, seed=1)
    off, dst = g.csr32()
    for m in (g.m + 1, g.m - 1):
        with pytest.raises(pr.PrError) as e:
            pr.pr_graph_create(g.n, m, off, dst)
        assert e.value.status == pr.PR_EINVAL


def test_graph_info_matches_table1_columns():
    g = gg.rmat(13, 8, dangling=0.15, unref=0.10, seed=2)
    s = g.stats()
    with gpu_graph(g) as G:
        I = G.info
        assert (I["n"], I["m"], I["n_d"], I["m_d"], I["n_u"]) == (s["n"], s["m"], s["n_d"], s["m_d"], s["n_u"])
        assert I["max_outdeg"] == s["max_outdeg"] and I["max_indeg"] == s["max_indeg"]
        assert I["ms_preprocess"] > 0


@pytest.mark.parametrize("bad", ["dup", "range", "offsets", "csc_mismatch"])
@pytest.mark.parametrize("on_device", (False, True))
def test_invalid_graphs_rejected(bad, on_device):
    g = gg.random_small(50, 3.0, 0.2, 0.1, seed=1)
    off, dst = [a.copy() for a in g.csr32()]
    ioff, isrc = [a.copy() for a in g.csc32()]
    if bad == "dup":
        r = int(np.argmax(np.diff(off)))
        dst[off[r] + 1] = dst[off[r]]
    elif bad == "range":
        dst[0] = g.n
    elif bad == "offsets":
        off[5], off[6] = off[6] + 1, off[5]
    else:
        isrc[0] = (isrc[0] + 1) % g.n
    arrs = [off, dst] + ([ioff, isrc] if bad == "csc_mismatch" else [None, None])
    if on_device:
        arrs = [None if a is None else torch.tensor(a, device="cuda") for a in arrs]
    with pytest.raises(pr.PrError) as e:
        pr.pr_graph_create(g.n, g.m, *arrs, mem_is_device=on_device)
    assert e.value.status == pr.PR_EINVAL


def test_invalid_solve_arguments():
    g = gg.cycle(5)
    with gpu_graph(g) as G:
        for c, eps in ((0.0, 1e-9), (1.0, 1e-9), (0.85, 0.0), (0.85, -1.0), (0.85, float("nan"))):
            with pytest.raises(pr.PrError) as e:
                G.solve(c, eps, pr.PR_IFP1)
            assert e.value.status == pr.PR_EINVAL
        for p in (np.array([1.0, -1.0, 0, 0, 0]), np.zeros(5), np.array([1.0, np.inf, 0, 0, 0])):
            with pytest.raises(pr.PrError) as e:
                G.solve(0.85, 1e-9, pr.PR_IFP2, p=p)
            assert e.value.status == pr.PR_EINVAL
        # the graph still works after errors
        out, st, status = G.solve(0.85, 1e-12, pr.PR_IFP2)
        assert status == pr.PR_OK and l1(out, np.full(5, 0.2)) < 1e-12


def test_round_cap_reports_not_converged():
    g = gg.rmat(12, 8, dangling=0.15, unref=0.1, seed=1)
    with gpu_graph(g) as G:
        out, st, status = G.solve(C, 1e-14, pr.PR_IFP1, opts=dict(max_rounds=3), check=False)
        assert status == pr.PR_ENOTCONV and st["rounds"] == 3
        assert abs(out.sum() - 1) < 1e-12
        out, st, status = G.solve(C, 1e-12, pr.PR_IFP1, opts=dict(xi_act=1.0), check=False)
        assert status == pr.PR_ENOTCONV and st["rounds"] == 0


@pytest.mark.parametrize("prec", (pr.PR_FP64, pr.PR_FP32, pr.PR_DF64))
def test_pull_is_deterministic_and_graph_matches_host_loop(prec):
    g = gg.rmat(13, 8, dangling=0.15, unref=0.1, seed=8)
    with gpu_graph(g) as G:
        for algo in ALGOS:
            eps = 1e-11 if prec != pr.PR_FP32 else 1e-7
            a = G.solve(C, eps, algo, prec, opts=dict(mode=pr.PR_MODE_PULL))[0]
            b = G.solve(C, eps, algo, prec, opts=dict(mode=pr.PR_MODE_PULL))[0]
            c = G.solve(C, eps, algo, prec, opts=dict(mode=pr.PR_MODE_PULL, use_graph=-1))[0]
            assert np.array_equal(a, b) and np.array_equal(a, c)


def long_rows_graph():
    """Rows of every length class of graph creation's row sorts (one lane up to
    32 entries, a warp up to 1024, a block up to 8192, one radix sort beyond):
    in-rows of 20000, 5000 and 500 entries and out-rows of 12000 and 3000 over
    a sparse random graph."""
    rng = np.random.default_rng(11)
    n = 30000
    src = [np.arange(1, 20001), np.arange(2, 5002), np.arange(3, 503), np.full(12000, 3), np.full(3000, 4),
           rng.integers(0, n, 90000)]
    dst = [np.zeros(20000, np.int64), np.full(5000, 1), np.full(500, 2), np.arange(4, 12004), np.arange(5, 3005),
           rng.integers(0, n, 90000)]
    return gg.from_edges(n, np.concatenate(src), np.concatenate(dst), drop_loops=True)


def shuffled_rows(off, ent, seed):
    """The entries of every row in a seeded random order."""
    rng = np.random.default_rng(seed)
    row = np.repeat(np.arange(off.size - 1), np.diff(off))
    return np.ascontiguousarray(ent[np.lexsort((rng.random(ent.size), row))])


@pytest.mark.parametrize("with_csc", (False, True))
def test_rows_of_every_length_in_any_order(with_csc):
    g = long_rows_graph()
    off, dst = g.csr32()
    ioff, isrc = g.csc32()
    dst_s, isrc_s = shuffled_rows(off, dst, 1), shuffled_rows(ioff, isrc, 2)
    assert not np.array_equal(dst_s, dst)
    truth = oracle.power(g, C, gg.p_uniform(g.n), tol=1e-15)[0]
    extra = (ioff, isrc_s) if with_csc else ()
    with pr.Graph(g.n, g.m, off, dst_s, *extra) as G, gpu_graph(g) as G0:
        assert G.info["max_indeg"] == g.indeg.max() >= 20000 and G.info["max_outdeg"] == g.outdeg.max() >= 12000
        for mode in (pr.PR_MODE_PUSH, pr.PR_MODE_PULL):
            out = G.solve(C, 1e-12, pr.PR_IFP2, pr.PR_FP64, opts=dict(mode=mode))[0]
            assert l1(out, truth) <= 1e-10, mode
        # the internal lists do not depend on the order of the caller's rows: the
        # deterministic pull rounds give the same bits on both graphs
        out = G.solve(C, 1e-12, pr.PR_IFP2, pr.PR_FP64, opts=dict(mode=pr.PR_MODE_PULL))[0]
        assert np.array_equal(out, G0.solve(C, 1e-12, pr.PR_IFP2, pr.PR_FP64, opts=dict(mode=pr.PR_MODE_PULL))[0])
    if with_csc:  # one source of the longest in-row replaced by a vertex with no edge to it
        bad = isrc_s.copy()
        absent = np.setdiff1d(np.arange(g.n), isrc[ioff[0]:ioff[1]])[-1]
        bad[ioff[0] + 7] = absent
        with pytest.raises(pr.PrError) as e:
            pr.pr_graph_create(g.n, g.m, off, dst_s, ioff, bad)
        assert e.value.status == pr.PR_EINVAL


def exact_graph(n, m, seed):
    """A graph of exactly m distinct edges (self loops allowed) on n vertices."""
    rng = np.random.default_rng(seed)
    code = rng.choice(n * n, size=m, replace=False)
    return gg.from_edges(n, code // n, code % n)


@pytest.mark.parametrize("n,m", [(2047, 4095), (2048, 4096), (2049, 4097), (3000, 8192), (4500, 12289),
                                 (4096, 20480), (20000, 61439)])
def test_graph_sizes_at_the_sort_tile_edges(n, m):
    """Graph creation sorts vertex keys in tiles of 2048 and edge keys in tiles
    of 4096: counts on either side of those edges, and several ragged tiles."""
    g = exact_graph(n, m, seed=n + m)
    assert g.m == m
    truth = oracle.power(g, C, gg.p_uniform(g.n), tol=1e-15)[0]
    ioff, isrc = g.csc32()
    for extra in ((), (ioff, isrc)):
        with pr.Graph(g.n, g.m, *g.csr32(), *extra) as G:
            I = G.info
            assert (I["m"], I["max_indeg"], I["max_outdeg"]) == (m, g.indeg.max(), g.outdeg.max())
            for mode in (pr.PR_MODE_PUSH, pr.PR_MODE_PULL):
                out = G.solve(C, 1e-12, pr.PR_IFP2, pr.PR_FP64, opts=dict(mode=mode))[0]
                assert l1(out, truth) <= 1e-10, (n, m, mode)


def test_torch_allocator_hook():
    g = gg.rmat(12, 8, dangling=0.15, unref=0.1, seed=2)
    truth = oracle.power(g, C, gg.p_uniform(g.n), tol=1e-15)[0]
    import gc
    gc.collect()
    torch.cuda.synchronize()
    pr.use_torch_allocator(True)
    try:
        before = torch.cuda.memory_allocated()
        with gpu_graph(g) as G:
            assert torch.cuda.memory_allocated() > before
            out, st, status = G.solve(C, 1e-11, pr.PR_IFP2)
            assert l1(out, truth) <= 1e-9
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before
    finally:
        pr.use_torch_allocator(False)


# ------------------------------------------------------------ full size
# the benchmark's stopping thresholds: IFP2 stops at an L1 error of about 1.2-1.35 x eps
# on these R-MAT graphs, so half of each gate leaves a margin of about 1.5
EPS_FP64 = 5e-10
EPS_FP32 = 5e-7


@pytest.fixture(scope="module")
def rmat22():
    """R-MAT scale 22 (4,194,304 vertices, edge factor 16), 20% dangling, 10% unreferenced,
    randomly relabelled: the single-graph benchmark workload.  The oracle runs the same
    algorithms at the same stopping thresholds, plus the Power method to 1e-13 (within
    L1 c/(1-c) 1e-13 = 5.7e-13 of the exact PageRank)."""
    g = gg.rmat(22, 16, dangling=0.20, unref=0.10, seed=1)
    p = gg.p_uniform(g.n)
    truth, it, dl, st = oracle.power(g, C, p, tol=1e-13)
    assert st == 0
    ref = {eps: oracle.ifp_rounds(IFP2, g, C, eps, p, trace=False) for eps in (EPS_FP64, EPS_FP32)}
    pw9 = oracle.power(g, C, p, tol=1e-9)[0]
    return g, truth, ref, pw9


@pytest.mark.slow
def test_fullsize_rmat22_bench_configuration(rmat22):
    g, truth, ref, pw9 = rmat22
    p = gg.p_uniform(g.n)
    with gpu_graph(g) as G:
        # the benchmark's solve: IFP2, IEEE FP64 and double-float, eps 5e-10, default options
        for prec in (pr.PR_FP64, pr.PR_DF64):
            out, st, status = G.solve(C, EPS_FP64, pr.PR_IFP2, prec)
            assert status == pr.PR_OK
            assert abs(st["rounds"] - ref[EPS_FP64]["rounds"]) <= 1
            assert l1(out, ref[EPS_FP64]["pi"]) <= 1e-9         # parity with the same algorithm
            err = l1(out, truth)
            assert err <= 1e-9, (prec, err)                     # the FP64 gate vs the exact PageRank
            assert err <= st["err_bound"] + 1e-12               # certified bound vs exact PageRank
            assert err <= oracle.eq2_residual(g, C, p, out) / (1 - C) + 1e-12
        # FP32 form (FP32 rounds, IEEE FP64 correction and rounds) at eps 5e-7
        out, st, status = G.solve(C, EPS_FP32, pr.PR_IFP2, pr.PR_FP32)
        assert status == pr.PR_OK and l1(out, ref[EPS_FP32]["pi"]) <= 1e-6
        err = l1(out, truth)
        assert err <= 1e-6, err                                 # the FP32 gate vs the exact PageRank
        assert err <= st["err_bound"] + 1e-9
        # Power at the same tolerance as the oracle's Power
        for prec in (pr.PR_FP64, pr.PR_DF64):
            out, st, status = G.solve(C, 1e-9, pr.PR_POWER, prec)
            assert status == pr.PR_OK and l1(out, pw9) <= 1e-9
            assert l1(out, truth) <= st["err_bound"] + 1e-12
        # push-only and pull-only delivery give the same result up to rounding
        for mode in (pr.PR_MODE_PUSH, pr.PR_MODE_PULL):
            out2, st2, _ = G.solve(C, EPS_FP64, pr.PR_IFP2, pr.PR_FP64, opts=dict(mode=mode))
            assert l1(out2, ref[EPS_FP64]["pi"]) <= 1e-9
            assert l1(out2, truth) <= 1e-9
