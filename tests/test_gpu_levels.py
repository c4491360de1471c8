"""Level-ordered IFP2 rounds (PR_MODE_LEVELS) against the oracle's
orc_ifp2_levels, through the C ABI.

The library assigns the levels itself from the degrees (pr_graph_create_ex);
oracle.gs_levels states the same rule, so with xi_act ~ 0 the per-round
frontier sizes and pushed-edge counts are integers the GPU reproduces
exactly, and R_t (residual left plus pushes in flight) agrees to rounding.
"""
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
    return float(np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)).sum())


def leveled(g, L):
    return pr.Graph(g.n, g.m, *g.csr32(), levels=L)


def hub_graph(n, seed):
    """ER edges plus a vertex pointing to everyone and one everyone points to:
    rows above the warp and CTA lane thresholds inside the levels."""
    base = gg.random_small(n, avg_deg=4.0, dangling=0.2, unref=0.1, seed=seed)
    src = list(np.repeat(np.arange(n), base.outdeg))
    dst = list(base.out_dst)
    nd = np.nonzero(base.outdeg > 0)[0]
    hub_out, hub_in = int(np.argmax(base.outdeg)), int(nd[1])
    src += [hub_out] * n + list(nd)
    dst += list(range(n)) + [hub_in] * len(nd)
    return gg.from_edges(n, np.array(src), np.array(dst), drop_loops=True)


GRAPHS = [
    ("small200", lambda: gg.random_small(200, 4.0, 0.2, 0.1, seed=1)),
    ("small3000", lambda: gg.random_small(3000, 6.0, 0.25, 0.1, seed=2)),
    ("rmat13", lambda: gg.rmat(13, 8, dangling=0.15, unref=0.10, seed=4)),
    ("hub20k", lambda: hub_graph(20000, 3)),
    # a row with more in-list entries than one block takes (kClusterRowMin =
    # 16384): served by a cluster of 8 blocks in the level-ordered rounds
    ("hub40k", lambda: hub_graph(40000, 4)),
]


def check_against_oracle(G, g, L, prec, eps, p=None, p_idx=None, p_dense=None, use_graph=0):
    pd = gg.p_uniform(g.n) if p_dense is None else p_dense
    lv = oracle.gs_levels(g, L)
    ref = oracle.ifp2_levels(g, C, eps, pd, lv, L, xi_act=1e-300)
    assert ref["status"] == 0
    # the stop decision compares R_t with eps: keep away from exact ties
    assert np.all(np.abs(ref["R"] / eps - 1) > 1e-6)
    k = ref["rounds"]
    out, st, status = G.solve(C, eps, pr.PR_IFP2, prec, p=p, p_idx=p_idx,
                              opts=dict(xi_act=1e-300, mode=pr.PR_MODE_LEVELS, trace_cap=k + 5,
                                        use_graph=use_graph))
    assert status == pr.PR_OK, pr.pr_last_error()
    assert st["rounds"] == k
    tr = st["trace"]
    assert np.array_equal(tr["F"][:k], ref["F"])
    assert np.array_equal(tr["E"][:k], ref["E"])
    nR = len(ref["R"])
    assert np.allclose(tr["R"][:nR], ref["R"], rtol=1e-11, atol=1e-300)
    assert st["resid_l1"] == pytest.approx(ref["R"][-1], rel=1e-11)
    assert st["err_bound"] == pytest.approx(2 * ref["R"][-1] / (1 - C), rel=1e-11)
    assert st["rounds_push"] == 0
    assert st["pushes"] == ref["F"].sum()
    assert st["edges_pushed"] == ref["E"].sum() + g.stats()["m_d"]
    assert l1(out, ref["pi"]) <= 1e-12
    return out, st, ref


@pytest.mark.parametrize("gcase", GRAPHS, ids=lambda c: c[0])
@pytest.mark.parametrize("L", (1, 4, 16))
@pytest.mark.parametrize("prec", (pr.PR_FP64, pr.PR_DF64))
def test_level_rounds_match_oracle_exactly(gcase, L, prec):
    g = gcase[1]()
    if gcase[0] == "hub40k":
        assert g.stats()["max_indeg"] > 16384
    with leveled(g, L) as G:
        assert G.info["levels"] == L
        check_against_oracle(G, g, L, prec, 1e-10)


@pytest.mark.parametrize("prec", (pr.PR_FP64, pr.PR_DF64))
def test_level_rounds_host_driven_and_profiled(prec):
    """Host-driven rounds and the profiled path run the same rounds."""
    g = gg.rmat(12, 8, dangling=0.2, unref=0.1, seed=3)
    with leveled(g, 8) as G:
        a, sa, _ = check_against_oracle(G, g, 8, prec, 1e-10, use_graph=-1)
        b, sb, _ = check_against_oracle(G, g, 8, prec, 1e-10)
        assert l1(a, b) == 0.0
        out, st, status = G.solve(C, 1e-10, pr.PR_IFP2, prec,
                                  opts=dict(mode=pr.PR_MODE_LEVELS, profile=1, xi_act=1e-300))
        assert status == pr.PR_OK and st["rounds"] == sb["rounds"]
        prof = st["profile"]
        # round 0 activates p; every later round is one group of level launches
        assert prof["k_activate"]["launches"] == 1
        assert prof["k_round_levels"]["launches"] == st["rounds"] - 1
        assert "k_push" not in prof and "k_round_pull" not in prof
        assert l1(out, b) <= 1e-13


@pytest.mark.parametrize("n", (3, 4, 9, 18))
def test_chain_drains_in_three_rounds(n):
    """Path 0->...->n-1, one level per inner vertex: two synchronous rounds,
    then one level-ordered round carries the residual to the dangling end."""
    g = gg.chain(n)
    y = (1 - C ** (np.arange(n) + 1)) / (n * (1 - C))
    L = n - 2
    with leveled(g, L) as G:
        for prec in (pr.PR_FP64, pr.PR_DF64):
            out, st, status = G.solve(C, 1e-300, pr.PR_IFP2, prec,
                                      opts=dict(xi_act=1e-300, mode=pr.PR_MODE_LEVELS, trace_cap=8))
            assert status == pr.PR_OK and st["rounds"] == 3 and st["resid_l1"] == 0.0
            assert l1(out, y / y.sum()) < 1e-14
            if n >= 4:
                assert list(st["trace"]["F"][:3]) == [n - 1, n - 2, n - 3]
                assert list(st["trace"]["E"][:3]) == [n - 2, n - 3, n - 4]


@pytest.mark.parametrize("k", (1, 64))
def test_ppr_sparse_seeds(k):
    g = gg.rmat(13, 8, dangling=0.15, unref=0.10, seed=5)
    idx, val = gg.p_seeds(g.n, k, seed=k)
    pd = gg.dense_from_sparse(g.n, idx, val)
    with leveled(g, 16) as G:
        check_against_oracle(G, g, 16, pr.PR_DF64, 1e-11, p=val, p_idx=idx, p_dense=pd / pd.sum())


@pytest.mark.parametrize("seed", (1, 2))
def test_fp32_form_and_certified_bound(seed):
    """FP32 level rounds, double-float correction, double-float level rounds."""
    g = gg.rmat(14, 8, dangling=0.15, unref=0.10, seed=seed)
    truth = oracle.power(g, C, gg.p_uniform(g.n), tol=1e-15)[0]
    with leveled(g, 16) as G:
        for eps in (1e-7, 1e-10):
            out, st, status = G.solve(C, eps, pr.PR_IFP2, pr.PR_FP32, opts=dict(mode=pr.PR_MODE_LEVELS))
            assert status == pr.PR_OK
            assert l1(out, truth) <= st["err_bound"] + 2e-7
        out, st, status = G.solve(C, 1e-11, pr.PR_IFP2, pr.PR_DF64, opts=dict(mode=pr.PR_MODE_LEVELS))
        assert status == pr.PR_OK and l1(out, truth) <= st["err_bound"] + 1e-13
        # the level-ordered rounds need fewer rounds than synchronous ones
        _, sync, _ = G.solve(C, 1e-11, pr.PR_IFP2, pr.PR_DF64, opts=dict(mode=pr.PR_MODE_PULL))
        assert st["rounds"] < sync["rounds"]


@pytest.mark.parametrize("L", (1, 3, 16))
def test_cluster_rows_in_every_precision(L):
    """A hub row above 16384 entries (an 8-block cluster) in the FP32 form,
    double-float and IEEE FP64, against the exact PageRank."""
    g = hub_graph(40000, 5)
    assert g.stats()["max_indeg"] > 16384
    truth = oracle.power(g, C, gg.p_uniform(g.n), tol=1e-15)[0]
    with leveled(g, L) as G:
        for prec, eps, slack in ((pr.PR_FP32, 1e-7, 2e-7), (pr.PR_DF64, 1e-11, 1e-13), (pr.PR_FP64, 1e-11, 1e-13)):
            out, st, status = G.solve(C, eps, pr.PR_IFP2, prec, opts=dict(mode=pr.PR_MODE_LEVELS))
            assert status == pr.PR_OK, pr.pr_last_error()
            assert l1(out, truth) <= st["err_bound"] + slack, (prec, l1(out, truth), st["err_bound"])


@pytest.mark.parametrize("mode", (pr.PR_MODE_AUTO, pr.PR_MODE_PUSH, pr.PR_MODE_PULL))
@pytest.mark.parametrize("algo", (pr.PR_IFP1, pr.PR_IFP2))
def test_leveled_graph_in_the_other_modes(mode, algo):
    """The level renumbering changes nothing for synchronous rounds."""
    g = gg.rmat(12, 8, dangling=0.2, unref=0.1, seed=7)
    ref = oracle.ifp_rounds(algo, g, C, 1e-10, gg.p_uniform(g.n), xi_act=1e-300)
    with leveled(g, 5) as G:
        out, st, status = G.solve(C, 1e-10, algo, pr.PR_DF64,
                                  opts=dict(xi_act=1e-300, mode=mode, trace_cap=ref["rounds"] + 5))
        assert status == pr.PR_OK and st["rounds"] == ref["rounds"]
        assert np.array_equal(st["trace"]["F"][:ref["rounds"]], ref["F"])
        assert l1(out, ref["pi"]) <= 1e-12
        pw, _, _ = G.solve(C, 1e-13, pr.PR_POWER, pr.PR_DF64)
        assert l1(pw, ref["pi"]) <= 1e-9


def test_level_mode_not_converged_status():
    g = gg.rmat(12, 8, dangling=0.2, unref=0.1, seed=3)
    lv = oracle.gs_levels(g, 4)
    with leveled(g, 4) as G:
        for cap in (1, 2, 3, 6):
            ref = oracle.ifp2_levels(g, C, 1e-14, gg.p_uniform(g.n), lv, 4, max_rounds=cap)
            assert ref["status"] == 1
            out, st, status = G.solve(C, 1e-14, pr.PR_IFP2, pr.PR_DF64,
                                      opts=dict(mode=pr.PR_MODE_LEVELS, max_rounds=cap), check=False)
            assert status == pr.PR_ENOTCONV and st["rounds"] == ref["rounds"], (cap, st["rounds"], ref["rounds"])
            assert l1(out, ref["pi"]) <= 1e-12


def test_level_mode_rejected_where_it_does_not_apply():
    g = gg.rmat(10, 8, dangling=0.2, unref=0.1, seed=1)
    with pr.Graph(g.n, g.m, *g.csr32()) as G:
        assert G.info["levels"] == 0
        _, _, s = G.solve(C, 1e-8, pr.PR_IFP2, opts=dict(mode=pr.PR_MODE_LEVELS), check=False)
        assert s == pr.PR_EINVAL and "levels" in pr.pr_last_error()
    with leveled(g, 4) as G:
        for algo in (pr.PR_IFP1, pr.PR_POWER):
            _, _, s = G.solve(C, 1e-8, algo, opts=dict(mode=pr.PR_MODE_LEVELS), check=False)
            assert s == pr.PR_EINVAL
        with pytest.raises(pr.PrError) as e:
            pr.pr_solve_batch([G], C, 1e-8, pr.PR_IFP2, opts=dict(mode=pr.PR_MODE_LEVELS))
        assert e.value.status == pr.PR_EINVAL
    for bad in (-1, 17):
        with pytest.raises(pr.PrError) as e:
            leveled(g, bad)
        assert e.value.status == pr.PR_EINVAL


def test_degenerate_graphs():
    """No edges, a single vertex, and a cycle (no dangling vertex, one level
    holds every vertex with in-edges)."""
    pe = gg.p_random(13, 5)
    pe /= pe.sum()
    with leveled(gg.empty(13), 4) as G:
        out, st, status = G.solve(C, 1e-12, pr.PR_IFP2, pr.PR_DF64, p=pe, opts=dict(mode=pr.PR_MODE_LEVELS))
        assert status == pr.PR_OK and l1(out, pe) < 1e-14
    with leveled(gg.empty(1), 1) as G:
        out, st, status = G.solve(C, 1e-12, pr.PR_IFP2, pr.PR_FP64, opts=dict(mode=pr.PR_MODE_LEVELS))
        assert status == pr.PR_OK and out[0] == 1.0
    g = gg.cycle(11)
    with leveled(g, 16) as G:
        check_against_oracle(G, g, 16, pr.PR_DF64, 1e-10)
