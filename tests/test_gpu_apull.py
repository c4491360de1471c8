"""Asynchronous pull rounds (PR_MODE_APULL): each non-dangling row recomputes
the residual it holds from the reserves (Eq. 4's identity), so pushes
committed earlier in the same round are taken at once, and commits all of it
when it is above xi_act -- the asynchronous scans of Sec. 3.2 without
atomics.  The schedule is the GPU's; the oracle's scans in id order
(orc_ifp_scan) are one schedule of it.  The tests check what holds for every
schedule: the certified bound against the exact PageRank (the stop test's R
bounds the residual left), fewer rounds than synchronous rounds, results
within the bounds of the oracle's schedule, and refusals."""
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


GRAPHS = [
    ("small200", lambda: gg.random_small(200, 4.0, 0.2, 0.1, seed=1, loops=True)),
    ("rmat13", lambda: gg.rmat(13, 8, dangling=0.15, unref=0.10, seed=4)),
    ("dag12", lambda: gg.rmat(12, 8, dangling=0.25, unref=0.0, dag_frac=0.9, seed=6)),
    ("er5000", lambda: gg.er(5000, 6.0, dangling=0.2, unref=0.1, seed=9)),
]


@pytest.mark.parametrize("gcase", GRAPHS, ids=lambda c: c[0])
@pytest.mark.parametrize("algo", (pr.PR_IFP1, pr.PR_IFP2))
@pytest.mark.parametrize("prec", (pr.PR_FP64, pr.PR_DF64))
def test_apull_within_the_certified_bound_and_faster(gcase, algo, prec):
    g = gcase[1]()
    p = gg.p_uniform(g.n)
    truth = oracle.power(g, C, p, tol=1e-15)[0]
    eps = 1e-11
    scan = oracle.ifp_scan(algo, g, C, eps, p)
    with pr.Graph(g.n, g.m, *g.csr32()) as G:
        _, sync, _ = G.solve(C, eps, algo, prec, opts=dict(mode=pr.PR_MODE_PULL))
        for use_graph in (0, -1, 0):  # the schedule differs between runs; every run must hold
            out, st, s = G.solve(C, eps, algo, prec, opts=dict(mode=pr.PR_MODE_APULL, use_graph=use_graph))
            assert s == pr.PR_OK, pr.pr_last_error()
            assert st["resid_l1"] <= eps and st["rounds_push"] == 0
            assert l1(out, truth) <= st["err_bound"] + 1e-13
            assert abs(float(np.sum(out)) - 1.0) < 1e-12
            assert st["rounds"] <= sync["rounds"]
            # the oracle's schedule (scans in id order) lands within both bounds
            assert l1(out, scan["pi"]) <= st["err_bound"] + oracle.certified_l1_bound(algo, C, scan["R"][-1]) + 1e-13


@pytest.mark.slow
def test_apull_saves_rounds_on_a_large_rmat():
    """Pushes are taken within a round when their source commits before the
    target's gather reads it: on a graph whose rows span several waves of the
    GPU's blocks (here R-MAT scale 20, about 0.4M non-dangling rows) that cuts
    the rounds well below the synchronous ones; on small graphs, whose rows all
    gather at once, the two nearly agree."""
    g = gg.rmat(20, 16, dangling=0.2, unref=0.1, seed=2)
    p = gg.p_uniform(g.n)
    truth = oracle.power(g, C, p, tol=1e-13)[0]
    with pr.Graph(g.n, g.m, *g.csr32()) as G:
        for prec in (pr.PR_FP64, pr.PR_DF64):
            _, sync, _ = G.solve(C, 1e-10, pr.PR_IFP2, prec, opts=dict(mode=pr.PR_MODE_PULL))
            out, ap, s = G.solve(C, 1e-10, pr.PR_IFP2, prec, opts=dict(mode=pr.PR_MODE_APULL))
            assert s == pr.PR_OK
            assert ap["rounds"] < 0.9 * sync["rounds"], (ap["rounds"], sync["rounds"])
            assert l1(out, truth) <= ap["err_bound"] + 1e-12


@pytest.mark.parametrize("prec", (pr.PR_FP64, pr.PR_DF64))
def test_apull_personalized_and_traces(prec):
    g = gg.rmat(13, 8, dangling=0.15, unref=0.10, seed=11)
    rng = np.random.default_rng(3)
    idx = rng.choice(g.n, size=17, replace=False).astype(np.int32)
    val = rng.uniform(0.5, 2.0, size=17)
    pv = np.zeros(g.n)
    np.add.at(pv, idx, val)
    pv /= pv.sum()
    truth = oracle.power(g, C, pv, tol=1e-15)[0]
    with pr.Graph(g.n, g.m, *g.csr32()) as G:
        for algo in (pr.PR_IFP1, pr.PR_IFP2):
            out, st, s = G.solve(C, 1e-11, algo, prec, p=val, p_idx=idx,
                                 opts=dict(mode=pr.PR_MODE_APULL, trace_cap=512))
            assert s == pr.PR_OK
            assert l1(out, truth) <= st["err_bound"] + 1e-13
            tr = st["trace"]
            nr = st["rounds"]
            assert tr["R"][nr - 1] == pytest.approx(st["resid_l1"], rel=0, abs=0)
            assert np.all(tr["mode"][:nr] == 2)
            assert 0 < tr["F"][0] <= 17  # round 0 commits the non-dangling seeds


def test_apull_chain_and_degenerate_graphs():
    n = 40
    y = (1 - C ** (np.arange(n) + 1)) / (n * (1 - C))
    with pr.Graph(n, n - 1, *gg.chain(n).csr32()) as G:
        for algo in (pr.PR_IFP1, pr.PR_IFP2):
            out, st, s = G.solve(C, 1e-14, algo, pr.PR_FP64, opts=dict(mode=pr.PR_MODE_APULL))
            assert s == pr.PR_OK and l1(out, y / y.sum()) < 1e-13
    for g in (gg.empty(6), gg.cycle(1), gg.in_star(9), gg.out_star(9)):
        truth = oracle.power(g, C, gg.p_uniform(g.n), tol=1e-15)[0]
        with pr.Graph(g.n, g.m, *g.csr32()) as G:
            for algo in (pr.PR_IFP1, pr.PR_IFP2):
                out, st, s = G.solve(C, 1e-12, algo, pr.PR_DF64, opts=dict(mode=pr.PR_MODE_APULL))
                assert s == pr.PR_OK and l1(out, truth) < 1e-10


def test_apull_round_cap_and_refusals():
    g = gg.rmat(12, 8, dangling=0.15, unref=0.10, seed=5)
    with pr.Graph(g.n, g.m, *g.csr32()) as G:
        out, st, s = G.solve(C, 1e-14, pr.PR_IFP2, pr.PR_FP64, opts=dict(mode=pr.PR_MODE_APULL, max_rounds=3))
        assert s == pr.PR_ENOTCONV and st["rounds"] == 3
        with pytest.raises(pr.PrError) as e:
            G.solve(C, 1e-9, pr.PR_POWER, pr.PR_FP64, opts=dict(mode=pr.PR_MODE_APULL))
        assert e.value.status == pr.PR_EINVAL


@pytest.mark.parametrize("gcase", GRAPHS, ids=lambda c: c[0])
@pytest.mark.parametrize("algo", (pr.PR_IFP1, pr.PR_IFP2))
def test_apull_fp32_form(gcase, algo):
    """PR_FP32 with asynchronous pull rounds: FP32 rounds to a residual of about
    8e-6 (or eps, if larger), then IEEE FP64 rounds from the reserve, whose first
    recompute corrects what the FP32 rounds left.  At the FP32 form's stop
    (5e-7) the result meets the FP32 gate; asked for 1e-11 it reaches FP64
    accuracy, within the certified bound."""
    g = gcase[1]()
    p = gg.p_uniform(g.n)
    truth = oracle.power(g, C, p, tol=1e-15)[0]
    with pr.Graph(g.n, g.m, *g.csr32()) as G:
        for eps, gate in ((5e-7, 1e-6), (1e-11, 1e-9)):
            for use_graph in (0, -1):
                out, st, s = G.solve(C, eps, algo, pr.PR_FP32, opts=dict(mode=pr.PR_MODE_APULL, use_graph=use_graph))
                assert s == pr.PR_OK, pr.pr_last_error()
                err = l1(out, truth)
                assert st["resid_l1"] <= eps and err <= gate, (eps, err)
                assert err <= st["err_bound"] + 1e-13
                assert abs(float(np.sum(out)) - 1.0) < 1e-12
                assert 0 < st["fp64_rounds"] < st["rounds"]


def test_apull_fp32_form_personalized_and_loose_stop():
    g = gg.rmat(13, 8, dangling=0.15, unref=0.10, seed=11)
    rng = np.random.default_rng(5)
    idx = rng.choice(g.n, size=9, replace=False).astype(np.int32)
    val = rng.uniform(0.5, 2.0, size=9)
    pv = np.zeros(g.n)
    np.add.at(pv, idx, val)
    pv /= pv.sum()
    truth = oracle.power(g, C, pv, tol=1e-15)[0]
    with pr.Graph(g.n, g.m, *g.csr32()) as G:
        for algo in (pr.PR_IFP1, pr.PR_IFP2):
            out, st, s = G.solve(C, 1e-10, algo, pr.PR_FP32, p=val, p_idx=idx, opts=dict(mode=pr.PR_MODE_APULL))
            assert s == pr.PR_OK and l1(out, truth) <= min(1e-9, st["err_bound"] + 1e-13)
            # a stop above the hand-over point: the FP32 rounds reach it, one FP64 round confirms it
            out, st, s = G.solve(C, 1e-4, algo, pr.PR_FP32, p=val, p_idx=idx, opts=dict(mode=pr.PR_MODE_APULL))
            assert s == pr.PR_OK and l1(out, truth) <= st["err_bound"] + 1e-12
            assert st["fp64_rounds"] >= 1


@pytest.mark.parametrize("c", (0.5, 0.95))
def test_apull_fp32_form_other_damping(c):
    """The hand-over point follows 1/(1-c): at c = 0.95 it is three times
    higher than at 0.85; the FP64 rounds still end at eps."""
    g = gg.rmat(12, 8, dangling=0.2, unref=0.1, seed=13)
    truth = oracle.power(g, c, gg.p_uniform(g.n), tol=1e-15)[0]
    with pr.Graph(g.n, g.m, *g.csr32()) as G:
        for algo in (pr.PR_IFP1, pr.PR_IFP2):
            out, st, s = G.solve(c, 1e-11, algo, pr.PR_FP32, opts=dict(mode=pr.PR_MODE_APULL))
            assert s == pr.PR_OK and st["resid_l1"] <= 1e-11
            assert l1(out, truth) <= st["err_bound"] + 1e-13
            assert 0 < st["fp64_rounds"] < st["rounds"]


def test_apull_fp32_form_slow_contraction():
    """A directed cycle at c = 0.99: the residual falls by only 1% a round, the
    FP32 rounds run long before the hand-over; the result is still the exact
    uniform vector."""
    n = 64
    with pr.Graph(n, n, *gg.cycle(n).csr32()) as G:
        for algo in (pr.PR_IFP1, pr.PR_IFP2):
            out, st, s = G.solve(0.99, 1e-10, algo, pr.PR_FP32, opts=dict(mode=pr.PR_MODE_APULL))
            assert s == pr.PR_OK and st["fp64_rounds"] > 0
            assert l1(out, np.full(n, 1.0 / n)) <= max(1e-10, st["err_bound"] + 1e-13)
