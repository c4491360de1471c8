"""Asynchronous push rounds (PR_MODE_ASYNC): each frontier vertex pushes all
of its residual at the moment it is processed, as the threads of Sec. 3.2
do, so the schedule decides how far mass travels within a round.  The
oracle runs one schedule (frontier in id order); the GPU's is another, so
the tests check what holds for every schedule: the certified error bound
against the exact PageRank, the stopping rule, round 0's frontier, a
residual that falls at least as fast as in synchronous rounds, exact results
where the arithmetic is exact, and refusals."""
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
    ("small200", lambda: gg.random_small(200, 4.0, 0.2, 0.1, seed=1)),
    ("rmat13", lambda: gg.rmat(13, 8, dangling=0.15, unref=0.10, seed=4)),
    ("dag12", lambda: gg.rmat(12, 8, dangling=0.25, unref=0.0, dag_frac=0.9, seed=6)),
]


@pytest.mark.parametrize("gcase", GRAPHS, ids=lambda c: c[0])
@pytest.mark.parametrize("algo", (pr.PR_IFP1, pr.PR_IFP2))
@pytest.mark.parametrize("prec", (pr.PR_FP64, pr.PR_DF64, pr.PR_FP32))
def test_async_rounds_within_the_certified_bound(gcase, algo, prec):
    g = gcase[1]()
    truth = oracle.power(g, C, gg.p_uniform(g.n), tol=1e-15)[0]
    eps = 1e-7 if prec == pr.PR_FP32 else 1e-11
    slack = 2e-7 if prec == pr.PR_FP32 else 1e-13
    with pr.Graph(g.n, g.m, *g.csr32()) as G:
        _, sync, _ = G.solve(C, eps, algo, prec, opts=dict(mode=pr.PR_MODE_PUSH, xi_act=1e-300))
        for use_graph in (0, -1, 0):  # the schedule differs between runs; every run must hold
            out, st, s = G.solve(C, eps, algo, prec, opts=dict(mode=pr.PR_MODE_ASYNC, xi_act=1e-300,
                                                               use_graph=use_graph))
            assert s == pr.PR_OK, pr.pr_last_error()
            assert st["resid_l1"] <= eps and st["rounds_pull"] == 0
            assert l1(out, truth) <= st["err_bound"] + slack
            assert abs(float(np.sum(out)) - 1.0) < 1e-12
            if prec != pr.PR_FP32:  # the FP32 form restarts its rounds after the correction
                assert st["rounds"] <= sync["rounds"]


@pytest.mark.parametrize("prec", (pr.PR_FP64, pr.PR_DF64))
def test_async_chain_is_exact(prec):
    """On a path all mass runs to the dangling end; whatever the schedule, the
    residual reaches exactly 0 within n - 1 rounds and the result is the
    closed form y_k = (1 - c^(k+1)) / (n (1 - c)), normalised."""
    n = 40
    g = gg.chain(n)
    y = (1 - C ** (np.arange(n) + 1)) / (n * (1 - C))
    with pr.Graph(g.n, g.m, *g.csr32()) as G:
        for algo in (pr.PR_IFP1, pr.PR_IFP2):
            out, st, s = G.solve(C, 1e-300, algo, prec, opts=dict(mode=pr.PR_MODE_ASYNC, xi_act=1e-300))
            assert s == pr.PR_OK and st["resid_l1"] == 0.0
            assert st["rounds"] <= n - 1
            assert l1(out, y / y.sum()) < 1e-14


def test_async_rounds_on_a_dag():
    """90% of the edges follow a topological order: mass pushed on within a
    round can run down several edges, never fewer than in a synchronous round."""
    g = gg.rmat(14, 8, dangling=0.25, unref=0.0, dag_frac=0.9, seed=2)
    with pr.Graph(g.n, g.m, *g.csr32()) as G:
        _, sync, _ = G.solve(C, 1e-10, pr.PR_IFP2, pr.PR_DF64, opts=dict(mode=pr.PR_MODE_PUSH))
        _, asy, s = G.solve(C, 1e-10, pr.PR_IFP2, pr.PR_DF64, opts=dict(mode=pr.PR_MODE_ASYNC))
        assert s == pr.PR_OK and asy["rounds"] <= sync["rounds"]


@pytest.mark.parametrize("k", (1, 16))
def test_async_ppr(k):
    g = gg.rmat(12, 8, dangling=0.2, unref=0.1, seed=5)
    idx, val = gg.p_seeds(g.n, k, seed=k)
    p = gg.dense_from_sparse(g.n, idx, val)
    truth = oracle.power(g, C, p / p.sum(), tol=1e-15)[0]
    with pr.Graph(g.n, g.m, *g.csr32()) as G:
        out, st, s = G.solve(C, 1e-11, pr.PR_IFP2, pr.PR_DF64, p=val, p_idx=idx, opts=dict(mode=pr.PR_MODE_ASYNC))
        assert s == pr.PR_OK and l1(out, truth) <= st["err_bound"] + 1e-13


@pytest.mark.parametrize("algo", (pr.PR_IFP1, pr.PR_IFP2))
@pytest.mark.parametrize("prec", (pr.PR_FP64, pr.PR_DF64))
def test_async_rounds_against_the_oracle_schedules(algo, prec):
    """Every schedule takes round 0's frontier before any push, so its size and
    its edges are those of the synchronous round.  With p >= 0 each frontier
    vertex then pushes at least its round-start residual: R after round 1 is
    at most the synchronous R, and R never rises.  The oracle's id-order
    schedule obeys the same rules; both results sit within the certified
    bound of each other's residual."""
    g = gg.rmat(13, 8, dangling=0.15, unref=0.10, seed=4)
    p = gg.p_uniform(g.n)
    eps = 1e-11
    sync = oracle.ifp_rounds(algo, g, C, eps, p, xi_act=1e-300)
    ido = oracle.ifp_async(algo, g, C, eps, p, xi_act=1e-300)
    assert ido["status"] == 0 and ido["R"][1] <= sync["R"][1]
    with pr.Graph(g.n, g.m, *g.csr32()) as G:
        out, st, s = G.solve(C, eps, algo, prec, opts=dict(mode=pr.PR_MODE_ASYNC, xi_act=1e-300,
                                                          trace_cap=sync["rounds"] + 5))
        assert s == pr.PR_OK
        k, tr = st["rounds"], st["trace"]
        assert k <= sync["rounds"]
        assert tr["F"][0] == sync["F"][0] and tr["E"][0] == sync["E"][0]
        assert abs(tr["R"][0] - sync["R"][0]) <= 1e-14 * sync["R"][0]
        assert tr["R"][1] <= sync["R"][1] * (1 + 1e-12)
        assert np.all(np.diff(tr["R"][:k + 1]) <= 1e-15 * tr["R"][0])
        bound = oracle.certified_l1_bound(algo, C, st["resid_l1"]) + oracle.certified_l1_bound(algo, C, ido["R"][-1])
        assert l1(out, ido["pi"]) <= bound + 1e-13


def test_async_refused_where_it_does_not_apply():
    g = gg.rmat(10, 8, dangling=0.2, unref=0.1, seed=1)
    with pr.Graph(g.n, g.m, *g.csr32()) as G:
        _, _, s = G.solve(C, 1e-8, pr.PR_POWER, opts=dict(mode=pr.PR_MODE_ASYNC), check=False)
        assert s == pr.PR_EINVAL
        with pytest.raises(pr.PrError) as e:
            pr.pr_solve_batch([G], C, 1e-8, pr.PR_IFP2, opts=dict(mode=pr.PR_MODE_ASYNC))
        assert e.value.status == pr.PR_EINVAL
        _, _, s = G.solve(C, 1e-8, pr.PR_IFP2, opts=dict(mode=6), check=False)
        assert s == pr.PR_EINVAL
