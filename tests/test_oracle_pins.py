"""Pins for the FP64 oracle: closed forms, library routines and invariants.

Every check here ties an oracle function to something other than itself:
a closed-form PageRank derived by hand from the definition (Eq. 1/2/4), the
dominant eigenvector of the Google matrix P'' computed by numpy's eigensolver,
mass conservation and the residual identity checked with scipy sparse
products, or the convergence structure of Sec. 3.3.1 (R_t = c^t on a cycle,
a DAG drains after its longest path).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import graphgen as gg
import oracle
from oracle import IFP1, IFP2

C = 0.85


def google_matrix(g, c, p):
    """Dense P'' = c(P + p d^T) + (1-c) p e^T, written from Sec. 2.1."""
    n = g.n
    P = np.zeros((n, n))
    od = g.outdeg
    for j in range(n):
        for e in range(g.out_off[j], g.out_off[j + 1]):
            P[g.out_dst[e], j] += 1.0 / od[j]
    d = (od == 0).astype(float)
    return c * (P + np.outer(p, d)) + (1 - c) * np.outer(p, np.ones(n))


def eig_pagerank(g, c, p):
    """pi = P'' pi, pi > 0, sum pi = 1 via numpy.linalg.eig (eigenvalue 1)."""
    w, V = np.linalg.eig(google_matrix(g, c, p))
    k = int(np.argmin(np.abs(w - 1.0)))
    v = np.real(V[:, k])
    return v / v.sum()


def sparse_P(g):
    """Column-stochastic P (dangling columns zero) as scipy CSR."""
    od = g.outdeg
    src = np.repeat(np.arange(g.n), od)
    vals = 1.0 / od[src]
    return sp.csr_matrix((vals, (g.out_dst, src)), shape=(g.n, g.n))


def l1(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).sum())


# ------------------------------------------------------------------ cycle
@pytest.mark.parametrize("n", [1, 2, 7, 50])
def test_cycle_uniform_all_methods(orc, n):
    g = gg.cycle(n)
    p = gg.p_uniform(n)
    truth = np.full(n, 1.0 / n)
    pi, it, dl, st = orc.power(g, C, p)
    assert st == 0 and l1(pi, truth) < 1e-14
    assert l1(orc.dense_solve(g, C, p), truth) < 1e-13
    for algo in (IFP1, IFP2):
        pi = orc.ifp_sequential(algo, g, C, 1e-14, p)[0]
        assert l1(pi, truth) < 1e-13
        out = orc.ifp_rounds(algo, g, C, 1e-12, p)
        assert out["status"] == 0 and l1(out["pi"], truth) < 1e-13


def test_cycle_round_count_is_log_eps_over_log_c(orc):
    """Sec. 3.3.1 with no dangling vertex: alpha(t) = 1, R_t = c^t exactly."""
    n = 11
    g = gg.cycle(n)
    for eps, expect in ((1e-10, 142), (1e-9, 128), (1e-6, 86)):
        assert math.ceil(math.log(eps) / math.log(C)) == expect
        out = orc.ifp_rounds(IFP1, g, C, eps, gg.p_uniform(n))
        assert out["rounds"] == expect
        R = out["R"]
        t = np.arange(R.size)
        assert np.allclose(R, C ** t, rtol=1e-12, atol=0)
        assert np.all(out["F"] == n) and np.all(out["E"] == n)


@pytest.mark.parametrize("v", [0, 3])
def test_cycle_personalized_closed_form(orc, v):
    """p = e_v on an n-cycle: pi_{v+k} = (1-c) c^k / (1 - c^n)."""
    n = 9
    g = gg.cycle(n)
    p = np.zeros(n)
    p[v] = 1.0
    k = (np.arange(n) - v) % n
    truth = (1 - C) * C ** k / (1 - C ** n)
    assert abs(truth.sum() - 1) < 1e-15
    assert l1(orc.power(g, C, p)[0], truth) < 1e-13
    assert l1(orc.dense_solve(g, C, p), truth) < 1e-14
    for algo in (IFP1, IFP2):
        out = orc.ifp_rounds(algo, g, C, 1e-14, p)
        assert l1(out["pi"], truth) < 1e-12


# ------------------------------------------------------------------ chain
@pytest.mark.parametrize("n", [2, 5, 40])
def test_chain_closed_form_and_finite_rounds(orc, n):
    """Path 0->...->n-1: y_k = (1 - c^(k+1)) / (n (1-c)), pi = y / sum y.

    It is a DAG, so synchronous IFP drains the non-dangling residual to exactly
    zero after n-1 rounds (longest path), whatever eps is (Sec. 3.3.3).
    """
    g = gg.chain(n)
    p = gg.p_uniform(n)
    y = (1 - C ** (np.arange(n) + 1)) / (n * (1 - C))
    truth = y / y.sum()
    assert l1(orc.power(g, C, p)[0], truth) < 1e-13
    assert l1(orc.dense_solve(g, C, p), truth) < 1e-14
    for algo in (IFP1, IFP2):
        out = orc.ifp_rounds(algo, g, C, 1e-300, p, xi_act=0.0)
        assert out["status"] == 0
        assert out["rounds"] == n - 1
        assert out["R"][-1] == 0.0
        assert l1(out["pi"], truth) < 1e-14
        pi = orc.ifp_sequential(algo, g, C, 0.0, p)[0]
        assert l1(pi, truth) < 1e-14


# ------------------------------------------------------------------ stars
@pytest.mark.parametrize("n", [2, 6, 33])
def test_out_star(orc, n):
    """Centre -> n-1 dangling leaves: y_c = 1/n, y_leaf = 1/n + c/(n(n-1))."""
    g = gg.out_star(n)
    p = gg.p_uniform(n)
    y = np.full(n, 1.0 / n + C / (n * (n - 1)))
    y[0] = 1.0 / n
    truth = y / y.sum()
    assert l1(orc.dense_solve(g, C, p), truth) < 1e-14
    assert l1(orc.power(g, C, p)[0], truth) < 1e-13
    for algo in (IFP1, IFP2):
        out = orc.ifp_rounds(algo, g, C, 1e-15, p)
        assert l1(out["pi"], truth) < 1e-14
    # IFP2 invalidates every edge of the star: phase 1 pushes nothing.
    out = orc.ifp_rounds(IFP2, g, C, 1e-15, p)
    assert out["E"].sum() == 0
    assert orc.ifp_rounds(IFP1, g, C, 1e-15, p)["E"].sum() == n - 1


@pytest.mark.parametrize("n", [2, 6, 33])
def test_in_star(orc, n):
    """n-1 leaves -> dangling centre: y_leaf = 1/n, y_c = 1/n + c(n-1)/n."""
    g = gg.in_star(n)
    p = gg.p_uniform(n)
    y = np.full(n, 1.0 / n)
    y[0] = 1.0 / n + C * (n - 1) / n
    truth = y / y.sum()
    assert l1(orc.dense_solve(g, C, p), truth) < 1e-14
    assert l1(orc.power(g, C, p)[0], truth) < 1e-13
    for algo in (IFP1, IFP2):
        assert l1(orc.ifp_rounds(algo, g, C, 1e-15, p)["pi"], truth) < 1e-14
        assert l1(orc.ifp_sequential(algo, g, C, 0.0, p)[0], truth) < 1e-14


def test_three_vertex_hand_example(orc):
    """0->1, 0->2, 1->2, vertex 2 dangling, uniform p.

    From Eq. 4 (dangling mass is not pushed): y = (I - cP)^{-1} p with
    y0 = 1/3, y1 = 1/3 + c y0/2, y2 = 1/3 + c y0/2 + c y1.
    """
    g = gg.from_edges(3, [0, 0, 1], [1, 2, 2])
    p = gg.p_uniform(3)
    y0 = 1 / 3
    y1 = 1 / 3 + C * y0 / 2
    y2 = 1 / 3 + C * y0 / 2 + C * y1
    truth = np.array([y0, y1, y2]) / (y0 + y1 + y2)
    assert l1(orc.dense_solve(g, C, p), truth) < 1e-15
    assert l1(orc.power(g, C, p)[0], truth) < 1e-13
    for algo in (IFP1, IFP2):
        assert l1(orc.ifp_rounds(algo, g, C, 1e-300, p, xi_act=0.0)["pi"], truth) < 1e-15
        assert l1(orc.ifp_sequential(algo, g, C, 0.0, p)[0], truth) < 1e-15


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_no_edges_gives_p(orc, seed):
    n = 13
    g = gg.empty(n)
    p = gg.p_random(n, seed)
    p = p / p.sum()
    assert l1(orc.dense_solve(g, C, p), p) < 1e-15
    assert l1(orc.power(g, C, p)[0], p) < 1e-15
    for algo in (IFP1, IFP2):
        out = orc.ifp_rounds(algo, g, C, 1e-12, p)
        assert out["rounds"] == 0 and l1(out["pi"], p) < 1e-15


# ------------------------------------------------------ library eigen solver
@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("c", [0.5, 0.85, 0.99])
def test_dense_and_power_match_numpy_eigenvector(orc, seed, c):
    g = gg.random_small(24, avg_deg=2.5, dangling=0.25, unref=0.15, seed=seed, loops=True)
    p = gg.p_random(g.n, seed + 10, zero_frac=0.3)
    p /= p.sum()
    truth = eig_pagerank(g, c, p)
    assert np.all(truth > -1e-15)
    pi_ge = orc.dense_solve(g, c, p)
    assert l1(pi_ge, truth) < 1e-12
    assert abs(pi_ge.sum() - 1) < 1e-13
    tol = 1e-15 if c < 0.9 else 1e-13  # the FP64 floor of ||delta||_1 grows with 1/(1-c)
    pi_pw, it, dl, st = orc.power(g, c, p, tol=tol, max_iter=200000)
    assert st == 0
    assert l1(pi_pw, truth) < c * tol / (1 - c) + 1e-12 / (1 - c)


# --------------------------------------------------- IFP vs dense, with bounds
@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("eps", [1e-4, 1e-8, 1e-12])
def test_ifp_rounds_within_certified_bound(orc, seed, eps):
    g = gg.random_small(150, avg_deg=4.0, dangling=0.2, unref=0.1, seed=seed)
    p = gg.p_uniform(g.n)
    truth = orc.dense_solve(g, C, p)
    for algo in (IFP1, IFP2):
        out = orc.ifp_rounds(algo, g, C, eps, p)
        assert out["status"] == 0
        R = out["R"][-1]
        assert R <= eps
        err = l1(out["pi"], truth)
        assert err <= oracle.certified_l1_bound(algo, C, R) + 1e-14


@pytest.mark.parametrize("seed", range(4))
def test_ifp_sequential_within_bound(orc, seed):
    """Alg. 2/3 stop with every non-dangling h_i <= xi, so R <= n_nd xi."""
    g = gg.random_small(120, avg_deg=4.0, dangling=0.2, unref=0.1, seed=seed)
    p = gg.p_uniform(g.n)
    truth = orc.dense_solve(g, C, p)
    n_nd = int((g.outdeg > 0).sum())
    for xi in (1e-6, 1e-10):
        for algo in (IFP1, IFP2):
            pi, scans, pushes, edges, st = orc.ifp_sequential(algo, g, C, xi, p)
            assert st == 0
            assert l1(pi, truth) <= oracle.certified_l1_bound(algo, C, n_nd * xi) + 1e-14


def test_ifp_sequential_paper_init_h_equals_one(orc):
    """Alg. 2/3 start from h_i = 1; the normalised result is the uniform-p PageRank."""
    g = gg.random_small(60, avg_deg=3.0, dangling=0.2, unref=0.1, seed=7)
    truth = orc.dense_solve(g, C, gg.p_uniform(g.n))
    for algo in (IFP1, IFP2):
        pi = orc.ifp_sequential(algo, g, C, 1e-13, np.ones(g.n))[0]
        assert l1(pi, truth) < 1e-10


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("seed", range(3))
def test_mass_and_residual_identity_every_round(orc, seed):
    """IFP1: sum x + sum r = 1 after every round; the final state satisfies
    r = p + c P~ s - s with s = x/(1-c) (checked with a scipy sparse product)."""
    g = gg.random_small(200, avg_deg=5.0, dangling=0.2, unref=0.1, seed=seed)
    p = gg.p_uniform(g.n)
    P = sparse_P(g)
    out = orc.ifp_rounds(IFP1, g, C, 1e-9, p)
    assert np.all(np.abs(out["mass"] - 1.0) < 1e-13)
    s = out["x"] / (1 - C)
    assert l1(out["r"], p + C * (P @ s) - s) < 1e-13
    # IFP2 phase 1 works on P with the rows of dangling vertices zeroed.
    nd = (g.outdeg > 0).astype(float)
    Pt = sp.diags(nd) @ P
    for max_rounds in (3, 10):
        o2 = orc.ifp_rounds(IFP2, g, C, 1e-30, p, max_rounds=max_rounds)
        assert o2["status"] == 1 and o2["rounds"] == max_rounds
        s2 = o2["x"] / (1 - C)
        r_nd = (p + C * (Pt @ s2) - s2) * nd
        assert l1(o2["r"] * nd, r_nd) < 1e-13


def test_residual_never_increases_in_fp64(orc):
    g = gg.random_small(200, avg_deg=5.0, dangling=0.2, unref=0.1, seed=11)
    for algo in (IFP1, IFP2):
        R = orc.ifp_rounds(algo, g, C, 1e-12, gg.p_uniform(g.n))["R"]
        assert np.all(np.diff(R) <= 1e-16)


def test_symmetric_vertices_equal(orc):
    """Two identical branches 0->1->3, 0->2->3 plus 3->0: pi_1 == pi_2."""
    g = gg.from_edges(4, [0, 0, 1, 2, 3], [1, 2, 3, 3, 0])
    p = gg.p_uniform(4)
    for pi in (orc.dense_solve(g, C, p), orc.power(g, C, p)[0],
               orc.ifp_rounds(IFP1, g, C, 1e-14, p)["pi"], orc.ifp_rounds(IFP2, g, C, 1e-14, p)["pi"]):
        assert abs(pi[1] - pi[2]) < 1e-15


def test_ifp2_pushes_fewer_edges_same_result(orc):
    """IFP2 saves the pushes into dangling vertices (Sec. 3.4), same limit."""
    g = gg.random_small(200, avg_deg=5.0, dangling=0.3, unref=0.1, seed=5)
    p = gg.p_uniform(g.n)
    a = orc.ifp_rounds(IFP1, g, C, 1e-13, p)
    b = orc.ifp_rounds(IFP2, g, C, 1e-13, p)
    assert b["E"].sum() < a["E"].sum()
    assert l1(a["pi"], b["pi"]) < 1e-11
    # In round 0 every non-dangling vertex is active with uniform p: IFP1 pushes
    # all m edges, IFP2 all but the m_d edges into dangling vertices.
    st = g.stats()
    assert a["E"][0] == st["m"] and b["E"][0] == st["m"] - st["m_d"]


def test_self_loops_keep_their_share(orc):
    """A self-loop is an ordinary edge of P: the snapshot rule keeps its mass."""
    g = gg.random_small(40, avg_deg=3.0, dangling=0.2, unref=0.1, seed=3, loops=True)
    assert any(g.out_dst[e] == i for i in range(g.n) for e in range(g.out_off[i], g.out_off[i + 1]))
    p = gg.p_uniform(g.n)
    truth = eig_pagerank(g, C, p)
    for algo in (IFP1, IFP2):
        assert l1(orc.ifp_rounds(algo, g, C, 1e-14, p)["pi"], truth) < 1e-12
        assert l1(orc.ifp_sequential(algo, g, C, 1e-16, p)[0], truth) < 1e-12


def test_eq2_residual(orc):
    g = gg.random_small(50, avg_deg=3.0, dangling=0.2, unref=0.1, seed=2)
    p = gg.p_uniform(g.n)
    pi = orc.dense_solve(g, C, p)
    assert orc.eq2_residual(g, C, p, pi) < 1e-15
    # With P' = cycle on 2 vertices, pi = (a, b): (I - cP')pi = (a - cb, b - ca).
    g2 = gg.cycle(2)
    p2 = np.array([0.5, 0.5])
    a, b = 0.7, 0.3
    expect = abs(a - C * b - (1 - C) * 0.5) + abs(b - C * a - (1 - C) * 0.5)
    assert abs(orc.eq2_residual(g2, C, p2, np.array([a, b])) - expect) < 1e-15


def test_power_iterations_match_contraction_rate(orc):
    """||pi_{k+1} - pi_k||_1 <= c^k ||pi_1 - pi_0||_1: the 210-iteration truth of Sec. 4
    reaches 0.85^210 ~ 1.5e-15."""
    g = gg.random_small(100, avg_deg=4.0, dangling=0.2, unref=0.1, seed=4)
    p = gg.p_uniform(g.n)
    d1 = orc.power(g, C, p, tol=0.0, max_iter=1)[2]
    for k in (10, 50, 100):
        dk = orc.power(g, C, p, tol=0.0, max_iter=k + 1)[2]
        assert dk <= C ** k * d1 * (1 + 1e-9) + 1e-16
    pi210 = orc.power(g, C, p, tol=0.0, max_iter=210)[0]
    assert l1(pi210, orc.dense_solve(g, C, p)) < 1e-13


def test_not_converged_and_stall_status(orc):
    g = gg.cycle(5)
    out = orc.ifp_rounds(IFP1, g, C, 1e-12, gg.p_uniform(5), max_rounds=4)
    assert out["status"] == 1 and out["rounds"] == 4
    out = orc.ifp_rounds(IFP1, g, C, 1e-12, gg.p_uniform(5), xi_act=1.0)
    assert out["status"] == 2 and out["rounds"] == 0


# ------------------------------------------------- level-ordered IFP2 rounds
@pytest.mark.parametrize("n", [2, 3, 4, 9, 40])
def test_levels_drain_a_chain_in_three_rounds(orc, n):
    """Path 0->...->n-1 with one level per vertex (the chain's vertices tie on
    the level key and fall in id order): two synchronous rounds, then one
    level-ordered round carries every residual to the end, where synchronous
    rounds need n-1 (the asynchronous scans of Sec. 3.2 on a DAG)."""
    g = gg.chain(n)
    p = gg.p_uniform(n)
    y = (1 - C ** (np.arange(n) + 1)) / (n * (1 - C))
    truth = y / y.sum()
    L = max(n - 2, 1)
    lv = oracle.gs_levels(g, L)
    if n > 2:
        assert list(lv[1:n - 1]) == list(range(n - 2)) and lv[0] == L and lv[n - 1] == -1
    out = orc.ifp2_levels(g, C, 1e-300, p, lv, L, xi_act=0.0)
    assert out["status"] == 0
    assert out["rounds"] == (1 if n == 2 else 3)
    assert l1(out["pi"], truth) < 1e-14
    if n >= 4:  # IFP2 never pushes into the dangling end: n-2, n-3, n-4 valid edges pushed
        assert list(out["E"]) == [n - 2, n - 3, n - 4]
        assert list(out["F"]) == [n - 1, n - 2, n - 3]


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("L", [1, 3, 16])
def test_levels_identity_and_bound(orc, seed, L):
    """The state after any level-ordered round satisfies
    r + r_pending = p + c P~ s - s on the non-dangling vertices (s = x/(1-c)),
    and the result is within 2R/(1-c) of the exact PageRank."""
    g = gg.random_small(200, avg_deg=5.0, dangling=0.2, unref=0.1, seed=seed)
    p = gg.p_uniform(g.n)
    P = sparse_P(g)
    nd = (g.outdeg > 0).astype(float)
    Pt = sp.diags(nd) @ P
    lv = oracle.gs_levels(g, L)
    truth = eig_pagerank(g, C, p)
    for max_rounds in (2, 3, 7):
        o = orc.ifp2_levels(g, C, 1e-30, p, lv, L, max_rounds=max_rounds)
        assert o["status"] == 1
        s = o["x"] / (1 - C)
        assert l1((o["r"] + o["r_pending"]) * nd, (p + C * (Pt @ s) - s) * nd) < 1e-13
    o = orc.ifp2_levels(g, C, 1e-10, p, lv, L)
    assert o["status"] == 0
    assert l1(o["pi"], truth) <= 2 * o["R"][-1] / (1 - C) + 1e-14
    # the stop test saw the whole residual of the state: delivered and in flight
    assert abs(o["R"][-1] - float(((np.abs(o["r"]) + np.abs(o["r_pending"])) * nd).sum())) < 1e-20


def test_levels_assignment_rule():
    """Ranks by floor(2^31 (in+1)/(in+out+2)), ties by id; unreferenced get L."""
    g = gg.from_edges(6, np.array([0, 0, 0, 1, 2, 3, 4], np.int32), np.array([1, 2, 3, 2, 3, 4, 1], np.int32))
    # in/out: v0 0/3 (unreferenced), v1 2/1, v2 2/1, v3 2/1, v4 1/1, v5 dangling, isolated
    lv = oracle.gs_levels(g, 4)
    assert lv[0] == 4 and lv[5] == -1
    # keys: v4: 2/4 -> 2^30 ; v1, v2, v3: 3/5 -> floor(0.6 * 2^31): v4 first, then 1, 2, 3
    assert list(lv[[4, 1, 2, 3]]) == [0, 1, 2, 3]


def test_levels_fewer_rounds_than_synchronous(orc):
    g = gg.rmat(12, 8, dangling=0.2, unref=0.1, seed=1)
    p = gg.p_uniform(g.n)
    sync = orc.ifp_rounds(IFP2, g, C, 1e-10, p)
    lv = oracle.gs_levels(g, 16)
    gs = orc.ifp2_levels(g, C, 1e-10, p, lv, 16)
    assert gs["rounds"] < 0.75 * sync["rounds"]
    assert l1(gs["pi"], sync["pi"]) < 2e-9


# --------------------------------------- asynchronous rounds in id order
def ordered_dag(n, avg_deg, seed, forward):
    """random_small's edges re-pointed so that every edge runs to a higher id
    (forward, self-loops dropped) or to a lower or equal id (self-loops kept)."""
    g = gg.random_small(n, avg_deg=avg_deg, dangling=0.2, unref=0.1, seed=seed, loops=True)
    src = np.repeat(np.arange(g.n), g.outdeg).astype(np.int32)
    dst = g.out_dst.astype(np.int32)
    lo, hi = np.minimum(src, dst), np.maximum(src, dst)
    if forward:
        keep = lo != hi
        return gg.from_edges(n, lo[keep], hi[keep])
    return gg.from_edges(n, hi, lo)


@pytest.mark.parametrize("n", [2, 3, 40])
def test_async_chain_drains_in_one_round(orc, n):
    """Path 0->...->n-1 taken in id order: each vertex passes on, in the same
    round, all that its predecessor just gave it, so one round carries every
    residual to the dangling end (synchronous rounds need n-1)."""
    g = gg.chain(n)
    y = (1 - C ** (np.arange(n) + 1)) / (n * (1 - C))
    for algo in (IFP1, IFP2):
        o = orc.ifp_async(algo, g, C, 0.0, gg.p_uniform(n), xi_act=0.0)
        assert o["status"] == 0 and o["rounds"] == 1 and o["R"][-1] == 0.0
        assert l1(o["pi"], y / y.sum()) < 1e-14
        assert orc.ifp_rounds(algo, g, C, 0.0, gg.p_uniform(n), xi_act=0.0)["rounds"] == n - 1


@pytest.mark.parametrize("seed", range(3))
def test_async_forward_dag_drains_in_one_round(orc, seed):
    """Every edge runs to a higher id: when a vertex's turn comes, all its
    in-neighbours have pushed, and nothing reaches it afterwards.  One round
    leaves no residual on a non-dangling vertex, and the result is the exact
    PageRank (eigenvector of the Google matrix)."""
    g = ordered_dag(120, 4.0, seed, forward=True)
    for p in (gg.p_uniform(g.n), gg.p_random(g.n, seed) / gg.p_random(g.n, seed).sum()):
        truth = eig_pagerank(g, C, p)
        for algo in (IFP1, IFP2):
            o = orc.ifp_async(algo, g, C, 0.0, p, xi_act=0.0)
            assert o["status"] == 0 and o["rounds"] == 1 and o["R"][-1] == 0.0
            assert l1(o["pi"], truth) < 1e-13


@pytest.mark.parametrize("seed", range(3))
def test_async_equals_synchronous_when_edges_point_down(orc, seed):
    """Every edge runs to a lower or equal id: a vertex receives nothing
    before its turn in a round, so the id-order schedule pushes exactly the
    round-start values, in the same order, as the synchronous rounds."""
    g = ordered_dag(150, 4.0, seed, forward=False)
    p = gg.p_random(g.n, seed + 10, zero_frac=0.3)
    p /= p.sum()
    for algo in (IFP1, IFP2):
        for cap in (1, 4, 100000):
            a = orc.ifp_async(algo, g, C, 1e-12, p, max_rounds=cap)
            s = orc.ifp_rounds(algo, g, C, 1e-12, p, max_rounds=cap)
            assert a["status"] == s["status"] and a["rounds"] == s["rounds"]
            for k in ("x", "r", "pi", "R", "F"):
                assert np.array_equal(a[k], s[k]), (algo, cap, k)


@pytest.mark.parametrize("seed", range(3))
def test_async_identity_and_mass_at_any_stop(orc, seed):
    """A push moves (1-c)v to the reserve and cv along the out-edges, whatever
    the schedule, so after any round: IFP1 keeps sum x + sum r = sum p and
    r = p + c P s - s (s = x/(1-c)); IFP2 keeps that identity on the
    non-dangling vertices with P~ (edges into dangling vertices dropped)."""
    g = gg.random_small(200, avg_deg=5.0, dangling=0.2, unref=0.1, seed=seed, loops=True)
    p = gg.p_uniform(g.n)
    P = sparse_P(g)
    nd = (g.outdeg > 0).astype(float)
    Pt = sp.diags(nd) @ P
    for cap in (1, 2, 5):
        o = orc.ifp_async(IFP1, g, C, 1e-30, p, max_rounds=cap)
        assert o["status"] == 1 and o["rounds"] == cap
        assert abs(o["x"].sum() + o["r"].sum() - 1.0) < 1e-14
        s = o["x"] / (1 - C)
        assert l1(o["r"], p + C * (P @ s) - s) < 1e-13
        o = orc.ifp_async(IFP2, g, C, 1e-30, p, max_rounds=cap)
        s = o["x"] / (1 - C)
        assert l1(o["r"] * nd, (p + C * (Pt @ s) - s) * nd) < 1e-13


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("eps", [1e-5, 1e-11])
def test_async_within_certified_bound(orc, seed, eps):
    """The bound depends only on the final residual, not on how it was
    reached: l1(pi, exact) <= 2cR/(1-c) (IFP1), 2R/(1-c) (IFP2)."""
    g = gg.random_small(150, avg_deg=4.0, dangling=0.2, unref=0.1, seed=seed)
    p = gg.p_random(g.n, seed, zero_frac=0.5)
    p /= p.sum()
    truth = eig_pagerank(g, C, p)
    for algo in (IFP1, IFP2):
        o = orc.ifp_async(algo, g, C, eps, p)
        assert o["status"] == 0 and o["R"][-1] <= eps
        assert l1(o["pi"], truth) <= oracle.certified_l1_bound(algo, C, o["R"][-1]) + 1e-14


@pytest.mark.parametrize("seed", range(3))
def test_async_residual_falls_at_least_as_fast_in_a_round(orc, seed):
    """With p >= 0 every residual stays >= 0, and a pushed amount of v lowers
    R by at least (1-c)v; a vertex of the frontier pushes at least its
    round-start value.  So R never rises, and after the first round it is no
    larger than after a synchronous round from the same start."""
    g = gg.random_small(200, avg_deg=5.0, dangling=0.2, unref=0.1, seed=seed)
    p = gg.p_random(g.n, seed, zero_frac=0.3)
    p /= p.sum()
    for algo in (IFP1, IFP2):
        a = orc.ifp_async(algo, g, C, 1e-12, p)
        s = orc.ifp_rounds(algo, g, C, 1e-12, p)
        assert np.all(np.diff(a["R"]) <= 0.0)
        assert a["R"][1] <= s["R"][1]
        assert np.all(a["r"] >= 0.0)


def test_async_statuses_and_rounds_on_rmat(orc):
    g = gg.rmat(11, 8, dangling=0.2, unref=0.1, seed=1)
    p = gg.p_uniform(g.n)
    for algo in (IFP1, IFP2):
        a = orc.ifp_async(algo, g, C, 1e-10, p)
        s = orc.ifp_rounds(algo, g, C, 1e-10, p)
        assert a["status"] == 0 and a["rounds"] < s["rounds"]
        assert l1(a["pi"], s["pi"]) <= oracle.certified_l1_bound(algo, C, 1e-10) * 2
    assert orc.ifp_async(IFP1, g, C, 1e-12, p, max_rounds=3)["status"] == 1
    o = orc.ifp_async(IFP1, g, C, 1e-12, p, xi_act=1.0)
    assert o["status"] == 2 and o["rounds"] == 0
    o = orc.ifp_async(IFP2, gg.empty(5), C, 1e-12, gg.p_uniform(5))
    assert o["status"] == 0 and o["rounds"] == 0 and l1(o["pi"], gg.p_uniform(5)) < 1e-15


@pytest.mark.parametrize("seed", range(3))
def test_ifp2_mass_with_phase2_at_any_stop(orc, seed):
    """IFP2 defers the pushes into dangling vertices: each push of v keeps
    (1-c)v, sends c v ndeg/deg to non-dangling targets, and leaves
    c v (deg - ndeg)/deg for phase 2 (Alg. 3), which hands it to the dangling
    targets in one step.  So once phase 2 has run, sum x + sum r = sum p at any
    stopping point, whatever the schedule."""
    g = gg.random_small(200, avg_deg=5.0, dangling=0.25, unref=0.1, seed=seed, loops=True)
    p = gg.p_random(g.n, seed, zero_frac=0.2)
    p /= p.sum()
    for run in (orc.ifp_rounds, orc.ifp_async):
        for cap in (1, 3, 100000):
            o = run(IFP2, g, C, 1e-13, p, max_rounds=cap)
            assert abs(o["x"].sum() + o["r"].sum() - 1.0) < 1e-14, (run.__name__, cap)


@pytest.mark.parametrize("n", [2, 5, 30])
def test_async_cycle_closed_form(orc, n):
    """Directed cycle 0->1->...->n-1->0, uniform p, frontier in id order.  In
    round 1 vertex k pushes everything it holds, (1 - c^(k+1))/(n(1-c)), so
    only vertex 0 keeps a residual: c(1 - c^n)/(n(1-c)).  From then on the
    frontier is the one vertex holding mass (the others received theirs after
    the round started), so each round moves it one step: R_t = c^(t-1) R_1.
    The result is still 1/n everywhere."""
    g = gg.cycle(n)
    for algo in (IFP1, IFP2):
        o = orc.ifp_async(algo, g, C, 1e-12, gg.p_uniform(n), xi_act=0.0)
        R1 = C * (1 - C ** n) / (n * (1 - C))
        t = np.arange(1, len(o["R"]))
        assert o["R"][0] == pytest.approx(1.0, abs=1e-15)
        assert np.allclose(o["R"][1:], R1 * C ** (t - 1), rtol=1e-12, atol=0)
        assert list(o["F"]) == [n] + [1] * (o["rounds"] - 1)
        assert o["rounds"] == 1 + int(math.ceil(math.log(1e-12 / R1) / math.log(C)))
        assert l1(o["pi"], np.full(n, 1.0 / n)) < 1e-11


# --------------------------------------- scans in id order (asynchronous pull rounds)
@pytest.mark.parametrize("n", [2, 3, 40])
def test_scan_chain_drains_in_one_scan(orc, n):
    """Path 0->...->n-1 in id order: each vertex passes on at its turn all its
    predecessor just gave it, so one scan carries every residual to the
    dangling end, exactly."""
    g = gg.chain(n)
    y = (1 - C ** (np.arange(n) + 1)) / (n * (1 - C))
    for algo in (IFP1, IFP2):
        o = orc.ifp_scan(algo, g, C, 0.0, gg.p_uniform(n), xi_act=0.0)
        assert o["status"] == 0 and o["rounds"] == 1 and o["R"][-1] == 0.0
        assert l1(o["pi"], y / y.sum()) < 1e-14


@pytest.mark.parametrize("seed", range(3))
def test_scan_forward_dag_drains_in_one_scan(orc, seed):
    """Every edge runs to a higher id: one scan leaves no residual on a
    non-dangling vertex and gives the exact PageRank."""
    g = ordered_dag(120, 4.0, seed, forward=True)
    p = gg.p_random(g.n, seed) / gg.p_random(g.n, seed).sum()
    truth = eig_pagerank(g, C, p)
    for algo in (IFP1, IFP2):
        o = orc.ifp_scan(algo, g, C, 0.0, p, xi_act=0.0)
        assert o["status"] == 0 and o["rounds"] == 1 and o["R"][-1] == 0.0
        assert l1(o["pi"], truth) < 1e-13


@pytest.mark.parametrize("seed", range(3))
def test_scan_equals_synchronous_when_edges_point_down(orc, seed):
    """Every edge runs to a lower or equal id: at its turn a vertex holds its
    scan-start value, and every vertex holding more than xi_act pushes, so a
    scan is one synchronous round: the same frontiers, residuals and result."""
    g = ordered_dag(150, 4.0, seed, forward=False)
    p = gg.p_random(g.n, seed + 10, zero_frac=0.3)
    p /= p.sum()
    for algo in (IFP1, IFP2):
        a = orc.ifp_scan(algo, g, C, 1e-12, p)
        s = orc.ifp_rounds(algo, g, C, 1e-12, p)
        assert a["status"] == s["status"] == 0 and a["rounds"] == s["rounds"]
        assert np.array_equal(a["F"], s["F"][:a["rounds"]])
        # the rounds trace R at each round's start (R_0 = 1), the scans at each scan's end
        assert np.allclose(a["R"], s["R"][1:a["rounds"] + 1], rtol=1e-13, atol=0)
        assert l1(a["pi"], s["pi"]) < 1e-15


@pytest.mark.parametrize("seed", range(3))
def test_scan_identity_mass_and_bound_at_any_stop(orc, seed):
    """After any number of scans the state is one of the rounds' states: IFP1
    keeps sum x + sum r = sum p; r = p + c P~ s - s (s = x/(1-c)) on the
    non-dangling vertices; the exact residual R never exceeds the bound the
    GPU stops on, and R never rises (p >= 0)."""
    g = gg.random_small(200, avg_deg=5.0, dangling=0.2, unref=0.1, seed=seed, loops=True)
    p = gg.p_random(g.n, seed, zero_frac=0.3)
    p /= p.sum()
    P = sparse_P(g)
    nd = (g.outdeg > 0).astype(float)
    Pt = sp.diags(nd) @ P
    for cap in (1, 2, 5):
        o = orc.ifp_scan(IFP1, g, C, 1e-30, p, max_rounds=cap)
        assert o["status"] == 1 and o["rounds"] == cap
        assert abs(o["x"].sum() + o["r"].sum() - 1.0) < 1e-14
        s = o["x"] / (1 - C)
        assert l1(o["r"], p + C * (P @ s) - s) < 1e-13
        assert np.all(o["R"] <= o["Rub"] * (1 + 1e-14))
        o = orc.ifp_scan(IFP2, g, C, 1e-30, p, max_rounds=cap)
        s = o["x"] / (1 - C)
        assert l1(o["r"] * nd, (p + C * (Pt @ s) - s) * nd) < 1e-13
        assert np.all(o["R"] <= o["Rub"] * (1 + 1e-14))
        assert np.all(np.diff(o["R"]) <= 0.0)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("eps", [1e-5, 1e-11])
def test_scan_within_certified_bound_and_faster(orc, seed, eps):
    g = gg.random_small(150, avg_deg=4.0, dangling=0.2, unref=0.1, seed=seed)
    p = gg.p_random(g.n, seed, zero_frac=0.5)
    p /= p.sum()
    truth = eig_pagerank(g, C, p)
    for algo in (IFP1, IFP2):
        o = orc.ifp_scan(algo, g, C, eps, p)
        assert o["status"] == 0 and o["R"][-1] <= eps
        assert l1(o["pi"], truth) <= oracle.certified_l1_bound(algo, C, o["R"][-1]) + 1e-14
        assert o["rounds"] < orc.ifp_rounds(algo, g, C, eps, p)["rounds"]


@pytest.mark.parametrize("n", [2, 5, 30])
def test_scan_cycle_closed_form(orc, n):
    """Directed cycle 0->1->...->n-1->0, uniform p.  In scan 1 vertex k pushes
    (1 - c^(k+1))/(n(1-c)), so only vertex 0 keeps c(1 - c^n)/(n(1-c)) = R_1.
    In every later scan that mass goes once around the cycle: R_t = c^(n(t-1)) R_1,
    with all n vertices pushing.  The bound the GPU stops on counts every
    push as possibly in flight: c times the mass pushed."""
    g = gg.cycle(n)
    for algo in (IFP1, IFP2):
        o = orc.ifp_scan(algo, g, C, 1e-12, gg.p_uniform(n), xi_act=0.0)
        R1 = C * (1 - C ** n) / (n * (1 - C))
        t = np.arange(1, o["rounds"] + 1)
        assert np.allclose(o["R"], R1 * C ** (n * (t - 1)), rtol=1e-12, atol=0)
        assert list(o["F"]) == [n] * o["rounds"]
        pushed1 = sum((1 - C ** (k + 1)) / (n * (1 - C)) for k in range(n))
        assert o["Rub"][0] == pytest.approx(C * pushed1, rel=1e-13)
        assert l1(o["pi"], np.full(n, 1.0 / n)) < 1e-11
