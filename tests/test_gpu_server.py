"""pr_server: continuous batching of IFP2 requests on resident graphs.

A request served in a mix of others (different graphs, sizes, damping
factors, personalization vectors, precisions, arrival times) must give the
result of the same solve done alone with pr_solve, and be within its
certified bound of the exact (personalized) PageRank from the FP64 oracle.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_03245_gb300 as pr  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pr.build()


def l1(a, b):
    return float(np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)).sum())


@pytest.fixture(scope="module")
def graphs():
    gl = [gg.rmat(14, 8, dangling=0.15, unref=0.10, seed=11),
          gg.er(4000, 5.0, dangling=0.2, unref=0.1, seed=12),
          gg.rmat(10, 16, dangling=0.3, unref=0.1, seed=13),
          gg.cycle(31), gg.in_star(50), gg.empty(7),
          gg.random_small(200, 3.0, 0.2, 0.1, seed=14)]
    hs = [pr.Graph(g.n, g.m, *g.csr32()) for g in gl]
    yield gl, hs
    for h in hs:
        h.close()


def request_mix(gl, seed=0):
    """(graph index, c, eps, prec, p, p_idx) for a mix of full and personalized requests."""
    rng = np.random.default_rng(seed)
    reqs = []
    for k, g in enumerate(gl):
        for prec in (pr.PR_DF64, pr.PR_FP32):
            eps = 1e-10 if prec == pr.PR_DF64 else 1e-9
            c = 0.85 if (k + prec) % 2 == 0 else 0.6
            reqs.append((k, c, eps, prec, None, None))
            if g.n >= 4:
                idx = rng.choice(g.n, size=min(3, g.n), replace=False).astype(np.int32)
                val = rng.uniform(0.5, 2.0, size=idx.size)
                reqs.append((k, c, eps, prec, val, idx))
    return reqs


def truth_of(g, c, p, p_idx):
    if p is None:
        pv = gg.p_uniform(g.n)
    else:
        pv = np.zeros(g.n)
        np.add.at(pv, p_idx, p)
        pv /= pv.sum()
    return oracle.power(g, c, pv, tol=1e-15)[0]


def test_server_mix_matches_alone_and_oracle(graphs):
    gl, hs = graphs
    reqs = request_mix(gl)
    with pr.Server(1 << 32) as S:
        tickets = [S.submit(hs[k], c, eps, prec, p, pi) for (k, c, eps, prec, p, pi) in reqs]
        results = [S.wait(t) for t in tickets]
    for (k, c, eps, prec, p, pi), (out, st, status) in zip(reqs, results):
        assert status == pr.PR_OK, (k, prec, st)
        assert abs(out.sum() - 1.0) < 1e-12
        alone, st1, s1 = hs[k].solve(c, eps, pr.PR_IFP2, prec, p=p, p_idx=pi)
        assert s1 == pr.PR_OK
        if prec == pr.PR_DF64:
            assert l1(out, alone) <= 1e-12, (k, l1(out, alone))
            assert abs(st["rounds"] - st1["rounds"]) <= 1
        else:
            assert l1(out, alone) <= st["err_bound"] + st1["err_bound"] + 1e-12, (k, l1(out, alone))
        truth = truth_of(gl[k], c, p, pi)
        assert l1(out, truth) <= st["err_bound"] + 1e-12, (k, prec, l1(out, truth), st["err_bound"])
        assert st["err_bound"] <= 2.0 * eps / (1.0 - c) + 1e-15


def test_server_staggered_arrivals(graphs):
    """Requests that arrive while others run join the running batch."""
    gl, hs = graphs
    with pr.Server(1 << 32) as S:
        first = [S.submit(hs[0], 0.85, 1e-11, pr.PR_DF64) for _ in range(3)]
        late = []
        for j in range(6):
            late.append(S.submit(hs[j % 3], 0.85, 1e-10, pr.PR_DF64 if j % 2 else pr.PR_FP32))
        outs = [S.wait(t) for t in first + late]
    ref = outs[0][0]
    for out, st, status in outs[:3]:
        assert status == pr.PR_OK
        assert l1(out, ref) <= 1e-13  # the same request three times
    for j, (out, st, status) in enumerate(outs[3:]):
        assert status == pr.PR_OK
        truth = truth_of(gl[j % 3], 0.85, None, None)
        assert l1(out, truth) <= st["err_bound"] + 1e-12


def test_server_budget_admission(graphs):
    """A budget that fits about one request at a time still serves them all."""
    gl, hs = graphs
    g0 = gl[0]
    one = 100 * g0.n  # bytes: above one DF64 request's state on this graph (about 63 n), below two
    with pr.Server(one) as S:
        tickets = [S.submit(hs[0], 0.85, 1e-10, pr.PR_DF64) for _ in range(4)]
        outs = [S.wait(t) for t in tickets]
    truth = truth_of(g0, 0.85, None, None)
    for out, st, status in outs:
        assert status == pr.PR_OK
        assert l1(out, truth) <= st["err_bound"] + 1e-12


def test_server_invalid_arguments(graphs):
    gl, hs = graphs
    with pytest.raises(pr.PrError) as e:
        pr.pr_server_create(0)
    assert e.value.status == pr.PR_EINVAL
    with pr.Server(1 << 30) as S:
        for bad in (dict(c=1.0, eps=1e-9, prec=pr.PR_DF64), dict(c=0.85, eps=0.0, prec=pr.PR_DF64),
                    dict(c=0.85, eps=1e-9, prec=pr.PR_FP64)):
            with pytest.raises(pr.PrError) as e:
                S.submit(hs[0], bad["c"], bad["eps"], bad["prec"])
            assert e.value.status == pr.PR_EINVAL
        with pytest.raises(pr.PrError) as e:
            S.submit(hs[0], 0.85, 1e-9, pr.PR_DF64, p=np.array([1.0]), p_idx=np.array([gl[0].n], np.int32))
        assert e.value.status == pr.PR_EINVAL
        st = pr.pr_stats()
        assert pr.lib().pr_server_poll(S.h, 12345, None, ctypes.byref(st)) == pr.PR_EINVAL  # unknown ticket
        with pytest.raises(ValueError):
            pr.pr_server_poll(S.h, 12345, 1)
        t = S.submit(hs[3], 0.85, 1e-9, pr.PR_DF64)
        # the output is checked against the request's graph, not a caller's n
        with pytest.raises(ValueError):
            pr.pr_server_poll(S.h, t, gl[3].n - 1, np.empty(gl[3].n - 1))
        with pytest.raises(ValueError):
            pr.pr_server_poll(S.h, t, None, np.empty(gl[3].n - 1))
        S.wait(t)
        assert pr.lib().pr_server_poll(S.h, t, None, ctypes.byref(st)) == pr.PR_EINVAL  # released by its poll
        with pytest.raises(ValueError):
            pr.pr_server_poll(S.h, t, gl[3].n)
    with pr.Server(4096) as S:  # one request needs more than the whole budget
        with pytest.raises(pr.PrError) as e:
            S.submit(hs[0], 0.85, 1e-9, pr.PR_DF64)
        assert e.value.status == pr.PR_EINVAL


def test_server_destroy_with_requests_in_flight(graphs):
    gl, hs = graphs
    S = pr.Server(1 << 32)
    for _ in range(8):
        S.submit(hs[0], 0.85, 1e-12, pr.PR_DF64)
    S.close()  # drops them; must not hang or leak device memory into later tests
    with pr.Server(1 << 32) as S2:
        out, st, status = S2.wait(S2.submit(hs[1], 0.85, 1e-10, pr.PR_DF64))
        assert status == pr.PR_OK


@pytest.fixture(scope="module")
def big():
    g = gg.rmat(16, 8, dangling=0.15, unref=0.10, seed=31)
    h = pr.Graph(g.n, g.m, *g.csr32())
    assert h.info["n_nd"] >= (1 << 14)  # large enough for column groups
    yield g, h
    h.close()


@pytest.mark.parametrize("prec", [pr.PR_FP32, pr.PR_DF64])
def test_server_column_groups_match_alone(big, prec):
    """Many requests on one large graph share gathers in column groups (more
    requests than one group holds, different seeds, damping factors and
    arrival times); each result equals the same solve alone."""
    g, h = big
    rng = np.random.default_rng(5 + prec)
    reqs = []
    for j in range(19):
        c = (0.85, 0.7, 0.9)[j % 3]
        if j % 5 == 4:
            reqs.append((c, None, None))  # full PageRank in the mix
        else:
            k = int(rng.integers(1, 65))
            idx = rng.choice(g.n, size=k, replace=False).astype(np.int32)
            reqs.append((c, rng.uniform(0.5, 1.5, size=k), idx))
    eps = 1e-10 if prec == pr.PR_DF64 else 1e-8
    with pr.Server(1 << 34) as S:
        first = [S.submit(h, c, eps, prec, p, pi) for (c, p, pi) in reqs[:11]]
        _ = S.wait(first[0])  # the rest arrive while the others run
        later = [S.submit(h, c, eps, prec, p, pi) for (c, p, pi) in reqs[11:]]
        results = [_] + [S.wait(t) for t in first[1:] + later]
    for (c, p, pi), (out, st, status) in zip(reqs, results):
        assert status == pr.PR_OK
        assert abs(out.sum() - 1.0) < 1e-12
        alone, st1, s1 = h.solve(c, eps, pr.PR_IFP2, prec, p=p, p_idx=pi)
        assert l1(out, alone) <= st["err_bound"] + st1["err_bound"] + 1e-12
        truth = truth_of(g, c, p, pi)
        assert l1(out, truth) <= st["err_bound"] + 1e-12, (l1(out, truth), st["err_bound"])
        if prec == pr.PR_DF64:
            # the same arithmetic as a pull-only solve alone (up to the order of the sums)
            alone_pull, st2, _ = h.solve(c, eps, pr.PR_IFP2, prec, p=p, p_idx=pi, opts=dict(mode=pr.PR_MODE_PULL))
            assert l1(out, alone_pull) <= 1e-12
            assert abs(st["rounds"] - st2["rounds"]) <= 1


def test_server_fp32_requests_meet_the_gate(big):
    """Served FP32-form requests (FP32 rounds, IEEE FP64 correction and rounds) at the
    benchmark's eps 5e-7 are within L1 1e-6 of their exact (personalized) PageRank,
    alone and in a mix of column-group and tile-engine requests."""
    g, h = big
    rng = np.random.default_rng(77)
    reqs = [(None, None)]
    for _ in range(9):
        k = int(rng.integers(1, 65))
        reqs.append((np.full(k, 1.0 / k), rng.choice(g.n, size=k, replace=False).astype(np.int32)))
    with pr.Server(1 << 34) as S:
        tickets = [S.submit(h, 0.85, 5e-7, pr.PR_FP32, p, pi) for p, pi in reqs]
        results = [S.wait(t) for t in tickets]
    for (p, pi), (out, st, status) in zip(reqs, results):
        assert status == pr.PR_OK
        assert st["fp64_rounds"] >= 0
        err = l1(out, truth_of(g, 0.85, p, pi))
        assert err <= 1e-6, err
