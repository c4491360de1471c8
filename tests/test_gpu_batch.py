"""pr_solve_batch: many graphs of uneven size in one persistent kernel per phase.

Each problem of a batch must give the result of the same solve done alone
(pr_solve with the same algorithm, precision, eps and options) -- the batch
changes the schedule, not the arithmetic -- and must be within the certified
bound of the exact PageRank from the FP64 oracle.
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


def mixed_graphs():
    """Uneven sizes and shapes: R-MAT of several scales, ER, fixed shapes, an empty graph."""
    return [gg.rmat(13, 8, dangling=0.15, unref=0.10, seed=1),
            gg.er(3000, 6.0, dangling=0.2, unref=0.1, seed=2),
            gg.rmat(10, 12, dangling=0.3, unref=0.1, seed=3),
            gg.cycle(17), gg.chain(25), gg.in_star(40), gg.out_star(40), gg.empty(9),
            gg.rmat(15, 8, dangling=0.15, unref=0.10, seed=4),
            gg.er(500, 20.0, dangling=0.1, unref=0.0, seed=5),
            gg.random_small(300, 3.0, 0.2, 0.1, seed=6)]


@pytest.fixture(scope="module")
def graphs():
    gl = mixed_graphs()
    hs = [pr.Graph(g.n, g.m, *g.csr32()) for g in gl]
    truths = [oracle.power(g, C, gg.p_uniform(g.n), tol=1e-15)[0] for g in gl]
    yield gl, hs, truths
    for h in hs:
        h.close()


@pytest.mark.parametrize("algo", (pr.PR_IFP1, pr.PR_IFP2))
@pytest.mark.parametrize("prec", (pr.PR_DF64, pr.PR_FP64, pr.PR_FP32))
@pytest.mark.parametrize("mode", (pr.PR_MODE_AUTO, pr.PR_MODE_PUSH, pr.PR_MODE_PULL))
def test_batch_matches_single_solves(graphs, algo, prec, mode):
    gl, hs, truths = graphs
    eps = 1e-10 if prec != pr.PR_FP32 else 1e-7
    opts = dict(mode=mode)
    outs, sts, status = pr.pr_solve_batch(hs, C, eps, algo, prec, opts=opts)
    assert status == pr.PR_OK
    tol_single = 1e-12 if prec != pr.PR_FP32 else 1e-6
    for k, (g, h, truth) in enumerate(zip(gl, hs, truths)):
        alone, st1, s1 = h.solve(C, eps, algo, prec, opts=opts)
        assert s1 == pr.PR_OK
        assert l1(outs[k], alone) <= tol_single, (k, l1(outs[k], alone))
        assert abs(sts[k]["rounds"] - st1["rounds"]) <= 1, (k, sts[k]["rounds"], st1["rounds"])
        assert l1(outs[k], truth) <= sts[k]["err_bound"] + (1e-12 if prec != pr.PR_FP32 else 2e-6)
        assert abs(outs[k].sum() - 1.0) < 1e-12


def test_batch_device_outputs_and_per_problem_parameters(graphs):
    gl, hs, truths = graphs
    cs = [0.85 if k % 2 == 0 else 0.5 for k in range(len(gl))]
    es = [1e-10 if k % 3 else 1e-8 for k in range(len(gl))]
    outs = [torch.empty(g.n, dtype=torch.float64, device="cuda") for g in gl]
    _, sts, status = pr.pr_solve_batch(hs, cs, es, pr.PR_IFP2, pr.PR_DF64, outs=outs)
    torch.cuda.synchronize()
    assert status == pr.PR_OK
    for k, (g, h) in enumerate(zip(gl, hs)):
        alone, st1, _ = h.solve(cs[k], es[k], pr.PR_IFP2, pr.PR_DF64)
        assert l1(outs[k].cpu().numpy(), alone) <= 1e-12
        truth = oracle.power(g, cs[k], gg.p_uniform(g.n), tol=1e-15)[0]
        assert l1(outs[k].cpu().numpy(), truth) <= sts[k]["err_bound"] + 1e-12


def test_batch_invalid_arguments(graphs):
    gl, hs, truths = graphs
    with pytest.raises(pr.PrError) as e:
        pr.pr_solve_batch(hs[:2], 1.5, 1e-9, pr.PR_IFP2)
    assert e.value.status == pr.PR_EINVAL
    with pytest.raises(pr.PrError) as e:
        pr.pr_solve_batch(hs[:2], 0.85, 1e-9, pr.PR_POWER)
    assert e.value.status == pr.PR_EINVAL


def test_batch_round_cap(graphs):
    gl, hs, truths = graphs
    outs, sts, status = pr.pr_solve_batch(hs, C, 1e-14, pr.PR_IFP1, pr.PR_DF64, opts=dict(max_rounds=3), check=False)
    assert status == pr.PR_ENOTCONV
    assert all(s["rounds"] <= 3 for s in sts)
    assert all(abs(o.sum() - 1.0) < 1e-12 for o in outs)
