"""Failures made on the host: an allocator that refuses after a number of
allocations (fault injection through the pr_set_allocator hook).  Every call
must return PR_ENOMEM with a message, leave nothing half-built, and the same
graph must solve correctly once allocations succeed again.  No kernel is made
to fault."""
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


class FailingAllocator:
    """Device allocations through torch's caching allocator; the allocation
    after the first `budget` returns NULL."""

    def __init__(self, budget):
        self.budget = budget
        self.count = 0
        self.live = 0

        def _alloc(nbytes, stream, ctx):
            self.count += 1
            if self.count > self.budget:
                return None
            self.live += 1
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)

        def _free(ptr, nbytes, stream, ctx):
            self.live -= 1
            torch.cuda.caching_allocator_delete(ptr)

        self.fns = (pr._ALLOC_FN(_alloc), pr._FREE_FN(_free))

    def __enter__(self):
        pr._check(pr.lib().pr_set_allocator(self.fns[0], self.fns[1], None))
        return self

    def __exit__(self, *a):
        pr._check(pr.lib().pr_set_allocator(pr._ALLOC_FN(), pr._FREE_FN(), None))


def l1(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).sum())


@pytest.fixture(scope="module")
def graph():
    g = gg.rmat(12, 8, dangling=0.2, unref=0.1, seed=41)
    return g, oracle.power(g, 0.85, gg.p_uniform(g.n), tol=1e-15)[0]


@pytest.mark.parametrize("budget", [0, 1, 2, 5, 9, 14, 20, 30])
def test_graph_create_and_solve_under_allocation_failure(graph, budget):
    g, truth = graph
    off, dst = g.csr32()
    created = None
    with FailingAllocator(budget) as fa:
        h = ctypes.c_void_p()
        st = pr.lib().pr_graph_create(g.n, g.m, off.ctypes.data, dst.ctypes.data, None, None, 0, None,
                                      ctypes.byref(h))
        if st != pr.PR_OK:
            assert st == pr.PR_ENOMEM, pr.pr_last_error()
            assert pr.pr_last_error()
            assert fa.live == 0  # everything it had allocated was released
        else:
            created = h
            for prec in (pr.PR_DF64, pr.PR_FP32, pr.PR_FP64):
                out, sts, s = pr.pr_solve(created, 0.85, 1e-10, pr.PR_IFP2, prec, check=False)
                assert s in (pr.PR_OK, pr.PR_ENOMEM), (s, pr.pr_last_error())
                if s == pr.PR_OK:
                    assert l1(out, truth) <= sts["err_bound"] + (2e-6 if prec == pr.PR_FP32 else 1e-12)
    if created is not None:
        # allocations work again: the same graph solves, in every precision
        for prec in (pr.PR_DF64, pr.PR_FP32, pr.PR_FP64):
            out, sts, s = pr.pr_solve(created, 0.85, 1e-10, pr.PR_IFP2, prec)
            assert s == pr.PR_OK
            assert l1(out, truth) <= sts["err_bound"] + 1e-12
        pr.pr_destroy(created)


def test_batch_under_allocation_failure(graph):
    g, truth = graph
    hs = [pr.Graph(g.n, g.m, *g.csr32()) for _ in range(3)]
    try:
        with FailingAllocator(0):
            with pytest.raises(pr.PrError) as e:
                pr.pr_solve_batch(hs, 0.85, 1e-10, pr.PR_IFP2, pr.PR_DF64)
            assert e.value.status == pr.PR_ENOMEM
        outs, sts, s = pr.pr_solve_batch(hs, 0.85, 1e-10, pr.PR_IFP2, pr.PR_DF64)
        assert s == pr.PR_OK
        for o, st in zip(outs, sts):
            assert l1(o, truth) <= st["err_bound"] + 1e-12
    finally:
        for h in hs:
            h.close()
