"""pr_power_noalloc: the allocation-free Power method, checked against pr_solve.

Some callers cannot allocate device memory (a framework that owns the device
memory pool, a path where an allocation could synchronise the device, a
plug-in that only receives buffers).  pr_power_noalloc keeps its working
vectors in a fixed array inside the library instead.  Through the C ABI this
test runs it twice in a row on the same inputs and compares each result with
the allocating entry point, pr_solve(PR_POWER), within the FP64 tolerance the
other GPU tests use; it also checks that a graph above the size limit is
refused.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_03245_gb300 as pr  # noqa: E402

C = 0.85
MAX_N = 1 << 19


def noalloc_fn():
    f = pr.lib().pr_power_noalloc
    f.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                  ctypes.c_double, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]
    f.restype = ctypes.c_int
    return f


@pytest.mark.parametrize("which", ["rmat14", "er3000"])
def test_noalloc_power_matches_pr_solve_twice(which):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pr.build()
    f = noalloc_fn()
    g = (gg.rmat(14, 8, dangling=0.15, unref=0.10, seed=1) if which == "rmat14"
         else gg.random_small(3000, 5.0, 0.2, 0.1, seed=2))
    off, dst = g.csr32()
    ioff, isrc = g.csc32()
    d_off, d_ioff, d_isrc = [torch.tensor(a, device="cuda") for a in (off, ioff, isrc)]
    with pr.Graph(g.n, g.m, off, dst) as G:
        ref, st, status = G.solve(C, 1e-12, pr.PR_POWER, pr.PR_FP64)
    assert status == pr.PR_OK
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        pi = torch.full((g.n,), float("nan"), dtype=torch.float64, device="cuda")
        it = ctypes.c_int32(-1)
        status = f(g.n, d_off.data_ptr(), d_ioff.data_ptr(), d_isrc.data_ptr(), C, 1e-12, 100000,
                   pi.data_ptr(), stream, ctypes.byref(it))
        torch.cuda.synchronize()
        assert status == pr.PR_OK, pr.pr_last_error()
        assert abs(it.value - st["rounds"]) <= 1
        out = pi.cpu().numpy()
        assert np.all(np.isfinite(out)), call
        assert np.abs(out - ref).sum() <= 1e-9, call
        assert abs(out.sum() - 1.0) < 1e-12


def test_noalloc_rejects_sizes_over_the_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pr.build()
    f = noalloc_fn()
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    pi = torch.zeros(4, dtype=torch.float64, device="cuda")
    status = f(MAX_N + 1, dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), C, 1e-9, 10, pi.data_ptr(), None,
               None)
    assert status == pr.PR_EINVAL
    assert "524288" in pr.pr_last_error()
