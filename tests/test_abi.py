"""Host-side checks of the C ABI: the library loads without a GPU, exports
every function include/pr.h declares, and rejects bad host input before
touching CUDA."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import graphgen as gg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def prlib():
    import paper_2302_03245_gb300 as pr
    pr.build()
    return pr


def declared_functions():
    text = open(os.path.join(ROOT, "include", "pr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(pr_[a-z_0-9]+)\s*\(", text)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pr_graph_create", "pr_solve", "pr_solve_ex", "pr_solve_batch", "pr_server_create",
                     "pr_server_submit", "pr_server_poll", "pr_server_destroy", "pr_graph_autotune",
                     "pr_destroy", "pr_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(prlib):
    lib = prlib.lib()
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", prlib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pr_\w+)", out))
    assert set(declared_functions()) <= exported


def test_header_compiles_as_c():
    src = "#include \"pr.h\"\nint main(void){pr_stats s; pr_opts o; pr_kernel_profile k; (void)s; (void)o; (void)k; return 0;}\n"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-x", "c",
                        "-", "-o", "/dev/null"], input=src, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_struct_layouts_match_binding(prlib):
    # offsets of the C structs as gcc lays them out, compared with ctypes
    src = r'''#include <stdio.h>
#include <stddef.h>
#include "pr.h"
int main(void){
 printf("%zu %zu %zu %zu %zu\n", sizeof(pr_stats), sizeof(pr_opts), sizeof(pr_graph_info), sizeof(pr_pvec), sizeof(pr_kernel_profile));
 printf("%zu %zu %zu\n", offsetof(pr_stats, ms), offsetof(pr_opts, trace_mode), offsetof(pr_graph_info, device_bytes));
 printf("%zu %zu %zu %zu\n", sizeof(pr_tuning), offsetof(pr_tuning, pull_ratio), offsetof(pr_tuning, bin_rows), offsetof(pr_tuning, pull_blocks));
 printf("%zu %zu %zu\n", sizeof(pr_server_stats), offsetof(pr_server_stats, groups), offsetof(pr_server_stats, ms_finish));
 printf("%zu %zu %zu\n", sizeof(pr_debug_report), offsetof(pr_debug_report, first_value), offsetof(pr_debug_report, max_identity_dev));
 return 0;}'''
    exe = os.path.join(ROOT, "tests", ".layout_probe")
    r = subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-x", "c", "-", "-o", exe], input=src,
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lines = subprocess.run([exe], capture_output=True, text=True).stdout.split("\n")
    os.remove(exe)
    sizes = list(map(int, lines[0].split()))
    offs = list(map(int, lines[1].split()))
    assert sizes == [ctypes.sizeof(prlib.pr_stats), ctypes.sizeof(prlib.pr_opts),
                     ctypes.sizeof(prlib.pr_graph_info), ctypes.sizeof(prlib.pr_pvec),
                     ctypes.sizeof(prlib.pr_kernel_profile)]
    assert offs == [prlib.pr_stats.ms.offset, prlib.pr_opts.trace_mode.offset,
                    prlib.pr_graph_info.device_bytes.offset]
    T = prlib.pr_tuning
    assert list(map(int, lines[2].split())) == [ctypes.sizeof(T), T.pull_ratio.offset, T.bin_rows.offset,
                                                T.pull_blocks.offset]
    S = prlib.pr_server_stats
    assert list(map(int, lines[3].split())) == [ctypes.sizeof(S), S.groups.offset, S.ms_finish.offset]
    D = prlib.pr_debug_report
    assert list(map(int, lines[4].split())) == [ctypes.sizeof(D), D.first_value.offset, D.max_identity_dev.offset]


@pytest.mark.parametrize("case", ["dup_free_but_bad_offsets", "range", "negative_n", "off0", "offn"])
def test_host_validation_without_gpu(prlib, case):
    g = gg.random_small(30, 3.0, 0.2, 0.1, seed=1)
    off, dst = [a.copy() for a in g.csr32()]
    n, m = g.n, g.m
    if case == "dup_free_but_bad_offsets":
        off[3], off[4] = off[4] + 1, off[3]
    elif case == "range":
        dst[-1] = n + 3
    elif case == "negative_n":
        n = 0
    elif case == "off0":
        off[0] = 1
    else:
        m = m + 1
    with pytest.raises(prlib.PrError) as e:
        prlib.pr_graph_create(n, m, off, dst)
    assert e.value.status == prlib.PR_EINVAL


def test_allocator_arguments_checked(prlib):
    lib = prlib.lib()
    st = lib.pr_set_allocator(prlib._ALLOC_FN(lambda a, b, c: None), prlib._FREE_FN(), None)
    assert st == prlib.PR_EINVAL
    assert lib.pr_set_allocator(prlib._ALLOC_FN(), prlib._FREE_FN(), None) == prlib.PR_OK


def test_output_arrays_checked_before_any_call(prlib):
    """Solve, batch and poll write n doubles into the caller's output: the
    binding refuses anything else before the library is called."""
    import numpy as np
    torch = pytest.importorskip("torch")
    on_device = prlib._on_device
    assert on_device(np.empty(5), 5) is False
    assert on_device(np.empty(8), 5) is False                      # longer is fine
    assert on_device(torch.empty(5, dtype=torch.float64), 5) is False
    with pytest.raises(TypeError):
        on_device(np.empty(5, np.float32), 5)
    with pytest.raises(TypeError):
        on_device(np.empty(10)[::2], 5)                             # not contiguous
    with pytest.raises(TypeError):
        on_device(torch.empty(5, dtype=torch.int64), 5)             # 8 bytes, not floating point
    with pytest.raises(TypeError):
        on_device(torch.empty(10, dtype=torch.float64)[::2], 5)
    with pytest.raises(ValueError):
        on_device(np.empty(4), 5)
    with pytest.raises(ValueError):
        on_device(torch.empty(4, dtype=torch.float64), 5)


def test_release_build_has_no_debug_checks(prlib):
    """libpr.so is the release build: the debug-build calls exist and refuse (no GPU needed)."""
    L = prlib.lib()
    if prlib.DEBUG:
        pytest.skip("PR_LIBRARY=debug loads the debug build")
    assert L.pr_is_debug_build() == 0
    assert L.pr_debug_inject(1) == prlib.PR_EINVAL
    rep = prlib.pr_debug_report()
    assert L.pr_debug_report_get(ctypes.byref(rep), 0) == prlib.PR_EINVAL
