"""Python binding of the GB300 IFP1 / IFP2 PageRank library (libpr.so).

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels.  The functions carry the C ABI's names (include/pr.h).  Host arrays
are numpy arrays; device arrays are torch CUDA tensors (their data_ptr() is
passed through).  PyTorch is used for device memory (optionally as the
library's allocator) and streams.

There is no CPU fallback: if libpr.so is missing or cannot be loaded the
functions raise, and a CUDA-less machine can only inspect the library.
With PR_LIBRARY=debug in the environment at first use, the debug build
libpr_debug.so (index and invariant checks, see include/pr.h) is loaded
instead.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEBUG = os.environ.get("PR_LIBRARY", "") == "debug"
LIB_PATH = os.path.join(HERE, "libpr_debug.so" if DEBUG else "libpr.so")

PR_OK, PR_EINVAL, PR_ENOMEM, PR_ECUDA, PR_ENOTCONV, PR_ETIMEOUT, PR_EAGAIN, PR_EBUSY, PR_ECHECK = range(9)
PR_POWER, PR_IFP1, PR_IFP2 = 0, 1, 2
PR_FP64, PR_FP32, PR_DF64 = 0, 1, 2
PR_MODE_AUTO, PR_MODE_PUSH, PR_MODE_PULL, PR_MODE_LEVELS, PR_MODE_ASYNC, PR_MODE_APULL = 0, 1, 2, 3, 4, 5
STATUS_NAMES = ["PR_OK", "PR_EINVAL", "PR_ENOMEM", "PR_ECUDA", "PR_ENOTCONV", "PR_ETIMEOUT", "PR_EAGAIN",
                "PR_EBUSY", "PR_ECHECK"]


class PrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class pr_pvec(ctypes.Structure):
    _fields_ = [("nnz", ctypes.c_int32), ("idx", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("is_device", ctypes.c_int32)]


class pr_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("rounds_push", ctypes.c_int32), ("rounds_pull", ctypes.c_int32),
                ("fp64_rounds", ctypes.c_int32), ("pushes", ctypes.c_int64), ("edges_pushed", ctypes.c_int64),
                ("edges_scanned", ctypes.c_int64), ("resid_l1", ctypes.c_double),
                ("dangling_mass", ctypes.c_double), ("err_bound", ctypes.c_double), ("ms", ctypes.c_double),
                ("p_scale", ctypes.c_double), ("launches", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


PR_K_ACTIVATE, PR_K_COMMIT, PR_K_PUSH, PR_K_PULL, PR_K_POWER, PR_K_OTHER, PR_K_LEVELS = range(7)
PR_K_KINDS = 8
KERNEL_NAMES = {PR_K_ACTIVATE: "k_activate", PR_K_COMMIT: "k_commit", PR_K_PUSH: "k_push",
                PR_K_PULL: "k_round_pull", PR_K_POWER: "k_sweep<OP_POWER>", PR_K_OTHER: "other",
                PR_K_LEVELS: "k_round_levels"}


class pr_kernel_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int32 * PR_K_KINDS), ("ms", ctypes.c_double * PR_K_KINDS)]

    def as_dict(self) -> dict:
        return {KERNEL_NAMES[k]: dict(launches=self.launches[k], ms=self.ms[k])
                for k in KERNEL_NAMES if self.launches[k]}


class pr_opts(ctypes.Structure):
    _fields_ = [("xi_act", ctypes.c_double), ("max_rounds", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("pull_ratio", ctypes.c_double), ("use_graph", ctypes.c_int32), ("trace_cap", ctypes.c_int32),
                ("trace_R", ctypes.c_void_p), ("trace_F", ctypes.c_void_p), ("trace_E", ctypes.c_void_p),
                ("trace_mode", ctypes.c_void_p), ("profile", ctypes.POINTER(pr_kernel_profile))]


class pr_graph_opts(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("reserved", ctypes.c_int32 * 7)]


class pr_graph_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_nd", ctypes.c_int32), ("n_ref", ctypes.c_int32),
                ("n_d", ctypes.c_int32), ("n_u", ctypes.c_int32), ("m", ctypes.c_int64), ("m_d", ctypes.c_int64),
                ("max_outdeg", ctypes.c_int32), ("max_indeg", ctypes.c_int32), ("ms_preprocess", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("levels", ctypes.c_int32), ("pad0", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class pr_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("finished", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("group_launches", ctypes.c_int64), ("tile_launches", ctypes.c_int64), ("groups", ctypes.c_int32),
                ("active", ctypes.c_int32), ("ms_admit", ctypes.c_double), ("ms_rounds", ctypes.c_double),
                ("ms_correct", ctypes.c_double), ("ms_finish", ctypes.c_double), ("queued_sum", ctypes.c_int64),
                ("running_sum", ctypes.c_int64), ("ms_tables", ctypes.c_double), ("ms_step_max", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class pr_tuning(ctypes.Structure):
    _fields_ = [("pull_thr", ctypes.c_int32 * 6), ("block_budget", ctypes.c_int32), ("pad0", ctypes.c_int32),
                ("pull_ratio", ctypes.c_double), ("bin_rows", ctypes.c_int32 * 7), ("pull_blocks", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {"pull_thr": list(self.pull_thr), "block_budget": self.block_budget, "pull_ratio": self.pull_ratio,
                "bin_rows": list(self.bin_rows), "pull_blocks": self.pull_blocks}


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


class pr_debug_report(ctypes.Structure):
    _fields_ = [("checks", ctypes.c_int64), ("fails", ctypes.c_int64), ("first_site", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("first_value", ctypes.c_int64), ("first_bound", ctypes.c_int64),
                ("max_mass_dev", ctypes.c_double), ("max_identity_dev", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force, debug=DEBUG)


def lib() -> ctypes.CDLL:
    """The loaded libpr.so; raises if it is not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2302_03245_gb300.build() first")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.pr_graph_create.argtypes = [i32, i64, P, P, P, P, ctypes.c_int, P, ctypes.POINTER(P)]
        L.pr_graph_create.restype = ctypes.c_int
        L.pr_graph_create_ex.argtypes = [i32, i64, P, P, P, P, ctypes.c_int, P, ctypes.POINTER(pr_graph_opts),
                                         ctypes.POINTER(P)]
        L.pr_graph_create_ex.restype = ctypes.c_int
        L.pr_graph_get_info.argtypes = [P, ctypes.POINTER(pr_graph_info)]
        L.pr_graph_get_info.restype = ctypes.c_int
        L.pr_graph_get_tuning.argtypes = [P, ctypes.POINTER(pr_tuning)]
        L.pr_graph_get_tuning.restype = ctypes.c_int
        L.pr_graph_set_tuning.argtypes = [P, ctypes.POINTER(pr_tuning)]
        L.pr_graph_set_tuning.restype = ctypes.c_int
        L.pr_graph_autotune.argtypes = [P, ctypes.c_int, dbl, ctypes.POINTER(pr_tuning), ctypes.c_char_p,
                                        ctypes.c_size_t]
        L.pr_graph_autotune.restype = ctypes.c_int
        L.pr_solve.argtypes = [P, dbl, dbl, ctypes.c_int, ctypes.c_int, ctypes.POINTER(pr_pvec), P, ctypes.c_int,
                               ctypes.POINTER(pr_stats)]
        L.pr_solve.restype = ctypes.c_int
        L.pr_solve_ex.argtypes = [P, dbl, dbl, ctypes.c_int, ctypes.c_int, ctypes.POINTER(pr_pvec),
                                  ctypes.POINTER(pr_opts), P, ctypes.c_int, ctypes.POINTER(pr_stats)]
        L.pr_solve_ex.restype = ctypes.c_int
        L.pr_solve_batch.argtypes = [ctypes.POINTER(P), i32, ctypes.POINTER(dbl), ctypes.POINTER(dbl), ctypes.c_int,
                                     ctypes.c_int, ctypes.POINTER(pr_pvec), ctypes.POINTER(pr_opts),
                                     ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(pr_stats)]
        L.pr_solve_batch.restype = ctypes.c_int
        L.pr_destroy.argtypes = [P]
        L.pr_destroy.restype = None
        L.pr_server_create.argtypes = [ctypes.c_size_t, P, ctypes.POINTER(P)]
        L.pr_server_create.restype = ctypes.c_int
        L.pr_server_submit.argtypes = [P, P, dbl, dbl, ctypes.c_int, ctypes.POINTER(pr_pvec), ctypes.POINTER(i64)]
        L.pr_server_submit.restype = ctypes.c_int
        L.pr_server_poll.argtypes = [P, i64, P, ctypes.POINTER(pr_stats)]
        L.pr_server_poll.restype = ctypes.c_int
        L.pr_server_destroy.argtypes = [P]
        L.pr_server_destroy.restype = None
        L.pr_server_get_stats.argtypes = [P, ctypes.POINTER(pr_server_stats)]
        L.pr_server_get_stats.restype = ctypes.c_int
        L.pr_last_error.restype = ctypes.c_char_p
        L.pr_version.restype = ctypes.c_char_p
        L.pr_set_allocator.argtypes = [_ALLOC_FN, _FREE_FN, P]
        L.pr_set_allocator.restype = ctypes.c_int
        L.pr_is_debug_build.restype = ctypes.c_int
        L.pr_debug_report_get.argtypes = [ctypes.POINTER(pr_debug_report), ctypes.c_int]
        L.pr_debug_report_get.restype = ctypes.c_int
        L.pr_debug_inject.argtypes = [i32]
        L.pr_debug_inject.restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status: int):
    if status != PR_OK:
        raise PrError(status, lib().pr_last_error().decode(errors="replace"))


def _ptr(a) -> int | None:
    """Address of a numpy array (host) or torch tensor (device or host)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _on_device(a, n: int | None = None) -> bool:
    """Whether an output array is device memory: True for a CUDA tensor, False
    for a numpy array or a host torch tensor (pinned or not).  The library
    writes n doubles there, so the array must be contiguous float64 with at
    least n elements."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("output arrays must be contiguous float64")
        size, dev = a.size, False
    else:
        if a.element_size() != 8 or not a.is_floating_point() or not a.is_contiguous():
            raise TypeError("output tensors must be contiguous float64")
        size, dev = a.numel(), bool(a.is_cuda)
    if n is not None and size < n:
        raise ValueError(f"output holds {size} values; the graph has {n} vertices")
    return dev


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def pr_last_error() -> str:
    return lib().pr_last_error().decode(errors="replace")


def pr_version() -> str:
    return lib().pr_version().decode()


def pr_graph_create(n: int, m: int, out_off, out_dst, in_off=None, in_src=None, mem_is_device: bool = False,
                    stream=None, levels: int = 0) -> ctypes.c_void_p:
    """Wraps pr_graph_create_ex.  Arrays are int32 numpy (host) or torch (device);
    levels > 0 prepares level-ordered rounds (PR_MODE_LEVELS)."""
    for a in (out_off, out_dst, in_off, in_src):
        if isinstance(a, np.ndarray) and (a.dtype != np.int32 or not a.flags.c_contiguous):
            raise TypeError("graph arrays must be contiguous int32")
    g = ctypes.c_void_p()
    o = pr_graph_opts()
    o.levels = int(levels)
    _check(lib().pr_graph_create_ex(int(n), int(m), _ptr(out_off), _ptr(out_dst), _ptr(in_off), _ptr(in_src),
                                    1 if mem_is_device else 0, _stream_handle(stream), ctypes.byref(o),
                                    ctypes.byref(g)))
    return g


def pr_graph_get_info(g) -> dict:
    info = pr_graph_info()
    _check(lib().pr_graph_get_info(g, ctypes.byref(info)))
    return info.as_dict()


def pr_graph_get_tuning(g) -> dict:
    t = pr_tuning()
    _check(lib().pr_graph_get_tuning(g, ctypes.byref(t)))
    return t.as_dict()


def pr_graph_set_tuning(g, pull_thr=None, block_budget=None, pull_ratio=0.0) -> dict:
    """Wraps pr_graph_set_tuning; unspecified fields keep the graph's values."""
    t = pr_tuning()
    _check(lib().pr_graph_get_tuning(g, ctypes.byref(t)))
    if pull_thr is not None:
        for k, v in enumerate(pull_thr):
            t.pull_thr[k] = int(v)
    if block_budget is not None:
        t.block_budget = int(block_budget)
    t.pull_ratio = float(pull_ratio)
    _check(lib().pr_graph_set_tuning(g, ctypes.byref(t)))
    return pr_graph_get_tuning(g)


def pr_graph_autotune(g, prec: int = PR_DF64, max_ms: float = 0.0) -> tuple[dict, str]:
    """Wraps pr_graph_autotune.  Returns (chosen tuning, trial report)."""
    t = pr_tuning()
    buf = ctypes.create_string_buffer(16384)
    _check(lib().pr_graph_autotune(g, int(prec), float(max_ms), ctypes.byref(t), buf, len(buf)))
    return t.as_dict(), buf.value.decode(errors="replace")


def graph_signature(info: dict) -> str:
    """Key of a tuning cache entry: the graph facts the launch parameters depend on."""
    return "n{n}_m{m}_nd{n_nd}_ref{n_ref}_md{m_d}_maxin{max_indeg}_maxout{max_outdeg}".format(**info)


def autotune_cached(g, cache_path: str, prec: int = PR_DF64, max_ms: float = 0.0) -> tuple[dict, str]:
    """Autotune g, or apply the tuning stored for a graph with the same signature
    (and the same GPU) in the JSON file cache_path; new results are added to it."""
    import json
    info = pr_graph_get_info(g)
    try:
        import torch
        dev = torch.cuda.get_device_name()
    except Exception:
        dev = "unknown"
    key = f"{dev}|{prec}|{graph_signature(info)}"
    try:
        with open(cache_path) as f:
            cache = json.load(f)
    except (OSError, ValueError):
        cache = {}
    if key in cache:
        e = cache[key]
        return pr_graph_set_tuning(g, e["pull_thr"], e["block_budget"], e["pull_ratio"]), "from cache"
    t, rep = pr_graph_autotune(g, prec, max_ms)
    cache[key] = {k: t[k] for k in ("pull_thr", "block_budget", "pull_ratio")}
    tmp = cache_path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, cache_path)
    return t, rep


def pr_destroy(g) -> None:
    if g is not None and g.value:
        lib().pr_destroy(g)
        g.value = None


def make_pvec(n: int, p=None, idx=None, is_device: bool = False):
    """pr_pvec for: None (uniform), a dense vector of length n, or (idx, val) sparse."""
    v = pr_pvec()
    keep = []
    if p is None and idx is None:
        v.nnz = -1
        return v, keep
    if idx is None:
        val = p if is_device else np.ascontiguousarray(p, dtype=np.float64)
        v.nnz, v.idx, v.val = n, None, _ptr(val)
        keep.append(val)
    else:
        ii = idx if is_device else np.ascontiguousarray(idx, dtype=np.int32)
        vv = p if is_device else np.ascontiguousarray(p, dtype=np.float64)
        v.nnz, v.idx, v.val = len(ii), _ptr(ii), _ptr(vv)
        keep += [ii, vv]
    v.is_device = 1 if is_device else 0
    return v, keep


def pr_solve(g, c: float, eps: float, algo: int, prec: int = PR_FP64, p=None, p_idx=None, out=None,
             p_is_device: bool = False, opts: dict | None = None, check: bool = True):
    """Wraps pr_solve_ex.  Returns (out, stats dict, status).

    out: None (a new host numpy array), a numpy float64 array, or a contiguous
    float64 torch tensor: a CUDA tensor is device output, a CPU (e.g. pinned)
    tensor host output.  opts: pr_opts fields by name; with
    trace_cap > 0 the per-round traces are returned in stats["trace"].
    """
    info = pr_graph_get_info(g)
    n = info["n"]
    pv, keep = make_pvec(n, p, p_idx, p_is_device)
    if out is None:
        out = np.empty(n, dtype=np.float64)
    out_dev = _on_device(out, n)
    st = pr_stats()
    o = pr_opts()
    trace = None
    prof = None
    if opts:
        for k, v in opts.items():
            if k in ("trace_cap", "profile"):
                continue
            setattr(o, k, v)
        if opts.get("profile"):
            prof = pr_kernel_profile()
            o.profile = ctypes.pointer(prof)
        cap = int(opts.get("trace_cap", 0))
        if cap > 0:
            trace = dict(R=np.zeros(cap), F=np.zeros(cap, np.int64), E=np.zeros(cap, np.int64),
                         mode=np.zeros(cap, np.int8))
            o.trace_cap = cap
            o.trace_R, o.trace_F = trace["R"].ctypes.data, trace["F"].ctypes.data
            o.trace_E, o.trace_mode = trace["E"].ctypes.data, trace["mode"].ctypes.data
    status = lib().pr_solve_ex(g, float(c), float(eps), int(algo), int(prec), ctypes.byref(pv), ctypes.byref(o),
                               _ptr(out), 1 if out_dev else 0, ctypes.byref(st))
    if check and status not in (PR_OK, PR_ENOTCONV):
        _check(status)
    d = st.as_dict()
    if trace is not None:
        d["trace"] = trace
    if prof is not None:
        d["profile"] = prof.as_dict()
    return out, d, status


def pr_solve_batch(graphs, c, eps, algo, prec=PR_DF64, outs=None, opts: dict | None = None, check: bool = True):
    """Wraps pr_solve_batch.  graphs: list of handles (or Graph objects); c, eps:
    scalars or per-graph sequences; outs: None (new host arrays), a list of numpy
    float64 arrays, or a list of float64 torch tensors, all on the device or all
    on the host.  Returns
    (outs, list of stats dicts, status)."""
    hs = [g.h if isinstance(g, Graph) else g for g in graphs]
    k = len(hs)
    ns = [pr_graph_get_info(h)["n"] for h in hs]
    cs = (ctypes.c_double * k)(*([float(c)] * k if np.isscalar(c) else [float(v) for v in c]))
    es = (ctypes.c_double * k)(*([float(eps)] * k if np.isscalar(eps) else [float(v) for v in eps]))
    if outs is None:
        outs = [np.empty(n, dtype=np.float64) for n in ns]
    dev = _on_device(outs[0], ns[0])
    if any(_on_device(o, n) != dev for o, n in zip(outs, ns)):
        raise TypeError("outs must all be device arrays or all host arrays")
    optr = (ctypes.c_void_p * k)(*[_ptr(o) for o in outs])
    harr = (ctypes.c_void_p * k)(*[h.value for h in hs])
    sts = (pr_stats * k)()
    o = pr_opts()
    for key, v in (opts or {}).items():
        setattr(o, key, v)
    status = lib().pr_solve_batch(harr, k, cs, es, int(algo), int(prec), None, ctypes.byref(o), optr,
                                  1 if dev else 0, sts)
    if check and status not in (PR_OK, PR_ENOTCONV):
        _check(status)
    return outs, [s.as_dict() for s in sts], status


# ------------------------------------------------------------------ serving
def pr_server_create(hbm_budget_bytes: int, stream=None) -> ctypes.c_void_p:
    """Wraps pr_server_create (current device; stream: torch stream, raw handle or None)."""
    s = ctypes.c_void_p()
    _check(lib().pr_server_create(int(hbm_budget_bytes), _stream_handle(stream), ctypes.byref(s)))
    return s


# vertex count of each ticket's graph, recorded at submit: pr_server_poll writes that
# many values, so the output is checked against it (not against a caller's number)
_TICKET_N: dict = {}


def pr_server_submit(server, g, c: float, eps: float, prec: int = PR_DF64, p=None, p_idx=None) -> int:
    """Wraps pr_server_submit; p/p_idx as in pr_solve (host only).  Returns the ticket."""
    n = pr_graph_get_info(g)["n"]
    pv, keep = make_pvec(n, p, p_idx, False)
    t = ctypes.c_int64()
    _check(lib().pr_server_submit(server, g, float(c), float(eps), int(prec), ctypes.byref(pv), ctypes.byref(t)))
    _TICKET_N[(server.value, t.value)] = n
    return t.value


def pr_server_poll(server, ticket: int, n: int | None = None, out=None):
    """Wraps pr_server_poll.  Returns None while the request runs (PR_EBUSY), else
    (out, stats dict, status) with status PR_OK or PR_ENOTCONV; raises on errors.
    The result has one value per vertex of the request's graph, recorded when the
    ticket was submitted through this binding; n, if given, must equal it.
    out: None (a new host array), a float64 numpy array, or a float64 torch tensor
    (host or CUDA) of at least that many values."""
    key = (server.value, int(ticket))
    if key not in _TICKET_N:
        raise ValueError(f"ticket {ticket} was not submitted to this server through this binding")
    n_req = _TICKET_N[key]
    if n is not None and int(n) != n_req:
        raise ValueError(f"ticket {ticket} is a request on a graph of {n_req} vertices, not {n}")
    if out is None:
        out = np.empty(n_req, dtype=np.float64)
    _on_device(out, n_req)  # the result is copied in: float64, contiguous, n_req values
    st = pr_stats()
    status = lib().pr_server_poll(server, int(ticket), _ptr(out), ctypes.byref(st))
    if status == PR_EBUSY:
        return None
    _TICKET_N.pop(key, None)
    if status not in (PR_OK, PR_ENOTCONV):
        _check(status)
    return out, st.as_dict(), status


def pr_server_get_stats(server) -> dict:
    st = pr_server_stats()
    _check(lib().pr_server_get_stats(server, ctypes.byref(st)))
    return st.as_dict()


def pr_server_destroy(server) -> None:
    if server is not None and server.value:
        for key in [k for k in _TICKET_N if k[0] == server.value]:
            del _TICKET_N[key]
        lib().pr_server_destroy(server)
        server.value = None


class Server:
    """RAII wrapper of a pr_server with a blocking wait()."""

    def __init__(self, hbm_budget_bytes: int, stream=None):
        self.h = pr_server_create(hbm_budget_bytes, stream)
        self._n = {}

    def submit(self, g, c, eps, prec=PR_DF64, p=None, p_idx=None) -> int:
        h = g.h if isinstance(g, Graph) else g
        t = pr_server_submit(self.h, h, c, eps, prec, p, p_idx)
        self._n[t] = _TICKET_N[(self.h.value, t)]
        return t

    def poll(self, ticket, out=None):
        r = pr_server_poll(self.h, ticket, None, out)
        if r is not None:
            self._n.pop(ticket, None)
        return r

    def wait(self, ticket, timeout_s: float = 120.0, sleep_s: float = 0.0005, out=None):
        import time
        t0 = time.monotonic()
        while True:
            r = self.poll(ticket, out)
            if r is not None:
                return r
            if time.monotonic() - t0 > timeout_s:
                raise TimeoutError(f"request {ticket} not finished after {timeout_s} s")
            time.sleep(sleep_s)

    def stats(self) -> dict:
        return pr_server_get_stats(self.h)

    def close(self):
        pr_server_destroy(self.h)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ------------------------------------------------------------ debug build
def pr_is_debug_build() -> bool:
    return bool(lib().pr_is_debug_build())


def pr_debug_report_get(reset: bool = False) -> dict:
    """The debug build's check report (raises PrError in a release build)."""
    r = pr_debug_report()
    _check(lib().pr_debug_report_get(ctypes.byref(r), 1 if reset else 0))
    return r.as_dict()


def pr_debug_inject(site: int) -> None:
    """Test hook of the debug build: the checks at `site` fail from the next solve on (0 = none)."""
    _check(lib().pr_debug_inject(int(site)))


# ------------------------------------------------------- torch allocator hook
_hooks = None


def use_torch_allocator(enable: bool = True) -> None:
    """Route the library's device allocations through torch's caching allocator."""
    global _hooks
    L = lib()
    if not enable:
        _check(L.pr_set_allocator(_ALLOC_FN(), _FREE_FN(), None))
        _hooks = None
        return
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)
        except Exception:
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    _hooks = (_ALLOC_FN(_alloc), _FREE_FN(_free))
    _check(L.pr_set_allocator(_hooks[0], _hooks[1], None))


class Graph:
    """RAII wrapper: pr_graph_create on construction, pr_destroy on close."""

    def __init__(self, n, m, out_off, out_dst, in_off=None, in_src=None, mem_is_device=False, stream=None,
                 levels=0):
        self.h = pr_graph_create(n, m, out_off, out_dst, in_off, in_src, mem_is_device, stream, levels)
        self.info = pr_graph_get_info(self.h)

    def solve(self, c, eps, algo, prec=PR_FP64, **kw):
        return pr_solve(self.h, c, eps, algo, prec, **kw)

    def tuning(self) -> dict:
        return pr_graph_get_tuning(self.h)

    def set_tuning(self, **kw) -> dict:
        return pr_graph_set_tuning(self.h, **kw)

    def autotune(self, prec=PR_DF64, max_ms=0.0, cache_path=None):
        if cache_path:
            return autotune_cached(self.h, cache_path, prec, max_ms)
        return pr_graph_autotune(self.h, prec, max_ms)

    def close(self):
        pr_destroy(self.h)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
