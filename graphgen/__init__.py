"""Seeded synthetic directed graphs and personalization vectors.

This module is the only code shared by the oracle tests and the CUDA-library
tests and benchmark.  It holds no PageRank arithmetic: it draws edges (R-MAT,
Erdos-Renyi, and a few fixed shapes with known PageRank), deletes the edges
that make a seeded set of vertices dangling or unreferenced, relabels
vertices, and returns compressed rows.  Out-lists (CSR) and in-lists (CSC)
are both sorted and free of duplicate edges, because the paper's adjacency
matrix is 0/1 (Sec. 2.1).

The statistics reported with each graph are the columns of the paper's
Table 1: n, m, n_d (dangling vertices), m_d (edges into dangling vertices)
and deg = m / n.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_SO = os.path.join(_HERE, "_graphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into a shared library next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        lib.gg_rmat.argtypes = [ctypes.c_int, i64, dbl, dbl, dbl, u64, P, P]
        lib.gg_er.argtypes = [i32, i64, u64, P, P]
        lib.gg_vertex_mask.argtypes = [i32, dbl, u64, u64, P]
        lib.gg_permutation.argtypes = [i32, u64, u64, P]
        lib.gg_relabel.argtypes = [i64, P, P, P]
        lib.gg_orient.argtypes = [i64, P, dbl, u64, P, P]
        lib.gg_filter.argtypes = [i64, P, P, P, P, ctypes.c_int]
        lib.gg_filter.restype = i64
        lib.gg_compress.argtypes = [i32, i64, P, P, P, P, P]
        lib.gg_compress.restype = i64
        lib.gg_transpose.argtypes = [i32, P, P, P, P]
        lib.gg_u01.argtypes = [u64, u64, u64]
        lib.gg_u01.restype = dbl
        lib.gg_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclasses.dataclass
class Graph:
    """A directed graph in compressed rows, vertex ids 0..n-1.

    out_off/out_dst: CSR (out-lists D(v), sorted); in_off/in_src: CSC (in-lists
    S(v), sorted).  Offsets are int64 here; the C ABI takes int32 offsets,
    which `csr32()` / `csc32()` provide.
    """
    n: int
    out_off: np.ndarray
    out_dst: np.ndarray
    in_off: np.ndarray
    in_src: np.ndarray
    name: str = ""
    recipe: dict = dataclasses.field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.out_off[-1])

    @property
    def outdeg(self) -> np.ndarray:
        return np.diff(self.out_off)

    @property
    def indeg(self) -> np.ndarray:
        return np.diff(self.in_off)

    def csr32(self):
        return self.out_off.astype(np.int32), self.out_dst

    def csc32(self):
        return self.in_off.astype(np.int32), self.in_src

    def stats(self) -> dict:
        """Table 1 columns (n, m, n_d, m_d, deg) plus unreferenced count n_u."""
        od, idg = self.outdeg, self.indeg
        dang = od == 0
        return {
            "n": self.n, "m": self.m,
            "n_d": int(dang.sum()),
            "m_d": int(idg[dang].sum()),
            "deg": (self.m / self.n) if self.n else 0.0,
            "n_u": int((idg == 0).sum()),
            "max_outdeg": int(od.max()) if self.n else 0,
            "max_indeg": int(idg.max()) if self.n else 0,
        }


def from_edges(n: int, src, dst, name: str = "edges", recipe: dict | None = None,
               drop_loops: bool = False) -> Graph:
    """Compressed rows from an edge list; repeated edges collapse to one."""
    L = _L()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = int(src.size)
    if drop_loops and m:
        src, dst = src.copy(), dst.copy()
        m = L.gg_filter(m, _p(src), _p(dst), None, None, 1)
        src, dst = src[:m], dst[:m]
    out_off = np.zeros(n + 1, np.int64)
    col = np.empty(max(m, 1), np.int32)
    tmp = np.empty(max(m, 1), np.int32)
    mm = L.gg_compress(n, m, _p(src), _p(dst), _p(out_off), _p(col), _p(tmp))
    out_dst = col[:mm].copy()
    del col, tmp
    in_off = np.zeros(n + 1, np.int64)
    in_src = np.empty(max(mm, 1), np.int32)
    L.gg_transpose(n, _p(out_off), _p(out_dst), _p(in_off), _p(in_src))
    return Graph(n, out_off, out_dst, in_off, in_src[:mm].copy(), name, dict(recipe or {}))


def _finish(n, src, dst, m, seed, dangling, unref, permute, name, recipe):
    """Delete out-edges of a seeded dangling set and in-edges of an independent
    unreferenced set, drop self-loops, optionally relabel, compress."""
    L = _L()
    drop_out = np.zeros(n, np.uint8)
    drop_in = np.zeros(n, np.uint8)
    if dangling > 0:
        L.gg_vertex_mask(n, dangling, seed, 1, _p(drop_out))
    if unref > 0:
        L.gg_vertex_mask(n, unref, seed, 2, _p(drop_in))
    m = L.gg_filter(m, _p(src), _p(dst), _p(drop_out), _p(drop_in), 1)
    src, dst = src[:m], dst[:m]
    if permute:
        perm = np.empty(n, np.int32)
        L.gg_permutation(n, seed, 2, _p(perm))
        L.gg_relabel(m, _p(perm), _p(src), _p(dst))
    return from_edges(n, src, dst, name=name, recipe=recipe)


def rmat(scale: int, edge_factor: float = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         dangling: float = 0.15, unref: float = 0.10, seed: int = 1, permute: bool = True,
         dag_frac: float | None = None, nverts: int | None = None, edges: int | None = None,
         undirected: bool = False) -> Graph:
    """Directed R-MAT graph on 2**scale vertices.

    `edge_factor * 2**scale` edges are sampled (or `edges` exactly); with
    `dag_frac` set, that share of edges is oriented forward in a seeded random
    order first; with `undirected`, every sampled edge is also taken reversed
    (a symmetric graph: no DAG structure before the deletions below).
    Self-loops and repeated edges are removed, then all out-edges
    of a seeded `dangling` share of vertices and all in-edges of an independent
    `unref` share are deleted, and the ids are randomly relabelled.  With
    `nverts` < 2**scale, vertices >= nverts and their edges are dropped.
    """
    L = _L()
    n = 1 << scale
    m = int(edges if edges is not None else round(edge_factor * n))
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    L.gg_rmat(scale, m, a, b, c, seed, _p(src), _p(dst))
    if dag_frac is not None:
        rank = np.empty(n, np.int32)
        L.gg_permutation(n, seed, 1, _p(rank))
        L.gg_orient(m, _p(rank), dag_frac, seed, _p(src), _p(dst))
    if nverts is not None and nverts < n:
        keep = (src < nverts) & (dst < nverts)
        src, dst = np.ascontiguousarray(src[keep]), np.ascontiguousarray(dst[keep])
        m, n = int(src.size), int(nverts)
    if undirected:
        src, dst = np.concatenate([src, dst]), np.concatenate([dst, src])
        m = int(src.size)
    recipe = dict(kind="rmat", scale=scale, edge_factor=edge_factor, abcd=(a, b, c, 1 - a - b - c),
                  dangling=dangling, unref=unref, seed=seed, permute=permute, dag_frac=dag_frac,
                  sampled_edges=int(m), nverts=n, undirected=bool(undirected))
    return _finish(n, src, dst, m, seed, dangling, unref, permute, f"rmat{scale}", recipe)


def er(n: int, avg_deg: float, dangling: float = 0.15, unref: float = 0.0, seed: int = 1,
       permute: bool = False) -> Graph:
    """Directed Erdos-Renyi G(n, m) with m = avg_deg * n sampled pairs."""
    L = _L()
    m = int(round(avg_deg * n))
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    L.gg_er(n, m, seed, _p(src), _p(dst))
    recipe = dict(kind="er", n=n, avg_deg=avg_deg, dangling=dangling, unref=unref, seed=seed)
    return _finish(n, src, dst, m, seed, dangling, unref, permute, f"er{n}", recipe)


# ---------------------------------------------------------------- fixed shapes
def cycle(n: int) -> Graph:
    """Directed cycle 0 -> 1 -> ... -> n-1 -> 0."""
    i = np.arange(n, dtype=np.int32)
    return from_edges(n, i, (i + 1) % n, name=f"cycle{n}")


def chain(n: int) -> Graph:
    """Directed path 0 -> 1 -> ... -> n-1 (vertex n-1 dangling, vertex 0 unreferenced)."""
    i = np.arange(n - 1, dtype=np.int32)
    return from_edges(n, i, i + 1, name=f"chain{n}")


def out_star(n: int) -> Graph:
    """Centre 0 with an edge to each of the n-1 leaves (the leaves are dangling)."""
    leaves = np.arange(1, n, dtype=np.int32)
    return from_edges(n, np.zeros(n - 1, np.int32), leaves, name=f"outstar{n}")


def in_star(n: int) -> Graph:
    """Each of the n-1 leaves has one edge to centre 0 (the centre is dangling)."""
    leaves = np.arange(1, n, dtype=np.int32)
    return from_edges(n, leaves, np.zeros(n - 1, np.int32), name=f"instar{n}")


def empty(n: int) -> Graph:
    return from_edges(n, np.zeros(0, np.int32), np.zeros(0, np.int32), name=f"empty{n}")


def random_small(n: int, avg_deg: float = 3.0, dangling: float = 0.2, unref: float = 0.1,
                 seed: int = 1, loops: bool = False) -> Graph:
    """Small random digraph for dense checks: ER pairs, optional self-loops kept."""
    L = _L()
    m = int(round(avg_deg * n))
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    L.gg_er(n, m, seed, _p(src), _p(dst))
    drop_out = np.zeros(n, np.uint8)
    drop_in = np.zeros(n, np.uint8)
    L.gg_vertex_mask(n, dangling, seed, 1, _p(drop_out))
    L.gg_vertex_mask(n, unref, seed, 2, _p(drop_in))
    m = L.gg_filter(m, _p(src), _p(dst), _p(drop_out), _p(drop_in), 0 if loops else 1)
    return from_edges(n, src[:m], dst[:m], name=f"small{n}s{seed}",
                      recipe=dict(kind="small", n=n, avg_deg=avg_deg, seed=seed, loops=loops))


# ------------------------------------------------------ personalization vectors
def p_uniform(n: int) -> np.ndarray:
    return np.full(n, 1.0 / n)


def p_seeds(n: int, k: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """k distinct seeded vertices with weight 1/k each (sparse form: idx, val)."""
    L = _L()
    idx = []
    seen = set()
    j = 0
    while len(idx) < k:
        v = int(L.gg_u01(seed, 500, j) * n)
        j += 1
        if v not in seen:
            seen.add(v)
            idx.append(v)
    idx = np.array(sorted(idx), np.int32)
    return idx, np.full(k, 1.0 / k)


def p_random(n: int, seed: int, zero_frac: float = 0.0) -> np.ndarray:
    """Dense random positive weights (a share zeroed), not normalised."""
    L = _L()
    u = np.array([L.gg_u01(seed, 600, i) for i in range(n)])
    z = np.array([L.gg_u01(seed, 601, i) < zero_frac for i in range(n)])
    u[z] = 0.0
    if u.sum() == 0:
        u[0] = 1.0
    return u


def dense_from_sparse(n: int, idx, val) -> np.ndarray:
    p = np.zeros(n)
    p[np.asarray(idx)] = np.asarray(val)
    return p


def num_threads() -> int:
    return int(_L().gg_num_threads())
