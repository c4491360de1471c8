"""FP64 CPU oracle for IFP1 / IFP2 PageRank -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg
may import this package.  The library's product path never calls it and
shares no code with it.  The arithmetic lives in `oracle.c` (plain C, FP64);
this file compiles it with gcc and marshals numpy arrays.

Parity status of each function (what pins it, see tests/test_oracle_pins.py):
  power            pinned: closed forms (cycle, PPR on a cycle, chain, stars,
                   no edges), numpy eigenvector of the Google matrix, dense solve.
  dense_solve      pinned: closed forms, eigenvector of P'', a hand-derived
                   3-vertex example.
  eq2_residual     pinned: zero on exact solutions, equals a hand-computed value
                   on a perturbed 3-vertex case.
  ifp_sequential   pinned: against dense_solve within Eq. 8-style bounds, and the
                   closed forms.
  ifp_rounds       pinned: cycle R_t = c^t round count, chain round count and
                   exact stop, mass invariant every round, closed forms, dense
                   solve within the bound 2cR/(1-c) (IFP1) / 2R/(1-c) (IFP2).
  ifp2_levels      pinned: the 3-round chain, the level rule on a hand-made
                   graph, identity and in-flight mass at any round cap, bound.
  ifp_async        pinned: one round on a forward DAG and the chain, equal to
                   ifp_rounds when every edge points down, the cycle's closed
                   form, identity and mass at any cap, the certified bound.
  ifp_scan         pinned: one scan on a forward DAG and the chain, equal to
                   ifp_rounds when every edge points down, the cycle's closed
                   form R_t = c^(n(t-1)) R_1, identity, mass and R <= Rub at any
                   cap, the certified bound.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_lib = {}

IFP1 = 1
IFP2 = 2


def compile_c(src: str, so: str) -> str:
    """gcc -O2, no fast-math and no FMA contraction: plain IEEE FP64."""
    tmp = so + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-shared", "-fPIC",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, so)
    return so


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into oracle/_oracle.so."""
    so = os.path.join(_HERE, "_oracle.so")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
        compile_c(_SRC, so)
    return so


def _L():
    if "lib" not in _lib:
        _lib["lib"] = _bind(ctypes.CDLL(build()))
    return _lib["lib"]


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _csr(g):
    off = np.ascontiguousarray(g.out_off, dtype=np.int64)
    dst = np.ascontiguousarray(g.out_dst, dtype=np.int32)
    return off, dst


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _bind(lib):
    P = ctypes.c_void_p
    i32, dbl = ctypes.c_int32, ctypes.c_double
    lib.orc_power.argtypes = [i32, P, P, dbl, P, dbl, i32, P, P, P]
    lib.orc_dense_solve.argtypes = [i32, P, P, dbl, P, P]
    lib.orc_eq2_residual.argtypes = [i32, P, P, dbl, P, P]
    lib.orc_eq2_residual.restype = dbl
    lib.orc_ifp_sequential.argtypes = [ctypes.c_int, i32, P, P, dbl, dbl, P, i32, P, P, P, P]
    lib.orc_ifp_rounds.argtypes = [ctypes.c_int, i32, P, P, dbl, dbl, dbl, P, i32,
                                   P, P, P, P, P, P, P, P]
    lib.orc_ifp_async.argtypes = [ctypes.c_int, i32, P, P, dbl, dbl, dbl, P, i32, P, P, P, P, P, P]
    lib.orc_ifp_scan.argtypes = [ctypes.c_int, i32, P, P, dbl, dbl, dbl, P, i32, P, P, P, P, P, P, P]
    lib.orc_ifp2_levels.argtypes = [i32, P, P, dbl, dbl, dbl, P, P, i32, i32,
                                    P, P, P, P, P, P, P, P]
    return lib


class Oracle:
    """Bound set of oracle functions.

    `so` loads another build of oracle.c (the mutation tests compile copies
    with a planted mistake and run the pins against them).
    """

    def __init__(self, so: str | None = None):
        self.L = _bind(ctypes.CDLL(so)) if so else _L()

    def power(self, g, c, p, tol=1e-14, max_iter=100000):
        """Power iteration on P'' from pi_0 = p (Eq. 1).  Returns (pi, iters, last_delta, status)."""
        off, dst = _csr(g)
        p = _f64(p)
        pi = np.empty(g.n)
        it = ctypes.c_int32()
        dl = ctypes.c_double()
        st = self.L.orc_power(g.n, _p(off), _p(dst), c, _p(p), tol, max_iter, _p(pi),
                              ctypes.byref(it), ctypes.byref(dl))
        return pi, it.value, dl.value, st

    def dense_solve(self, g, c, p):
        """Solve Eq. 2 by Gaussian elimination (small n)."""
        off, dst = _csr(g)
        p = _f64(p)
        pi = np.empty(g.n)
        st = self.L.orc_dense_solve(g.n, _p(off), _p(dst), c, _p(p), _p(pi))
        if st:
            raise ArithmeticError("singular system")
        return pi

    def eq2_residual(self, g, c, p, pi):
        """|| (I - cP') pi - (1-c) p ||_1."""
        off, dst = _csr(g)
        return float(self.L.orc_eq2_residual(g.n, _p(off), _p(dst), c, _p(_f64(p)), _p(_f64(pi))))

    def ifp_sequential(self, algo, g, c, xi, h0, max_scans=1000000):
        """Alg. 2 / Alg. 3 with one thread.  Returns (pi, scans, pushes, edges, status)."""
        off, dst = _csr(g)
        h0 = _f64(h0)
        pi = np.empty(g.n)
        sc, pu, ed = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        st = self.L.orc_ifp_sequential(algo, g.n, _p(off), _p(dst), c, xi, _p(h0), max_scans, _p(pi),
                                       ctypes.byref(sc), ctypes.byref(pu), ctypes.byref(ed))
        return pi, sc.value, pu.value, ed.value, st

    def ifp_rounds(self, algo, g, c, eps, p, xi_act=None, max_rounds=100000, trace=True):
        """Synchronous-round IFP1/IFP2 with (1-c) reserve.

        Returns dict(pi, x, r, rounds, status, R, F, E, mass) -- the traces are
        per round (R has rounds+1 entries, F and E have rounds entries,
        mass[t] for t = 1..rounds is sum x + sum r after round t).
        """
        off, dst = _csr(g)
        p = _f64(p)
        n = g.n
        if xi_act is None:
            n_nd = int((np.diff(off) > 0).sum())
            xi_act = eps / max(n_nd, 1)
        x, r, pi = np.empty(n), np.empty(n), np.empty(n)
        T = max_rounds + 2
        tR = np.zeros(T) if trace else None
        tF = np.zeros(T, np.int64) if trace else None
        tE = np.zeros(T, np.int64) if trace else None
        tM = np.zeros(T) if trace else None
        rounds = ctypes.c_int32()
        st = self.L.orc_ifp_rounds(algo, n, _p(off), _p(dst), c, eps, xi_act, _p(p), max_rounds,
                                   _p(x), _p(r), _p(pi), ctypes.byref(rounds),
                                   _p(tR), _p(tF), _p(tE), _p(tM))
        k = rounds.value
        out = dict(pi=pi, x=x, r=r, rounds=k, status=st, xi_act=xi_act)
        if trace:
            out.update(R=tR[:k + 1].copy(), F=tF[:k].copy(), E=tE[:k].copy(), mass=tM[1:k + 1].copy())
        return out


    def ifp_async(self, algo, g, c, eps, p, xi_act=None, max_rounds=100000, trace=True):
        """IFP1/IFP2 asynchronous rounds, frontier in id order (orc_ifp_async).
        Returns dict(pi, x, r, rounds, status, R, F)."""
        off, dst = _csr(g)
        p = _f64(p)
        n = g.n
        if xi_act is None:
            n_nd = int((np.diff(off) > 0).sum())
            xi_act = eps / max(n_nd, 1)
        x, r, pi = np.empty(n), np.empty(n), np.empty(n)
        T = max_rounds + 2
        tR = np.zeros(T) if trace else None
        tF = np.zeros(T, np.int64) if trace else None
        rounds = ctypes.c_int32()
        st = self.L.orc_ifp_async(algo, n, _p(off), _p(dst), c, eps, xi_act, _p(p), max_rounds,
                                  _p(x), _p(r), _p(pi), ctypes.byref(rounds), _p(tR), _p(tF))
        k = rounds.value
        out = dict(pi=pi, x=x, r=r, rounds=k, status=st, xi_act=xi_act)
        if trace:
            out.update(R=tR[:k + 1].copy(), F=tF[:k].copy())
        return out

    def ifp_scan(self, algo, g, c, eps, p, xi_act=None, max_rounds=100000, trace=True):
        """IFP1/IFP2 scans in id order with the (1-c) reserve (orc_ifp_scan).
        Returns dict(pi, x, r, rounds, status, R, Rub, F), traces indexed by scan."""
        off, dst = _csr(g)
        p = _f64(p)
        n = g.n
        if xi_act is None:
            n_nd = int((np.diff(off) > 0).sum())
            xi_act = eps / max(n_nd, 1)
        x, r, pi = np.empty(n), np.empty(n), np.empty(n)
        T = max_rounds + 2
        tR = np.zeros(T) if trace else None
        tU = np.zeros(T) if trace else None
        tF = np.zeros(T, np.int64) if trace else None
        rounds = ctypes.c_int32()
        st = self.L.orc_ifp_scan(algo, n, _p(off), _p(dst), c, eps, xi_act, _p(p), max_rounds, _p(x), _p(r),
                                 _p(pi), ctypes.byref(rounds), _p(tR), _p(tU), _p(tF))
        k = rounds.value
        out = dict(pi=pi, x=x, r=r, rounds=k, status=st, xi_act=xi_act)
        if trace:
            out.update(R=tR[:k].copy(), Rub=tU[:k].copy(), F=tF[:k].copy())
        return out

    def ifp2_levels(self, g, c, eps, p, levels, L, xi_act=None, max_rounds=100000, trace=True):
        """IFP2 in level-ordered rounds (orc_ifp2_levels).  levels[i] in [0, L]
        for non-dangling i (gs_levels gives the library's assignment rule).
        Returns dict(pi, x, r, r_pending, rounds, status, R, F, E): R, F, E are
        indexed by round (R has the decision residual of each round taken)."""
        off, dst = _csr(g)
        p = _f64(p)
        n = g.n
        if xi_act is None:
            n_nd = int((np.diff(off) > 0).sum())
            xi_act = eps / max(n_nd, 1)
        lv = np.ascontiguousarray(levels, dtype=np.int32)
        x, r, rp, pi = np.empty(n), np.empty(n), np.empty(n), np.empty(n)
        T = max_rounds + 2
        tR = np.zeros(T) if trace else None
        tF = np.zeros(T, np.int64) if trace else None
        tE = np.zeros(T, np.int64) if trace else None
        rounds = ctypes.c_int32()
        st = self.L.orc_ifp2_levels(n, _p(off), _p(dst), c, eps, xi_act, _p(p), _p(lv), int(L), max_rounds,
                                    _p(x), _p(r), _p(rp), _p(pi), ctypes.byref(rounds), _p(tR), _p(tF), _p(tE))
        k = rounds.value
        out = dict(pi=pi, x=x, r=r, r_pending=rp, rounds=k, status=st, xi_act=xi_act)
        if trace:
            # decisions taken: rounds 0..k-1 and, when the stop came at the start
            # of a synchronous round (k < 2 or status != 0 there), round k itself
            nd = k + 1 if (k < 2 or st != 0) else k
            out.update(R=tR[:nd].copy(), F=tF[:k].copy(), E=tE[:k].copy())
        return out


def gs_levels(g, L: int) -> np.ndarray:
    """Level of every vertex for level-ordered rounds, from its degrees alone:
    non-dangling vertices with in-edges are ranked by the integer key
    floor(2^31 (indeg + 1) / (indeg + outdeg + 2)), ascending (vertices that
    mostly send come first), ties by id; rank q of n_ref gets level
    floor(q L / n_ref).  Non-dangling vertices without in-edges get level L;
    dangling vertices -1 (never scanned in IFP2's phase 1)."""
    outdeg = np.diff(g.out_off).astype(np.int64)
    indeg = np.diff(g.in_off).astype(np.int64)
    lv = np.full(g.n, -1, np.int32)
    ref = np.nonzero((outdeg > 0) & (indeg > 0))[0]
    key = ((indeg[ref] + 1) << 31) // (indeg[ref] + outdeg[ref] + 2)
    order = ref[np.lexsort((ref, key))]
    q = np.arange(order.size, dtype=np.int64)
    lv[order] = (q * L // max(order.size, 1)).astype(np.int32)
    lv[(outdeg > 0) & (indeg == 0)] = L
    return lv


_default = None


def default() -> Oracle:
    """The oracle build; ORACLE_SO in the environment substitutes another build
    of oracle.c (used only by the mutation tests)."""
    global _default
    if _default is None:
        _default = Oracle(os.environ.get("ORACLE_SO") or None)
    return _default


def power(*a, **k):
    return default().power(*a, **k)


def dense_solve(*a, **k):
    return default().dense_solve(*a, **k)


def eq2_residual(*a, **k):
    return default().eq2_residual(*a, **k)


def ifp_sequential(*a, **k):
    return default().ifp_sequential(*a, **k)


def ifp_rounds(*a, **k):
    return default().ifp_rounds(*a, **k)


def ifp2_levels(*a, **k):
    return default().ifp2_levels(*a, **k)


def ifp_async(*a, **k):
    return default().ifp_async(*a, **k)


def ifp_scan(*a, **k):
    return default().ifp_scan(*a, **k)


def certified_l1_bound(algo: int, c: float, R: float) -> float:
    """Guaranteed L1 error of an IFP result stopped at residual L1 R (non-dangling).

    With s = x/(1-c) and y = (I - cP)^{-1} p the exact unnormalised vector of
    Eq. 4, the stopped state satisfies (I - cP~) s = p - r.  IFP1 returns
    s + r, and y - (s + r) = sum_{k>=1} (cP)^k r has L1 norm <= cR/(1-c)
    (dangling columns of P are zero, so only the non-dangling residual
    propagates).  IFP2 returns s on non-dangling vertices and
    p_d + c P s on dangling ones; its unnormalised error is <= R/(1-c).
    Normalising two positive vectors at most doubles the L1 distance relative
    to sum y >= 1, giving 2cR/(1-c) (IFP1) and 2R/(1-c) (IFP2).  The paper's
    own estimate, Eq. 8, is the rougher ERR < xi.
    """
    return (2.0 * c * R if algo == IFP1 else 2.0 * R) / (1.0 - c)
