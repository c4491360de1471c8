"""The seeded generators of `graphgen`, data-parallel in PyTorch (any device).

Every function here produces exactly the graph its namesake in `graphgen`
produces from the same arguments: the random draws are the same
counter-based hash (SplitMix64 finaliser) evaluated on int64 tensors, the
permutation is the same sort by keys, and the compressed rows are sorted and
free of repeated edges in the same way.  On a GPU this makes graphs of
hundreds of millions of edges in well under a second, so benchmarks can build
their inputs on the device.  Like `graphgen`, it holds no PageRank arithmetic.
"""
from __future__ import annotations

import dataclasses

import torch

_M64 = (1 << 64) - 1


def _s64(v: int) -> int:
    """A 64-bit pattern as the signed int64 torch stores."""
    v &= _M64
    return v - (1 << 64) if v >> 63 else v


def _lsr(z: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (z >> k) & ((1 << (64 - k)) - 1)


_G = _s64(0x9E3779B97F4A7C15)
_C1 = _s64(0xBF58476D1CE4E5B9)
_C2 = _s64(0x94D049BB133111EB)


def _mix64(z: torch.Tensor) -> torch.Tensor:
    z = z + _G
    z = (z ^ _lsr(z, 30)) * _C1
    z = (z ^ _lsr(z, 27)) * _C2
    return z ^ _lsr(z, 31)


def _mix64_int(z: int) -> int:
    z = (z + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def draw(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """64-bit draws for (seed, stream, idx) as int64 bit patterns."""
    base = _s64(_mix64_int((seed * 0x2545F4914F6CDD1D + stream) & _M64))
    return _mix64(idx.to(torch.int64) ^ base)


def draw_u01(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return _lsr(draw(seed, stream, idx), 11).to(torch.float64) * (1.0 / 9007199254740992.0)


CHUNK = 1 << 25  # edges drawn per pass (bounds the int64 temporaries)


def _chunks(m: int, device):
    step = CHUNK
    for lo in range(0, m, step):
        yield lo, torch.arange(lo, min(m, lo + step), device=device, dtype=torch.int64)


def rmat_edges(scale: int, m: int, a: float, b: float, c: float, seed: int, device):
    ta = int(a * 65536.0 + 0.5)
    tb = int((a + b) * 65536.0 + 0.5)
    tc = int((a + b + c) * 65536.0 + 0.5)
    src = torch.empty(m, dtype=torch.int32, device=device)
    dst = torch.empty(m, dtype=torch.int32, device=device)
    for lo, e in _chunks(m, device):
        s = torch.zeros_like(e)
        d = torch.zeros_like(e)
        bits = None
        for lv in range(scale):
            if lv % 4 == 0:
                bits = draw(seed, 1 + lv // 4, e)
            u = bits & 0xFFFF
            bits = _lsr(bits, 16)
            sb = (u >= tb).to(torch.int64)
            db = ((u >= ta) & (u < tb) | (u >= tc)).to(torch.int64)
            s = (s << 1) | sb
            d = (d << 1) | db
        src[lo:lo + e.numel()] = s.to(torch.int32)
        dst[lo:lo + e.numel()] = d.to(torch.int32)
    return src, dst


def er_edges(n: int, m: int, seed: int, device):
    src = torch.empty(m, dtype=torch.int32, device=device)
    dst = torch.empty(m, dtype=torch.int32, device=device)
    for lo, e in _chunks(m, device):
        h = draw(seed, 100, e)
        src[lo:lo + e.numel()] = (((h & 0xFFFFFFFF) * n) >> 32).to(torch.int32)
        dst[lo:lo + e.numel()] = ((_lsr(h, 32) * n) >> 32).to(torch.int32)
    return src, dst


def vertex_mask(n: int, frac: float, seed: int, stream: int, device) -> torch.Tensor:
    return draw_u01(seed, 200 + stream, torch.arange(n, device=device)) < frac


def permutation(n: int, seed: int, stream: int, device) -> torch.Tensor:
    """perm[i] = rank of vertex i's key (the sort definition of graphgen)."""
    keys = _lsr(draw(seed, 300 + stream, torch.arange(n, device=device)), 1)
    order = torch.sort(keys, stable=True).indices
    perm = torch.empty(n, dtype=torch.int32, device=device)
    perm[order] = torch.arange(n, device=device, dtype=torch.int32)
    return perm


def orient(src, dst, rank, frac: float, seed: int):
    m = src.numel()
    for lo, e in _chunks(m, src.device):
        hi = lo + e.numel()
        s, d = src[lo:hi], dst[lo:hi]
        flip = (draw_u01(seed, 400, e) < frac) & (rank[s.long()] > rank[d.long()])
        s2 = torch.where(flip, d, s)
        d2 = torch.where(flip, s, d)
        src[lo:hi], dst[lo:hi] = s2, d2
    return src, dst


@dataclasses.dataclass
class TGraph:
    """Compressed rows on a torch device: the counterpart of graphgen.Graph."""
    n: int
    out_off: torch.Tensor  # int64 [n+1]
    out_dst: torch.Tensor  # int32 [m]
    in_off: torch.Tensor
    in_src: torch.Tensor
    name: str = ""
    recipe: dict = dataclasses.field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.out_off[-1])

    def csr32(self):
        return self.out_off.to(torch.int32), self.out_dst

    def csc32(self):
        return self.in_off.to(torch.int32), self.in_src

    def stats(self) -> dict:
        od = self.out_off.diff()
        idg = self.in_off.diff()
        dang = od == 0
        return {"n": self.n, "m": self.m, "n_d": int(dang.sum()), "m_d": int(idg[dang].sum()),
                "deg": self.m / self.n if self.n else 0.0, "n_u": int((idg == 0).sum()),
                "max_outdeg": int(od.max()) if self.n else 0, "max_indeg": int(idg.max()) if self.n else 0}

    def to_host(self):
        import graphgen
        return graphgen.Graph(self.n, self.out_off.cpu().numpy(), self.out_dst.cpu().numpy(),
                              self.in_off.cpu().numpy(), self.in_src.cpu().numpy(), self.name, dict(self.recipe))


def _rows(n: int, key: torch.Tensor, val: torch.Tensor):
    """Rows grouped by key, sorted by val inside, repeated pairs dropped."""
    k = torch.unique(key.to(torch.int64) * n + val.to(torch.int64))  # sorted
    rk = (k // n).to(torch.int64)
    col = (k % n).to(torch.int32)
    off = torch.zeros(n + 1, dtype=torch.int64, device=key.device)
    off[1:] = torch.cumsum(torch.bincount(rk, minlength=n), 0)
    return off, col, rk


def from_edges(n: int, src, dst, name="edges", recipe=None) -> TGraph:
    out_off, out_dst, rows = _rows(n, src, dst)
    in_off, in_src, _ = _rows(n, out_dst, rows)
    return TGraph(n, out_off, out_dst, in_off, in_src, name, dict(recipe or {}))


def _finish(n, src, dst, seed, dangling, unref, permute, name, recipe):
    dev = src.device
    keep = src != dst
    if dangling > 0:
        keep &= ~vertex_mask(n, dangling, seed, 1, dev)[src.long()]
    if unref > 0:
        keep &= ~vertex_mask(n, unref, seed, 2, dev)[dst.long()]
    src, dst = src[keep], dst[keep]
    if permute:
        perm = permutation(n, seed, 2, dev)
        src, dst = perm[src.long()], perm[dst.long()]
    return from_edges(n, src, dst, name=name, recipe=recipe)


def rmat(scale: int, edge_factor: float = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         dangling: float = 0.15, unref: float = 0.10, seed: int = 1, permute: bool = True,
         dag_frac: float | None = None, nverts: int | None = None, edges: int | None = None,
         undirected: bool = False, device="cuda") -> TGraph:
    """graphgen.rmat on a torch device (same arguments, same graph)."""
    n = 1 << scale
    m = int(edges if edges is not None else round(edge_factor * n))
    src, dst = rmat_edges(scale, m, a, b, c, seed, device)
    if dag_frac is not None:
        rank = permutation(n, seed, 1, device)
        src, dst = orient(src, dst, rank, dag_frac, seed)
    if nverts is not None and nverts < n:
        keep = (src < nverts) & (dst < nverts)
        src, dst = src[keep], dst[keep]
        m, n = int(src.numel()), int(nverts)
    if undirected:
        src, dst = torch.cat([src, dst]), torch.cat([dst, src])
        m = int(src.numel())
    recipe = dict(kind="rmat", scale=scale, edge_factor=edge_factor, abcd=(a, b, c, 1 - a - b - c),
                  dangling=dangling, unref=unref, seed=seed, permute=permute, dag_frac=dag_frac,
                  sampled_edges=int(m), nverts=n, undirected=bool(undirected))
    return _finish(n, src, dst, seed, dangling, unref, permute, f"rmat{scale}", recipe)


def er(n: int, avg_deg: float, dangling: float = 0.15, unref: float = 0.0, seed: int = 1,
       permute: bool = False, device="cuda") -> TGraph:
    """graphgen.er on a torch device."""
    m = int(round(avg_deg * n))
    src, dst = er_edges(n, m, seed, device)
    recipe = dict(kind="er", n=n, avg_deg=avg_deg, dangling=dangling, unref=unref, seed=seed)
    return _finish(n, src, dst, seed, dangling, unref, permute, f"er{n}", recipe)
