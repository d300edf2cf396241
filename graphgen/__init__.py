"""Seeded synthetic graph generators shared by the oracle tests and the GPU path.

This module produces *inputs only*: symmetric CSR graphs (int64 row offsets,
uint32 column ids stored in int32 tensors, optional float32 edge weights).  It
contains none of the compression method's arithmetic -- no Philox, no
sampling thresholds, no triangle logic -- so the CPU oracle and the CUDA
library can both consume its output without sharing any method code.

Every random quantity is a pure function of (seed, stream, counter) computed
with a 32-bit integer mixer on int64 tensors, so a graph is bit-identical
whether it is generated on the CPU or on a CUDA device.  All multiplier
constants are below 2**31, so no intermediate product overflows int64.

Generators:
  * ``rmat``      -- R-MAT (Chakrabarti, Zhan, Faloutsos 2004) recursive-quadrant
                     edges, self-loops dropped, vertex ids permuted by a seeded
                     bijection, symmetrised and deduplicated.
  * ``chung_lu``  -- power-law expected-degree graph (Chung & Lu 2002): i.i.d.
                     endpoint pairs drawn proportionally to integer weights.
  * ``rgg3d``     -- 3-D random geometric graph on the unit torus, integer
                     coordinates so the distance test is exact.
  * ``attach_weights`` -- edge weights k * 2**-24, k uniform in {1..2**24},
                     keyed by the canonical endpoint pair so both arcs agree.
  * small fixtures (complete graphs, cycles, stars, bowtie, diamond, G(n, q)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

M32 = 0xFFFFFFFF

# stream identifiers keep the draws of different generator stages independent
_S_RMAT = 0x0152A7
_S_PERM = 0x0BE3A1
_S_CL_A = 0x0C1A01
_S_CL_B = 0x0C1A02
_S_RGG = 0x0466D3
_S_WGT = 0x0E1647


@dataclass
class CSR:
    """Symmetric CSR: rows sorted ascending, no self-loops, no duplicates."""

    n: int
    off: torch.Tensor  # int64 [n+1]
    col: torch.Tensor  # int32 [nnz] holding uint32 ids (< 2**31 here)
    w: Optional[torch.Tensor] = None  # float32 [nnz] or None

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    @property
    def m(self) -> int:
        return self.nnz // 2

    def to(self, device) -> "CSR":
        return CSR(self.n, self.off.to(device), self.col.to(device),
                   None if self.w is None else self.w.to(device))

    def numpy(self):
        return (self.off.cpu().numpy(), self.col.cpu().numpy().view(np.uint32),
                None if self.w is None else self.w.cpu().numpy())


# ---------------------------------------------------------------------------
# counter-based integer mixing (device agnostic)
# ---------------------------------------------------------------------------

def _mix32(x: torch.Tensor) -> torch.Tensor:
    """A 32-bit avalanche mixer on int64 tensors whose values lie in [0, 2**32)."""
    x = x ^ (x >> 16)
    x = (x * 0x7FEB352D) & M32
    x = x ^ (x >> 15)
    x = (x * 0x68E31DA5) & M32
    x = x ^ (x >> 16)
    x = (x * 0x2C1B3C6D) & M32
    x = x ^ (x >> 12)
    return x


def draw32(seed, stream: int, ctr: torch.Tensor, sub: int = 0) -> torch.Tensor:
    """Uniform 32-bit values (int64 tensor) for counters ``ctr`` (int64, >= 0).
    ``seed`` is an int or an int64 tensor broadcastable against ``ctr``."""
    if isinstance(seed, torch.Tensor):
        s = _mix32(((seed & M32) ^ ((seed >> 32) * 0x5851F42D)) & M32)
    else:
        s = _mix32(torch.full((), ((seed & M32) ^ (seed >> 32) * 0x5851F42D) & M32,
                              dtype=torch.int64, device=ctr.device))
    s = _mix32((s + stream) & M32)
    h = _mix32((s + (ctr & M32)) & M32)
    h = _mix32((h + ((ctr >> 32) & M32) + 0x3C6EF372) & M32)
    return _mix32((h + sub * 0x1B873593) & M32)


# ---------------------------------------------------------------------------
# CSR assembly
# ---------------------------------------------------------------------------

def csr_from_edges(n: int, src: torch.Tensor, dst: torch.Tensor) -> CSR:
    """Symmetrise, drop self-loops and duplicates, and build a sorted CSR."""
    keep = src != dst
    src, dst = src[keep], dst[keep]
    keys = torch.cat([src * n + dst, dst * n + src])
    del src, dst
    keys = torch.unique(keys)  # sorted
    rows = keys // n
    col = (keys - rows * n).to(torch.int32)
    del keys
    cnt = torch.bincount(rows, minlength=n)
    del rows
    off = torch.zeros(n + 1, dtype=torch.int64, device=col.device)
    off[1:] = torch.cumsum(cnt, 0)
    return CSR(n, off, col)


def _permutation(n: int, seed: int, device) -> torch.Tensor:
    """A seeded bijection of [0, n): ids ordered by a hash, ties by id."""
    v = torch.arange(n, dtype=torch.int64, device=device)
    h = draw32(seed, _S_PERM, v)
    order = torch.argsort(h * n + v)  # unique keys -> deterministic everywhere
    perm = torch.empty_like(order)
    perm[order] = v
    return perm


# ---------------------------------------------------------------------------
# R-MAT
# ---------------------------------------------------------------------------

def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 1, device="cpu", permute: bool = True,
         chunk: int = 1 << 26) -> CSR:
    """R-MAT graph with n = 2**scale and edge_factor * n generated edges."""
    n = 1 << scale
    total = edge_factor * n
    ta = int(math.floor(a * 2**32))
    tab = int(math.floor((a + b) * 2**32))
    tabc = int(math.floor((a + b + c) * 2**32))
    srcs, dsts = [], []
    for start in range(0, total, chunk):
        i = torch.arange(start, min(total, start + chunk), dtype=torch.int64, device=device)
        s = torch.zeros_like(i)
        d = torch.zeros_like(i)
        for lvl in range(scale):
            r = draw32(seed, _S_RMAT, i, lvl)
            sb = (r >= tab).to(torch.int64)                 # quadrants c, d: lower half
            db = ((r >= ta) & (r < tab)) | (r >= tabc)     # quadrants b, d: right half
            s = s * 2 + sb
            d = d * 2 + db.to(torch.int64)
        srcs.append(s)
        dsts.append(d)
    src = torch.cat(srcs)
    dst = torch.cat(dsts)
    del srcs, dsts
    if permute:
        perm = _permutation(n, seed, device)
        src, dst = perm[src], perm[dst]
    return csr_from_edges(n, src, dst)


def rmat_batch(scales, efs, seeds, a: float = 0.57, b: float = 0.19, c: float = 0.19, device="cpu"):
    """Many R-MAT graphs at once, as one disjoint union CSR.

    Graph i equals rmat(scales[i], efs[i], seed=seeds[i]) exactly; its vertices
    occupy [vbase[i], vbase[i] + 2**scales[i]) of the union.  Returns
    (union CSR, vbase, abase) with abase[i] = offset of graph i's first arc."""
    G = len(scales)
    sc = torch.tensor(scales, dtype=torch.int64, device=device)
    ef = torch.tensor(efs, dtype=torch.int64, device=device)
    sd = torch.tensor(seeds, dtype=torch.int64, device=device)
    nv = torch.ones_like(sc) << sc
    vbase = torch.zeros(G, dtype=torch.int64, device=device)
    vbase[1:] = torch.cumsum(nv, 0)[:-1]
    n_total = int(nv.sum().item())
    counts = ef * nv
    gi = torch.repeat_interleave(torch.arange(G, device=device), counts)
    start = torch.cumsum(counts, 0) - counts
    ei = torch.arange(gi.numel(), dtype=torch.int64, device=device) - start[gi]
    ta = int(math.floor(a * 2**32))
    tab = int(math.floor((a + b) * 2**32))
    tabc = int(math.floor((a + b + c) * 2**32))
    es, eg, ek = sc[gi], sd[gi], ei
    src = torch.zeros_like(ei)
    dst = torch.zeros_like(ei)
    for lvl in range(int(sc.max().item())):
        live = lvl < es
        r = draw32(eg, _S_RMAT, ek, lvl)
        sb = (r >= tab).to(torch.int64)
        db = (((r >= ta) & (r < tab)) | (r >= tabc)).to(torch.int64)
        src = torch.where(live, src * 2 + sb, src)
        dst = torch.where(live, dst * 2 + db, dst)
    # per-graph seeded permutation: rank of (hash, id) inside each graph
    vg = torch.repeat_interleave(torch.arange(G, device=device), nv)
    vl = torch.arange(n_total, dtype=torch.int64, device=device) - vbase[vg]
    h = draw32(sd[vg], _S_PERM, vl)
    if int(sc.max().item()) > 20:
        raise ValueError("rmat_batch supports scales up to 20")
    # lexicographic (graph, hash, id) by two stable sorts (the packed key would overflow)
    o1 = torch.argsort(h * (1 << 20) + vl, stable=True)
    order = o1[torch.argsort(vg[o1], stable=True)]
    perm = torch.empty_like(order)
    perm[order] = torch.arange(n_total, dtype=torch.int64, device=device)
    # perm maps union id -> union position; positions within a graph are contiguous
    src = perm[vbase[gi] + src]
    dst = perm[vbase[gi] + dst]
    g = csr_from_edges(n_total, src, dst)
    abase = g.off[vbase]
    return g, vbase.cpu().tolist(), abase.cpu().tolist()


def batch_member(union: CSR, vbase, i: int, n_i: int) -> CSR:
    """Graph i of a disjoint union as a standalone CSR (local ids)."""
    lo, hi = vbase[i], vbase[i] + n_i
    off = union.off[lo:hi + 1] - union.off[lo]
    col = union.col[int(union.off[lo]):int(union.off[hi])] - lo
    return CSR(n_i, off.clone(), col.clone(), None)


# ---------------------------------------------------------------------------
# Chung-Lu
# ---------------------------------------------------------------------------

def chung_lu(log2n: int, gamma: float = 2.1, mean_degree: float = 32.0, seed: int = 1,
             device="cpu", i0: float = 10.0, weight_bits: int = 20) -> CSR:
    """Chung-Lu power-law graph: mean_degree/2 * n endpoint pairs drawn i.i.d. with
    P(v) proportional to w_v, w_v ~ (v + i0)^(-1/(gamma-1)) scaled to the mean degree
    and capped at sqrt(sum w).  Integer cumulative weights keep the draw exact."""
    n = 1 << log2n
    wv = np.power(np.arange(n, dtype=np.float64) + i0, -1.0 / (gamma - 1.0))
    wv *= mean_degree * n / wv.sum()
    wv = np.minimum(wv, math.sqrt(wv.sum()))
    wq = np.maximum(1, np.round(wv * (1 << weight_bits) / wv.max() * 1.0).astype(np.int64))
    cum = torch.from_numpy(np.cumsum(wq)).to(device)
    total_w = int(cum[-1].item())
    pairs = int(mean_degree * n // 2)
    srcs, dsts = [], []
    chunk = 1 << 26
    for start in range(0, pairs, chunk):
        i = torch.arange(start, min(pairs, start + chunk), dtype=torch.int64, device=device)
        ends = []
        for stream in (_S_CL_A, _S_CL_B):
            hi = draw32(seed, stream, i, 0)
            lo = draw32(seed, stream, i, 1)
            r = ((hi << 31) | (lo >> 1)) % total_w
            ends.append(torch.searchsorted(cum, r, right=True))
        srcs.append(ends[0])
        dsts.append(ends[1])
    src = torch.cat(srcs)
    dst = torch.cat(dsts)
    perm = _permutation(n, seed, device)
    return csr_from_edges(n, perm[src], perm[dst])


# ---------------------------------------------------------------------------
# 3-D random geometric graph
# ---------------------------------------------------------------------------

def rgg3d(log2n: int, mean_degree: float = 48.0, seed: int = 1, device="cpu",
          coord_bits: int = 20, chunk_points: int = 1 << 20) -> CSR:
    """n points with integer coordinates in [0, 2**coord_bits)^3 on a torus; an edge
    joins points at (integer) squared distance < R2, where n * 4/3 pi r^3 = mean_degree."""
    n = 1 << log2n
    L = 1 << coord_bits
    r = (mean_degree * 3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    R = r * L
    R2 = int(math.floor(R * R))
    G = max(3, int(L // math.ceil(R)))  # cells per dimension, side >= R
    side = -(-L // G)
    v = torch.arange(n, dtype=torch.int64, device=device)
    xyz = torch.stack([draw32(seed, _S_RGG, v, k) >> (32 - coord_bits) for k in range(3)], 1)
    cell3 = xyz // side
    cell = (cell3[:, 0] * G + cell3[:, 1]) * G + cell3[:, 2]
    order = torch.argsort(cell * n + v)
    cell_sorted = cell[order]
    starts = torch.searchsorted(cell_sorted, torch.arange(G**3 + 1, device=device))
    srcs, dsts = [], []
    offsets = [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)]
    for p0 in range(0, n, chunk_points):
        pts = torch.arange(p0, min(n, p0 + chunk_points), dtype=torch.int64, device=device)
        c3 = cell3[pts]
        for dx, dy, dz in offsets:
            nc = ((c3[:, 0] + dx) % G * G + (c3[:, 1] + dy) % G) * G + (c3[:, 2] + dz) % G
            lo, hi = starts[nc], starts[nc + 1]
            cnt = hi - lo
            rep = torch.repeat_interleave(torch.arange(pts.numel(), device=device), cnt)
            base = torch.repeat_interleave(lo - torch.cumsum(cnt, 0) + cnt, cnt)
            idx = base + torch.arange(rep.numel(), device=device)
            q = order[idx]
            p = pts[rep]
            dd = (xyz[p] - xyz[q]).abs()
            dd = torch.minimum(dd, L - dd)
            d2 = (dd * dd).sum(1)
            ok = (d2 < R2) & (p < q)
            srcs.append(p[ok])
            dsts.append(q[ok])
    src = torch.cat(srcs)
    dst = torch.cat(dsts)
    return csr_from_edges(n, src, dst)


# ---------------------------------------------------------------------------
# edge weights
# ---------------------------------------------------------------------------

def attach_weights(g: CSR, seed: int = 1) -> CSR:
    """Weights k * 2**-24 with k uniform in {1..2**24}, keyed by the canonical
    endpoint pair, so both arcs of an edge carry the same value and sums are exact."""
    dev = g.col.device
    rows = torch.repeat_interleave(torch.arange(g.n, dtype=torch.int32 if g.n < 2**31 else torch.int64, device=dev),
                                   g.off[1:] - g.off[:-1])
    w = torch.empty(g.nnz, dtype=torch.float32, device=dev)
    chunk = 1 << 27  # bounds the int64 temporaries on very large graphs
    for s0 in range(0, g.nnz, chunk):
        r = rows[s0:s0 + chunk].to(torch.int64)
        c = g.col[s0:s0 + chunk].to(torch.int64)
        k = (draw32(seed, _S_WGT, torch.minimum(r, c) * g.n + torch.maximum(r, c)) & 0xFFFFFF) + 1
        w[s0:s0 + chunk] = (k.to(torch.float64) * 2.0**-24).to(torch.float32)
    return CSR(g.n, g.off, g.col, w)


# ---------------------------------------------------------------------------
# small fixtures
# ---------------------------------------------------------------------------

def from_edge_list(n: int, edges) -> CSR:
    if len(edges) == 0:
        z = torch.zeros(0, dtype=torch.int64)
        return csr_from_edges(n, z, z)
    e = torch.tensor(edges, dtype=torch.int64)
    return csr_from_edges(n, e[:, 0], e[:, 1])


def biclique_matched(k: int) -> CSR:
    """K_{k,k} (left ids 0..k-1, right ids k..2k-1) plus a perfect matching of
    the left side (k even).  The left vertices get degree k + 1, so in the
    degree order every right vertex has all k left vertices above it
    (out-degree k), and each matching edge closes a triangle with every right
    vertex: k/2 * k triangles over k*k + k/2 edges."""
    left = torch.arange(k, dtype=torch.int64).repeat_interleave(k)
    right = k + torch.arange(k, dtype=torch.int64).repeat(k)
    ml = torch.arange(0, k - 1, 2, dtype=torch.int64)
    return csr_from_edges(2 * k, torch.cat([left, ml]), torch.cat([right, ml + 1]))


def hubs_over_leaves(k: int, h: int) -> CSR:
    """h hubs joined to k middle vertices; each middle vertex also has k
    leaves and a matching partner (k even), so it ranks above the hubs in the
    degree order: every hub has out-degree k, and the k/2 matching edges close
    a triangle with every hub (k/2 * h triangles)."""
    mid = torch.arange(k, dtype=torch.int64)
    hubs = k + torch.arange(h, dtype=torch.int64)
    leaves = k + h + torch.arange(k * k, dtype=torch.int64)
    ml = torch.arange(0, k - 1, 2, dtype=torch.int64)
    src = torch.cat([mid.repeat_interleave(h), mid.repeat_interleave(k), ml])
    dst = torch.cat([hubs.repeat(k), leaves, ml + 1])
    return csr_from_edges(k + h + k * k, src, dst)


def complete(k: int) -> CSR:
    return from_edge_list(k, [(i, j) for i in range(k) for j in range(i + 1, k)])


def cycle(k: int) -> CSR:
    return from_edge_list(k, [(i, (i + 1) % k) for i in range(k)])


def path(k: int) -> CSR:
    return from_edge_list(k, [(i, i + 1) for i in range(k - 1)])


def star(k: int) -> CSR:
    """Centre 0 with k leaves."""
    return from_edge_list(k + 1, [(0, i) for i in range(1, k + 1)])


def bowtie() -> CSR:
    """Two triangles sharing only vertex 2."""
    return from_edge_list(5, [(0, 1), (0, 2), (1, 2), (2, 3), (2, 4), (3, 4)])


def diamond() -> CSR:
    """Two triangles sharing the edge {1, 2}."""
    return from_edge_list(4, [(0, 1), (0, 2), (1, 2), (1, 3), (2, 3)])


def gnp(n: int, q: float, seed: int = 1) -> CSR:
    """Erdos-Renyi G(n, q) from the counter mixer (upper-triangle pairs)."""
    iu = torch.triu_indices(n, n, 1)
    ctr = iu[0].to(torch.int64) * n + iu[1].to(torch.int64)
    r = draw32(seed, 0x06A901, ctr)
    keep = r < int(q * 2**32)
    return csr_from_edges(n, iu[0][keep].to(torch.int64), iu[1][keep].to(torch.int64))


def disjoint_union(*gs: CSR) -> CSR:
    srcs, dsts, base = [], [], 0
    for g in gs:
        rows = torch.repeat_interleave(torch.arange(g.n, dtype=torch.int64), g.off[1:] - g.off[:-1])
        srcs.append(rows + base)
        dsts.append(g.col.to(torch.int64) + base)
        base += g.n
    return csr_from_edges(base, torch.cat(srcs), torch.cat(dsts))
