"""Full-size checks on the power-law and geometric workloads:
Chung-Lu with 2^26 vertices (exponent 2.1, mean degree 32, weights k*2^-24)
under max-weight TR at p = 1, and a 3-D random geometric graph with 2^24
points (mean degree 48, triangle-dense) under the TR kernels.

At these sizes the oracle answers sampled edges one by one (the union kernels'
deletion of an edge depends only on the triangles through it).  For the
Chung-Lu graph the oracle's Kruskal MST weight and component count of H are
compared exactly with the values it computed for G (stored by
tests/golden/make_golden.py chung_lu26_mst): max-weight TR keeps both
(Sec. 6, Others).  The cycle property is also checked on sampled deleted
edges: each must be the heaviest edge, under (weight, lo, hi), of a triangle
of G.
"""
import os

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from tests.digest import csr_digest, read_golden

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import paper_1912_08950_gb300 as m

    return m


@pytest.fixture(scope="module")
def ctx(sg):
    c = sg.Context(0)
    yield c
    c.close()


def _host(g):
    off, col, w = g.numpy()
    return (g.n, np.ascontiguousarray(off), np.ascontiguousarray(col), None if w is None else np.ascontiguousarray(w))


def _sample_arcs(off, col, k, seed):
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, col.size, size=k)
    rows = np.searchsorted(off, idx, side="right") - 1
    return rows.astype(np.int64), col[idx].astype(np.int64)


def _has(off, col, x, y):
    lo, hi = off[x], off[x + 1]
    k = np.searchsorted(col[lo:hi], y)
    return k < hi - lo and col[lo + k] == y


def _weight(off, col, w, x, y):
    lo, hi = off[x], off[x + 1]
    return w[lo + np.searchsorted(col[lo:hi], y)]


def _is_max_of_a_triangle(off, col, w, x, y):
    lo, hi = min(x, y), max(x, y)
    wxy = (_weight(off, col, w, x, y), lo, hi)
    common = np.intersect1d(col[off[x]:off[x + 1]], col[off[y]:off[y + 1]], assume_unique=True)
    for z in common:
        z = int(z)
        a = (_weight(off, col, w, x, z), min(x, z), max(x, z))
        b = (_weight(off, col, w, y, z), min(y, z), max(y, z))
        if a < wxy and b < wxy:
            return True
    return False


def _union_parity(sg, G, host, kernel, p, seed, samples):
    n, off, col, w = host
    H = sg.compress(G, kernel, p, seed)
    hoff, hcol, hw = H.download()
    rows, cols = _sample_arcs(off, col, samples, 17)
    for x, y in zip(rows, cols):
        deleted = oracle.tr_union_edge_deleted(host, kernel, p, seed, int(x), int(y))
        assert _has(hoff, hcol, int(x), int(y)) == (not deleted), (kernel, x, y)
    return H, hoff, hcol, hw


def test_chung_lu_26_maxw(sg, ctx):
    g = gg.attach_weights(gg.chung_lu(26, 2.1, 32.0, seed=1, device="cuda"), seed=1)
    torch.cuda.synchronize()
    G = sg.Graph.from_csr(ctx, g, copy=True)
    host = _host(g)
    del g
    torch.cuda.empty_cache()
    n, off, col, w = host
    gold = read_golden(os.path.join(GOLDEN, "chung_lu26_mst.txt"))
    assert gold["graph"] == [str(n), str(col.size), csr_digest(off, col, w)], "generator output changed"
    H, hoff, hcol, hw = _union_parity(sg, G, host, "tr_maxw", 1.0, 3, 2000)
    # H is a subgraph with G's components and G's MST weight, both from the oracle
    assert np.all(np.diff(hoff) <= np.diff(off))
    h_host = (n, hoff, hcol, hw)
    assert oracle.cc_count(h_host) == int(gold["cc"][0])
    assert oracle.mst_weight_units(h_host) == int(gold["mst_units"][0])
    assert sg.cc_count(H) == int(gold["cc"][0]) and sg.cc_count(G) == int(gold["cc"][0])
    # sampled deleted edges are triangle maxima (cycle property => MST weight kept)
    rows, cols = _sample_arcs(off, col, 20000, 23)
    checked = 0
    for x, y in zip(rows, cols):
        x, y = int(x), int(y)
        if not _has(hoff, hcol, x, y):
            assert _is_max_of_a_triangle(off, col, w, x, y)
            checked += 1
            if checked >= 300:
                break
    assert checked > 0
    H.free()
    G.free()


def test_rgg_24_tr_kernels(sg, ctx):
    g = gg.attach_weights(gg.rgg3d(24, 48.0, seed=1, device="cuda"), seed=1)
    torch.cuda.synchronize()
    G = sg.Graph.from_csr(ctx, g, copy=True)
    host = _host(g)
    del g
    torch.cuda.empty_cache()
    n, off, col, w = host
    deg = np.diff(off)
    assert 40 < deg.mean() < 56
    cc_g = oracle.cc_count(host)
    assert sg.cc_count(G) == cc_g
    for kernel, p in (("tr_maxw", 1.0), ("tr_random", 0.5)):
        H, hoff, hcol, _ = _union_parity(sg, G, host, kernel, p, 5, 1500)
        if kernel == "tr_maxw":
            # components kept (Sec. 6): the oracle counts them in H
            assert oracle.cc_count((n, hoff, hcol, None)) == cc_g
        H.free()
    # edge-once: invariants that hold at any size
    H = sg.compress(G, "tr_eo", 0.5, 5)
    hoff, hcol, _ = H.download()
    dh = np.diff(hoff)
    assert np.all(deg - dh <= deg // 2)
    assert (off[-1] - hoff[-1]) // 2 <= (off[-1] // 2) / 3
    assert oracle.cc_count((n, hoff, hcol, None)) == cc_g
    rows, cols = _sample_arcs(off, col, 5000, 29)
    for x, y in zip(rows, cols):
        x, y = int(x), int(y)
        if not _has(hoff, hcol, x, y):
            assert np.intersect1d(hcol[hoff[x]:hoff[x + 1]], hcol[hoff[y]:hoff[y + 1]]).size > 0
    H.free()
    G.free()
