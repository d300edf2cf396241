"""Parity at the full R-MAT scale-22 size (edge factor 16, seed 1), in the
launch configuration the benchmark times.  Edge kernels are compared with the
whole oracle output; union TR on sampled edges answered one by one by the
oracle; Edge-Once TR through the invariants that hold at any size (2-spanner,
edge-disjoint acceptance => at most m/3 deletions and degree drop <= d/2,
preserved components) plus exact parity at scale 16."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle

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


@pytest.fixture(scope="module")
def big(sg, ctx):
    g = gg.rmat(22, 16, seed=1, device="cuda")
    G = sg.Graph.from_csr(ctx, g, copy=True)
    yield g.to("cpu"), G
    G.free()


@pytest.mark.parametrize("kern", ["uniform", "spectral_avgdeg", "spectral_logn"])
def test_edge_kernels_full_graph(sg, big, kern):
    g, G = big
    H = sg.compress(G, kern, 0.5, 1)
    off, col, _ = H.download()
    o_off, o_col, _ = oracle.compress(g, kern, 0.5, 1)
    assert np.array_equal(off, o_off) and np.array_equal(col, o_col)
    H.free()


def _edge_sample(g, k, seed):
    off, col, _ = g.numpy()
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, col.size, size=k)
    rows = np.searchsorted(off, idx, side="right") - 1
    return rows, col[idx].astype(np.int64)


def _has_edge(off, col, x, y):
    lo, hi = off[x], off[x + 1]
    k = np.searchsorted(col[lo:hi], y)
    return k < hi - lo and col[lo + k] == y


@pytest.mark.parametrize("kern", ["tr_random", "tr_p2", "tr_mincount"])
def test_tr_union_sampled_edges(sg, big, kern):
    g, G = big
    H = sg.compress(G, kern, 0.5, 1)
    off, col, _ = H.download()
    rows, cols = _edge_sample(g, 3000, 5)
    for x, y in zip(rows, cols):
        deleted = oracle.tr_union_edge_deleted(g, kern, 0.5, 1, int(x), int(y))
        assert _has_edge(off, col, int(x), int(y)) == (not deleted)
    assert 0 < col.size < g.nnz
    H.free()


@pytest.mark.parametrize("kern,p", [("tr_eo", 0.2), ("tr_eo", 0.5), ("tr_eo", 0.8), ("tr_eo_mincount", 0.5)])
def test_tr_eo_invariants_full_size(sg, big, kern, p):
    g, G = big
    H = sg.compress(G, kern, p, 1)
    off, col, _ = H.download()
    goff, gcol, _ = g.numpy()
    dg, dh = np.diff(goff), np.diff(off)
    assert np.all(dh <= dg) and np.all(dg - dh <= dg // 2)
    assert (g.nnz - col.size) // 2 <= g.m / 3
    cc = oracle.cc_count(g)
    assert oracle.cc_count((g.n, off, col, None)) == cc and sg.cc_count(H) == sg.cc_count(G) == cc
    # sampled deleted edges keep a 2-path in H
    rows, cols = _edge_sample(g, 20000, 7)
    checked = 0
    for x, y in zip(rows, cols):
        x, y = int(x), int(y)
        if _has_edge(off, col, x, y):
            continue
        nx = col[off[x]:off[x + 1]]
        ny = col[off[y]:off[y + 1]]
        assert np.intersect1d(nx, ny).size > 0
        checked += 1
    assert checked > 0
    H.free()


def test_tr_eo_exact_scale16(sg, ctx):
    g = gg.rmat(16, 16, seed=1)
    G = sg.Graph.from_csr(ctx, g)
    H = sg.compress(G, "tr_eo", 0.5, 1)
    off, col, _ = H.download()
    o_off, o_col, _ = oracle.compress(g, "tr_eo", 0.5, 1)
    assert np.array_equal(off, o_off) and np.array_equal(col, o_col)
    H.free()
    G.free()


def test_analytics_full_size(sg, big):
    g, G = big
    H = sg.compress(G, "tr_eo", 0.5, 1)
    d = sg.divergence(G, H)
    off, col, _ = H.download()
    P, rp = oracle.pagerank(g)
    Q, rq = oracle.pagerank((g.n, off, col, None))
    # FP64 residuals of the FP32 iterates: within 2e-5 sum(x) of the oracle's
    assert abs(d["pr_residual_g"] - rp) <= 2e-5 and abs(d["pr_residual_h"] - rq) <= 2e-5
    x, _ = sg.pagerank(G)
    rel = np.abs(x.cpu().numpy().astype(np.float64) - P) / P
    assert rel.max() <= 1e-5, rel.max()
    kl = oracle.kl_divergence(P, Q)
    assert abs(d["kl_bits"] - kl) <= 1e-5 * kl + 1e-12, (d["kl_bits"], kl)
    assert d["cc_g"] == oracle.cc_count(g)
    assert d["cc_h"] == oracle.cc_count((g.n, off, col, None))
    H.free()
