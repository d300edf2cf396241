"""Vertex-level accuracy metrics (Sec. 5) on the GPU vs the oracle:
BFS levels and critical edges (Sec. 5.3), A_REN counts (Sec. 5.2.2) and the
per-vertex triangle counts they are taken over -- all integer results, so
every comparison is exact.  Score vectors for A_REN are the same float32
arrays on both sides."""
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


GRAPHS = {
    "path": gg.path(40), "odd_cycle": gg.cycle(41), "K6": gg.complete(6), "star": gg.star(30),
    "two_parts": gg.disjoint_union(gg.rmat(8, 8, seed=3), gg.cycle(9), gg.from_edge_list(4, [])),
    "rmat12": gg.rmat(12, 16, seed=2), "rmat14": gg.rmat(14, 16, seed=1),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_bfs_levels_and_critical_edges(sg, ctx, name):
    g = GRAPHS[name]
    G = sg.Graph.from_csr(ctx, g)
    for root in sorted({0, g.n // 2, g.n - 1}):
        lev = sg.bfs_levels(G, root).cpu().numpy().astype(np.int64)
        assert np.array_equal(lev, oracle.bfs_levels(g, root))
        assert sg.critical_edges(G, root) == oracle.critical_edges(g, root)
    G.free()


def test_bfs_bottom_up_steps(sg, ctx):
    # a hub reaches most vertices in one step, so the middle levels run bottom-up
    g = gg.chung_lu(14, 2.1, 32.0, seed=4)
    G = sg.Graph.from_csr(ctx, g)
    root = int(np.argmax(np.diff(g.numpy()[0])))
    lev = sg.bfs_levels(G, root).cpu().numpy().astype(np.int64)
    want = oracle.bfs_levels(g, root)
    assert np.array_equal(lev, want)
    assert np.bincount(want[want >= 0]).max() * 32 > g.n
    assert sg.critical_edges(G, root) == oracle.critical_edges(g, root)
    G.free()


@pytest.mark.parametrize("name", ["K6", "two_parts", "rmat12", "rmat14"])
def test_vertex_triangle_counts(sg, ctx, name):
    g = GRAPHS[name]
    G = sg.Graph.from_csr(ctx, g)
    t = sg.vertex_triangle_counts(G).cpu().numpy()
    assert np.array_equal(t, oracle.vertex_triangle_counts(g))
    G.free()


def test_vertex_triangle_counts_chunked_tables(sg, ctx):
    g = gg.complete(600)  # N+(u) fills most of a 1024-entry table
    G = sg.Graph.from_csr(ctx, g)
    t = sg.vertex_triangle_counts(G).cpu().numpy()
    assert np.all(t == 599 * 598 // 2)
    G.free()


@pytest.mark.parametrize("hub_launch", [True, False])
def test_vertex_triangle_counts_long_out_lists(sg, ctx, hub_launch):
    # out-degree 1100: 1100 such vertices go to the hub launch; 40 are too few
    # for it and the main launch takes their N+(u) in two chunks
    if hub_launch:
        g, k, h = gg.biclique_matched(1100), 1100, 1100
    else:
        g, k, h = gg.hubs_over_leaves(1100, 40), 1100, 40
    G = sg.Graph.from_csr(ctx, g)
    t = sg.vertex_triangle_counts(G).cpu().numpy()
    G.free()
    assert np.array_equal(t, oracle.vertex_triangle_counts(g))
    assert int(t.sum()) == 3 * (k // 2) * h


@pytest.mark.parametrize("seed", [1, 2])
def test_reordered_neighbours(sg, ctx, seed):
    g = GRAPHS["rmat14"]
    G = sg.Graph.from_csr(ctx, g)
    rng = np.random.default_rng(seed)
    x = rng.random(g.n, dtype=np.float32)
    y = x.copy()
    flip = rng.random(g.n) < 0.3
    y[flip] = rng.random(int(flip.sum()), dtype=np.float32)
    y[rng.random(g.n) < 0.1] = 0.5  # ties on one side
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    assert sg.reordered_neighbours(G, xd, yd) == oracle.reordered_neighbours(g, x, y)
    assert sg.reordered_neighbours(G, xd, xd) == 0
    G.free()


@pytest.mark.parametrize("kern", ["tr_random", "tr_eo", "uniform"])
def test_accuracy_matches_oracle(sg, ctx, kern):
    g = GRAPHS["rmat14"]
    G = sg.Graph.from_csr(ctx, g)
    H = sg.compress(G, kern, 0.5, 3)
    r = sg.accuracy(G, H)
    off, col, _ = H.download()
    h = (g.n, off, col, None)
    # the same float32 PageRank vectors feed the oracle's count
    P = sg.pagerank(G)[0].cpu().numpy()
    Q = sg.pagerank(H)[0].cpu().numpy()
    assert r["pr_reordered"] == oracle.reordered_neighbours(g, P, Q)
    assert r["tc_reordered"] == oracle.reordered_neighbours(g, oracle.vertex_triangle_counts(g),
                                                            oracle.vertex_triangle_counts(h))
    deg = np.diff(g.numpy()[0])
    assert r["root"] == int(np.argmax(deg))
    assert r["critical_g"] == oracle.critical_edges(g, r["root"])
    assert r["critical_h"] == oracle.critical_edges(h, r["root"])
    assert r["m_g"] == g.m and abs(r["pr_aren"] - r["pr_reordered"] / g.m) < 1e-15
    assert 0.0 < r["critical_fraction"] <= 1.5
    H.free()
    G.free()


def test_accuracy_identity(sg, ctx):
    g = GRAPHS["rmat12"]
    G = sg.Graph.from_csr(ctx, g)
    r = sg.accuracy(G, G, root=5)
    assert r["pr_reordered"] == 0 and r["tc_reordered"] == 0
    assert r["critical_g"] == r["critical_h"] and r["critical_fraction"] == 1.0 and r["root"] == 5
    G.free()


def test_accuracy_full_size(sg, ctx):
    g = gg.rmat(22, 16, seed=1, device="cuda")
    torch.cuda.synchronize()
    G = sg.Graph.from_csr(ctx, g, copy=True)
    host = (g.n, g.off.cpu().numpy(), g.col.cpu().numpy().view(np.uint32), None)
    del g
    torch.cuda.empty_cache()
    H = sg.compress(G, "tr_eo", 0.5, 1)
    r = sg.accuracy(G, H)
    off, col, _ = H.download()
    assert r["critical_g"] == oracle.critical_edges(host, r["root"])
    assert r["critical_h"] == oracle.critical_edges((host[0], off, col, None), r["root"])
    # per-vertex triangle counts: they sum to 3T, and sampled low-degree vertices match brute force
    t = sg.vertex_triangle_counts(G).cpu().numpy()
    assert int(t.sum()) == 3 * sg.triangle_count(G)
    goff, gcol = host[1], host[2]
    deg = np.diff(goff)
    rng = np.random.default_rng(7)
    cand = np.flatnonzero((deg >= 2) & (deg <= 60))
    for v in rng.choice(cand, size=200, replace=False):
        nb = gcol[goff[v]:goff[v + 1]]
        k = 0
        for a in nb:
            k += np.intersect1d(nb, gcol[goff[a]:goff[a + 1]], assume_unique=True).size
        assert t[v] == k // 2
    assert 0 <= r["pr_aren"] <= 1 and 0 <= r["tc_aren"] <= 1
    H.free()
    G.free()
