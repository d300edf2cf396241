"""low_degree (Listing 1; Sec. 4.4) on the GPU vs the oracle, bit for bit:
vertex count, renumbered CSR, carried weights and the new-to-old id map."""
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


def _check(sg, ctx, g):
    G = sg.Graph.from_csr(ctx, g)
    H, nto = sg.low_degree(G, return_map=True)
    k, o_off, o_col, new_id = oracle.low_degree(g)
    off, col, w = H.download()
    assert H.n == k
    assert np.array_equal(off, o_off) and np.array_equal(col, o_col)
    old = np.flatnonzero(new_id >= 0)
    assert np.array_equal(nto.cpu().numpy().view(np.uint32).astype(np.int64), old)
    if g.w is not None:
        gw = g.numpy()[2]
        goff, gcol, _ = g.numpy()
        # every kept arc carries the weight of its arc in G
        for i in range(0, H.n, max(1, H.n // 50)):
            x = old[i]
            for j in range(off[i], off[i + 1]):
                y = old[col[j]]
                gj = goff[x] + np.searchsorted(gcol[goff[x]:goff[x + 1]], y)
                assert w[j] == gw[gj]
    H.free()
    G.free()
    return k


SMALL = {
    "path": gg.path(12), "star": gg.star(9), "cycle": gg.cycle(9), "K5": gg.complete(5),
    "isolated": gg.from_edge_list(7, []), "edge": gg.from_edge_list(4, [(0, 3)]),
    "mixed": gg.disjoint_union(gg.from_edge_list(3, []), gg.path(2), gg.cycle(4), gg.star(5)),
    "gnp": gg.gnp(300, 0.004, 2),
}


@pytest.mark.parametrize("name", sorted(SMALL))
def test_low_degree_small(sg, ctx, name):
    _check(sg, ctx, SMALL[name])


def test_low_degree_empty_graph(sg, ctx):
    assert _check(sg, ctx, gg.from_edge_list(0, [])) == 0


@pytest.mark.parametrize("scale,ef,seed", [(12, 4, 1), (14, 16, 2), (16, 2, 3)])
def test_low_degree_rmat(sg, ctx, scale, ef, seed):
    # low edge factors leave many degree-1 vertices; several vertex tiles and a ragged tail
    _check(sg, ctx, gg.rmat(scale, ef, seed=seed))


def test_low_degree_weighted(sg, ctx):
    _check(sg, ctx, gg.attach_weights(gg.rmat(12, 2, seed=5), seed=5))


def test_low_degree_full_size(sg, ctx):
    g = gg.rmat(22, 16, seed=1, device="cuda")
    torch.cuda.synchronize()
    G = sg.Graph.from_csr(ctx, g, copy=True)
    H, nto = sg.low_degree(G, return_map=True)
    goff = g.off.cpu().numpy()
    deg = np.diff(goff)
    keep = np.flatnonzero(deg >= 2)
    assert H.n == keep.size
    assert np.array_equal(nto.cpu().numpy().view(np.uint32).astype(np.int64), keep)
    # H's degrees: kept vertices lose exactly their degree-1 neighbours
    off, col, _ = H.download()
    gcol = g.col.cpu().numpy().view(np.uint32)
    rng = np.random.default_rng(3)
    for i in rng.integers(0, H.n, size=200):
        x = keep[i]
        nb = gcol[goff[x]:goff[x + 1]]
        want = np.searchsorted(keep, nb[deg[nb] >= 2])
        assert np.array_equal(col[off[i]:off[i + 1]], want)
    H.free()
    G.free()
