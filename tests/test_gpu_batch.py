"""Batched compression: every graph of the batch must come out bit for bit as
it does from sg_compress alone (and as the oracle computes it)."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

EDGE_TR = ["uniform", "tr_random", "spectral_logn", "tr_p2", "spectral_avgdeg"]


@pytest.fixture(scope="module")
def sg():
    import paper_1912_08950_gb300 as m

    return m


@pytest.fixture(scope="module")
def ctx(sg):
    c = sg.Context(0)
    yield c
    c.close()


def _graphs(count, weighted, seed0):
    rng = np.random.default_rng(seed0)
    out = []
    for i in range(count):
        s = int(rng.integers(3, 12))
        ef = int(rng.integers(2, 20))
        g = gg.rmat(s, ef, seed=seed0 + i)
        out.append(gg.attach_weights(g, seed=i + 1) if weighted else g)
    out.insert(count // 2, gg.from_edge_list(0, []) if not weighted else gg.attach_weights(gg.complete(4)))
    out.insert(count // 3, gg.attach_weights(gg.from_edge_list(6, [])) if weighted else gg.from_edge_list(6, []))
    return out


def _check_batch(sg, ctx, graphs, kernels, ps, seeds, want_weights=False):
    G = [sg.Graph.from_csr(ctx, g) for g in graphs]
    B = sg.Batch(ctx, G)
    outs = B.compress(kernels, ps, seeds, want_weights)
    for i, (g, h) in enumerate(zip(graphs, outs)):
        off, col, w = h.download()
        solo = sg.compress(G[i], kernels[i], ps[i], seeds[i], want_weights)
        s_off, s_col, s_w = solo.download()
        solo.free()
        assert np.array_equal(off, s_off), (i, kernels[i])
        assert np.array_equal(col, s_col), (i, kernels[i])
        if s_w is not None and w is not None:
            assert np.array_equal(w.view(np.uint32), s_w.view(np.uint32)), (i, kernels[i])
        if i % 5 == 0:
            o_off, o_col, _ = oracle.compress(g, kernels[i], ps[i], seeds[i], want_weights)
            assert np.array_equal(off, o_off) and np.array_equal(col, o_col)
    info = B.info()
    assert info["vertices"] == sum(g.n for g in graphs)
    return B, G


def test_batch_matches_solo_unweighted(sg, ctx):
    graphs = _graphs(40, False, 100)
    n = len(graphs)
    kernels = [EDGE_TR[i % len(EDGE_TR)] for i in range(n)]
    ps = [(0.2, 0.5, 0.8)[i % 3] for i in range(n)]
    seeds = [i + 1 for i in range(n)]
    B, G = _check_batch(sg, ctx, graphs, kernels, ps, seeds, want_weights=True)
    # a second call with new parameters reuses the tuned CUDA graph
    kernels2 = kernels[::-1]
    seeds2 = [s * 7 + 3 for s in seeds]
    outs = B.compress(kernels2, ps, seeds2)
    for i in range(n):
        off, col, _ = outs[i].download()
        solo = sg.compress(G[i], kernels2[i], ps[i], seeds2[i])
        s_off, s_col, _ = solo.download()
        solo.free()
        assert np.array_equal(off, s_off) and np.array_equal(col, s_col)
    B.free()


def test_batch_matches_solo_weighted_maxw(sg, ctx):
    graphs = _graphs(24, True, 300)
    n = len(graphs)
    kernels = [("tr_maxw", "tr_random", "uniform", "spectral_avgdeg")[i % 4] for i in range(n)]
    ps = [1.0 if k == "tr_maxw" else 0.5 for k in kernels]
    seeds = [11 * i + 5 for i in range(n)]
    B, _ = _check_batch(sg, ctx, graphs, kernels, ps, seeds)
    B.free()


def test_batch_long_out_lists_are_chunked(sg, ctx):
    # a batch has no hub launch: the biclique's out-degree-1100 vertices are
    # taken by the main launch's tables in chunks
    graphs = [gg.rmat(8, 8, seed=3), gg.biclique_matched(1100), gg.complete(30)]
    kernels = ["tr_random", "tr_random", "tr_p2"]
    B, _ = _check_batch(sg, ctx, graphs, kernels, [0.5, 0.7, 0.4], [1, 2, 3])
    B.free()


def test_batch_rejects_edge_once(sg, ctx):
    G = [sg.Graph.from_csr(ctx, gg.complete(5))]
    B = sg.Batch(ctx, G)
    for kern in ("tr_eo", "tr_eo_maxw", "tr_eo_mincount", "tr_mincount"):
        with pytest.raises(sg.SgError) as e:
            B.compress([kern], [0.5], [1])
        assert e.value.status == sg.SG_ERR_UNSUPPORTED
    B.free()


def test_batch_edge_kernel_graphs_before_triangle_graphs(sg, ctx):
    # Large graphs with edge kernels first, triangle kernels last: those
    # graphs are not oriented, so the in-arc room of the later vertices sits
    # beyond nnz/2 -- the in-arc records must cover all nnz.
    graphs = [gg.rmat(s, 16, seed=40 + i) for i, s in enumerate((14, 13, 14, 12, 13, 12))]
    kernels = ["uniform", "spectral_avgdeg", "uniform", "tr_random", "tr_p2", "tr_random"]
    ps = [0.5, 0.5, 0.3, 0.6, 0.5, 0.9]
    seeds = [3, 4, 5, 6, 7, 8]
    B, _ = _check_batch(sg, ctx, graphs, kernels, ps, seeds)
    # and with the order reversed
    outs = B.compress(kernels[::-1], ps[::-1], seeds[::-1])
    for i, h in enumerate(outs):
        off, col, _ = h.download()
        o_off, o_col, _ = oracle.compress(graphs[i], kernels[::-1][i], ps[::-1][i], seeds[::-1][i])
        assert np.array_equal(off, o_off) and np.array_equal(col, o_col)
    B.free()


def test_batch_at_benchmark_scale_range(sg, ctx):
    """Three hundred R-MAT graphs drawn like the 4096-graph benchmark batch
    (scale round(8 + 8u), edge factor 8..32, per-graph seed and p, kernels
    uniform / spectral / union TR round-robin): every output equals its solo
    run, every 10th the oracle's (union TR only up to scale 14, to keep the
    oracle's time bounded)."""
    count = 300
    rng = np.random.default_rng(11)
    scales = [int(round(8 + 8 * x)) for x in rng.random(count)]
    efs = [int(e) for e in rng.integers(8, 33, size=count)]
    seeds = [i + 1 for i in range(count)]
    ps = [float(x) for x in rng.choice([0.2, 0.5, 0.8], size=count)]
    kernels = [("uniform", "spectral_avgdeg", "tr_random")[i % 3] for i in range(count)]
    u, vbase, _ = gg.rmat_batch(scales, efs, seeds, device="cuda")
    graphs = [gg.batch_member(u, vbase, i, 1 << scales[i]) for i in range(count)]
    G = [sg.Graph.from_csr(ctx, g) for g in graphs]
    B = sg.Batch(ctx, G)
    outs = B.compress(kernels, ps, seeds)
    for i in range(count):
        off, col, _ = outs[i].download()
        solo = sg.compress(G[i], kernels[i], ps[i], seeds[i])
        s_off, s_col, _ = solo.download()
        solo.free()
        assert np.array_equal(off, s_off) and np.array_equal(col, s_col), (i, scales[i], kernels[i])
        if i % 10 == 0 and (kernels[i] != "tr_random" or scales[i] <= 14):
            o_off, o_col, _ = oracle.compress(graphs[i].to("cpu"), kernels[i], ps[i], seeds[i])
            assert np.array_equal(off, o_off) and np.array_equal(col, o_col), (i, scales[i], kernels[i])
    assert B.info()["vertices"] == sum(g.n for g in graphs)
    B.free()
    for g in G:
        g.free()
