"""CUDA path vs the CPU oracle, through the C-ABI.

Compressed edge sets must match bit for bit (integer work); PageRank values
and the KL divergence must lie within 1e-5 relative of the FP64 oracle
(|kl - kl*| <= 1e-5 kl* + 1e-12); component counts must match exactly.
"""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

KERNELS = ["uniform", "spectral_logn", "spectral_avgdeg", "tr_random", "tr_eo", "tr_p2", "tr_mincount",
           "tr_eo_mincount"]
WKERNELS = ["tr_maxw", "tr_eo_maxw"]


@pytest.fixture(scope="module")
def sg():
    import paper_1912_08950_gb300 as m

    return m


@pytest.fixture(scope="module")
def ctx(sg):
    assert torch.cuda.is_available()
    c = sg.Context(0)
    yield c
    c.close()


def _same(sg, ctx, g, kern, p, seed, want_weights=False):
    G = sg.Graph.from_csr(ctx, g)
    H = sg.compress(G, kern, p, seed, want_weights)
    off, col, w = H.download()
    o_off, o_col, o_w = oracle.compress(g, kern, p, seed, want_weights)
    assert np.array_equal(off, o_off), f"{kern} p={p} seed={seed}: offsets differ"
    assert np.array_equal(col, o_col), f"{kern} p={p} seed={seed}: columns differ"
    if o_w is not None or w is not None:
        assert w is not None and o_w is not None
        assert np.array_equal(w.view(np.uint32), o_w.view(np.uint32)), f"{kern}: weights differ"
    H.free()
    G.free()
    return off, col


# ------------------------------------------------------------- small graphs
SMALL = {
    "K3": gg.complete(3), "K4": gg.complete(4), "K7": gg.complete(7), "bowtie": gg.bowtie(),
    "diamond": gg.diamond(), "star": gg.star(40), "path": gg.path(50), "cycle": gg.cycle(33),
    "isolated": gg.from_edge_list(9, []), "one_edge": gg.from_edge_list(5, [(1, 3)]),
    "gnp": gg.gnp(90, 0.2, 3), "union": gg.disjoint_union(gg.complete(5), gg.star(7), gg.path(4), gg.complete(3)),
}


@pytest.mark.parametrize("name", sorted(SMALL))
@pytest.mark.parametrize("kern", KERNELS)
def test_small_graphs_bit_exact(sg, ctx, name, kern):
    for p, seed in ((0.0, 1), (0.5, 2), (1.0, 3)):
        _same(sg, ctx, SMALL[name], kern, p, seed)


def test_empty_vertex_set(sg, ctx):
    g = gg.from_edge_list(0, [])
    for kern in KERNELS:
        _same(sg, ctx, g, kern, 0.5, 1)


# ------------------------------------------------- R-MAT scale 14 (workload)
def _sparse_rows(n, m, seed):
    """n vertices, m random edges: most rows empty, the rest of degree 1-3."""
    rng = np.random.default_rng(seed)
    a = rng.integers(0, n, size=m)
    b = rng.integers(0, n, size=m)
    keep = a != b
    return gg.csr_from_edges(n, torch.from_numpy(a[keep]), torch.from_numpy(b[keep]))


@pytest.mark.parametrize("kern", KERNELS)
def test_sparse_rows_bit_exact(sg, ctx, kern):
    # a 256-arc warp span holds well over 32 row starts and long runs of empty
    # rows, so every compaction's row search takes several batches of starts,
    # and tiles begin and end inside runs of empty rows
    for n, m, seed in ((200_000, 3_000, 1), (20_000, 9_000, 2), (4_100, 4_100, 3)):
        g = _sparse_rows(n, m, seed)
        for p, s in ((0.5, 7), (1.0, 8)):
            _same(sg, ctx, g, kern, p, s)


@pytest.fixture(scope="module")
def rmat14():
    return gg.rmat(14, 16, seed=1)


@pytest.mark.parametrize("kern", ["uniform", "tr_random"])
def test_rmat14_named_workload(sg, ctx, rmat14, kern):
    _same(sg, ctx, rmat14, kern, 0.5, 1)


@pytest.mark.parametrize("kern", KERNELS)
@pytest.mark.parametrize("p", [0.2, 0.5, 0.8])
def test_rmat14_all_kernels(sg, ctx, rmat14, kern, p):
    _same(sg, ctx, rmat14, kern, p, 7)


@pytest.mark.parametrize("kern", ["spectral_logn", "spectral_avgdeg"])
def test_spectral_weights_bit_exact(sg, ctx, rmat14, kern):
    _same(sg, ctx, rmat14, kern, 0.5, 3, want_weights=True)


@pytest.mark.parametrize("kern", WKERNELS + ["uniform", "tr_random", "tr_eo", "tr_p2", "tr_mincount", "tr_eo_mincount"])
def test_weighted_bit_exact(sg, ctx, kern):
    g = gg.attach_weights(gg.rmat(12, 16, seed=4), seed=4)
    _same(sg, ctx, g, kern, 0.6, 5)
    _same(sg, ctx, g, kern, 1.0, 6)


def test_maxw_preserves_mst(sg, ctx):
    g = gg.attach_weights(gg.rmat(13, 16, seed=2), seed=2)
    G = sg.Graph.from_csr(ctx, g)
    for kern in WKERNELS:
        H = sg.compress(G, kern, 1.0, 9)
        off, col, w = H.download()
        assert oracle.mst_weight_units((g.n, off, col, w)) == oracle.mst_weight_units(g)
        assert sg.cc_count(H) == oracle.cc_count(g)
        H.free()


def test_rmat_seeds_and_scales(sg, ctx):
    for scale, ef, seed in ((8, 8, 11), (11, 32, 12), (12, 4, 13), (15, 16, 14)):
        g = gg.rmat(scale, ef, seed=seed)
        for kern in KERNELS:
            _same(sg, ctx, g, kern, 0.5, seed)


def test_chung_lu_and_rgg(sg, ctx):
    cl = gg.attach_weights(gg.chung_lu(13, 2.1, 32.0, seed=1), seed=1)
    rg = gg.attach_weights(gg.rgg3d(12, 48.0, seed=1), seed=1)
    for g in (cl, rg):
        for kern in ["tr_maxw", "tr_eo", "tr_random", "uniform"]:
            _same(sg, ctx, g, kern, 1.0 if kern == "tr_maxw" else 0.5, 2)


def test_triangle_count(sg, ctx, rmat14):
    for g in (rmat14, SMALL["K7"], SMALL["gnp"], SMALL["path"], gg.rgg3d(11, 48.0, seed=2)):
        G = sg.Graph.from_csr(ctx, g)
        assert sg.triangle_count(G) == oracle.triangle_count(g)
        G.free()


def _eo_run(sg, ctx, g, kern, p, seed, cap):
    ctx.set_eo_list_capacity(cap)
    try:
        ctx.stats(reset=True)
        _same(sg, ctx, g, kern, p, seed)
        return ctx.stats(reset=True)
    finally:
        ctx.set_eo_list_capacity(0)


def test_work_model(sg, ctx):
    # W (shorter list per arc) and W+ (N+(v) per arc u->v) recounted in numpy
    # from the degree order (d_u, u) < (d_v, v)
    g = gg.rmat(12, 16, seed=6)
    off, col, _ = g.numpy()
    off = off.astype(np.int64)
    col = col.astype(np.int64)
    deg = np.diff(off)
    src = np.repeat(np.arange(g.n), deg)
    key = deg * (1 << 32) + np.arange(g.n)
    fwd = key[src] < key[col]
    s_, d_ = src[fwd], col[fwd]
    dp = np.bincount(s_, minlength=g.n)
    G = sg.Graph.from_csr(ctx, g)
    w = sg.tr_work(G)
    G.free()
    assert w["m"] == fwd.sum()
    assert w["forward_probes"] == int(dp[d_].sum())
    # a table owner with d+ < 2 closes no triangle, so its arcs are not streamed
    owner = np.where(dp[d_] <= dp[s_], s_, d_)
    shorter = np.minimum(dp[s_], dp[d_])
    assert w["probes"] == int(shorter[dp[owner] >= 2].sum())
    assert w["head_arcs"] == int((dp[s_] < dp[d_]).sum())


@pytest.mark.parametrize("cap", [-1, 4096, 60000, 250000, 0])
@pytest.mark.parametrize("kern", ["tr_eo", "tr_eo_maxw", "tr_eo_mincount"])
def test_eo_list_capacity_does_not_change_result(sg, ctx, kern, cap):
    # -1: enumerate every round.  Small caps: a listing pass that runs out of
    # room in its first bucket only bids, and later passes list the buckets
    # that fit (a window of the schedule), list again above the window once
    # it is decided, and so on.  0: automatic (everything fits)
    g = gg.attach_weights(gg.rmat(13, 16, seed=8), seed=8)
    st = _eo_run(sg, ctx, g, kern, 0.7, 4, cap)
    # every pass but a last one that finds nothing live ends in a round
    assert 1 <= st["eo_passes"] <= st["eo_rounds"] + 1
    if cap == 0:
        assert st["eo_passes"] == 1 and st["eo_list_passes"] == 1
    if cap == -1:
        assert st["eo_listed"] == 0 and st["eo_list_passes"] == 0
        assert st["eo_passes"] == st["eo_rounds"] + 1


def test_eo_workspace_reuse_and_release(sg, ctx):
    # repeated calls reuse the context's list workspaces; releasing them in
    # between changes nothing but the allocations
    g = gg.rmat(12, 16, seed=4)
    first = _same(sg, ctx, g, "tr_eo", 0.5, 3)
    again = _same(sg, ctx, g, "tr_eo", 0.5, 3)
    ctx.release_workspace()
    after = _same(sg, ctx, g, "tr_eo", 0.5, 3)
    for x, y in ((first, again), (first, after)):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])


def test_eo_list_windows(sg, ctx):
    # caps between the first bucket and the whole list: some pass lists a
    # window of the schedule and a later pass lists the triangles above it
    g = gg.rmat(14, 16, seed=5)
    relisted = 0
    for cap in (30000, 100000, 300000, 1000000):
        st = _eo_run(sg, ctx, g, "tr_eo", 0.6, 9, cap)
        assert st["eo_list_passes"] <= st["eo_passes"] <= st["eo_rounds"] + 1
        relisted += st["eo_list_passes"] >= 2
    assert relisted > 0


def test_deterministic_repeats(sg, ctx, rmat14):
    G = sg.Graph.from_csr(ctx, rmat14)
    ref = None
    for _ in range(3):
        H = sg.compress(G, "tr_eo", 0.5, 42)
        out = H.download()[1]
        H.free()
        if ref is None:
            ref = out
        assert np.array_equal(ref, out)
    G.free()


# ---------------------------------------------------------------- analytics
def _pr_check(sg, ctx, g):
    G = sg.Graph.from_csr(ctx, g)
    x, r = sg.pagerank(G)
    ref, rr = oracle.pagerank(g)
    x = x.cpu().numpy().astype(np.float64)
    rel = np.abs(x - ref) / ref
    assert rel.max() <= 1e-5, rel.max()
    # the residual ||x50 - x49||_1 in FP64: both FP32 iterates lie within
    # 1e-5 relative of the FP64 ones, so it is within 2e-5 sum(x) = 2e-5
    assert abs(r - rr) <= 2e-5, (r, rr)
    G.free()


def test_pagerank_residual_star_two_iterations(sg, ctx):
    # the hand-worked two-update star (see the oracle's pin): FP32 values, FP64 residual
    k, d = 5, 0.85
    n = k + 1
    b = (1 - d) / n
    c1, l1 = b + d * k / n, b + d / (n * k)
    c2, l2 = b + d * k * l1, b + d * c1 / k
    want = abs(c2 - c1) + k * abs(l2 - l1)
    G = sg.Graph.from_csr(ctx, gg.star(k))
    x, r = sg.pagerank(G, d, 2)
    _, rr = oracle.pagerank(gg.star(k), d, 2)
    assert abs(r - want) <= 1e-5 * want and abs(r - rr) <= 1e-5 * rr
    G.free()


@pytest.mark.parametrize("name", ["star", "cycle", "union", "gnp", "isolated"])
def test_pagerank_small(sg, ctx, name):
    _pr_check(sg, ctx, SMALL[name])


def test_pagerank_rmat14(sg, ctx, rmat14):
    _pr_check(sg, ctx, rmat14)


def test_pagerank_regular_is_uniform(sg, ctx):
    G = sg.Graph.from_csr(ctx, gg.cycle(64))
    x, _ = sg.pagerank(G)
    assert torch.all(x == x[0]) and abs(float(x[0]) - 1 / 64) < 1e-9
    G.free()


@pytest.mark.parametrize("kern,p", [("uniform", 0.5), ("tr_eo", 0.5), ("tr_random", 0.8), ("spectral_avgdeg", 0.5)])
def test_divergence_rmat14(sg, ctx, rmat14, kern, p):
    G = sg.Graph.from_csr(ctx, rmat14)
    H = sg.compress(G, kern, p, 3)
    d = sg.divergence(G, H)
    off, col, _ = H.download()
    ref = oracle.divergence(rmat14, (rmat14.n, off, col, None))
    assert abs(d["kl_bits"] - ref["kl_bits"]) <= 1e-5 * ref["kl_bits"] + 1e-12, (d["kl_bits"], ref["kl_bits"])
    assert d["cc_g"] == ref["cc_g"] and d["cc_h"] == ref["cc_h"]
    assert d["m_g"] == rmat14.m and d["m_h"] == col.size // 2
    assert abs(d["pr_residual_g"] - ref["pr_residual_g"]) <= 2e-5
    assert abs(d["pr_residual_h"] - ref["pr_residual_h"]) <= 2e-5
    H.free()
    G.free()


def test_kl_of_identity_is_zero(sg, ctx, rmat14):
    G = sg.Graph.from_csr(ctx, rmat14)
    assert sg.divergence(G, G)["kl_bits"] == 0.0
    G.free()


def test_cc_labels(sg, ctx):
    g = SMALL["union"]
    G = sg.Graph.from_csr(ctx, g)
    cnt, lab = sg.cc_count(G, labels=True)
    n_ref, lab_ref = oracle.cc_count(g, return_labels=True)
    assert cnt == n_ref
    assert np.array_equal(lab.cpu().numpy().astype(np.int64), lab_ref)
    G.free()


@pytest.mark.parametrize("shape", ["forest", "no_giant", "giant_plus_specks"])
def test_cc_sampled_giant(sg, ctx, shape):
    # the giant-component guess from sampled roots decides only which rows are
    # skipped: counts and labels must match the oracle whatever the shape
    rng = np.random.default_rng(7)
    if shape == "forest":  # 3000 random trees of 1-60 vertices
        parts, base = [], 0
        for _ in range(3000):
            k = int(rng.integers(1, 61))
            par = base + (rng.integers(0, np.arange(1, k), size=k - 1) if k > 1 else np.zeros(0, np.int64))
            parts.append(np.stack([base + np.arange(1, k), par], 1) if k > 1 else np.zeros((0, 2), np.int64))
            base += k
        e = np.concatenate(parts)
        g = gg.csr_from_edges(base, torch.from_numpy(e[:, 0]), torch.from_numpy(e[:, 1]))
    elif shape == "no_giant":  # 20000 disjoint edges and 5000 isolated vertices
        a_ = torch.arange(0, 40000, 2)
        g = gg.csr_from_edges(45000, a_, a_ + 1)
    else:  # a giant R-MAT core, small cliques and isolated vertices
        core = gg.rmat(14, 8, seed=3)
        g = gg.disjoint_union(core, *[gg.complete(int(k)) for k in rng.integers(1, 6, size=400)],
                              gg.from_edge_list(3000, []))
    G = sg.Graph.from_csr(ctx, g)
    cnt, lab = sg.cc_count(G, labels=True)
    n_ref, lab_ref = oracle.cc_count(g, return_labels=True)
    assert cnt == n_ref
    assert np.array_equal(lab.cpu().numpy().astype(np.int64), lab_ref)
    G.free()


# --------------------------------------------------------- argument checks
def test_errors(sg, ctx):
    g = gg.rmat(8, 8, seed=1)
    G = sg.Graph.from_csr(ctx, g)
    for bad in (-0.1, 1.5, float("nan")):
        with pytest.raises(sg.SgError) as e:
            sg.compress(G, "uniform", bad, 1)
        assert e.value.status == sg.SG_ERR_INVALID_ARG
    with pytest.raises(sg.SgError) as e:
        sg.compress(G, "tr_maxw", 0.5, 1)
    assert e.value.status == sg.SG_ERR_NEEDS_WEIGHTS
    with pytest.raises(sg.SgError) as e:
        sg.compress(G, 99, 0.5, 1)
    assert e.value.status == sg.SG_ERR_INVALID_ARG
    G.free()
    # offsets that do not end at nnz fail validation
    off = torch.tensor([0, 1, 1, 1], dtype=torch.int64)
    with pytest.raises(sg.SgError) as e:
        sg.Graph.from_tensors(ctx, 3, off.cuda(), torch.tensor([1, 2], dtype=torch.int32).cuda(), validate=True)
    assert e.value.status == sg.SG_ERR_INVALID_GRAPH
    # an asymmetric CSR fails validation
    bad = gg.CSR(3, torch.tensor([0, 1, 2, 2]), torch.tensor([1, 2], dtype=torch.int32))
    with pytest.raises(sg.SgError) as e:
        sg.Graph.from_csr(ctx, bad, validate=True)
    assert e.value.status == sg.SG_ERR_INVALID_GRAPH
    # an unsorted row fails validation
    bad = gg.CSR(3, torch.tensor([0, 2, 3, 4]), torch.tensor([2, 1, 0, 0], dtype=torch.int32))
    with pytest.raises(sg.SgError):
        sg.Graph.from_csr(ctx, bad, validate=True)
    # the context is still usable afterwards
    G = sg.Graph.from_csr(ctx, g, validate=True)
    _ = sg.compress(G, "uniform", 0.5, 1)
    G.free()


@pytest.mark.parametrize("kern,p", [("tr_random", 0.3), ("tr_eo", 0.5), ("tr_eo", 1.0), ("tr_p2", 0.4),
                                    ("tr_mincount", 0.6), ("tr_eo_mincount", 1.0)])
def test_chunked_heavy_tables(sg, ctx, kern, p):
    # K600: out-degrees up to 599 fill most of a 1024-entry table (the hub
    # launch and the chunked paths have tests of their own below)
    g = gg.complete(600)
    _same(sg, ctx, g, kern, p, 12)
    G = sg.Graph.from_csr(ctx, g)
    assert sg.triangle_count(G) == 600 * 599 * 598 // 6
    G.free()


@pytest.mark.parametrize("kern,p", [("tr_random", 0.3), ("tr_eo", 0.5), ("tr_eo", 1.0), ("tr_p2", 0.4),
                                    ("tr_mincount", 0.6), ("tr_eo_mincount", 1.0), ("tr_maxw", 1.0)])
def test_hub_tables(sg, ctx, kern, p):
    # every right vertex of the matched biclique has out-degree 1100: longer
    # than the main launch's tables, so the hub launch handles them (1100
    # hubs, more than the SMs)
    g = gg.attach_weights(gg.biclique_matched(1100), seed=3)
    _same(sg, ctx, g, kern, p, 5)
    G = sg.Graph.from_csr(ctx, g)
    assert sg.triangle_count(G) == 550 * 1100
    w = sg.tr_work(G)
    assert w["max_out_degree"] == 1100 and w["triangles"] == 550 * 1100
    G.free()


def test_hub_tables_chunked(sg, ctx):
    # out-degree 4100 exceeds even the hub table, which then takes N+(u) in
    # chunks (the oracle needs about a minute for this graph)
    g = gg.biclique_matched(4100)
    _same(sg, ctx, g, "tr_random", 0.5, 8)
    G = sg.Graph.from_csr(ctx, g)
    assert sg.triangle_count(G) == 2050 * 4100
    G.free()


@pytest.mark.parametrize("kern", ["tr_random", "tr_eo"])
def test_few_hubs_chunked_in_main_launch(sg, ctx, kern):
    # 40 hubs of out-degree 1100 are too few for a hub launch: the main
    # launch takes their N+(u) in two chunks.  Each of the 1100 vertices below
    # the hubs gets 1100 leaves and a matching partner, so it ranks above them.
    k, h = 1100, 40
    g = gg.hubs_over_leaves(k, h)
    G = sg.Graph.from_csr(ctx, g)
    w = sg.tr_work(G)
    assert w["max_out_degree"] == k and w["triangles"] == (k // 2) * h
    G.free()
    _same(sg, ctx, g, kern, 0.6, 2)


def test_edge_triangle_counts_through_mincount(sg, ctx):
    # at p = 1 every triangle is selected, so min-count TR deletes exactly the
    # per-triangle minima of the counts -- a wrong count anywhere shows up
    g = gg.rmat(13, 32, seed=21)
    _same(sg, ctx, g, "tr_mincount", 1.0, 2)
    _same(sg, ctx, g, "tr_eo_mincount", 1.0, 2)


def test_p2_at_p1_on_disjoint_triangles(sg, ctx):
    k = 3000
    g = gg.disjoint_union(*[gg.complete(3)] * k)
    G = sg.Graph.from_csr(ctx, g)
    H = sg.compress(G, "tr_p2", 1.0, 5)
    off, col, _ = H.download()
    assert col.size == 2 * k
    H.free()
    G.free()
