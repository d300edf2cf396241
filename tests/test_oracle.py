"""Pins for the CPU oracle: values and properties fixed by the paper, by the
published Philox definition and by the mathematics -- never by the oracle
itself and never by the CUDA path."""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components, minimum_spanning_tree
from scipy.stats import entropy

import graphgen as gg
import oracle
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _edges_of(n, res):
    off, col, _ = res
    return brute.edge_set_arrays(n, off, col)


def _scipy(g, weighted=False):
    off, col, w = g.numpy()
    data = w.astype(np.float64) if weighted else np.ones(col.size)
    return sp.csr_matrix((data, col.astype(np.int64), off), shape=(g.n, g.n))


# --------------------------------------------------------------------------
# Philox4x32-10: published known-answer vectors (Salmon et al. SC'11)
# --------------------------------------------------------------------------
def test_philox_known_answers():
    rows = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            lhs, rhs = line.split("->")
            ins = [int(t, 16) for t in lhs.split()]
            want = [int(t, 16) for t in rhs.split()]
            got = oracle.philox4x32_10(ins[:4], ins[4:6])
            assert [int(v) for v in got] == want
            rows += 1
    assert rows == 3


def test_threshold_edges():
    assert oracle.threshold(0.0) == 0
    assert oracle.threshold(1.0) == 2**32
    assert oracle.threshold(0.5) == 2**31
    assert oracle.threshold(0.25) == 2**30


# --------------------------------------------------------------------------
# triangle enumeration (Sec. 4.3): brute force and closed forms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,q,seed", [(12, 0.5, 1), (20, 0.4, 2), (30, 0.3, 3), (40, 0.25, 4), (64, 0.15, 5)])
def test_triangles_match_brute_force(n, q, seed):
    g = gg.gnp(n, q, seed)
    want = brute.triangles(n, brute.edge_set(g))
    got = [tuple(int(v) for v in t) for t in oracle.triangle_list(g)]
    assert got == want  # same set, both in lexicographic order
    assert oracle.triangle_count(g) == len(want)


@pytest.mark.parametrize("k", [3, 4, 5, 6, 7, 8, 12])
def test_triangles_complete_graph(k):
    assert oracle.triangle_count(gg.complete(k)) == math.comb(k, 3)


@pytest.mark.parametrize("g", [gg.path(10), gg.star(9), gg.cycle(8), gg.cycle(9), gg.from_edge_list(6, [(0, 3), (0, 4), (0, 5), (1, 3), (1, 4), (2, 5)])])
def test_triangle_free_families(g):
    assert oracle.triangle_count(g) == 0


def test_triangle_count_invariant_under_permutation():
    a = gg.rmat(9, 8, seed=3, permute=False)
    b = gg.rmat(9, 8, seed=3, permute=True)
    assert oracle.triangle_count(a) == oracle.triangle_count(b) > 0


# --------------------------------------------------------------------------
# uniform sampling (Listing 1 random_uniform; Sec. 4.2.2)
# --------------------------------------------------------------------------
def test_uniform_p0_p1():
    g = gg.rmat(10, 8, seed=2)
    off, col, _ = oracle.compress(g, "uniform", 0.0, 7)
    assert col.size == 0 and np.all(off == 0)
    off, col, _ = oracle.compress(g, "uniform", 1.0, 7)
    assert np.array_equal(col, g.numpy()[1]) and np.array_equal(off, g.numpy()[0])


def test_uniform_output_is_symmetric_subgraph():
    g = gg.rmat(11, 8, seed=4)
    E = brute.edge_set(g)
    off, col, _ = oracle.compress(g, "uniform", 0.37, 11)
    H = _edges_of(g.n, (off, col, None))
    assert H <= E
    # symmetric: every kept edge appears as both arcs
    assert col.size == 2 * len(H)


def test_uniform_expected_kept_fraction():
    # E|E'| = p m (each edge stays with probability p), within 5 sigma over seeds
    g = gg.rmat(10, 8, seed=5)
    m = g.m
    for p in (0.2, 0.5, 0.8):
        kept = [oracle.compress(g, "uniform", p, s)[1].size // 2 for s in range(1, 41)]
        mean = np.mean(kept)
        sigma = math.sqrt(m * p * (1 - p) / len(kept))
        assert abs(mean - p * m) < 5 * sigma, (p, mean, p * m)


def test_uniform_triangles_scale_as_p_cubed():
    # a triangle survives iff its three (independent) edges do: E T' = p^3 T
    g = gg.rmat(10, 16, seed=6)
    T = oracle.triangle_count(g)
    p = 0.5
    vals = []
    for s in range(1, 21):
        off, col, _ = oracle.compress(g, "uniform", p, s)
        vals.append(oracle.triangle_count((g.n, off, col, None)))
    assert abs(np.mean(vals) / (p**3 * T) - 1) < 0.05


# --------------------------------------------------------------------------
# spectral sparsification (Listing 1 spectral_sparsify; Sec. 4.2.1)
# --------------------------------------------------------------------------
def test_spectral_star_identity_with_unit_weights():
    g = gg.star(40)  # every edge has min degree 1 <= Y = p ln 41
    for kern, p in (("spectral_logn", 0.5), ("spectral_logn", 1.0)):
        off, col, w = oracle.compress(g, kern, p, 3, want_weights=True)
        assert np.array_equal(col, g.numpy()[1])
        assert np.all(w == 1.0)


def _spectral_probs(g, kern, p):
    off, col, _ = g.numpy()
    deg = np.diff(off)
    Y = p * math.log(g.n) if kern == "spectral_logn" else p * g.m / g.n
    probs = {}
    for x in range(g.n):
        for y in col[off[x]:off[x + 1]]:
            y = int(y)
            if x < y:
                probs[(x, y)] = min(1.0, Y / min(deg[x], deg[y]))
    return probs


@pytest.mark.parametrize("kern,p", [("spectral_logn", 0.5), ("spectral_avgdeg", 0.5), ("spectral_avgdeg", 0.2)])
def test_spectral_expectations(kern, p):
    # E|E'| = sum p_e and E[sum of kept weights] = m (each edge gives p_e * 1/p_e)
    g = gg.rmat(10, 16, seed=8)
    probs = _spectral_probs(g, kern, p)
    pe = np.array(list(probs.values()))
    kept, wsum = [], []
    S = 30
    for s in range(1, S + 1):
        off, col, w = oracle.compress(g, kern, p, s, want_weights=True)
        kept.append(col.size // 2)
        wsum.append(w.astype(np.float64).sum() / 2)
    var_k = (pe * (1 - pe)).sum()
    assert abs(np.mean(kept) - pe.sum()) < 5 * math.sqrt(var_k / S)
    var_w = ((1 - pe) / pe).sum()  # Var of (1/p) Bernoulli(p) is (1-p)/p
    assert abs(np.mean(wsum) - g.m) < 5 * math.sqrt(var_w / S)


def test_spectral_keeps_low_degree_edges():
    # edges whose min degree is <= Y always stay (p_e = 1)
    g = gg.rmat(10, 16, seed=9)
    probs = _spectral_probs(g, "spectral_avgdeg", 0.5)
    off, col, _ = oracle.compress(g, "spectral_avgdeg", 0.5, 5)
    H = _edges_of(g.n, (off, col, None))
    for e, pe in probs.items():
        if pe == 1.0:
            assert e in H


# --------------------------------------------------------------------------
# Triangle p-1-Reduction, union semantics (Listing 1 p-1-reduction; Sec. 4.3)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,q,seed", [(16, 0.5, 1), (30, 0.35, 2), (48, 0.2, 3)])
@pytest.mark.parametrize("p", [0.3, 1.0])
def test_tr_random_matches_brute_force(n, q, seed, p):
    g = gg.gnp(n, q, seed)
    E = brute.edge_set(g)
    got = _edges_of(n, oracle.compress(g, "tr_random", p, seed + 100))
    assert got == brute.tr_union(n, E, p, seed + 100)


def test_tr_single_triangle():
    g = gg.complete(3)
    for s in range(1, 30):
        off, col, _ = oracle.compress(g, "tr_random", 1.0, s)
        assert col.size == 4  # exactly one of the three edges removed
        r = brute.draw(s, 0, 1, 2, brute.TAG_TRI)
        k = (int(r[1]) * 3) >> 32
        gone = [(0, 1), (0, 2), (1, 2)][k]
        assert gone not in _edges_of(3, (off, col, None))


def test_tr_choice_is_uniform():
    # disjoint triangles: each selected triangle loses one edge, position u.a.r.
    k = 600
    g = gg.disjoint_union(*[gg.complete(3)] * k)
    off, col, _ = oracle.compress(g, "tr_random", 1.0, 17)
    H = _edges_of(g.n, (off, col, None))
    counts = np.zeros(3)
    for t in range(k):
        a, b, c = 3 * t, 3 * t + 1, 3 * t + 2
        missing = [e for e in [(a, b), (a, c), (b, c)] if e not in H]
        assert len(missing) == 1
        counts[[(a, b), (a, c), (b, c)].index(missing[0])] += 1
    chi2 = ((counts - k / 3) ** 2 / (k / 3)).sum()
    assert chi2 < 13.8  # chi^2_2 at p = 0.001


def test_tr_selection_rate():
    k = 2000
    g = gg.disjoint_union(*[gg.complete(3)] * k)
    p = 0.3
    off, col, _ = oracle.compress(g, "tr_random", p, 5)
    removed = (g.nnz - col.size) // 2
    assert abs(removed - p * k) < 5 * math.sqrt(k * p * (1 - p))


@pytest.mark.parametrize("g", [gg.path(12), gg.star(10), gg.cycle(10), gg.rmat(8, 2, seed=1)])
def test_tr_identity_on_triangle_free_or_p0(g):
    for kern in ("tr_random", "tr_eo"):
        off, col, _ = oracle.compress(g, kern, 0.0, 3)
        assert np.array_equal(col, g.numpy()[1])
    if oracle.triangle_count(g) == 0:
        for kern in ("tr_random", "tr_eo"):
            off, col, _ = oracle.compress(g, kern, 1.0, 3)
            assert np.array_equal(col, g.numpy()[1])


def test_tr_deletes_only_triangle_edges():
    g = gg.rmat(10, 8, seed=12)
    E = brute.edge_set(g)
    in_tri = set()
    for a, b, c in (tuple(int(v) for v in t) for t in oracle.triangle_list(g)):
        in_tri.update([(a, b), (a, c), (b, c)])
    for kern in ("tr_random", "tr_eo"):
        H = _edges_of(g.n, oracle.compress(g, kern, 0.7, 4))
        assert (E - H) <= in_tri


# --------------------------------------------------------------------------
# max-weight TR: the MST weight and CC are preserved (Sec. 4.3; Sec. 6)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kern", ["tr_maxw", "tr_eo_maxw"])
@pytest.mark.parametrize("scale,ef,p", [(9, 8, 1.0), (10, 16, 1.0), (10, 16, 0.4)])
def test_maxw_preserves_mst_and_cc(kern, scale, ef, p):
    g = gg.attach_weights(gg.rmat(scale, ef, seed=scale))
    off, col, w = oracle.compress(g, kern, p, 21)
    h = gg.CSR(g.n, __import__("torch").from_numpy(off), __import__("torch").from_numpy(col.view(np.int32)),
               __import__("torch").from_numpy(w))
    G = _scipy(g, True)
    H = _scipy(h, True)
    mst_g = minimum_spanning_tree(G).sum()
    mst_h = minimum_spanning_tree(H).sum()
    assert mst_g == pytest.approx(mst_h, rel=0, abs=1e-6)
    assert oracle.mst_weight_units(g) == oracle.mst_weight_units(h)
    assert round(mst_g * 2**24) == oracle.mst_weight_units(g)
    assert connected_components(G)[0] == connected_components(H)[0]


def test_maxw_k3_deletes_heaviest():
    g = gg.attach_weights(gg.complete(3), seed=4)
    W = brute.weights(g)
    heaviest = max(W, key=lambda e: (W[e], e))
    off, col, w = oracle.compress(g, "tr_maxw", 1.0, 1)
    H = _edges_of(3, (off, col, None))
    assert H == set(W) - {heaviest}


def test_maxw_matches_brute_force():
    g = gg.attach_weights(gg.gnp(30, 0.35, 7), seed=7)
    E, W = brute.edge_set(g), brute.weights(g)
    got = _edges_of(30, oracle.compress(g, "tr_maxw", 0.6, 9))
    assert got == brute.tr_union(30, E, 0.6, 9, W)
    got = _edges_of(30, oracle.compress(g, "tr_eo_maxw", 0.6, 9))
    assert got == brute.tr_eo(30, E, 0.6, 9, W)[0]


# --------------------------------------------------------------------------
# Edge-Once TR (Sec. 4.3; Sec. 6 Edge-Once p-1-TR)
# --------------------------------------------------------------------------
def test_eo_k4_leaves_five_edges():
    # any two triangles of K4 share an edge: exactly one is accepted
    for s in range(1, 40):
        off, col, _ = oracle.compress(gg.complete(4), "tr_eo", 1.0, s)
        assert col.size == 10


def test_eo_bowtie_and_diamond():
    for s in range(1, 20):
        assert oracle.compress(gg.bowtie(), "tr_eo", 1.0, s)[1].size == 12 - 4
        assert oracle.compress(gg.diamond(), "tr_eo", 1.0, s)[1].size == 10 - 2


@pytest.mark.parametrize("n,q,seed,p", [(16, 0.6, 1, 1.0), (30, 0.4, 2, 0.5), (48, 0.3, 3, 0.8), (64, 0.2, 4, 1.0)])
def test_eo_matches_brute_force(n, q, seed, p):
    g = gg.gnp(n, q, seed)
    E = brute.edge_set(g)
    want, accepted = brute.tr_eo(n, E, p, seed)
    off, col, _, acc = oracle.compress(g, "tr_eo", p, seed, return_accepted=True)
    assert _edges_of(n, (off, col, None)) == want
    acc_edges = set()
    for a, b, c in accepted:
        acc_edges.update([(a, b), (a, c), (b, c)])
    goff, gcol, _ = g.numpy()
    mask_edges = {(min(x, int(gcol[i])), max(x, int(gcol[i]))) for x in range(n) for i in range(goff[x], goff[x + 1]) if acc[i]}
    assert mask_edges == acc_edges


@pytest.mark.parametrize("scale,ef,p,seed", [(10, 16, 1.0, 1), (10, 16, 0.5, 2), (11, 8, 0.8, 3)])
def test_eo_invariants(scale, ef, p, seed):
    g = gg.rmat(scale, ef, seed=seed)
    E = brute.edge_set(g)
    off, col, _, acc = oracle.compress(g, "tr_eo", p, seed, return_accepted=True)
    H = _edges_of(g.n, (off, col, None))
    D = E - H
    adjH = [set() for _ in range(g.n)]
    for a, b in H:
        adjH[a].add(b)
        adjH[b].add(a)
    # 2-spanner: every deleted {u,v} keeps a 2-path u-w-v (Sec. 6, shortest paths)
    for u, v in D:
        assert adjH[u] & adjH[v]
    # at most one third of the edges can go (Sec. 6 / Sec. 7 discussion)
    assert len(D) <= len(E) / 3
    # CC preserved (Sec. 6 "Others")
    G = _scipy(g)
    Hm = sp.csr_matrix((np.ones(col.size), col.astype(np.int64), off), shape=(g.n, g.n))
    assert connected_components(G)[0] == connected_components(Hm)[0]
    # degree drops by at most floor(d/2) (Sec. 6, degree)
    dg = np.diff(g.numpy()[0])
    dh = np.diff(off)
    assert np.all(dg - dh <= dg // 2)
    # every deleted edge is an accepted-triangle edge, and accepted triangles are
    # edge-disjoint: deleted edges are exactly one per accepted triangle
    goff, gcol, _ = g.numpy()
    n_acc_edges = int(acc.sum()) // 2
    assert n_acc_edges == 3 * len(D)


def test_eo_maximal():
    # every selected triangle not accepted shares an edge with an accepted one
    g = gg.rmat(9, 16, seed=5)
    p, seed = 0.6, 8
    off, col, _, acc = oracle.compress(g, "tr_eo", p, seed, return_accepted=True)
    goff, gcol, _ = g.numpy()
    considered = {(min(x, int(gcol[i])), max(x, int(gcol[i]))) for x in range(g.n) for i in range(goff[x], goff[x + 1]) if acc[i]}
    for a, b, c in (tuple(int(v) for v in t) for t in oracle.triangle_list(g)):
        r = brute.draw(seed, a, b, c, brute.TAG_TRI)
        if int(r[0]) < brute.thr(p):
            assert {(a, b), (a, c), (b, c)} & considered


def test_eo_removes_no_more_than_union():
    g = gg.rmat(10, 16, seed=3)
    for p in (0.2, 0.5, 0.8):
        ku = oracle.compress(g, "tr_random", p, 4)[1].size
        ke = oracle.compress(g, "tr_eo", p, 4)[1].size
        assert ke >= ku


# --------------------------------------------------------------------------
# per-edge union query agrees with the whole-graph kernels
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kern", ["tr_random", "tr_maxw", "tr_p2", "tr_mincount"])
def test_union_edge_query(kern):
    g = gg.attach_weights(gg.rmat(9, 16, seed=2))
    E = brute.edge_set(g)
    H = _edges_of(g.n, oracle.compress(g, kern, 0.5, 6))
    for (x, y) in sorted(E):
        assert oracle.tr_union_edge_deleted(g, kern, 0.5, 6, x, y) == ((x, y) not in H)
        assert oracle.tr_union_edge_deleted(g, kern, 0.5, 6, y, x) == ((x, y) not in H)


# --------------------------------------------------------------------------
# PageRank, KL divergence, connected components (Table 1; Sec. 5.2.3)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("g", [gg.cycle(7), gg.complete(6), gg.cycle(40)])
def test_pagerank_regular_graph_is_uniform(g):
    x, r = oracle.pagerank(g)
    assert np.allclose(x, 1.0 / g.n, rtol=1e-14, atol=0)


def _pr_fixed_point(g, d):
    # independent closed form: solve x = (1-d)/n 1 + d (A D^-1 x + (dangling.x)/n 1)
    n = g.n
    A = _scipy(g).toarray()
    deg = A.sum(0)
    M = np.zeros((n, n))
    for u in range(n):
        if deg[u] > 0:
            M[:, u] = A[:, u] / deg[u]
        else:
            M[:, u] = 1.0 / n
    return np.linalg.solve(np.eye(n) - d * M, np.full(n, (1 - d) / n))


@pytest.mark.parametrize("g", [gg.star(9), gg.disjoint_union(gg.path(5), gg.complete(4), gg.from_edge_list(3, [])), gg.rmat(6, 4, seed=3)])
def test_pagerank_fixed_point(g):
    x, r = oracle.pagerank(g, 0.85, 400)
    assert np.allclose(x, _pr_fixed_point(g, 0.85), rtol=1e-10, atol=0)
    assert abs(x.sum() - 1) < 1e-12


def test_pagerank_star_closed_form():
    # centre c, k leaves: x_c = (1-d)/n + d k x_l, x_l = (1-d)/n + d x_c / k
    k, d = 7, 0.85
    n = k + 1
    b = (1 - d) / n
    xc = (b + d * k * b) / (1 - d * d)
    xl = b + d * xc / k
    x, _ = oracle.pagerank(gg.star(k), d, 400)
    assert x[0] == pytest.approx(xc, rel=1e-12)
    assert np.allclose(x[1:], xl, rtol=1e-12)


def test_pagerank_residual_zero_on_power_of_two_cycle():
    # n and every degree powers of two: 1/n, the shares x/d and their sums are
    # exact in binary, and (1 - d)/n + d/n rounds to 1/n, so no update moves x
    x, r = oracle.pagerank(gg.cycle(16), 0.85, 50)
    assert np.all(x == 1.0 / 16) and r == 0.0


def test_pagerank_residual_star_two_iterations():
    # hand-worked: from x0 = 1/n, one update gives the centre
    # (1-d)/n + d k/n and each leaf (1-d)/n + d/(n k); the second update uses
    # those; the residual is the L1 norm of the second update's change
    k, d = 5, 0.85
    n = k + 1
    b = (1 - d) / n
    c1, l1 = b + d * k / n, b + d / (n * k)
    c2, l2 = b + d * k * l1, b + d * c1 / k
    want = abs(c2 - c1) + k * abs(l2 - l1)
    x, r = oracle.pagerank(gg.star(k), d, 2)
    assert x[0] == pytest.approx(c2, rel=1e-14) and np.allclose(x[1:], l2, rtol=1e-14)
    assert r == pytest.approx(want, rel=1e-12)
    # one update: the change from the uniform start
    _, r1 = oracle.pagerank(gg.star(k), d, 1)
    assert r1 == pytest.approx(abs(c1 - 1 / n) + k * abs(l1 - 1 / n), rel=1e-12)


def test_pagerank_residual_shrinks_by_damping():
    # the update is a contraction with factor d in L1: r_{t+1} <= d r_t
    g = gg.rmat(8, 8, seed=2)
    rs = [oracle.pagerank(g, 0.85, t)[1] for t in range(1, 12)]
    assert all(b <= 0.85 * a * (1 + 1e-9) for a, b in zip(rs, rs[1:]))


def test_pagerank_is_distribution_with_dangling():
    g = gg.rmat(12, 8, seed=4)  # has isolated vertices
    x, r = oracle.pagerank(g)
    assert abs(x.sum() - 1.0) < 1e-12
    assert np.all(x >= 0.15 / g.n * (1 - 1e-12))


def test_kl_identities():
    rng = np.random.default_rng(1)
    P = rng.random(100)
    Q = rng.random(100)
    assert oracle.kl_divergence(P, P) == 0.0
    assert oracle.kl_divergence(P, Q) == pytest.approx(entropy(P, Q, base=2), rel=1e-12)
    assert oracle.kl_divergence(P, Q) > 0
    # two-point closed form
    a, b = 0.3, 0.6
    want = a * math.log2(a / b) + (1 - a) * math.log2((1 - a) / (1 - b))
    assert oracle.kl_divergence([a, 1 - a], [b, 1 - b]) == pytest.approx(want, rel=1e-14)


def test_kl_grows_with_compression():
    # more compression -> larger KL (Sec. 7 discussion of Table 8), on average
    g = gg.rmat(11, 16, seed=7)
    P, _ = oracle.pagerank(g)
    kls = []
    for p in (0.9, 0.6, 0.3):
        off, col, _ = oracle.compress(g, "uniform", p, 3)
        Q, _ = oracle.pagerank((g.n, off, col, None))
        kls.append(oracle.kl_divergence(P, Q))
    assert kls[0] < kls[1] < kls[2]


@pytest.mark.parametrize("parts", [[gg.complete(4), gg.path(3), gg.cycle(5)], [gg.star(3)] * 5, [gg.from_edge_list(7, [])]])
def test_cc_disjoint_unions(parts):
    g = gg.disjoint_union(*parts)
    want = sum(connected_components(_scipy(p))[0] for p in parts)
    assert oracle.cc_count(g) == want


def test_cc_matches_scipy():
    g = gg.rmat(13, 4, seed=9)
    assert oracle.cc_count(g) == connected_components(_scipy(g))[0]


def test_divergence_of_identity_is_zero():
    g = gg.rmat(10, 8, seed=1)
    d = oracle.divergence(g, g)
    assert d["kl_bits"] == 0.0 and d["cc_g"] == d["cc_h"]



# --------------------------------------------------------------------------
# Triangle p-2-Reduction and Min-Count TR (Sec. 4.3 x = 2; "CT", Sec. 7)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,q,seed", [(16, 0.5, 1), (30, 0.35, 2), (48, 0.2, 3)])
@pytest.mark.parametrize("p", [0.4, 1.0])
def test_new_tr_kernels_match_brute_force(n, q, seed, p):
    g = gg.gnp(n, q, seed)
    E = brute.edge_set(g)
    assert _edges_of(n, oracle.compress(g, "tr_p2", p, seed)) == brute.tr_p2(n, E, p, seed)
    assert _edges_of(n, oracle.compress(g, "tr_mincount", p, seed)) == brute.tr_mincount(n, E, p, seed)
    assert _edges_of(n, oracle.compress(g, "tr_eo_mincount", p, seed)) == brute.tr_eo_mincount(n, E, p, seed)


def test_p2_single_triangle_keeps_one_edge():
    g = gg.complete(3)
    for s in range(1, 20):
        off, col, _ = oracle.compress(g, "tr_p2", 1.0, s)
        assert col.size == 2
        r = brute.draw(s, 0, 1, 2, brute.TAG_TRI)
        assert _edges_of(3, (off, col, None)) == {[(0, 1), (0, 2), (1, 2)][(int(r[1]) * 3) >> 32]}


def test_p2_on_disjoint_triangles():
    k = 500
    g = gg.disjoint_union(*[gg.complete(3)] * k)
    off, col, _ = oracle.compress(g, "tr_p2", 1.0, 9)
    assert col.size == 2 * k  # one edge of every triangle left


def test_mincount_tie_and_choice():
    # K3: every edge lies in one triangle; ties go to the smallest pair {0,1}
    off, col, _ = oracle.compress(gg.complete(3), "tr_mincount", 1.0, 5)
    assert _edges_of(3, (off, col, None)) == {(0, 2), (1, 2)}
    # diamond: {1,2} lies in two triangles, so it is never the one deleted
    for s in range(1, 10):
        H = _edges_of(4, oracle.compress(gg.diamond(), "tr_mincount", 1.0, s))
        assert (1, 2) in H


def test_mincount_deletes_least_covered_edge():
    g = gg.rmat(9, 16, seed=4)
    E = brute.edge_set(g)
    cnt = brute.edge_triangle_counts(g.n, E)
    H = _edges_of(g.n, oracle.compress(g, "tr_mincount", 1.0, 2))
    for a, b, c in (tuple(int(v) for v in t) for t in oracle.triangle_list(g)):
        es = [(a, b), (a, c), (b, c)]
        gone = [e for e in es if e not in H]
        # the triangle's own choice is deleted (others may be deleted by other triangles)
        assert min(es, key=lambda e: (cnt[e], e)) in gone


def test_ct_is_edge_once_packing():
    # same accepted set as EO, so the same number of deletions; CC preserved
    g = gg.rmat(10, 16, seed=6)
    a = oracle.compress(g, "tr_eo", 0.5, 3)[1].size
    b = oracle.compress(g, "tr_eo_mincount", 0.5, 3)
    assert a == b[1].size
    Hm = sp.csr_matrix((np.ones(b[1].size), b[1].astype(np.int64), b[0]), shape=(g.n, g.n))
    assert connected_components(_scipy(g))[0] == connected_components(Hm)[0]


# --------------------------------------------------------------------------
# single-vertex kernel low_degree (Listing 1; Sec. 4.4)
# --------------------------------------------------------------------------
def _low_edges(res):
    k, off, col, _ = res
    return brute.edge_set_arrays(k, off, col)


@pytest.mark.parametrize("n,q,seed", [(20, 0.08, 1), (40, 0.05, 2), (60, 0.03, 3), (30, 0.3, 4)])
def test_low_degree_matches_brute_force(n, q, seed):
    g = gg.gnp(n, q, seed)
    k, E2 = brute.low_degree(n, brute.edge_set(g))
    res = oracle.low_degree(g)
    assert res[0] == k and _low_edges(res) == E2
    # new ids are increasing in the old ids and -1 exactly for degree <= 1
    deg = np.diff(g.numpy()[0])
    nid = res[3]
    assert np.array_equal(nid < 0, deg <= 1)
    kept = nid[nid >= 0]
    assert np.array_equal(kept, np.arange(k))


def test_low_degree_closed_forms():
    # a path loses its two ends and keeps a path of n - 2 vertices
    k, off, col, _ = oracle.low_degree(gg.path(10))
    assert k == 8 and col.size == 2 * 7
    # a star keeps only its centre, now isolated (one pass over input degrees)
    k, off, col, _ = oracle.low_degree(gg.star(9))
    assert k == 1 and col.size == 0
    # cycles and cliques are unchanged
    for g in (gg.cycle(11), gg.complete(6)):
        k, off, col, _ = oracle.low_degree(g)
        o, c, _ = g.numpy()
        assert k == g.n and np.array_equal(off, o) and np.array_equal(col, c)
    # isolated vertices and isolated edges vanish
    k, off, col, _ = oracle.low_degree(gg.disjoint_union(gg.from_edge_list(3, []), gg.path(2), gg.cycle(4)))
    assert k == 4 and col.size == 8


# --------------------------------------------------------------------------
# BFS critical edges (Sec. 5.3) and reordered neighbours A_REN (Sec. 5.2.2)
# --------------------------------------------------------------------------
def _hops(g, root):
    from scipy.sparse.csgraph import shortest_path
    d = shortest_path(_scipy(g), unweighted=True, indices=root)
    return np.where(np.isinf(d), -1, d).astype(np.int64)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_bfs_levels_match_scipy(seed):
    g = gg.rmat(10, 8, seed=seed)
    for root in (0, 5, g.n - 1):
        assert np.array_equal(oracle.bfs_levels(g, root), _hops(g, root))


@pytest.mark.parametrize("seed", [1, 2])
def test_critical_edges_brute_force(seed):
    g = gg.disjoint_union(gg.rmat(9, 8, seed=seed), gg.cycle(7))
    for root in (0, 3, g.n - 2):
        h = _hops(g, root)
        E = brute.edge_set(g)
        want = sum(1 for a, b in E if h[a] >= 0 and h[b] >= 0 and abs(h[a] - h[b]) == 1)
        assert oracle.critical_edges(g, root) == want


def test_critical_edges_closed_forms():
    assert oracle.critical_edges(gg.cycle(10), 0) == 10      # even cycle: every edge
    assert oracle.critical_edges(gg.cycle(11), 4) == 10      # odd cycle: all but the far edge
    assert oracle.critical_edges(gg.complete(7), 2) == 6     # clique: only the root's edges
    assert oracle.critical_edges(gg.path(9), 4) == 8         # a tree: every edge
    st = gg.star(6)
    assert oracle.critical_edges(st, 0) == st.m and oracle.critical_edges(st, st.n - 1) == st.m  # a tree
    # a second component is never reached
    assert oracle.critical_edges(gg.disjoint_union(gg.path(4), gg.complete(5)), 0) == 3


def test_reordered_neighbours():
    g = gg.rmat(10, 8, seed=3)
    rng = np.random.default_rng(1)
    x = rng.random(g.n, dtype=np.float32)
    y = rng.random(g.n, dtype=np.float32)
    E = brute.edge_set(g)
    assert oracle.reordered_neighbours(g, x, y) == brute.reordered(E, x, y)
    assert oracle.reordered_neighbours(g, x, x) == 0
    # reversing the order flips every edge whose endpoints differ in score
    differ = sum(1 for a, b in E if x[a] != x[b])
    assert oracle.reordered_neighbours(g, x, -x) == differ
    # a tie on one side and an order on the other counts as reordered
    assert oracle.reordered_neighbours(g, np.zeros(g.n, np.float32), x) == differ


def test_vertex_triangle_counts():
    g = gg.gnp(40, 0.3, 7)
    t = oracle.vertex_triangle_counts(g)
    want = np.zeros(g.n, dtype=np.int64)
    for a, b, c in brute.triangles(g.n, brute.edge_set(g)):
        want[[a, b, c]] += 1
    assert np.array_equal(t, want)
    assert t.sum() == 3 * oracle.triangle_count(g)
    assert np.all(oracle.vertex_triangle_counts(gg.complete(7)) == 15)  # C(6,2)


def test_reordered_neighbours_integer_scores():
    g = gg.rmat(9, 8, seed=2)
    x = oracle.vertex_triangle_counts(g)
    h = oracle.compress(g, "tr_random", 0.5, 1)
    y = oracle.vertex_triangle_counts((g.n, h[0], h[1], None))
    E = brute.edge_set(g)
    assert oracle.reordered_neighbours(g, x, y) == brute.reordered(E, x, y)
    assert oracle.reordered_neighbours(g, x, x) == 0
