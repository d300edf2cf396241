"""Brute-force restatements on tiny graphs, written independently of the oracle.

Triangles come from itertools over vertex triples, edges from a Python set,
so an indexing or merge mistake in the oracle's enumerator cannot hide here.
Random draws use the oracle's Philox only, which is itself pinned to the
published known-answer vectors.
"""
import itertools

import numpy as np

import oracle

TAG_EDGE = 0x45444745
TAG_TRI = 0x54524931


def edge_set(g):
    off, col, _ = g.numpy()
    E = set()
    for x in range(g.n):
        for y in col[off[x]:off[x + 1]]:
            E.add((min(x, int(y)), max(x, int(y))))
    return E


def edge_set_arrays(n, off, col):
    E = set()
    for x in range(n):
        for y in col[off[x]:off[x + 1]]:
            E.add((min(x, int(y)), max(x, int(y))))
    return E


def weights(g):
    off, col, w = g.numpy()
    W = {}
    for x in range(g.n):
        for i in range(off[x], off[x + 1]):
            y = int(col[i])
            W[(min(x, y), max(x, y))] = float(w[i])
    return W


def triangles(n, E):
    adj = [set() for _ in range(n)]
    for a, b in E:
        adj[a].add(b)
        adj[b].add(a)
    out = []
    for a, b, c in itertools.combinations(range(n), 3):
        if b in adj[a] and c in adj[a] and c in adj[b]:
            out.append((a, b, c))
    return out


def draw(seed, a, b, c, tag):
    return oracle.philox4x32_10([a, b, c, tag], [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF])


def thr(p):
    return min(2**32, int(np.floor(p * 2**32)))


def tr_union(n, E, p, seed, W=None):
    D = set()
    for a, b, c in triangles(n, E):
        r = draw(seed, a, b, c, TAG_TRI)
        if int(r[0]) >= thr(p):
            continue
        es = [(a, b), (a, c), (b, c)]
        if W is None:
            k = (int(r[1]) * 3) >> 32
        else:
            k = max(range(3), key=lambda i: (W[es[i]], es[i]))
        D.add(es[k])
    return E - D


def tr_eo(n, E, p, seed, W=None):
    sel = []
    for a, b, c in triangles(n, E):
        r = draw(seed, a, b, c, TAG_TRI)
        if int(r[0]) < thr(p):
            sel.append((int(r[2]), a, b, c, int(r[1])))
    sel.sort()
    considered, D, accepted = set(), set(), []
    for r2, a, b, c, r1 in sel:
        es = [(a, b), (a, c), (b, c)]
        if any(e in considered for e in es):
            continue
        considered.update(es)
        accepted.append((a, b, c))
        k = ((r1 * 3) >> 32) if W is None else max(range(3), key=lambda i: (W[es[i]], es[i]))
        D.add(es[k])
    return E - D, accepted


def edge_triangle_counts(n, E):
    cnt = {e: 0 for e in E}
    for a, b, c in triangles(n, E):
        for e in ((a, b), (a, c), (b, c)):
            cnt[e] += 1
    return cnt


def tr_p2(n, E, p, seed):
    """Each selected triangle keeps only the edge its draw r1 names."""
    D = set()
    for a, b, c in triangles(n, E):
        r = draw(seed, a, b, c, TAG_TRI)
        if int(r[0]) >= thr(p):
            continue
        es = [(a, b), (a, c), (b, c)]
        keep = (int(r[1]) * 3) >> 32
        D.update(e for i, e in enumerate(es) if i != keep)
    return E - D


def tr_mincount(n, E, p, seed):
    cnt = edge_triangle_counts(n, E)
    D = set()
    for a, b, c in triangles(n, E):
        r = draw(seed, a, b, c, TAG_TRI)
        if int(r[0]) < thr(p):
            es = [(a, b), (a, c), (b, c)]
            D.add(min(es, key=lambda e: (cnt[e], e)))
    return E - D


def tr_eo_mincount(n, E, p, seed):
    cnt = edge_triangle_counts(n, E)
    sel = []
    for a, b, c in triangles(n, E):
        r = draw(seed, a, b, c, TAG_TRI)
        if int(r[0]) < thr(p):
            sel.append((int(r[2]), a, b, c))
    sel.sort()
    considered, D = set(), set()
    for r2, a, b, c in sel:
        es = [(a, b), (a, c), (b, c)]
        if any(e in considered for e in es):
            continue
        considered.update(es)
        D.add(min(es, key=lambda e: (cnt[e], e)))
    return E - D


def low_degree(n, E):
    """Induced subgraph on the vertices of degree >= 2, renumbered by id."""
    deg = [0] * n
    for a, b in E:
        deg[a] += 1
        deg[b] += 1
    keep = [v for v in range(n) if deg[v] >= 2]
    new = {v: i for i, v in enumerate(keep)}
    return len(keep), {(new[a], new[b]) for a, b in E if a in new and b in new}


def reordered(E, x, y):
    sgn = lambda p, q: int(p > q) - int(p < q)
    return sum(1 for a, b in E if sgn(x[a], x[b]) != sgn(y[a], y[b]))
