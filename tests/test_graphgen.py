"""The synthetic inputs are valid simple symmetric CSR graphs with the
requested shapes (R-MAT, Chung-Lu, 3-D random geometric)."""
import numpy as np
import pytest
import torch

import graphgen as gg


def _check_csr(g):
    off, col, w = g.numpy()
    assert off[0] == 0 and off[-1] == col.size and np.all(np.diff(off) >= 0)
    rows = np.repeat(np.arange(g.n), np.diff(off))
    assert np.all(col < g.n)
    assert not np.any(rows == col), "self-loop"
    key = rows.astype(np.int64) * g.n + col
    assert np.all(np.diff(key) > 0), "rows not strictly sorted / duplicates"
    rev = col.astype(np.int64) * g.n + rows
    assert np.array_equal(np.sort(rev), key), "not symmetric"
    if w is not None:
        order = np.argsort(rev)
        assert np.array_equal(w[order], w), "weights differ between arcs"


@pytest.mark.parametrize("scale,ef", [(8, 8), (12, 16)])
def test_rmat_valid(scale, ef):
    g = gg.rmat(scale, ef, seed=1)
    _check_csr(g)
    assert g.n == 2**scale and 0 < g.m <= ef * 2**scale


def test_rmat_deterministic_and_seeded():
    a, b, c = gg.rmat(10, 8, seed=1), gg.rmat(10, 8, seed=1), gg.rmat(10, 8, seed=2)
    assert torch.equal(a.col, b.col) and torch.equal(a.off, b.off)
    assert not (a.col.numel() == c.col.numel() and torch.equal(a.col, c.col))


def test_rmat_skew():
    # a = 0.57 concentrates edges: the max degree far exceeds the mean
    g = gg.rmat(14, 16, seed=1)
    deg = np.diff(g.numpy()[0])
    assert deg.max() > 20 * deg.mean()


def test_chung_lu_valid_power_law():
    g = gg.chung_lu(12, 2.1, 32.0, seed=1)
    _check_csr(g)
    deg = np.diff(g.numpy()[0])
    assert 10 < deg.mean() < 40 and deg.max() > 5 * deg.mean()


def test_rgg_valid_and_triangle_dense():
    g = gg.rgg3d(12, 48.0, seed=1)
    _check_csr(g)
    deg = np.diff(g.numpy()[0])
    assert 35 < deg.mean() < 60


def test_weights_symmetric_in_range():
    g = gg.attach_weights(gg.rmat(10, 8, seed=3), seed=5)
    _check_csr(g)
    w = g.w.numpy()
    assert np.all(w > 0) and np.all(w <= 1)
    k = w.astype(np.float64) * 2**24
    assert np.all(k == np.round(k))


def test_rmat_batch_equals_individual_graphs():
    scales, efs, seeds = [5, 8, 3, 7, 8], [4, 16, 8, 2, 32], [11, 12, 13, 14, 15]
    u, vbase, abase = gg.rmat_batch(scales, efs, seeds)
    _check_csr(u)
    for i, (s, e, sd) in enumerate(zip(scales, efs, seeds)):
        one = gg.rmat(s, e, seed=sd)
        mem = gg.batch_member(u, vbase, i, 1 << s)
        assert torch.equal(mem.off, one.off) and torch.equal(mem.col, one.col), i
        assert abase[i] == int(u.off[vbase[i]])


def test_structured_hub_generators():
    # the matched biclique: k*k + k/2 edges, left degree k + 1, right degree k
    g = gg.biclique_matched(10)
    off, col, _ = g.numpy()
    deg = np.diff(off)
    assert g.m == 100 + 5 and np.all(deg[:10] == 11) and np.all(deg[10:] == 10)
    # hubs over leaves: every middle vertex outranks the hubs
    h = gg.hubs_over_leaves(6, 2)
    off, col, _ = h.numpy()
    deg = np.diff(off)
    assert h.n == 6 + 2 + 36 and h.m == 12 + 36 + 3
    assert np.all(deg[:6] == 2 + 6 + 1) and np.all(deg[6:8] == 6) and np.all(deg[8:] == 1)

