"""The error contract on the GPU, with no fault: every failure here is a
bounded device-side wait that runs out, or a device error word that the
host reads after a stream sync.  After each error the context is used
again and must give the oracle's result."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import paper_1912_08950_gb300 as m

    return m


@pytest.mark.parametrize("kern", ["uniform", "spectral_avgdeg", "tr_random", "tr_eo"])
def test_scan_wait_runs_out_and_the_context_recovers(sg, kern):
    ctx = sg.Context(0)
    # about 3,450 chunks of 256 arcs: the chunk scan runs over four tiles of
    # 1024 chunks, and tile 1 waits on tile 0
    g = gg.rmat(15, 16, seed=3)
    G = sg.Graph.from_csr(ctx, g)
    ctx.set_scan_hold(4096)  # tile 0 never publishes; a wait gives up after 4096 polls
    with pytest.raises(sg.SgError) as ei:
        sg.compress(G, kern, 0.5, 1)
    assert ei.value.status == sg.SG_ERR_TIMEOUT
    assert b"gave up" in sg.lib().sg_last_error()
    ctx.set_scan_hold(0)
    H = sg.compress(G, kern, 0.5, 1)
    off, col, _ = H.download()
    o_off, o_col, _ = oracle.compress(g, kern, 0.5, 1)
    assert np.array_equal(off, o_off) and np.array_equal(col, o_col)
    H.free()
    G.free()
    ctx.close()


def _stash_overflow_graph():
    """Vertex 0 with 24 out-neighbours that all hash to slots 0 and 1 of its
    128-slot table under both cuckoo hash functions (multipliers 0x9E3779B1
    and 0x85EBCA77, slot = top 7 bits): two fit, the other 22 overflow the
    16-entry stash.  Each neighbour gets 30 private leaves, so that it ranks
    above vertex 0 in the degree order."""
    w = np.arange(1, 1 << 21, dtype=np.uint64)
    s1 = ((w * 0x9E3779B1) & 0xFFFFFFFF) >> 25
    s2 = ((w * 0x85EBCA77) & 0xFFFFFFFF) >> 25
    keys = [int(x) for x in w[(s1 < 2) & (s2 < 2)][:24]]
    base = max(keys) + 1
    edges = [(0, k) for k in keys]
    for i, k in enumerate(keys):
        edges += [(k, base + 30 * i + j) for j in range(30)]
    return gg.from_edge_list(base + 30 * len(keys), edges)


def test_cuckoo_stash_overflow_is_reported(sg):
    ctx = sg.Context(0)
    g = _stash_overflow_graph()
    G = sg.Graph.from_csr(ctx, g)
    with pytest.raises(sg.SgError) as ei:
        sg.triangle_count(G)
    assert ei.value.status == sg.SG_ERR_CUDA
    assert b"stash" in sg.lib().sg_last_error()
    G.free()
    # the context keeps working
    k = gg.complete(7)
    K = sg.Graph.from_csr(ctx, k)
    assert sg.triangle_count(K) == 35
    H = sg.compress(K, "tr_random", 1.0, 2)
    off, col, _ = H.download()
    o_off, o_col, _ = oracle.compress(k, "tr_random", 1.0, 2)
    assert np.array_equal(off, o_off) and np.array_equal(col, o_col)
    H.free()
    K.free()
    ctx.close()
