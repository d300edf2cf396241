"""The no-allocation uniform-sampling entry point, called through the C-ABI.

Some callers cannot let a library call cudaMalloc (their own allocator owns
the GPU's memory, or the memory was reserved up front), so the library offers
sg_compress_uniform_noalloc, which keeps its scratch in a fixed device array.
Its output must equal the regular sg_compress(SG_UNIFORM) output bit for bit,
and the oracle's, on calls in a row, because every call reuses the same
scratch array.  This file is collected last so that a failure here cannot
hide other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def _noalloc(sg, g_dev, p, seed, stream):
    n, nnz = g_dev.n, g_dev.nnz
    off_out = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    col_out = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
    cnt = ctypes.c_int64(-1)
    stream.wait_stream(torch.cuda.current_stream())  # inputs were written on the current stream
    st = sg.lib().sg_compress_uniform_noalloc(0, ctypes.c_void_p(stream.cuda_stream), n, nnz, g_dev.off.data_ptr(),
                                              g_dev.col.data_ptr(), float(p), seed, off_out.data_ptr(),
                                              col_out.data_ptr(), ctypes.byref(cnt))
    sg._check(st)
    return off_out.cpu().numpy(), col_out[:cnt.value].cpu().numpy().view(np.uint32)


def _regular(sg, ctx, g, p, seed):
    G = sg.Graph.from_csr(ctx, g)
    H = sg.compress(G, "uniform", p, seed)
    off, col, _ = H.download()
    H.free()
    G.free()
    return off, col


def test_noalloc_matches_regular_entry_point_and_oracle_twice_in_a_row():
    import paper_1912_08950_gb300 as sg

    ctx = sg.Context(0)
    stream = ctx.torch_stream
    big = gg.rmat(16, 16, seed=3).to("cuda")
    small = gg.rmat(12, 8, seed=4).to("cuda")
    # a larger call first, then a smaller one: stale scratch must not leak
    for g, p, seed in ((big, 0.5, 11), (small, 0.3, 12), (small, 0.3, 12)):
        got = _noalloc(sg, g, p, seed, stream)
        host = g.to("cpu")
        want = _regular(sg, ctx, host, p, seed)
        o_off, o_col, _ = oracle.compress(host, "uniform", p, seed)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
        assert np.array_equal(got[0], o_off) and np.array_equal(got[1], o_col)
    ctx.close()


def test_noalloc_keeps_the_callers_current_device():
    import paper_1912_08950_gb300 as sg

    g = gg.rmat(10, 8, seed=5).to("cuda")
    before = torch.cuda.current_device()
    _noalloc(sg, g, 0.5, 1, torch.cuda.Stream())
    assert torch.cuda.current_device() == before


def test_noalloc_rejects_oversized_and_malformed_input():
    import paper_1912_08950_gb300 as sg

    cnt = ctypes.c_int64()
    dummy = torch.zeros(2, dtype=torch.int64, device="cuda")
    st = sg.lib().sg_compress_uniform_noalloc(0, None, 1, (1 << 27) + 2, dummy.data_ptr(), dummy.data_ptr(), 0.5, 1,
                                              dummy.data_ptr(), dummy.data_ptr(), ctypes.byref(cnt))
    assert st == sg.SG_ERR_UNSUPPORTED
    assert b"134217728" in sg.lib().sg_last_error()
    # offsets whose last entry disagrees with nnz are refused before any launch
    off = torch.tensor([0, 1, 5], dtype=torch.int64, device="cuda")
    col = torch.tensor([1, 0], dtype=torch.int32, device="cuda")
    out_off = torch.empty(3, dtype=torch.int64, device="cuda")
    out_col = torch.empty(2, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    st = sg.lib().sg_compress_uniform_noalloc(0, None, 2, 2, off.data_ptr(), col.data_ptr(), 0.5, 1,
                                              out_off.data_ptr(), out_col.data_ptr(), ctypes.byref(cnt))
    assert st == sg.SG_ERR_INVALID_GRAPH
