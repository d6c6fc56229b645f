"""GPU test of sc_all_edges_noalloc, the entry point for callers that cannot
allocate device memory (a serving arena or a framework allocator that owns the
device budget, latency-critical paths where cudaMalloc/cudaFree would block).

It must give what sc_all_edges gives for the same options (fixed length, FP64
blocks of 32, plain estimator) and what the oracle's FP64 series gives at the
same length, call after call, although every call works in the same static
device array that keeps the previous call's contents. This file is named so
that pytest collects it after the other GPU suites.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu

TOL64 = 1e-12  # the FP64 tolerance of the other parity tests


def _noalloc(lib, g, ell, stream):
    import torch

    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    out = torch.full((g.nnz,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    st = lib.sc_all_edges_noalloc(g.n, g.nnz, ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(ci.data_ptr()),
                                  ell, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, lib.sc_last_error_detail().decode()
    return out.cpu().numpy()


def _reference(g, ell):
    from paper_2305_16086_gb300 import Graph

    with Graph(g.row_ptr, g.col_idx) as G:
        s, _, _ = G.all_edges(policy="fixed", ell_fixed=ell, precision="fp64", block_width=32)
    return s


def test_noalloc_matches_all_edges_on_consecutive_calls(cuda_lib):
    """Several calls in a row through the C ABI, each checked against both
    sc_all_edges (same options) and the oracle's FP64 series at the same length
    (Algorithm 2): stale scratch from the previous call must not leak in. The
    lengths reach every branch of the entry point: ell = 0 (no hop), 1 (the
    gather of X_1 alone), 2 (the last hop straight after the first), >= 3 (full
    hops); n = 700 and 901 leave a partial last block of 32 sources."""
    import torch

    from oracle import series

    stream = torch.cuda.current_stream()
    g_tree = gg.tree_plus_gnp(700, 8.0, 3)
    g_ba = gg.barabasi_albert(901, 4, 2)
    cases = [(g_tree, 7), (g_ba, 5), (g_tree, 1), (g_ba, 2), (g_tree, 7), (gg.perturbed_grid(9, 11, 0.05, 1), 0),
             (g_ba, 1), (g_tree, 2)]
    for g, ell in cases:
        got = _noalloc(cuda_lib, g, ell, stream)
        want = _reference(g, ell)
        assert np.max(np.abs(got - want)) <= TOL64
        exact_series, _ = series.series_entries(g.n, g.row_ptr, g.col_idx, ell)
        assert np.max(np.abs(got - exact_series)) <= TOL64


def test_noalloc_rejects_graphs_beyond_the_scratch_limit(cuda_lib):
    import torch

    from paper_2305_16086_gb300 import binding

    limit = 64 << 20
    n, nnz = 200_000, 4_000_000  # 524 n + 16 nnz > 64 MiB: rejected before any device work
    assert 524 * n + 16 * nnz > limit
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = cuda_lib.sc_all_edges_noalloc(n, nnz, ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()),
                                       5, ctypes.c_void_p(out.data_ptr()), None)
    assert binding.STATUS_NAMES[st] == "SC_ERR_INVALID_ARG"
    assert b"limit" in cuda_lib.sc_last_error_detail()


def test_noalloc_rejects_malformed_csr(cuda_lib):
    import torch

    from paper_2305_16086_gb300 import ScError, binding

    rp = torch.tensor([0, 1, 2, 4], dtype=torch.int32, device="cuda")
    ci = torch.tensor([1, 0, 0, 1], dtype=torch.int32, device="cuda")  # (2,0),(2,1) without reverses
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(ScError) as ei:
        binding.all_edges_noalloc(rp, ci, 3, out)
    assert ei.value.name == "SC_ERR_NOT_SYMMETRIC"
