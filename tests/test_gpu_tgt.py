"""GPU parity of the TGT path (Algorithm 2) through the C ABI against the oracle.

Tolerances:
  * FP64 probability blocks vs the FP64 series oracle at the same tau: 1e-12
    (only summation order differs; each p carries O(l u) relative error,
    u = 2^-53, and s_hat sums at most 2 (tau + 1) terms of magnitude <= 1).
  * FP32 blocks with FP64 accumulation: 2e-6 absolute on s_hat (each stored p
    has relative error <= (l + 1) 2^-24 plus the chunked summation's).
  * BF16 blocks: 3e-2 absolute on s_hat (reported variant).
  * Any precision vs the exact resistance (O1): the method's eps (Thm. 3.2).
  * Integer outputs (tau per entry, structural flags): exact.
"""
import numpy as np
import pytest

import graphgen as gg
from oracle import exact, series, truncation

pytestmark = pytest.mark.gpu

TOL64, TOL32, TOLBF16 = 1e-12, 2e-6, 3e-2


def _graph(cuda_lib, g, **kw):
    from paper_2305_16086_gb300 import Graph

    return Graph(g.row_ptr, g.col_idx, **kw)


# --------------------------------------------------------------------------- ingest
def _expect_status(g_rp, g_ci, name, **kw):
    from paper_2305_16086_gb300 import Graph, ScError

    with pytest.raises(ScError) as ei:
        Graph(np.asarray(g_rp, np.int32), np.asarray(g_ci, np.int32), **kw)
    assert ei.value.name == name, str(ei.value)


def test_create_rejects_malformed_csr(cuda_lib):
    # path 0-1-2 is rp [0,1,3,4], ci [1,0,2,1]
    _expect_status([0, 3, 1, 4], [1, 0, 2, 1], "SC_ERR_BAD_CSR")          # row_ptr decreasing
    _expect_status([0, 1, 3, 5], [1, 0, 2, 1], "SC_ERR_BAD_CSR")          # row_ptr[n] != nnz
    _expect_status([0, 1, 3, 4], [1, 0, 7, 1], "SC_ERR_BAD_CSR")          # column out of range
    _expect_status([0, 1, 3, 4], [1, 2, 0, 1], "SC_ERR_BAD_CSR")          # row not sorted
    _expect_status([0, 2, 4, 5], [0, 1, 0, 2, 1], "SC_ERR_SELF_LOOP")
    _expect_status([0, 2, 4, 5], [1, 1, 0, 2, 1], "SC_ERR_DUPLICATE_EDGE")
    _expect_status([0, 1, 3, 3], [1, 0, 2], "SC_ERR_ISOLATED_NODE")
    _expect_status([0, 1, 2, 4], [1, 0, 0, 1], "SC_ERR_NOT_SYMMETRIC")
    g = gg.from_edges(6, [0, 1, 3, 4], [1, 2, 4, 5])
    _expect_status(g.row_ptr, g.col_idx, "SC_ERR_DISCONNECTED")
    g = gg.cycle(6)
    _expect_status(g.row_ptr, g.col_idx, "SC_ERR_BIPARTITE", reject_bipartite=True)


@pytest.mark.parametrize("maker,bip", [(lambda: gg.cycle(8), 1), (lambda: gg.cycle(7), 0),
                                       (lambda: gg.grid(5, 7), 1), (lambda: gg.random_tree(50, 1), 1),
                                       (lambda: gg.petersen(), 0), (lambda: gg.barabasi_albert(500, 3, 0), 0)])
def test_info(cuda_lib, maker, bip):
    g = maker()
    with _graph(cuda_lib, g) as G:
        info = G.info()
    assert info["n"] == g.n and info["nnz"] == g.nnz and info["m"] == g.m
    assert info["min_degree"] == g.degree.min() and info["max_degree"] == g.degree.max()
    assert info["bipartite"] == bip
    # BFS depth from node 0 = eccentricity of node 0
    import scipy.sparse as sp
    from scipy.sparse.csgraph import shortest_path

    a = sp.csr_matrix((np.ones(g.nnz), g.col_idx, g.row_ptr), shape=(g.n, g.n))
    ecc = int(shortest_path(a, unweighted=True, indices=[0]).max())
    assert info["diameter_lb"] == ecc


def test_device_pointer_input(cuda_lib):
    import torch

    g = gg.tree_plus_gnp(300, 6.0, 2)
    from paper_2305_16086_gb300 import Graph

    with Graph(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda()) as G:
        s, _, _ = G.all_edges(policy="fixed", ell_fixed=5, precision="fp64")
    ref, _ = series.series_entries(g.n, g.row_ptr, g.col_idx, 5)
    assert np.max(np.abs(s - ref)) < TOL64


# --------------------------------------------------------------------------- lambda / tau
LAMBDA_GRAPHS = [
    lambda: gg.tree_plus_gnp(2000, 10.0, 0), lambda: gg.barabasi_albert(3000, 4, 1),
    lambda: gg.petersen(), lambda: gg.cycle(9), lambda: gg.complete(12),
    lambda: gg.perturbed_grid(20, 20, 0.05, 3), lambda: gg.gnp_lcc(1500, 6.0, 2),
]


@pytest.mark.parametrize("maker", LAMBDA_GRAPHS)
def test_lambda_matches_oracle(cuda_lib, maker):
    g = maker()
    lp, lm, _ = truncation.spectrum_extremes(g.n, g.row_ptr, g.col_idx)
    with _graph(cuda_lib, g) as G:
        bip = G.info()["bipartite"]
        lam = G.estimate_lambda()
        tight = G.estimate_lambda(tol=1e-10, max_iter=min(g.n, 2500))
    want_minus = -lp if bip else lm  # bipartite: the -1 mode is deflated; the spectrum is symmetric
    # default tolerance: Ritz values lie inside the spectrum, within their residual of it, and
    # lambda_star (with the residual margin) is at least the true value
    assert lam["converged"] == 1
    assert lp - lam["residual_plus"] - 1e-12 <= lam["lambda_plus"] <= lp + 1e-10
    assert want_minus - 1e-10 <= lam["lambda_minus"] <= want_minus + lam["residual_minus"] + 1e-12
    assert lam["lambda_star"] >= max(abs(lp), abs(want_minus)) - 1e-12
    # tight tolerance: the extremes themselves
    assert tight["converged"] == 1
    assert abs(tight["lambda_plus"] - lp) < 1e-9 and abs(tight["lambda_minus"] - want_minus) < 1e-9


@pytest.mark.parametrize("eps", [1e-2, 1e-3])
@pytest.mark.parametrize("maker", [lambda: gg.tree_plus_gnp(2000, 10.0, 0), lambda: gg.barabasi_albert(3000, 4, 1)])
def test_truncation_matches_oracle(cuda_lib, maker, eps):
    g = maker()
    with _graph(cuda_lib, g) as G:
        lam = G.estimate_lambda()
        ell, per_src, per_entry = G.truncation_length(eps)
    tau = truncation.tau_entries(g.n, g.row_ptr, g.col_idx, eps, lam["lambda_star"])
    diff = np.flatnonzero(tau != per_entry)
    if diff.size:  # only a last-ulp difference of log() at an exact integer boundary may flip a length
        d = g.degree
        rows = g.entry_rows()
        f = truncation.f_edge(d[rows[diff]], d[g.col_idx[diff]], eps, lam["lambda_star"])
        x = 1.0 / d[rows[diff]] + 1.0 / d[g.col_idx[diff]] - 2.0 / (d[rows[diff]] * d[g.col_idx[diff]])
        raw = np.log(x / (eps * (1 - lam["lambda_star"] ** 2))) / np.log(1 / lam["lambda_star"]) - 1
        assert np.all(np.abs(raw - np.round(raw)) < 1e-9), (diff.size, f)
    assert ell == int(per_entry.max()) == int(per_src.max())
    assert np.array_equal(per_src, truncation.tau_per_source(g.n, g.row_ptr, per_entry))


# --------------------------------------------------------------------------- the series
SERIES_GRAPHS = [
    lambda: gg.tree_plus_gnp(600, 8.0, 1),
    lambda: gg.barabasi_albert(900, 5, 3),
    lambda: gg.lollipop(9, 30),
    lambda: gg.perturbed_grid(13, 17, 0.05, 4),
    lambda: gg.complete(40),
]


@pytest.mark.parametrize("maker", SERIES_GRAPHS)
@pytest.mark.parametrize("tau", [1, 4, 9])
def test_fp64_series_matches_oracle(cuda_lib, maker, tau):
    g = maker()
    ref, _ = series.series_entries(g.n, g.row_ptr, g.col_idx, tau)
    with _graph(cuda_lib, g) as G:
        s, _, rep = G.all_edges(policy="fixed", ell_fixed=tau, precision="fp64")
    assert np.max(np.abs(s - ref)) < TOL64
    rev = series.reverse_entries(g.n, g.row_ptr, g.col_idx)
    assert np.array_equal(s, s[rev])  # both directions bitwise equal
    assert abs(rep["foster_sum"] - 0.5 * ref.sum()) < 1e-9


@pytest.mark.parametrize("B,vpl,heavy,slices", [(32, 1, 128, 0), (32, 2, 4, 1), (32, 4, 7, 2), (64, 1, 3, 0),
                                                (64, 2, 128, 1), (128, 2, 5, 0), (128, 4, 128, 3),
                                                (32, -1, 0, 0), (64, -1, 0, 2), (128, -1, 0, 1)])
def test_fp64_every_kernel_variant(cuda_lib, B, vpl, heavy, slices):
    g = gg.barabasi_albert(700, 6, 5)  # hubs above the small heavy thresholds; 700 % B != 0
    ref, _ = series.series_entries(g.n, g.row_ptr, g.col_idx, 7)
    with _graph(cuda_lib, g) as G:
        s, _, rep = G.all_edges(policy="fixed", ell_fixed=7, precision="fp64", block_width=B, rows_split=vpl,
                                heavy_threshold=heavy, max_slices=slices)
    assert rep["block_width"] == B and rep["rows_split"] == vpl
    assert np.max(np.abs(s - ref)) < TOL64
    if vpl == -1:  # the TMA-gather kernel sums in the same order as the SIMT kernel
        with _graph(cuda_lib, g) as G:
            s1, _, _ = G.all_edges(policy="fixed", ell_fixed=7, precision="fp64", block_width=B, rows_split=1 if B < 128 else 2)
        assert np.array_equal(s, s1)


@pytest.mark.parametrize("prec,tol", [("fp32", TOL32), ("bf16", TOLBF16)])
@pytest.mark.parametrize("B,vpl", [(32, 1), (64, 1), (64, 2), (128, 1), (128, 4), (32, -1), (64, -1), (128, -1)])
def test_low_precision_blocks(cuda_lib, prec, tol, B, vpl):
    g = gg.barabasi_albert(1100, 5, 7)
    ref, _ = series.series_entries(g.n, g.row_ptr, g.col_idx, 7)
    with _graph(cuda_lib, g) as G:
        s, _, _ = G.all_edges(policy="fixed", ell_fixed=7, precision=prec, block_width=B, rows_split=vpl,
                              heavy_threshold=16)
    err = np.max(np.abs(s - ref))
    assert err < tol, err


def test_bitwise_deterministic_and_independent_of_launch_shape(cuda_lib):
    g = gg.barabasi_albert(2000, 6, 11)
    outs = []
    with _graph(cuda_lib, g) as G:
        for B, vpl, heavy, sl in [(64, 1, 128, 0), (64, 1, 128, 0), (32, 4, 9, 1), (128, 1, 40, 2), (128, 2, 1000, 0),
                                  (64, -1, 0, 0), (32, -1, 0, 3), (128, -1, 0, 0), (64, 0, 0, 0)]:
            s, _, rep = G.all_edges(policy="fixed", ell_fixed=9, precision="fp32", block_width=B, rows_split=vpl,
                                    heavy_threshold=heavy, max_slices=sl)
            outs.append((s, rep["foster_sum"]))
    for s, f in outs[1:]:
        assert np.array_equal(s, outs[0][0]) and f == outs[0][1]


# --------------------------------------------------------------------------- eps guarantee
def test_config_small_tree_gnp_within_eps(cuda_lib):
    """n = 2,000 tree + G(n,p), avg degree 10, FP64, eps = 1e-3: every edge
    within eps of the exact value (dense Cholesky oracle), and a lower bound."""
    g = gg.tree_plus_gnp(2000, 10.0, 0)
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    with _graph(cuda_lib, g) as G:
        lam = G.estimate_lambda()
        for prec, pol in [("fp64", "global"), ("fp64", "per_edge"), ("fp32", "global"), ("fp32", "per_edge")]:
            s, _, rep = G.all_edges(eps=1e-3, policy=pol, precision=prec)
            err = s - r
            assert np.max(np.abs(err)) <= 1e-3, (prec, pol, np.max(np.abs(err)))
            if prec == "fp64":
                assert np.all(err <= 1e-12)  # odd truncation: a lower bound
            # the series oracle at the same lengths
            tau = truncation.tau_entries(g.n, g.row_ptr, g.col_idx, 1e-3, lam["lambda_star"])
            if pol == "global":
                tau = np.full_like(tau, tau.max())
            ref, _ = series.series_entries(g.n, g.row_ptr, g.col_idx, tau)
            assert np.max(np.abs(s - ref)) < (TOL64 if prec == "fp64" else TOL32)
            assert rep["ell_global"] == tau.max()
            assert abs(rep["foster_sum"] - 0.5 * s.sum()) < 1e-8
            assert (g.n - 1) - rep["foster_sum"] >= -1e-9  # lower bound on every edge


def test_end_corrected_bipartite_and_tail_bound(cuda_lib):
    g = gg.perturbed_grid(14, 15, 0.05, 6)
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    with _graph(cuda_lib, g) as G:
        lam = G.estimate_lambda()
        for tau in (9, 41):
            s, b, rep = G.all_edges(policy="fixed", ell_fixed=tau, precision="fp64", estimator="end_corrected")
            ref, q = series.series_entries(g.n, g.row_ptr, g.col_idx, tau, end_corrected=True)
            assert np.max(np.abs(s - ref)) < TOL64
            want_b = series.tail_bound(q, 1.0, lam["lambda_plus"] + lam["residual_plus"], True)
            assert np.max(np.abs(b - want_b) / np.maximum(want_b, 1e-300)) < 1e-9
            assert np.all(r - s >= -1e-12) and np.all(r - s <= b + 1e-12)
            assert abs(rep["max_tail_bound"] - b.max()) < 1e-15


def test_global_policy_rejects_bipartite(cuda_lib):
    from paper_2305_16086_gb300 import ScError

    g = gg.grid(6, 6)
    with _graph(cuda_lib, g) as G:
        with pytest.raises(ScError) as ei:
            G.all_edges(policy="global")
    assert ei.value.name == "SC_ERR_UNSUPPORTED"
