"""GPU parity of the windowed blocks (the frontier of Algorithm 2 kept as an
interval of rows) against the full-graph blocks and the oracle.

  * windowed == full, bit for bit: the window only skips rows whose value is
    exactly zero and the summation order of a row does not depend on it;
  * on grid-numbered graphs the automatic choice windows the blocks and moves
    fewer bytes;
  * against the FP64 series oracle at the same length: 1e-12 (FP64 blocks),
    2e-6 (FP32 blocks);
  * a small perturbed lattice (bipartite, slow mixing): at the shortest odd
    length whose end-corrected series is within eps of the exact values
    (found with the oracle), the GPU result is within eps too.
"""
import numpy as np
import pytest

import graphgen as gg
from oracle import exact, series

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 2e-6


def _graph(g):
    from paper_2305_16086_gb300 import Graph

    return Graph(g.row_ptr, g.col_idx)


@pytest.mark.parametrize("maker,estimator", [
    (lambda: gg.perturbed_grid(40, 50, 0.05, 3), "end_corrected"),
    (lambda: gg.barabasi_albert(2000, 4, 5), "plain"),
    (lambda: gg.tree_plus_gnp(1500, 10.0, 2), "plain"),
])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_windowed_equals_full_bitwise(cuda_lib, maker, estimator, precision):
    g = maker()
    with _graph(g) as G:
        kw = dict(policy="fixed", ell_fixed=9, precision=precision, estimator=estimator, eps=1e-3)
        s_w, b_w, rep_w = G.all_edges(windows=True, heavy_threshold=64, **kw)
        s_f, b_f, rep_f = G.all_edges(windows=False, heavy_threshold=64, **kw)
    assert rep_w["windowed"] == 1 and rep_f["windowed"] == 0
    assert np.array_equal(s_w, s_f)
    if b_w is not None:
        assert np.array_equal(b_w, b_f)


@pytest.mark.parametrize("B", [32, 64, 128])
def test_windowed_block_widths_agree(cuda_lib, B):
    g = gg.perturbed_grid(60, 70, 0.05, 4)
    with _graph(g) as G:
        s, _, rep = G.all_edges(windows=True, policy="fixed", ell_fixed=11, precision="fp64",
                                estimator="end_corrected", block_width=B)
        s0, _, _ = G.all_edges(windows=False, policy="fixed", ell_fixed=11, precision="fp64",
                               estimator="end_corrected", block_width=32)
    assert rep["block_width"] == B
    assert np.array_equal(s, s0)


def test_grid_auto_windows_match_oracle(cuda_lib):
    g = gg.perturbed_grid(120, 150, 0.05, 6)  # bandwidth 150, n = 18000
    tau = 21
    rng = np.random.default_rng(1)
    k = rng.choice(g.nnz, 300, replace=False)
    rows = np.searchsorted(g.row_ptr, k, side="right") - 1
    src = np.unique(np.concatenate([rows, g.col_idx[k]]))
    ref, _ = series.series_entries(g.n, g.row_ptr, g.col_idx, tau, sources=src, end_corrected=True)
    with _graph(g) as G:
        s64, _, rep64 = G.all_edges(policy="fixed", ell_fixed=tau, precision="fp64", estimator="end_corrected")
        s32, _, rep32 = G.all_edges(policy="fixed", ell_fixed=tau, precision="fp32", estimator="end_corrected")
        _, _, rep_full = G.all_edges(policy="fixed", ell_fixed=tau, precision="fp32", estimator="end_corrected",
                                     windows=False)
    assert rep64["windowed"] == 1 and rep32["windowed"] == 1
    assert rep32["hop_bytes"] < 0.7 * rep_full["hop_bytes"]
    assert np.max(np.abs(s64[k] - ref[k])) <= TOL64
    assert np.max(np.abs(s32[k] - ref[k])) <= TOL32


def test_small_lattice_within_eps_at_empirical_length(cuda_lib):
    """Slow-mixing bipartite lattice: the a-priori length is unusable
    (lambda_plus near 1), so the length is the shortest odd one whose
    end-corrected series is within eps of the exact values."""
    g = gg.perturbed_grid(24, 30, 0.05, 7)
    eps = 1e-2
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)

    def ok(t):
        s, _ = series.series_entries(g.n, g.row_ptr, g.col_idx, t, end_corrected=True)
        return np.max(np.abs(s - r)) <= eps

    hi = 1
    while not ok(hi):  # doubling, then bisection over odd lengths
        hi = 2 * hi + 1
        assert hi < 20000
    lo = (hi - 1) // 2  # fails (or 0)
    while hi - lo > 2:
        mid = lo + ((hi - lo) // 2) | 1
        mid = mid if mid < hi else hi - 2
        if mid <= lo:
            break
        if ok(mid):
            hi = mid
        else:
            lo = mid
    ell = hi
    with _graph(g) as G:
        s32, _, rep = G.all_edges(policy="fixed", ell_fixed=ell, precision="fp32", estimator="end_corrected",
                                  windows=True)
    assert np.max(np.abs(s32 - r)) <= eps + TOL32
    assert np.all(s32 <= r + TOL32)  # odd length, end-corrected: still a lower bound


def test_learned_policy_windowed_equals_full(cuda_lib):
    from paper_2305_16086_gb300 import binding
    from oracle import learned

    train = gg.barabasi_albert(2500, 5, 21)
    test_g = gg.barabasi_albert(3000, 5, 22)
    init = np.random.default_rng(3).normal(0, 0.2, learned.NPARAM).astype(np.float32)
    with _graph(train) as Gt:
        Gt.estimate_lambda()
        model, _ = binding.mlp_train([Gt], init, epochs=200, lr=1e-2, eps=1e-3, precision="fp32")
    with _graph(test_g) as G:
        G.estimate_lambda()
        binding.mlp_load(G, model)
        s_w, _, rep_w = G.all_edges(policy="learned", precision="fp32", windows=True)
        s_f, _, rep_f = G.all_edges(policy="learned", precision="fp32", windows=False)
    assert rep_w["windowed"] == 1
    assert np.array_equal(s_w, s_f)
    # windowed blocks hold sources of one length, so no source runs extra hops
    assert rep_w["source_hops"] <= rep_f["source_hops"]


def test_windowed_bf16_from_hop_equals_full(cuda_lib):
    g = gg.perturbed_grid(50, 60, 0.05, 8)
    with _graph(g) as G:
        kw = dict(policy="fixed", ell_fixed=21, precision="bf16", bf16_from_hop=6, estimator="end_corrected")
        s_w, _, rep_w = G.all_edges(windows=True, **kw)
        s_f, _, rep_f = G.all_edges(windows=False, **kw)
    assert rep_w["windowed"] == 1 and rep_f["windowed"] == 0
    assert np.array_equal(s_w, s_f)
