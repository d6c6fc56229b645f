"""GPU parity of TGT+ (Algorithm 4) through the C ABI against the oracle.

The walk tail uses the same counter-based Philox streams on both sides, so
with FP64 blocks the GPU and the oracle draw identical walks: the walk counts
(integers decided in FP64 on both sides) must agree exactly and s_hat up to
rounding (1e-10). Against the exact resistance the bar is eps (Theorem 4.4,
with probability at least 1 - delta).
"""
import numpy as np
import pytest

import graphgen as gg
from oracle import exact, series, tgtplus, truncation

pytestmark = pytest.mark.gpu


def _graph(g):
    from paper_2305_16086_gb300 import Graph

    return Graph(g.row_ptr, g.col_idx)


def _oracle_tgt_plus(g, eps, lam_star, tt, seed, gamma=10):
    tau = truncation.tau_entries(g.n, g.row_ptr, g.col_idx, eps / 2, lam_star)
    ghat = np.zeros(g.nnz)
    walks = 0
    for i in range(g.n):
        a, b = g.row_ptr[i], g.row_ptr[i + 1]
        gi, R, _ = tgtplus.tgt_plus_half(g.n, g.row_ptr, g.col_idx, i, tau[a:b], tt, eps, 1.0 / g.n, gamma, seed, g.m)
        ghat[a:b] = gi / g.degree[i]
        walks += int(R.sum())
    rev = series.reverse_entries(g.n, g.row_ptr, g.col_idx)
    return ghat + ghat[rev], walks, tau


def _oracle_switch(g, eps, lam_star, gamma=10):
    """First hop l (>= 1) at which Eq. 14, summed over all sources, holds."""
    tau = truncation.tau_entries(g.n, g.row_ptr, g.col_idx, eps / 2, lam_star)
    L = int(tau.max())
    cols = [np.eye(g.n)[:, i] for i in range(g.n)]
    P = np.zeros((g.n, g.n))
    for r in range(g.n):
        nb = g.col_idx[g.row_ptr[r]:g.row_ptr[r + 1]]
        P[r, nb] = 1.0 / len(nb)
    X = np.eye(g.n)
    for ell in range(1, L):
        X = P @ X  # column i = p_ell(., v_i)
        lhs = sum(tgtplus.frontier_volume(g.row_ptr, X[:, i]) for i in range(g.n))
        rhs = 0
        for i in range(g.n):
            p = X[:, i]
            for k in range(g.row_ptr[i], g.row_ptr[i + 1]):
                Lw = int(tau[k]) - ell
                if Lw > 0:
                    chi = tgtplus.calchi(g.row_ptr, g.col_idx, p, i, int(g.col_idx[k]), Lw, gamma)
                    rhs += tgtplus.walk_count(chi, g.degree[i], g.m, 1.0 / g.n, eps)
        if lhs > rhs:
            return ell
    return L


@pytest.mark.parametrize("seed", [3, 1234567890123])
def test_tgt_plus_fp64_matches_oracle_walk_for_walk(cuda_lib, seed):
    g = gg.tree_plus_gnp(160, 7.0, 5)
    eps = 0.05
    with _graph(g) as G:
        lam = G.estimate_lambda()
        s, _, rep = G.all_edges(eps=eps, mode="tgt_plus", policy="per_edge", precision="fp64", seed=seed,
                                switch="paper")
    assert rep["tt_min"] == rep["tt_max"]  # one launch holds every source of this graph
    tt = rep["tt_min"]
    assert tt == _oracle_switch(g, eps, lam["lambda_star"])  # Eq. 14, evaluated by the oracle
    ref, walks, tau = _oracle_tgt_plus(g, eps, lam["lambda_star"], tt, seed)
    if tt < tau.max():
        assert rep["walks"] == walks > 0
    assert np.max(np.abs(s - ref)) < 1e-10
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    assert np.max(np.abs(s - r)) <= eps


def test_tgt_plus_deterministic_per_seed(cuda_lib):
    g = gg.barabasi_albert(1500, 4, 2)
    with _graph(g) as G:
        kw = dict(eps=0.02, mode="tgt_plus", policy="per_edge", precision="fp32", switch="paper")
        a, _, ra = G.all_edges(seed=9, **kw)
        b, _, rb = G.all_edges(seed=9, **kw)
        c, _, rc = G.all_edges(seed=10, **kw)
    assert np.array_equal(a, b) and ra["walks"] == rb["walks"]
    assert not np.array_equal(a, c)
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    assert np.max(np.abs(a - r)) <= 0.02 and np.max(np.abs(c - r)) <= 0.02


@pytest.mark.parametrize("gamma", [0, 3, 16])
def test_tgt_plus_gamma_variants_within_eps(cuda_lib, gamma):
    g = gg.tree_plus_gnp(400, 8.0, 7)
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    with _graph(g) as G:
        s, _, rep = G.all_edges(eps=0.05, mode="tgt_plus", policy="per_edge", precision="fp64", gamma=gamma, seed=1,
                                switch="paper")
    assert np.max(np.abs(s - r)) <= 0.05


@pytest.mark.slow
def test_tgt_plus_ba_200k_sampled(cuda_lib):
    """Barabasi-Albert n = 200,000, m0 = 10, FP32 blocks, eps = 1e-3: sampled
    edges vs CG within eps, and the traversal stops before the full length."""
    g = gg.barabasi_albert(200_000, 10, 1)
    rng = np.random.default_rng(1)
    e = g.edges()
    pick = e[rng.choice(e.shape[0], size=120, replace=False)]
    k = exact.entry_of_edges(g.n, g.row_ptr, g.col_idx, pick)
    with _graph(g) as G:
        G.estimate_lambda()
        s, _, rep = G.all_edges(eps=1e-3, mode="tgt_plus", policy="per_edge", precision="fp32", seed=5)
    r = exact.exact_cg(g.n, g.row_ptr, g.col_idx, pick)
    assert np.max(np.abs(s[k] - r)) <= 1e-3
    assert rep["tt_max"] <= rep["ell_global"]


def test_tgt_plus_cost_rule_walks_replace_remaining_hops(cuda_lib):
    """With the cost rule the traversal may stop early; the result stays within eps."""
    g = gg.rmat(12, 16, seed=3)
    _, _, lam = truncation.spectrum_extremes(g.n, g.row_ptr, g.col_idx)
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx) if g.n <= 4000 else None
    with _graph(g) as G:
        s, _, rep = G.all_edges(eps=0.02, mode="tgt_plus", policy="per_edge", precision="fp32", seed=2)
    if r is not None:
        assert np.max(np.abs(s - r)) <= 0.02


@pytest.mark.parametrize("maker,kw", [
    (lambda: gg.barabasi_albert(3000, 5, 41), dict(policy="global", precision="fp32", switch="paper")),
    (lambda: gg.barabasi_albert(2600, 6, 42), dict(policy="per_edge", precision="fp64", switch="cost", block_width=32)),
    (lambda: gg.tree_plus_gnp(2200, 7.0, 43), dict(policy="global", precision="bf16", switch="per_source",
                                                   block_width=64)),
    (lambda: gg.rmat(12), dict(policy="global", precision="fp32", switch="paper", gamma=3)),
    (lambda: gg.rmat(11), dict(policy="global", precision="fp32", switch="paper", gamma=0)),
    # every column of K_n is one value off the source: thousands of ties at the threshold, so the
    # candidate buffer overflows and the column is scanned in full inside the kernel
    (lambda: gg.complete(2500), dict(policy="fixed", ell_fixed=5, precision="fp64", switch="paper")),
])
def test_threshold_topgamma_scan_equals_full_scan(cuda_lib, maker, kw):
    """The switch test's top-gamma candidates (Algorithm 3) from the entries at or
    above the gamma-th largest tile maximum give what the scan of every row
    gives: the same walk counts, switch hops and walks, bit for bit."""
    g = maker()
    with _graph(g) as G:
        base = dict(eps=5e-3, mode="tgt_plus", seed=9, **kw)
        s, _, rep = G.all_edges(**base)
        f, _, rep_f = G.all_edges(full_topgamma_scan=True, **base)
    assert rep["switch_tests"] > 0
    assert np.array_equal(s, f)
    for key in ("walks", "walk_steps", "tt_min", "tt_max", "switch_tests"):
        assert rep[key] == rep_f[key], key
