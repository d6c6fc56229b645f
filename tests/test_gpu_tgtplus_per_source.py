"""GPU parity of TGT+ with the per-source switch (SC_SWITCH_PER_SOURCE,
Algorithm 4's loop with Eq. 14 tested per source) against the oracle's
per-source TGT+ (oracle.tgtplus.switch_hop, tgt_plus_half). The walk streams
are keyed by (entry, walk, side, step), so with FP64 blocks the result equals
the oracle's walk for walk (1e-10); against the exact resistance the bar is
eps (Theorem 4.4).
"""
import numpy as np
import pytest

import graphgen as gg
from oracle import exact, series, tgtplus, truncation

pytestmark = pytest.mark.gpu


def _graph(g):
    from paper_2305_16086_gb300 import Graph

    return Graph(g.row_ptr, g.col_idx)


@pytest.mark.parametrize("seed", [3, 77])
def test_per_source_switch_matches_oracle_walk_for_walk(cuda_lib, seed):
    """SC_SWITCH_PER_SOURCE: each source switches at its own Eq. 14 hop
    (oracle: tgtplus.switch_hop) and draws its walks from its own column; the
    Philox streams are keyed by (entry, walk, side, step), so the FP64 result
    equals the oracle's walk for walk."""
    g = gg.tree_plus_gnp(160, 7.0, 5)
    eps = 0.05
    with _graph(g) as G:
        lam = G.estimate_lambda()
        s, _, rep = G.all_edges(eps=eps, mode="tgt_plus", policy="per_edge", precision="fp64", seed=seed,
                                switch="per_source")
    tau = truncation.tau_entries(g.n, g.row_ptr, g.col_idx, eps / 2, lam["lambda_star"])
    ghat = np.zeros(g.nnz)
    walks, steps, tts = 0, 0, []
    for i in range(g.n):
        a, b = g.row_ptr[i], g.row_ptr[i + 1]
        tt = tgtplus.switch_hop(g.n, g.row_ptr, g.col_idx, i, tau[a:b], eps, 1.0 / g.n, 10, g.m)
        gi, R, _ = tgtplus.tgt_plus_half(g.n, g.row_ptr, g.col_idx, i, tau[a:b], tt, eps, 1.0 / g.n, 10, seed, g.m)
        ghat[a:b] = gi / g.degree[i]
        walks += int(R.sum())
        steps += int(np.sum(2 * R * np.maximum(tau[a:b] - tt, 0)))  # both walks of a pair, tau_ij - tt steps each
        tts.append(tt)
    ref = ghat + ghat[series.reverse_entries(g.n, g.row_ptr, g.col_idx)]
    assert (rep["tt_min"], rep["tt_max"]) == (min(tts), max(tts))
    assert rep["walks"] == walks
    assert rep["walk_steps"] == steps
    assert np.max(np.abs(s - ref)) < 1e-10
    assert np.max(np.abs(s - exact.exact_dense(g.n, g.row_ptr, g.col_idx))) <= eps


def test_per_source_switch_within_eps_fp32(cuda_lib):
    g = gg.barabasi_albert(1500, 4, 2)
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    with _graph(g) as G:
        s, _, rep = G.all_edges(eps=0.02, mode="tgt_plus", policy="per_edge", precision="fp32", seed=4,
                                switch="per_source")
    assert np.max(np.abs(s - r)) <= 0.02
    assert rep["tt_min"] <= rep["tt_max"]
