"""GPU tests of TGT+ at learned lengths (SC_MODE_TGT_PLUS with SC_ELL_LEARNED):
Algorithm 4's traversal and walks at the per-source lengths the MLP predicts,
each edge's truncation certified after the run by the one-even-hop bound
(lam*^(tau + 1 - l) / (1 - lam*) t_l(e) <= eps / 2) and extended where it
fails. With the per-source switch and FP64 blocks the result equals the
oracle's composition (oracle.tgtplus.tgt_plus_learned) walk for walk (1e-10);
every configuration is within eps of the exact values. The eigenvalue bound
is the oracle's, given to the library (sc_graph_set_lambda), so both sides
start from the same lambda*.
"""
import math

import numpy as np
import pytest

import graphgen as gg
from oracle import exact, tgtplus, truncation

pytestmark = pytest.mark.gpu


def _graph(g):
    from paper_2305_16086_gb300 import Graph

    return Graph(g.row_ptr, g.col_idx)


def _constant_model(L0):
    """A model whose output is log(L0 - 1/4) for every source: the predicted
    length is L0 (odd) on both sides, half a unit from any rounding boundary."""
    from paper_2305_16086_gb300 import binding

    m = np.zeros(binding.MLP_MODEL_FLOATS, dtype=np.float32)
    m[binding.MLP_PARAMS - 1] = math.log(L0 - 0.25)  # b3
    m[binding.MLP_PARAMS + binding.MLP_FEATURES:] = 1.0  # feature standard deviations
    return m


@pytest.mark.parametrize("L0,seed", [(1, 7), (3, 21)])
def test_matches_the_oracle_walk_for_walk(cuda_lib, L0, seed):
    from paper_2305_16086_gb300 import binding

    g = gg.tree_plus_gnp(180, 6.0, 9)
    eps = 0.05
    lp, lm, ls = truncation.spectrum_extremes(g.n, g.row_ptr, g.col_idx)
    cap = int(truncation.tau_entries(g.n, g.row_ptr, g.col_idx, eps / 2, ls).max())
    with _graph(g) as G:
        G.set_lambda(lp, lm, ls)
        binding.mlp_load(G, _constant_model(L0))
        assert np.all(binding.mlp_predict(G, cap) == L0)
        s, _, rep = G.all_edges(eps=eps, mode="tgt_plus", policy="learned", precision="fp64", switch="per_source",
                                seed=seed)
    ref, tau, tt, rounds, seen = tgtplus.tgt_plus_learned(g.n, g.row_ptr, g.col_idx, np.full(g.n, L0), cap, eps, ls,
                                                         1.0 / g.n, 10, seed, g.m)
    assert np.max(np.abs(s - ref)) < 1e-10
    assert rounds >= 1 and rep["extension_rounds"] == rounds
    assert (rep["tt_min"], rep["tt_max"]) == seen  # over every run, reruns included
    assert np.max(np.abs(s - exact.exact_dense(g.n, g.row_ptr, g.col_idx))) <= eps


def test_trained_model_fp32_within_eps_and_cheaper_than_eq6(cuda_lib):
    """A model trained on one Barabasi-Albert graph, applied to another with
    FP32 blocks and the cost switch rule: within eps, fewer source-hops than
    TGT+ at the lengths of Eq. 6 (eps / 2)."""
    from paper_2305_16086_gb300 import binding

    train = gg.barabasi_albert(3000, 6, 31)
    test_g = gg.barabasi_albert(4000, 6, 32)
    eps = 2e-3
    init = np.random.default_rng(0).normal(0.0, 0.2, binding.MLP_PARAMS).astype(np.float32)
    with _graph(train) as Gt:
        Gt.estimate_lambda()
        model, _ = binding.mlp_train([Gt], init, epochs=300, lr=1e-2, eps=eps / 2, precision="fp32")
    r = exact.exact_dense(test_g.n, test_g.row_ptr, test_g.col_idx)
    with _graph(test_g) as G:
        G.estimate_lambda()
        binding.mlp_load(G, model)
        s, _, rep = G.all_edges(eps=eps, mode="tgt_plus", policy="learned", precision="fp32", seed=3)
        s6, _, rep6 = G.all_edges(eps=eps, mode="tgt_plus", policy="global", precision="fp32", seed=3)
    assert np.max(np.abs(s - r)) <= eps and np.max(np.abs(s6 - r)) <= eps
    assert rep["walks"] < rep6["walks"]


def test_rmat_bf16_within_eps_on_sampled_edges(cuda_lib):
    """The composite of the R-MAT workload at scale 14: TGT+ walk tail, learned
    lengths, BF16 storage from hop 8 on; sampled edges against CG."""
    from paper_2305_16086_gb300 import binding

    g = gg.rmat(14)
    t = gg.rmat(13, seed=15)
    eps = 1e-3
    init = np.random.default_rng(1).normal(0.0, 0.2, binding.MLP_PARAMS).astype(np.float32)
    with _graph(t) as Gt:
        Gt.estimate_lambda()
        model, _ = binding.mlp_train([Gt], init, epochs=300, lr=1e-2, eps=eps / 2, precision="fp32")
    rng = np.random.default_rng(4)
    e = g.edges()
    pick = e[rng.choice(e.shape[0], size=300, replace=False)]
    k = exact.entry_of_edges(g.n, g.row_ptr, g.col_idx, pick)
    with _graph(g) as G:
        G.estimate_lambda()
        binding.mlp_load(G, model)
        s, _, rep = G.all_edges(eps=eps, mode="tgt_plus", policy="learned", precision="bf16", seed=5)
    r = exact.exact_cg(g.n, g.row_ptr, g.col_idx, pick)
    assert np.max(np.abs(s[k] - r)) <= eps
    assert rep["walks"] > 0 and rep["tt_min"] >= 1
