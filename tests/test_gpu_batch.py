"""GPU parity of the batched traversal (sc_batch_all_edges) over many
independent graphs of uneven size.

  * each graph's values equal, bit for bit, those of sc_all_edges on that
    graph alone (the batch changes which rows a launch visits, never the
    summation order);
  * against the FP64 series oracle at each graph's length: 1e-12 (FP64
    blocks), 2e-6 (FP32 blocks);
  * non-bipartite graphs at their own Eq. 6 length: within eps of the exact
    values; bipartite lattices take a given length (their Eq. 6 length does
    not exist);
  * per-graph reports (length, Foster sum) and the rejected requests.
"""
import math

import numpy as np
import pytest

import graphgen as gg
from oracle import exact, series

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 2e-6


def _mixed(count, nmin, nmax, seed):
    """The uneven-size recipe of the batched workload at a smaller size range:
    n log-uniform in [nmin, nmax]; G(n, 8/(n-1)), Barabasi-Albert m=5 and
    perturbed lattices in turn."""
    return gg.batch_graphs(count, nmin, nmax, base_seed=seed)


def _graphs(gs):
    from paper_2305_16086_gb300 import Graph

    return [Graph(g.row_ptr, g.col_idx) for g in gs]


def _close(Gs):
    for G in Gs:
        G.close()


def _lengths(gs, grid_ell):
    return [grid_ell if g.meta.get("bipartite") else 0 for g in gs]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_equals_single_graph_runs(cuda_lib, precision):
    from paper_2305_16086_gb300 import binding

    gs = _mixed(9, 150, 1200, 40)
    Gs = _graphs(gs)
    try:
        ells = _lengths(gs, 31)
        outs, reps = binding.batch_all_edges(Gs, ells, eps=1e-3, precision=precision, estimator="end_corrected")
        again, _ = binding.batch_all_edges(Gs, ells, eps=1e-3, precision=precision, estimator="end_corrected")
        for i, (g, G) in enumerate(zip(gs, Gs)):
            ell = reps[i]["ell_global"]
            s, _, rep = G.all_edges(policy="fixed", ell_fixed=ell, precision=precision, estimator="end_corrected")
            assert np.array_equal(outs[i], s), i
            assert np.array_equal(outs[i], again[i]), i
            assert reps[i]["foster_sum"] == pytest.approx(0.5 * np.sum(outs[i]), rel=1e-12)
            if g.meta.get("bipartite"):
                assert ell == 31
            else:
                ref_ell, _, _ = G.truncation_length(1e-3)
                assert ell == ref_ell
    finally:
        _close(Gs)


def test_batch_matches_oracle_and_eps(cuda_lib):
    from paper_2305_16086_gb300 import binding

    eps = 1e-3
    gs = _mixed(12, 200, 1500, 50)
    Gs = _graphs(gs)
    try:
        ells = _lengths(gs, 41)
        s64, reps = binding.batch_all_edges(Gs, ells, eps=eps, precision="fp64", estimator="end_corrected")
        s32, _ = binding.batch_all_edges(Gs, ells, eps=eps, precision="fp32", estimator="end_corrected")
    finally:
        _close(Gs)
    for i, g in enumerate(gs):
        ell = reps[i]["ell_global"]
        ref, _ = series.series_entries(g.n, g.row_ptr, g.col_idx, ell, end_corrected=True)
        assert np.max(np.abs(s64[i] - ref)) <= TOL64, i
        assert np.max(np.abs(s32[i] - ref)) <= TOL32, i
        if not g.meta.get("bipartite"):
            r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
            assert np.max(np.abs(s32[i] - r)) <= eps, i
            assert np.all(s64[i] <= r + 1e-12), i  # odd length: lower bound


def test_batch_uneven_sizes_sampled(cuda_lib):
    """The uneven-size recipe over a wider range (n up to 6000): sampled
    edges per graph against the series oracle, and the exact values by CG
    for the non-bipartite graphs."""
    from paper_2305_16086_gb300 import binding

    eps = 1e-3
    gs = _mixed(30, 1000, 6000, 60)
    Gs = _graphs(gs)
    try:
        ells = _lengths(gs, 201)
        s32, reps = binding.batch_all_edges(Gs, ells, eps=eps, precision="fp32", estimator="end_corrected")
    finally:
        _close(Gs)
    rng = np.random.default_rng(7)
    for i, g in enumerate(gs):
        k = rng.choice(g.nnz, 12, replace=False)
        rows = np.searchsorted(g.row_ptr, k, side="right") - 1
        src = np.unique(np.concatenate([rows, g.col_idx[k]]))
        ell = reps[i]["ell_global"]
        ref, _ = series.series_entries(g.n, g.row_ptr, g.col_idx, ell, sources=src, end_corrected=True)
        assert np.max(np.abs(s32[i][k] - ref[k])) <= TOL32, i
        if not g.meta.get("bipartite"):
            pairs = np.stack([rows, g.col_idx[k]], axis=1)
            r = exact.exact_cg(g.n, g.row_ptr, g.col_idx, pairs)
            assert np.max(np.abs(s32[i][k] - r)) <= eps, i


def test_batch_rejections(cuda_lib):
    from paper_2305_16086_gb300 import ScError, binding

    gs = [gg.barabasi_albert(300, 3, 1), gg.perturbed_grid(10, 12, 0.05, 2)]
    Gs = _graphs(gs)
    try:
        with pytest.raises(ScError) as ei:
            binding.batch_all_edges(Gs, None, eps=1e-3)  # the lattice has no Eq. 6 length
        assert ei.value.name == "SC_ERR_UNSUPPORTED"
        with pytest.raises(ScError) as ei:
            binding.batch_all_edges(Gs, [0, 21], eps=1e-3, mode="tgt_plus")
        assert ei.value.name == "SC_ERR_UNSUPPORTED"
        with pytest.raises(ScError) as ei:  # no model loaded
            binding.batch_all_edges(Gs, None, eps=1e-3, policy="learned", estimator="end_corrected", ell_cap=63)
        assert ei.value.name == "SC_ERR_INVALID_ARG"
        with pytest.raises(ScError) as ei:
            binding.batch_all_edges(Gs, [0, -3], eps=1e-3)
        assert ei.value.name == "SC_ERR_INVALID_ARG"
        outs, reps = binding.batch_all_edges(Gs, [0, 21], eps=1e-3, precision="fp64", estimator="end_corrected")
        assert reps[1]["ell_global"] == 21 and reps[0]["ell_global"] >= 1
    finally:
        _close(Gs)


def _mixed_model(eps):
    """One model for the three families, trained on one graph of each."""
    from paper_2305_16086_gb300 import Graph, binding

    ts = [gg.gnp_lcc(1500, 8.0, 31), gg.barabasi_albert(1500, 5, 32), gg.perturbed_grid(36, 40, 0.05, 33)]
    Gt = [Graph(t.row_ptr, t.col_idx) for t in ts]
    try:
        for G, t in zip(Gt, ts):
            G.estimate_lambda(allow_unconverged=bool(t.meta.get("bipartite")))
        init = np.random.default_rng(0).normal(0.0, 0.2, binding.MLP_PARAMS).astype(np.float32)
        model, _ = binding.mlp_train(Gt, init, epochs=300, lr=1e-2, eps=eps, precision="fp32", ell_cap=2047)
    finally:
        _close(Gt)
    return model


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_learned_batch_equals_single_runs(cuda_lib, precision):
    """The learned policy inside a batch: each graph's values, length report
    and certification flag equal those of sc_all_edges on that graph alone with
    the same model, bit for bit (an edge's length sequence depends only on its
    own graph's values); every graph within eps of the dense oracle."""
    from paper_2305_16086_gb300 import binding

    eps = 1e-3
    model = _mixed_model(eps)
    gs = _mixed(9, 1000, 2500, 70)
    Gs = _graphs(gs)
    kw = dict(eps=eps, precision=precision, estimator="end_corrected", policy="learned", ell_cap=2047,
              block_width=64, rows_split=1)
    try:
        for G in Gs:
            G.estimate_lambda(allow_unconverged=True)
            binding.mlp_load(G, model)
        outs, reps = binding.batch_all_edges(Gs, None, **kw)
        singles = [G.all_edges(**kw) for G in Gs]
    finally:
        _close(Gs)
    assert max(r["extension_rounds"] for _, _, r in singles) >= 1  # the check extended something
    assert reps[0]["extension_rounds"] == max(r["extension_rounds"] for _, _, r in singles)
    for i, (g, out, rep, (s1, _, r1)) in enumerate(zip(gs, outs, reps, singles)):
        assert np.array_equal(out, s1), i
        assert rep["ell_global"] == r1["ell_global"], i  # the cap
        assert (rep["ell_min_source"], rep["ell_max_source"]) == (r1["ell_min_source"], r1["ell_max_source"]), i
        assert rep["uncertified"] == r1["uncertified"] == (1 if g.meta.get("bipartite") else 0), i
        r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
        assert np.max(np.abs(out - r)) <= eps, (i, g.name)
