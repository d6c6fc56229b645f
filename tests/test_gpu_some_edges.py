"""GPU tests of sc_some_edges (s_hat at listed CSR entries only, the source loop
of Algorithm 2 restricted to their endpoints): each value equals the one
sc_all_edges gives at that entry, bit for bit, for the policies and modes
whose per-source work does not depend on the block (TGT with every length
policy, windowed blocks, TGT+ with the per-source switch)."""
import numpy as np
import pytest

import graphgen as gg
from oracle import series

pytestmark = pytest.mark.gpu


def _graph(g):
    from paper_2305_16086_gb300 import Graph

    return Graph(g.row_ptr, g.col_idx)


def _pick(g, count, seed):
    rng = np.random.default_rng(seed)
    return rng.choice(g.nnz, size=count, replace=True).astype(np.int64)


@pytest.mark.parametrize("kw", [dict(policy="global", precision="fp32"), dict(policy="per_edge", precision="fp64"),
                                dict(policy="global", precision="bf16", block_width=64),
                                dict(policy="fixed", ell_fixed=8, precision="fp32", estimator="end_corrected"),
                                dict(mode="tgt_plus", policy="global", precision="fp64", switch="per_source",
                                     seed=3)])
def test_equals_all_edges_at_the_listed_entries(cuda_lib, kw):
    from paper_2305_16086_gb300 import binding

    g = gg.barabasi_albert(3000, 5, 17)
    ent = _pick(g, 300, 1)
    with _graph(g) as G:
        full, _, _ = G.all_edges(eps=2e-3, **kw)
        part, rep = binding.some_edges(G, ent, eps=2e-3, **kw)
    assert np.array_equal(part, full[ent])
    assert rep["foster_sum"] == pytest.approx(part.sum(), rel=1e-12)
    assert rep["source_hops"] < 0.5 * g.n * rep["ell_max_source"]  # only the listed entries' endpoints ran


def test_learned_policy(cuda_lib):
    from paper_2305_16086_gb300 import binding

    t = gg.barabasi_albert(2000, 6, 5)
    g = gg.barabasi_albert(2500, 6, 6)
    with _graph(t) as Gt:
        Gt.estimate_lambda()
        init = np.random.default_rng(1).normal(0.0, 0.2, binding.MLP_PARAMS).astype(np.float32)
        model, _ = binding.mlp_train([Gt], init, epochs=100, lr=1e-2, eps=1e-3, precision="fp32")
    ent = _pick(g, 200, 2)
    with _graph(g) as G:
        G.estimate_lambda()
        binding.mlp_load(G, model)
        full, _, _ = G.all_edges(eps=1e-3, policy="learned", precision="fp32")
        part, _ = binding.some_edges(G, ent, eps=1e-3, policy="learned", precision="fp32")
    assert np.array_equal(part, full[ent])


def test_windowed_lattice_and_device_output(cuda_lib):
    import torch

    from paper_2305_16086_gb300 import binding

    g = gg.perturbed_grid(60, 70, 0.05, 3)
    ent = _pick(g, 150, 3)
    out = torch.empty(ent.size, dtype=torch.float64, device="cuda")
    with _graph(g) as G:
        kw = dict(policy="fixed", ell_fixed=31, precision="fp64", estimator="end_corrected", windows=True)
        full, _, rf = G.all_edges(**kw)
        binding.some_edges(G, ent, out=out, **kw)
        _, rp = binding.some_edges(G, ent, **kw)
    assert rf["windowed"] == 1 and rp["windowed"] == 1
    assert np.array_equal(out.cpu().numpy(), full[ent])
    ref, _ = series.series_entries(g.n, g.row_ptr, g.col_idx, 31, end_corrected=True)
    assert np.max(np.abs(out.cpu().numpy() - ref[ent])) < 1e-12


def test_rejects_entries_out_of_range(cuda_lib):
    from paper_2305_16086_gb300 import ScError, binding

    g = gg.barabasi_albert(300, 3, 1)
    with _graph(g) as G:
        for bad in ([g.nnz], [-1], []):
            with pytest.raises(ScError) as ei:
                binding.some_edges(G, np.asarray(bad, dtype=np.int64), policy="fixed", ell_fixed=3)
            assert ei.value.name == "SC_ERR_INVALID_ARG"
