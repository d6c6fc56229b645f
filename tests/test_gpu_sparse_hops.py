"""GPU tests of the hops a block computes only where they can be non-zero or
are read: hop 3 from the non-zero values of X_2 (k_hop_sparse) and hop L-1 on
the sources' two-hop balls (k_hop_ball, ahead of the sparse last hop). Both
keep the full hop's summation order, so sc_all_edges with SC_OPT_SPARSE_HOPS
must give bit for bit what it gives with every hop run in full, for every
precision, block width, lane split, heavy-row threshold and slice count; and
the FP64 result must match the oracle's series (Algorithm 2) at 1e-12.
"""
import numpy as np
import pytest

import graphgen as gg
from oracle import series

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _graph(g):
    from paper_2305_16086_gb300 import Graph

    return Graph(g.row_ptr, g.col_idx)


GRAPHS = [lambda: gg.barabasi_albert(2000, 6, 11), lambda: gg.tree_plus_gnp(900, 9.0, 4), lambda: gg.rmat(12),
          lambda: gg.perturbed_grid(23, 31, 0.05, 6)]


@pytest.mark.parametrize("maker", GRAPHS)
@pytest.mark.parametrize("ell", [3, 4, 5, 6, 7, 10])
def test_sparse_hops_equal_full_hops_fp32(cuda_lib, maker, ell):
    g = maker()
    with _graph(g) as G:
        kw = dict(policy="fixed", ell_fixed=ell, precision="fp32", windows=False, time_kernels=True)
        s, _, rep = G.all_edges(sparse_hops=True, **kw)
        d, _, rep_d = G.all_edges(**kw)
    assert np.array_equal(s, d)
    assert rep["foster_sum"] == rep_d["foster_sum"]
    kc = rep["kernel_classes"]
    assert (kc["sparse_hop"]["launches"] > 0) == (ell >= 5)
    assert (kc["ball_hop"]["launches"] > 0) == (ell >= 4)
    assert rep_d["kernel_classes"]["sparse_hop"]["launches"] == 0 and rep_d["kernel_classes"]["ball_hop"]["launches"] == 0
    # the full hops replaced: two fewer dense launches per block from L = 5 on
    assert rep["kernel_classes"]["dense_hop"]["launches"] < rep_d["kernel_classes"]["dense_hop"]["launches"] or ell < 4


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("B,vpl,heavy,slices", [(32, 1, 12, 0), (64, 2, 5, 2), (128, 4, 20, 0), (128, 2, 1000, 3),
                                                (64, -1, 0, 0)])
def test_every_width_split_and_heavy_threshold(cuda_lib, prec, B, vpl, heavy, slices):
    g = gg.barabasi_albert(1500, 7, 3)  # hubs above the small heavy thresholds; 1500 % B != 0
    with _graph(g) as G:
        kw = dict(policy="fixed", ell_fixed=7, precision=prec, block_width=B, rows_split=vpl, heavy_threshold=heavy,
                  max_slices=slices, bf16_from_hop=1)
        s, _, _ = G.all_edges(sparse_hops=True, **kw)
        d, _, _ = G.all_edges(**kw)
    assert np.array_equal(s, d)
    if prec == "fp64":
        ref, _ = series.series_entries(g.n, g.row_ptr, g.col_idx, 7)
        assert np.max(np.abs(s - ref)) < TOL64


def test_bf16_switch_hop_keeps_full_hops_around_it(cuda_lib):
    """With bf16 storage from hop 8 on, hop L - 1 = 8 changes storage and stays
    a full hop; hop 3 is still sparse."""
    g = gg.barabasi_albert(1200, 5, 8)
    with _graph(g) as G:
        kw = dict(policy="fixed", ell_fixed=9, precision="bf16", time_kernels=True)
        s, _, rep = G.all_edges(sparse_hops=True, **kw)
        d, _, _ = G.all_edges(**kw)
    assert np.array_equal(s, d)
    kc = rep["kernel_classes"]
    assert kc["sparse_hop"]["launches"] > 0 and kc["ball_hop"]["launches"] == 0


def test_learned_and_per_edge_policies(cuda_lib):
    """Per-source lengths (sources of one block run the longest of them) and
    the learned policy's records of hops tau - 1 and tau go through the same
    kernels."""
    from paper_2305_16086_gb300 import binding

    g = gg.barabasi_albert(3000, 6, 21)
    t = gg.barabasi_albert(2500, 6, 22)
    with _graph(t) as Gt:
        Gt.estimate_lambda()
        init = np.random.default_rng(0).normal(0.0, 0.2, binding.MLP_PARAMS).astype(np.float32)
        model, _ = binding.mlp_train([Gt], init, epochs=60, lr=1e-2, eps=1e-3, precision="fp32")
    with _graph(g) as G:
        G.estimate_lambda()
        binding.mlp_load(G, model)
        for policy in ("per_edge", "learned"):
            s, _, rep = G.all_edges(eps=1e-3, policy=policy, precision="fp32", sparse_hops=True)
            d, _, rep_d = G.all_edges(eps=1e-3, policy=policy, precision="fp32")
            assert np.array_equal(s, d), policy
            assert rep["source_hops"] == rep_d["source_hops"]


def test_tgt_plus_with_sparse_hop_3(cuda_lib):
    """TGT+ reads X_l in full at its switch tests: hop 3 may still come from
    X_2's non-zero values (it stores the full X_3), the ball hop is not used."""
    g = gg.barabasi_albert(2500, 5, 31)
    with _graph(g) as G:
        G.estimate_lambda()
        kw = dict(eps=2e-3, mode="tgt_plus", policy="global", precision="fp64", seed=5, time_kernels=True)
        s, _, rep = G.all_edges(sparse_hops=True, **kw)
        d, _, rep_d = G.all_edges(**kw)
    assert np.array_equal(s, d) and rep["walks"] == rep_d["walks"]
    assert rep["kernel_classes"]["ball_hop"]["launches"] == 0
