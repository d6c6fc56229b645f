"""GPU tests of the learned length on bipartite graphs (lambda* = 1: no bound,
no a-priori length). The end-corrected series is accepted per edge by the
power-law tail estimate of the pair sums q(tau) = t_{tau+1} + t_{tau+2} and
extended (tau <- 2 tau + 1, at most ell_cap) where the estimate exceeds eps;
the run is labelled uncertified. With FP64 blocks the values and the rounds
equal the oracle's loop (oracle.learned.learned_bipartite) within 1e-10, the
labels equal oracle.learned.estimated_lengths, and a model trained on one
perturbed lattice keeps another within eps of the exact values with fewer
source-hops than the shortest global length that does.
"""
import numpy as np
import pytest

import graphgen as gg
from oracle import exact, learned, series

pytestmark = pytest.mark.gpu


def _graph(g):
    from paper_2305_16086_gb300 import Graph

    return Graph(g.row_ptr, g.col_idx)


def _csr(g):
    return g.n, g.row_ptr, g.col_idx


def _constant_model(L0):
    import math

    from paper_2305_16086_gb300 import binding

    m = np.zeros(binding.MLP_MODEL_FLOATS, dtype=np.float32)
    m[binding.MLP_PARAMS - 1] = math.log(L0 - 0.25)
    m[binding.MLP_PARAMS + binding.MLP_FEATURES:] = 1.0
    return m


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_estimated_lengths_match_the_oracle(cuda_lib, precision):
    from paper_2305_16086_gb300 import binding

    g = gg.perturbed_grid(24, 30, 0.05, 2)
    eps, cap = 1e-2, 61
    with _graph(g) as G:
        pe, ps = binding.estimated_lengths(G, eps, cap, precision)
    ref = learned.estimated_lengths(*_csr(g), eps, cap)
    if precision == "fp64":
        assert np.array_equal(pe, ref)
    else:  # an fp32 block moves an estimate near eps across it on a few entries only
        assert np.mean(pe != ref) < 0.01
    assert np.array_equal(ps, learned.source_labels(g.n, g.row_ptr, pe))


@pytest.mark.parametrize("windows", [False, True])
@pytest.mark.parametrize("L0", [5, 21])
def test_constant_model_matches_the_oracle_loop(cuda_lib, windows, L0):
    from paper_2305_16086_gb300 import binding

    g = gg.perturbed_grid(40, 50, 0.05, 7)
    eps, cap = 1e-2, 255
    with _graph(g) as G:
        G.estimate_lambda(allow_unconverged=True)
        binding.mlp_load(G, _constant_model(L0))
        s, est, rep = G.all_edges(eps=eps, policy="learned", precision="fp64", estimator="end_corrected",
                                  ell_cap=cap, windows=windows)
    ref, tau, rounds = learned.learned_bipartite(g.n, g.row_ptr, g.col_idx, np.full(g.n, L0), cap, eps)
    assert np.max(np.abs(s - ref)) < 1e-10
    assert rep["extension_rounds"] == rounds and rep["uncertified"] == 1
    assert rep["windowed"] == (1 if windows else 0)
    assert np.all((est <= eps) | (tau == cap))
    r = exact.exact_dense(*_csr(g))
    assert np.all(s <= r + 1e-12) and np.max(r - s) <= eps


def test_windowed_equals_full_bit_for_bit(cuda_lib):
    from paper_2305_16086_gb300 import binding

    g = gg.perturbed_grid(30, 90, 0.05, 4)
    with _graph(g) as G:
        G.estimate_lambda(allow_unconverged=True)
        binding.mlp_load(G, _constant_model(7))
        kw = dict(eps=1e-2, policy="learned", precision="fp32", estimator="end_corrected", ell_cap=127)
        s_w, _, rw = G.all_edges(windows=True, **kw)
        s_f, _, rf = G.all_edges(windows=False, **kw)
    assert rw["windowed"] == 1 and rf["windowed"] == 0
    assert np.array_equal(s_w, s_f)


def _empirical_length(g, r, eps, L):
    """The shortest odd global length whose end-corrected series is within eps
    of the exact values on every edge."""
    T = learned.hop_terms(*_csr(g), L)
    rev = series.reverse_entries(*_csr(g))
    full = T + T[rev]
    cs = np.cumsum(full, axis=1)
    for t in range(1, L - 1, 2):
        if np.max(r - (cs[:, t] + 0.5 * full[:, t + 1])) <= eps:
            return t
    raise AssertionError("no global length up to L")


def test_trained_model_within_eps_and_fewer_hops_than_the_global_length(cuda_lib):
    from paper_2305_16086_gb300 import binding

    train = gg.perturbed_grid(60, 60, 0.05, 11)
    test_g = gg.perturbed_grid(50, 80, 0.05, 12)
    eps, cap = 1e-2, 511
    init = np.random.default_rng(0).normal(0.0, 0.2, binding.MLP_PARAMS).astype(np.float32)
    with _graph(train) as Gt:
        Gt.estimate_lambda(allow_unconverged=True)
        model, curve = binding.mlp_train([Gt], init, epochs=300, lr=1e-2, eps=eps, precision="fp32", ell_cap=cap)
    assert curve[-1] < 0.5 * curve[0]
    W1 = model[:binding.MLP_PARAMS][:32 * 6].reshape(32, 6)
    assert np.all(W1[:, 2] == 0.0) and np.all(W1[:, 5] == 0.0)  # no triangles on a lattice: constant, ignored
    r = exact.exact_dense(*_csr(test_g))
    with _graph(test_g) as G:
        G.estimate_lambda(allow_unconverged=True)
        binding.mlp_load(G, model)
        s, _, rep = G.all_edges(eps=eps, policy="learned", precision="fp32", estimator="end_corrected",
                                ell_cap=cap)
    assert rep["uncertified"] == 1
    assert np.max(r - s) <= eps and np.all(s <= r + 1e-6)
    ell_emp = _empirical_length(test_g, r, eps, 600)
    assert rep["source_hops"] < test_g.n * (ell_emp + 2)


def test_refusals(cuda_lib):
    from paper_2305_16086_gb300 import ScError, binding

    g = gg.perturbed_grid(12, 14, 0.05, 1)
    with _graph(g) as G:
        G.estimate_lambda(allow_unconverged=True)
        binding.mlp_load(G, _constant_model(5))
        for kw, name in [(dict(estimator="plain", ell_cap=63), "SC_ERR_UNSUPPORTED"),
                         (dict(estimator="end_corrected"), "SC_ERR_INVALID_ARG"),
                         (dict(estimator="end_corrected", ell_cap=64), "SC_ERR_INVALID_ARG"),
                         (dict(estimator="end_corrected", ell_cap=63, mode="tgt_plus"), "SC_ERR_UNSUPPORTED")]:
            with pytest.raises(ScError) as ei:
                G.all_edges(eps=1e-2, policy="learned", **kw)
            assert ei.value.name == name, kw
    h = gg.barabasi_albert(300, 3, 2)
    with _graph(h) as H:
        with pytest.raises(ScError) as ei:
            binding.estimated_lengths(H, 1e-2, 61)
        assert ei.value.name == "SC_ERR_UNSUPPORTED"
