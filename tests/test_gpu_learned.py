"""GPU parity of the learned per-source length (features, labels, MLP, policy).

  * features: float32 of the oracle's FP64 values (relative 1e-5);
  * certified lengths with FP64 blocks: equal to the oracle's, except where the
    bound sits within rounding of eps;
  * MLP loss and gradient (FP32) against the FP64 oracle (relative 1e-3);
  * training on the GPU lowers the loss like the oracle's training;
  * the learned policy: every edge within eps of the exact value and a
    truncated series at an odd length, and fewer source-hops than the global
    length (the gain the network brings).
"""
import numpy as np
import pytest

import graphgen as gg
from oracle import exact, learned, series, truncation

pytestmark = pytest.mark.gpu


def _graph(g):
    from paper_2305_16086_gb300 import Graph

    return Graph(g.row_ptr, g.col_idx)


def _csr(g):
    return g.n, g.row_ptr, g.col_idx


@pytest.mark.parametrize("maker", [lambda: gg.barabasi_albert(900, 5, 2), lambda: gg.tree_plus_gnp(700, 8.0, 4),
                                   lambda: gg.lollipop(8, 20)])
def test_features_match_oracle(cuda_lib, maker):
    from paper_2305_16086_gb300 import binding

    g = maker()
    with _graph(g) as G:
        lam = G.estimate_lambda()
        F = binding.source_features(G)
    ref = learned.features(*_csr(g))
    assert np.allclose(F, ref, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("maker", [lambda: gg.barabasi_albert(800, 5, 3), lambda: gg.gnp_lcc(600, 6.0, 1)])
@pytest.mark.parametrize("eps", [1e-2, 1e-3])
def test_certified_lengths_match_oracle(cuda_lib, maker, eps):
    from paper_2305_16086_gb300 import binding

    g = maker()
    with _graph(g) as G:
        lam = G.estimate_lambda()
        pe, ps, cap = binding.certified_lengths(G, eps, "fp64")
    ref = learned.certified_lengths(*_csr(g), eps, lam["lambda_star"], cap)
    diff = np.flatnonzero(pe != ref)
    if diff.size:  # only where the bound equals eps to rounding
        T = learned.hop_terms(*_csr(g), cap)
        rev = series.reverse_entries(*_csr(g))
        full = T + T[rev]
        f = lam["lambda_star"] ** 2 / (1 - lam["lambda_star"] ** 2)
        t = np.minimum(pe[diff], ref[diff])
        b = f * (full[diff, t - 1] + full[diff, t])
        assert np.all(np.abs(b - eps) <= 1e-12 * eps), diff.size
    assert np.array_equal(ps, learned.source_labels(g.n, g.row_ptr, pe))


def test_mlp_loss_and_gradient_match_oracle(cuda_lib):
    from paper_2305_16086_gb300 import binding

    rng = np.random.default_rng(5)
    N = 1000
    F = rng.normal(size=(N, 6)) * 2 + 1
    mu, sd = F.mean(axis=0), F.std(axis=0)
    theta = rng.normal(0, 0.3, learned.NPARAM)
    t = rng.normal(size=N)
    model = np.concatenate([theta, mu, sd]).astype(np.float32)
    loss, grad = binding.mlp_loss_grad(model, F.astype(np.float32), t.astype(np.float32))
    X = (F.astype(np.float32) - mu.astype(np.float32)) / sd.astype(np.float32)
    ref_loss, ref_grad = learned.loss_and_grad(theta.astype(np.float32).astype(np.float64), X.astype(np.float64), t.astype(np.float32))
    assert abs(loss - ref_loss) <= 1e-4 * abs(ref_loss)
    scale = np.max(np.abs(ref_grad))
    assert np.max(np.abs(grad - ref_grad)) <= 1e-3 * scale


def test_training_on_gpu_tracks_the_oracle(cuda_lib):
    from paper_2305_16086_gb300 import binding

    g = gg.barabasi_albert(1500, 5, 8)
    rng = np.random.default_rng(2)
    init = rng.normal(0, 0.2, learned.NPARAM).astype(np.float32)
    epochs = 200
    with _graph(g) as G:
        lam = G.estimate_lambda()
        model, curve = binding.mlp_train([G], init, epochs=epochs, lr=1e-2, eps=1e-3, precision="fp64")
        _, _, cap = binding.certified_lengths(G, 1e-3, "fp64")
    assert curve[-1] < 0.3 * curve[0]
    # the oracle's training from the same start on its own features and labels
    F = learned.features(*_csr(g))
    y = np.log(learned.source_labels(g.n, g.row_ptr, learned.certified_lengths(*_csr(g), 1e-3, lam["lambda_star"], cap)))
    mu, sd = learned.standardise(F)
    X = (F - mu) / sd
    theta = init.astype(np.float64)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    ref = []
    for t in range(1, epochs + 1):
        loss, gr = learned.loss_and_grad(theta, X, y)
        ref.append(loss)
        theta, m, v = learned.adam_step(theta, gr, m, v, t, lr=1e-2)
    assert abs(curve[0] - ref[0]) <= 1e-4 * ref[0]
    assert abs(curve[-1] - ref[-1]) <= 0.15 * ref[-1] + 1e-4


def test_learned_policy_within_eps_and_cheaper(cuda_lib):
    """Train on one Barabasi-Albert graph, apply to another of the family."""
    from paper_2305_16086_gb300 import binding

    train = gg.barabasi_albert(3000, 6, 11)
    test_g = gg.barabasi_albert(4000, 6, 12)
    eps = 1e-3
    rng = np.random.default_rng(0)
    init = rng.normal(0, 0.2, learned.NPARAM).astype(np.float32)
    with _graph(train) as Gt:
        Gt.estimate_lambda()
        model, curve = binding.mlp_train([Gt], init, epochs=400, lr=1e-2, eps=eps, precision="fp32")
    r = exact.exact_dense(*_csr(test_g))
    with _graph(test_g) as G:
        lam = G.estimate_lambda()
        binding.mlp_load(G, model)
        s_l, b_l, rep_l = G.all_edges(eps=eps, policy="learned", precision="fp64")
        s_g, _, rep_g = G.all_edges(eps=eps, policy="global", precision="fp64")
    assert np.max(np.abs(s_l - r)) <= eps
    assert np.all(s_l <= r + 1e-12)  # odd lengths: lower bounds
    # every edge certified by its bound or run to the a-priori length
    cap = rep_g["ell_global"]
    S = {t: series.series_entries(*_csr(test_g), t)[0] for t in range(1, cap + 1, 2)}
    matched = np.zeros(test_g.nnz, dtype=bool)
    for t, st in S.items():
        matched |= np.abs(s_l - st) < 1e-12
    assert matched.all()  # each value is the truncated series at some odd length
    assert rep_l["source_hops"] < rep_g["source_hops"]  # the gain: fewer hops than the global length
