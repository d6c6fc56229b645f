"""Pins for the learned-length oracle: features, certified lengths, MLP and Adam.

  * features against their definitions on named graphs, against P^2 and P^3,
    and unchanged on two disjoint copies of a graph (no dependence on size);
  * per-hop terms against the series oracle and exact matrix powers;
  * certified lengths: the bound holds at tau_e, fails at tau_e - 2, and the
    truncated series at tau_e is within eps of the exact value;
  * the MLP gradient against central finite differences; Adam's first step
    against its closed form;
  * the bipartite tail estimate against brute-force power-law sums, a
    geometric tail, its special cases and the exact remainder on a lattice;
    its labels by two routes; its extension loop within eps.
"""
import numpy as np
import pytest

import graphgen as gg
from oracle import exact, learned, series, truncation


def _P(g):
    P = np.zeros((g.n, g.n))
    for r in range(g.n):
        nb = g.col_idx[g.row_ptr[r]:g.row_ptr[r + 1]]
        P[r, nb] = 1.0 / len(nb)
    return P


def test_features_on_named_graphs():
    F = learned.features(*_csr(gg.complete(6)))
    assert np.allclose(F[:, 2], 1.0) and np.allclose(F[:, 0], np.log(5)) and np.allclose(F[:, 1], np.log(5))
    assert np.allclose(F[:, 3], 0.0)  # regular: the neighbours' mean degree is the mean degree
    assert np.allclose(F[:, 5], 4 / 25)  # K6: from i, 5 first steps, 4 closing second steps, 1/5 each
    F = learned.features(*_csr(gg.star(5)))
    assert F[0, 2] == 0.0 and np.allclose(F[1:, 2], 0.0)  # no triangles; leaves have d = 1
    # mean degree 10/6: the center's neighbours have degree 1, a leaf's neighbour degree 5
    assert np.isclose(F[0, 3], np.log(1 / (10 / 6))) and np.allclose(F[1:, 3], np.log(5 / (10 / 6)))
    assert np.allclose(F[:, 5], 0.0)  # a tree has no 3-cycles
    g = gg.barbell(4, 1)  # K4 - K4 joined by one edge: corner nodes lose clustering
    F = learned.features(*_csr(g))
    assert np.isclose(F[0, 2], 1.0) and np.isclose(F[3, 2], 3 / 6)


def test_features_by_hand_on_lollipop():
    # K4 on {0, 1, 2, 3} and the path 3 - 4 - 5: degrees 3, 3, 3, 4, 2, 1; n = 6, 2m = 16
    F = learned.features(*_csr(gg.lollipop(4, 2)))
    assert np.allclose(F[:, 0], np.log([3, 3, 3, 4, 2, 1]))
    assert np.allclose(F[:, 1], np.log([3, 3, 3, 2, 1, 2]))  # smallest neighbour degree
    assert np.allclose(F[:, 2], [1, 1, 1, 3 / 6, 0, 0])
    mean_nb = np.array([10 / 3, 10 / 3, 10 / 3, 11 / 4, 5 / 2, 2 / 1])
    assert np.allclose(F[:, 3], np.log(mean_nb / (16 / 6)))
    assert np.allclose(F[:, 4], [(1 / 3 + 1 / 3 + 1 / 4) / 3] * 3 + [(3 / 3 + 1 / 2) / 4, (1 / 4 + 1) / 2, 1 / 2])
    # p_3(0,0): the triangles at 0 are (0,1,2), (0,1,3), (0,2,3), each walked both ways:
    # 2 (1/(3*3) + 1/(3*4) + 1/(3*4)) / 3; node 3: triangles (3,0,1), (3,0,2), (3,1,2): 2 (3/9) / 4
    p3_0 = 2 * (1 / 9 + 1 / 12 + 1 / 12) / 3
    assert np.allclose(F[:, 5], [p3_0] * 3 + [2 * (3 / 9) / 4, 0.0, 0.0])


@pytest.mark.parametrize("seed", [0, 1])
def test_p2_feature_is_two_step_return_probability(seed):
    g = gg.tree_plus_gnp(50, 5.0, seed)
    F = learned.features(*_csr(g))
    P = _P(g)
    assert np.allclose(F[:, 4], np.diag(P @ P), atol=1e-14)
    assert np.allclose(F[:, 5], np.diag(P @ P @ P), atol=1e-14)


def test_features_do_not_depend_on_the_graph_size():
    """Two disjoint copies of a graph (as a larger graph of the family) give
    every node the features it has in one copy."""
    g = gg.tree_plus_gnp(60, 5.0, 3)
    e = g.edges()
    two = gg.from_edges(2 * g.n, np.concatenate([e[:, 0], e[:, 0] + g.n]), np.concatenate([e[:, 1], e[:, 1] + g.n]))
    F1 = learned.features(*_csr(g))
    F2 = learned.features(*_csr(two))
    assert np.allclose(F2[:g.n], F1, atol=1e-14) and np.allclose(F2[g.n:], F1, atol=1e-14)


def test_hop_terms_match_series_and_powers():
    g = gg.tree_plus_gnp(40, 4.0, 3)
    L = 6
    T = learned.hop_terms(*_csr(g), L)
    P = _P(g)
    d = g.degree
    rows = g.entry_rows()
    Pl = [np.linalg.matrix_power(P, l) for l in range(L + 1)]
    for k in range(0, g.nnz, 7):
        i, j = rows[k], g.col_idx[k]
        for l in range(L + 1):
            assert abs(T[k, l] - (Pl[l][i, i] - Pl[l][j, i]) / d[i]) < 1e-14
    gsum, t1, t2 = series.half_sums(*_csr(g), 3, extra_steps=2)
    assert np.allclose(gsum, T[:, :4].sum(axis=1), atol=1e-14)
    assert np.allclose(t1, T[:, 4], atol=1e-15) and np.allclose(t2, T[:, 5], atol=1e-15)


@pytest.mark.parametrize("maker", [lambda: gg.barabasi_albert(600, 5, 1), lambda: gg.tree_plus_gnp(500, 8.0, 2),
                                   lambda: gg.gnp_lcc(500, 6.0, 3)])
@pytest.mark.parametrize("eps", [1e-2, 1e-3])
def test_certified_lengths(maker, eps):
    g = maker()
    _, _, lam = truncation.spectrum_extremes(*_csr(g))
    cap = int(truncation.tau_entries(*_csr(g), eps, lam).max())
    tau = learned.certified_lengths(*_csr(g), eps, lam, cap)
    assert np.all(tau % 2 == 1) and np.all(tau <= cap)
    rev = series.reverse_entries(*_csr(g))
    assert np.array_equal(tau, tau[rev])
    T = learned.hop_terms(*_csr(g), cap)
    full = T + T[rev]
    f = lam * lam / (1 - lam * lam)
    idx = np.arange(g.nnz)
    below = tau < cap
    assert np.all(f * (full[idx, tau - 1] + full[idx, tau])[below] <= eps)
    prev = tau - 2
    has_prev = prev >= 1
    assert np.all(f * (full[idx, prev - 1] + full[idx, prev])[has_prev] > eps)
    s, _ = series.series_entries(*_csr(g), tau)
    r = exact.exact_dense(*_csr(g))
    assert np.max(np.abs(s - r)) <= eps
    labels = learned.source_labels(g.n, g.row_ptr, tau)
    assert labels.max() <= cap and labels.mean() < cap  # the certified lengths are shorter on average


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = rng.normal(0, 0.3, learned.NPARAM)
    X = rng.normal(size=(40, learned.NF))
    t = rng.normal(size=40)
    loss, grad = learned.loss_and_grad(theta, X, t)
    h = 1e-6
    for p in rng.choice(learned.NPARAM, size=60, replace=False):
        e = np.zeros_like(theta)
        e[p] = h
        fd = (learned.loss_and_grad(theta + e, X, t)[0] - learned.loss_and_grad(theta - e, X, t)[0]) / (2 * h)
        assert abs(fd - grad[p]) <= 1e-7 + 1e-5 * abs(fd)


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    theta, m, v = learned.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.1)
    assert np.allclose(theta, -0.1 * g / (np.abs(g) + 1e-8))


def test_prediction_rounds_to_an_odd_length_with_a_quarter_slack():
    """With every weight zero the network outputs its last bias b3: exp(b3)
    maps to the smallest odd integer >= exp(b3) - 1/4, clipped to [1, cap]."""
    F = np.zeros((1, learned.NF))
    mu, sd = np.zeros(learned.NF), np.ones(learned.NF)
    for e, cap, want in ((0.3, 9, 1), (1.2, 9, 1), (1.3, 9, 3), (3.2, 9, 3), (3.3, 9, 5), (4.76, 9, 5), (5.2, 9, 5),
                         (5.3, 9, 7), (8.5, 7, 7), (1e6, 7, 7), (40.0, 8, 9)):
        theta = np.zeros(learned.NPARAM)
        theta[-1] = np.log(e)
        assert learned.predict_lengths(theta, F, mu, sd, cap)[0] == want, (e, cap)
    theta = np.zeros(learned.NPARAM)
    theta[-1] = 800.0  # exp overflows to inf
    assert learned.predict_lengths(theta, F, mu, sd, 7)[0] == 7


def test_training_reduces_loss_and_predictions_are_odd():
    g = gg.barabasi_albert(800, 5, 4)
    lp, _, lam = truncation.spectrum_extremes(*_csr(g))
    cap = int(truncation.tau_entries(*_csr(g), 1e-3, lam).max())
    labels = learned.source_labels(g.n, g.row_ptr, learned.certified_lengths(*_csr(g), 1e-3, lam, cap))
    F = learned.features(*_csr(g))
    mu, sd = learned.standardise(F)
    X = (F - mu) / sd
    y = np.log(labels)
    rng = np.random.default_rng(1)
    theta = rng.normal(0, 0.2, learned.NPARAM)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    l0 = learned.loss_and_grad(theta, X, y)[0]
    for t in range(1, 301):
        loss, grad = learned.loss_and_grad(theta, X, y)
        theta, m, v = learned.adam_step(theta, grad, m, v, t, lr=1e-2)
    assert loss < 0.2 * l0
    L = learned.predict_lengths(theta, F, mu, sd, cap)
    assert np.all(L % 2 == 1) and L.min() >= 1 and L.max() <= cap


def _csr(g):
    return g.n, g.row_ptr, g.col_idx


# ---------------------------------------------------------------------------
# bipartite graphs: the power-law tail estimate and the extension loop
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("p", [1.5, 2.0, 3.0])
@pytest.mark.parametrize("tau", [11, 51, 301])
def test_tail_estimate_sums_a_power_law(p, tau):
    """Pair sums a(x) = x^-p at x = tau+1, tau+3, ...: the estimate from
    q(tau-2), q(tau) recovers their sum (brute force to 2e6 terms plus the
    integral of the rest) within the midpoint rule's error p(p+1)/(8 tau^2)."""
    q_prev, q = (tau - 1.0) ** -p, (tau + 1.0) ** -p
    est = learned.tail_estimate(np.array([q_prev]), np.array([q]), tau)[0]
    i = np.arange(2_000_000, dtype=np.float64)
    far = tau + 1.0 + 2.0 * i.size
    brute = np.sum((tau + 1.0 + 2.0 * i) ** -p) + far ** (1.0 - p) / (2.0 * (p - 1.0))
    assert abs(est / brute - 1.0) <= p * (p + 1.0) / (8.0 * tau * tau)


@pytest.mark.parametrize("mu", [0.1, 0.5, 0.9])
@pytest.mark.parametrize("tau", [11, 101])
def test_tail_estimate_overshoots_a_geometric_tail(mu, tau):
    """Pair sums falling by a fixed ratio mu per two hops sum to q / (1 - mu);
    the power-law fit never falls below that (it reads a faster-falling ratio
    as a steeper power), or is infinite when the fitted power is <= 1."""
    est = learned.tail_estimate(np.array([1.0 / mu]), np.array([1.0]), tau)[0]
    assert est >= 1.0 / (1.0 - mu)


def test_tail_estimate_special_cases():
    est = learned.tail_estimate(np.array([1.0, 1.0, 0.0, 1.0, 1.0, 1.0, np.nan, 1.1]),
                                np.array([0.0, -1e-20, 1.0, 1.0, 2.0, 0.5, 1.0, 1.0]),
                                np.array([5, 5, 5, 5, 5, 1, 5, 5]))
    assert est[0] == 0.0 and est[1] == 0.0  # nothing left (or rounding below zero)
    assert np.isinf(est[2])  # no earlier pair to fit
    assert np.isinf(est[3]) and np.isinf(est[4])  # no decay, or growth: p <= 1
    assert np.isinf(est[5])  # tau = 1 has no pair before it
    assert np.isinf(est[6])
    assert np.isinf(est[7])  # decay too slow to sum (p = ln 1.1 / ln 1.5 < 1)


def _lattice():
    return gg.perturbed_grid(24, 30, 0.05, 2)


def test_tail_estimate_on_a_perturbed_lattice():
    """Against the exact remainder of the end-corrected series (grounded
    Laplacian): from hop 21 on the estimate is never below 0.8 of it (the
    diffusive decay it is made for), and the geometric fit of the same pair
    sums falls to about half of it."""
    g = _lattice()
    r = exact.exact_dense(*_csr(g))
    L = 160
    T = learned.hop_terms(*_csr(g), L)
    rev = series.reverse_entries(*_csr(g))
    full = T + T[rev]
    cs = np.cumsum(full, axis=1)
    geo_min = np.inf
    for t in range(21, L - 2, 10):
        true = r - (cs[:, t] + 0.5 * full[:, t + 1])
        qp, q = full[:, t - 1] + full[:, t], full[:, t + 1] + full[:, t + 2]
        est = learned.tail_estimate(qp, q, t)
        m = true > 1e-9
        assert np.all(true > -1e-12)  # the remainder is non-negative (lower bound)
        assert np.min(est[m] / true[m]) >= 0.8
        geo = q / (2.0 * (1.0 - np.sqrt(q / qp)))
        geo_min = min(geo_min, np.min(geo[m] / true[m]))
    assert geo_min < 0.6


def test_estimated_lengths_two_routes():
    """The labels from the recorded hop terms equal a search over odd tau with
    the series oracle's own pair sums q(tau) (Algorithm 2 at each length)."""
    g = _lattice()
    eps, cap = 1e-2, 61
    tau = learned.estimated_lengths(*_csr(g), eps, cap)
    assert np.all(tau % 2 == 1) and np.all((tau >= 3) & (tau <= cap))
    rev = series.reverse_entries(*_csr(g))
    assert np.array_equal(tau, tau[rev])
    q = {t: series.series_entries(*_csr(g), t, end_corrected=True)[1] for t in range(1, cap + 1, 2)}
    want = np.full(g.nnz, cap)
    done = np.zeros(g.nnz, dtype=bool)
    for t in range(3, cap + 1, 2):
        ok = ~done & (learned.tail_estimate(q[t - 2], q[t], t) <= eps)
        want[ok] = t
        done |= ok
    assert np.array_equal(tau, want)


def test_learned_bipartite_within_eps():
    """The extension loop from a short constant length: every edge ends at an
    odd length whose estimate passed (or the cap), the values are the
    end-corrected series there, and all are within eps of the exact values."""
    g = _lattice()
    eps, cap = 1e-2, 255
    s, tau, rounds = learned.learned_bipartite(g.n, g.row_ptr, g.col_idx, np.full(g.n, 5), cap, eps)
    assert rounds >= 2
    assert np.all(tau % 2 == 1) and np.all(tau <= cap)
    assert np.mean(tau) < 0.5 * cap  # accepted well below the cap, not run out to it
    ref, q = series.series_entries(*_csr(g), tau, end_corrected=True)
    assert np.array_equal(s, ref)
    _, qp = series.series_entries(*_csr(g), tau - 2, end_corrected=True)
    est = learned.tail_estimate(qp, q, tau)
    assert np.all((est <= eps) | (tau == cap))
    r = exact.exact_dense(*_csr(g))
    assert np.all(s <= r + 1e-12) and np.max(r - s) <= eps
