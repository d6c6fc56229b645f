"""Pins for the TGT+ oracle (O3): Philox, walk estimator, CalChi, walk counts.

  * Philox4x32-10 against the published known-answer vectors (golden file).
  * Lemma 4.1 (g_tau = g_tt + g_{tt->tau}) and the unbiasedness of X (Eq. 11)
    against exact matrix powers.
  * Lemma 4.3 / Eq. 17 against exhaustive enumeration of every walk.
  * rho_hat >= rho (Eq. 16 by brute force), and a case where Algorithm 3's
    rho_hat, taken literally, falls below rho.
  * Eq. 13's Hoeffding guarantee over many seeds.
"""
import itertools
import math
import os

import numpy as np
import pytest

import graphgen as gg
from oracle import exact, philox, series, tgtplus

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    n = 0
    for line in open(os.path.join(GOLDEN, "philox_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        out = philox.philox4x32_10(*w[:6])
        assert [int(v) for v in out] == w[6:]
        n += 1
    assert n == 3


def test_uniform_index_range_and_ends():
    for d in (1, 2, 3, 7, 1000, 2259):
        assert philox.uniform_index(0, d) == 0
        assert philox.uniform_index(2**32 - 1, d) == d - 1
        u = np.arange(0, 2**32, 2**32 // 4096, dtype=np.uint64)
        idx = philox.uniform_index(u, d)
        assert idx.min() >= 0 and idx.max() <= d - 1


def _dense_P(g):
    P = np.zeros((g.n, g.n))
    for r in range(g.n):
        nb = g.col_idx[g.row_ptr[r]:g.row_ptr[r + 1]]
        P[r, nb] = 1.0 / len(nb)
    return P


def test_lemma_4_1_and_unbiased_walk_estimator():
    g = gg.tree_plus_gnp(12, 3.5, 2)
    P = _dense_P(g)
    i = 0
    j = int(g.col_idx[g.row_ptr[0]])
    k = int(g.row_ptr[0])
    tau, tt = 9, 3
    d_i = g.degree[i]
    Pl = [np.linalg.matrix_power(P, l) for l in range(tau + 1)]
    g_tau = sum(Pl[l][i, i] - Pl[l][j, i] for l in range(tau + 1))
    g_tt = sum(Pl[l][i, i] - Pl[l][j, i] for l in range(tt + 1))
    p = Pl[tt][:, i]  # p_tt(x, v_i)
    assert np.allclose(tgtplus.source_column(g.n, g.row_ptr, g.col_idx, i, tt), p, rtol=0, atol=1e-15)
    # Eq. 10 (times d_i): sum_x p_tt(x,i) sum_{l=1}^{tau-tt} (p_l(i,x) - p_l(j,x))
    g_tail = sum(p[x] * (Pl[l][i, x] - Pl[l][j, x]) for x in range(g.n) for l in range(1, tau - tt + 1))
    assert abs(g_tau - (g_tt + g_tail)) < 1e-14
    # the series oracle agrees with the exact powers for g_tau
    gh, _, _ = series.half_sums(g.n, g.row_ptr, g.col_idx, tau, sources=[i], extra_steps=0)
    assert abs(gh[k] * d_i - g_tau) < 1e-13
    # Monte Carlo mean of X d_i -> g_tail
    R = 200_000
    est = tgtplus.walk_estimate(g.row_ptr, g.col_idx, p, i, j, tau - tt, k, R, seed=7)
    si = tgtplus.walk_sums(g.row_ptr, g.col_idx, p, i, tau - tt, k, 4000, 0, 7)
    sj = tgtplus.walk_sums(g.row_ptr, g.col_idx, p, j, tau - tt, k, 4000, 1, 7)
    sigma = np.std(si - sj)
    assert abs(est - g_tail) < 5 * sigma / math.sqrt(R)
    # tgt_plus_half with these lengths reproduces g_tt + walk mean
    gp, Rk, chi = tgtplus.tgt_plus_half(g.n, g.row_ptr, g.col_idx, i,
                                        np.full(d_i, tau), tt, 0.05, 1.0 / g.n, 10, 7, g.m)
    assert Rk[0] == tgtplus.walk_count(chi[0], d_i, g.m, 1.0 / g.n, 0.05)
    est_k = tgtplus.walk_estimate(g.row_ptr, g.col_idx, p, i, j, tau - tt, k, int(Rk[0]), 7)
    assert abs(gp[0] - (g_tt + est_k)) < 1e-12


def _all_walks(g, start, L):
    walks = [[start]]
    for _ in range(L):
        walks = [w + [int(y)] for w in walks for y in g.col_idx[g.row_ptr[w[-1]]:g.row_ptr[w[-1] + 1]]]
    return [w[1:] for w in walks]


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("L", [1, 2, 4])
def test_lemma_4_3_bounds_by_enumeration(seed, L):
    g = gg.tree_plus_gnp(9, 3.0, seed)
    rng = np.random.default_rng(seed)
    p = rng.random(g.n) ** 3  # uneven values so that the bounds are exercised
    rho = tgtplus.rho_exact(g.row_ptr, g.col_idx, p)
    rh = tgtplus.rho_hat(g.row_ptr, g.col_idx, p, 3)
    assert rh >= rho - 1e-15
    for i in range(g.n):
        for j in g.col_idx[g.row_ptr[i]:g.row_ptr[i + 1]].tolist():
            lb_i, ub_i = tgtplus.lemma43(g.row_ptr, g.col_idx, p, i, L, rh)
            lb_j, ub_j = tgtplus.lemma43(g.row_ptr, g.col_idx, p, j, L, rh)
            si = [p[w].sum() for w in _all_walks(g, i, L)]
            sj = [p[w].sum() for w in _all_walks(g, j, L)]
            assert min(si) >= lb_i - 1e-12 and max(si) <= ub_i + 1e-12
            assert min(sj) >= lb_j - 1e-12 and max(sj) <= ub_j + 1e-12
            chi = tgtplus.calchi(g.row_ptr, g.col_idx, p, i, j, L, 3)
            span = max(si) - min(sj) - (min(si) - max(sj))
            assert span <= chi + 1e-12  # X d_i lies in an interval of width chi


def test_rho_hat_upper_bound_and_literal_counterexample():
    # path 0-1-2-3 plus 4 attached to 3; candidates C = {0, 2, 3} (gamma = 3)
    g = gg.from_edges(5, [0, 1, 2, 3], [1, 2, 3, 4])
    p = np.array([0.50, 0.09, 0.10, 0.10, 0.01])
    rho = tgtplus.rho_exact(g.row_ptr, g.col_idx, p)          # edge (0,1): 0.59
    literal = tgtplus.rho_hat(g.row_ptr, g.col_idx, p, 3, literal=True)  # only (2,3) inside C: 0.20
    safe = tgtplus.rho_hat(g.row_ptr, g.col_idx, p, 3)
    assert literal < rho <= safe
    rng = np.random.default_rng(3)
    for _ in range(200):
        h = gg.tree_plus_gnp(30, 4.0, int(rng.integers(1 << 30)))
        q = rng.random(h.n) ** 4
        for gamma in (1, 2, 5, 10):
            assert tgtplus.rho_hat(h.row_ptr, h.col_idx, q, gamma) >= tgtplus.rho_exact(h.row_ptr, h.col_idx, q) - 1e-15


def test_eq15_gamma_zero():
    g = gg.cycle(7)
    p = np.linspace(0.0, 0.3, 7)
    assert tgtplus.calchi(g.row_ptr, g.col_idx, p, 0, 1, 5, 0) == pytest.approx(2 * 5 * 0.3)


def test_walk_count_formula_and_hoeffding():
    # Eq. 13 is the least Hoeffding count for deviation eps/4 with range chi/d_i
    # and failure probability delta/m per half-edge estimate
    for chi, d, m, delta, eps in ((0.02, 7, 1000, 1e-3, 0.01), (0.05, 7, 1000, 1e-3, 0.01),
                                  (0.3, 2, 50_000, 2e-5, 1e-3), (1e-3, 40, 10, 0.1, 0.05)):
        R = tgtplus.walk_count(chi, d, m, delta, eps)
        assert 2 * math.exp(-2 * R * (eps / 4) ** 2 / (chi / d) ** 2) <= delta / m * (1 + 1e-9)
        assert R == 1 or 2 * math.exp(-2 * (R - 1) * (eps / 4) ** 2 / (chi / d) ** 2) > delta / m
    # empirical: over many seeds the estimate stays within eps/4 of its mean
    g = gg.tree_plus_gnp(40, 5.0, 4)
    i = 3
    j = int(g.col_idx[g.row_ptr[i]])
    k = int(g.row_ptr[i])
    tt, L = 2, 4
    p = tgtplus.source_column(g.n, g.row_ptr, g.col_idx, i, tt)
    chi = tgtplus.calchi(g.row_ptr, g.col_idx, p, i, j, L, 10)
    eps = 0.02
    R = tgtplus.walk_count(chi, g.degree[i], g.m, 1.0 / g.n, eps)
    P = _dense_P(g)
    exact_tail = sum(p[x] * (np.linalg.matrix_power(P, l)[i, x] - np.linalg.matrix_power(P, l)[j, x])
                     for x in range(g.n) for l in range(1, L + 1))
    devs = [abs(tgtplus.walk_estimate(g.row_ptr, g.col_idx, p, i, j, L, k, R, s) - exact_tail) / g.degree[i]
            for s in range(60)]
    assert max(devs) <= eps / 4


def test_full_tgt_plus_within_eps_on_small_graph():
    g = gg.tree_plus_gnp(60, 6.0, 5)
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    from oracle import truncation

    _, _, lam = truncation.spectrum_extremes(g.n, g.row_ptr, g.col_idx)
    eps = 0.05
    tau = truncation.tau_entries(g.n, g.row_ptr, g.col_idx, eps / 2, lam)  # Algorithm 4 sets the lengths for eps / 2
    ghat = np.zeros(g.nnz)
    for i in range(g.n):
        a, b = g.row_ptr[i], g.row_ptr[i + 1]
        gi, _, _ = tgtplus.tgt_plus_half(g.n, g.row_ptr, g.col_idx, i, tau[a:b], 3, eps, 1.0 / g.n, 10, 11, g.m)
        ghat[a:b] = gi / g.degree[i]
    rev = series.reverse_entries(g.n, g.row_ptr, g.col_idx)
    s = ghat + ghat[rev]
    assert np.max(np.abs(s - r)) <= eps


def _reach_exactly(g, i, ell):
    """Nodes at the end of some walk of exactly ell steps from v_i (boolean
    matrix powers, no probabilities)."""
    a = np.zeros((g.n, g.n), dtype=bool)
    a[g.entry_rows(), g.col_idx] = True
    cur = np.zeros(g.n, dtype=bool)
    cur[i] = True
    for _ in range(ell):
        cur = a[cur].any(axis=0)
    return cur


@pytest.mark.parametrize("maker", [lambda: gg.tree_plus_gnp(50, 4.0, 2), lambda: gg.grid(5, 6),
                                   lambda: gg.lollipop(6, 4)])
def test_frontier_volume_is_the_degree_of_the_exact_reach(maker):
    """Eq. 14's left side: the support of p_l(., v_i) is the set reached by a
    walk of exactly l steps (on a bipartite graph one side of the ball only)."""
    g = maker()
    for i in (0, g.n // 2, g.n - 1):
        for ell in range(0, 7):
            p = tgtplus.source_column(g.n, g.row_ptr, g.col_idx, i, ell)
            assert tgtplus.frontier_volume(g.row_ptr, p) == int(g.degree[_reach_exactly(g, i, ell)].sum())


def test_per_source_switch_is_the_first_hop_where_eq14_holds():
    """tgtplus.switch_hop against Eq. 14 evaluated from columns of matrix
    powers of P: it fails at every earlier hop and holds at the switch, which
    is never past the source's longest length; a large eps switches sooner."""
    from oracle import truncation

    g = gg.tree_plus_gnp(70, 5.0, 4)
    _, _, lam = truncation.spectrum_extremes(g.n, g.row_ptr, g.col_idx)
    P = np.zeros((g.n, g.n))
    P[g.entry_rows(), g.col_idx] = 1.0 / g.degree[g.entry_rows()]
    for eps in (0.02, 0.2):
        tau = truncation.tau_entries(g.n, g.row_ptr, g.col_idx, eps / 2, lam)
        tts = []
        for i in range(0, g.n, 7):
            a, b = g.row_ptr[i], g.row_ptr[i + 1]
            tt = tgtplus.switch_hop(g.n, g.row_ptr, g.col_idx, i, tau[a:b], eps, 1.0 / g.n, 10, g.m)
            assert 0 <= tt <= tau[a:b].max()
            col = np.zeros(g.n)
            col[i] = 1.0
            for ell in range(tt + 1):
                lhs = int(g.degree[col != 0].sum())
                rhs = sum(tgtplus.walk_count(tgtplus.calchi(g.row_ptr, g.col_idx, col, i, int(g.col_idx[k]),
                                                            int(tau[k]) - ell, 10), g.degree[i], g.m, 1.0 / g.n, eps)
                          for k in range(a, b) if tau[k] - ell > 0)
                assert (lhs > rhs) == (ell == tt), (i, ell, tt)
                col = P @ col  # p_{ell+1}(x, v_i) = P^(ell+1)[x, v_i] = sum_y P[x, y] p_ell(y, v_i)
            tts.append(tt)
        if eps == 0.02:
            tts_small = tts
    assert np.mean(tts) <= np.mean(tts_small)


def test_tgt_plus_with_per_source_switch_within_eps():
    """Theorem 4.4 with Algorithm 4's per-source switch (fixed seeds)."""
    from oracle import truncation

    g = gg.tree_plus_gnp(60, 6.0, 5)
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    _, _, lam = truncation.spectrum_extremes(g.n, g.row_ptr, g.col_idx)
    eps = 0.05
    tau = truncation.tau_entries(g.n, g.row_ptr, g.col_idx, eps / 2, lam)
    ghat = np.zeros(g.nnz)
    walks = 0
    for i in range(g.n):
        a, b = g.row_ptr[i], g.row_ptr[i + 1]
        tt = tgtplus.switch_hop(g.n, g.row_ptr, g.col_idx, i, tau[a:b], eps, 1.0 / g.n, 10, g.m)
        gi, R, _ = tgtplus.tgt_plus_half(g.n, g.row_ptr, g.col_idx, i, tau[a:b], tt, eps, 1.0 / g.n, 10, 13, g.m)
        ghat[a:b] = gi / g.degree[i]
        walks += int(R.sum())
    rev = series.reverse_entries(g.n, g.row_ptr, g.col_idx)
    assert walks > 0
    assert np.max(np.abs(ghat + ghat[rev] - r)) <= eps


# ---------------------------------------------------------------- TGT+ at learned lengths
@pytest.mark.parametrize("maker", [lambda: gg.tree_plus_gnp(40, 5.0, 3), lambda: gg.barabasi_albert(45, 3, 2),
                                   lambda: gg.barbell(6, 2)])
def test_even_hop_bound_holds_against_the_exact_tail(maker):
    """tail past odd tau (exact resistance minus the series at tau) <= the
    one-even-hop bound lam*^(tau + 1 - l) / (1 - lam*) t_l(e) for every even
    l <= tau + 1, with lam* the spectral radius past lambda_1 from a dense
    eigendecomposition."""
    from oracle import learned

    g = maker()
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    deg = g.degree.astype(float)
    A = np.zeros((g.n, g.n))
    A[g.entry_rows(), g.col_idx] = 1.0
    N = A / np.sqrt(np.outer(deg, deg))
    ev = np.sort(np.linalg.eigvalsh(N))
    lam = max(abs(ev[0]), abs(ev[-2]))
    T = learned.hop_terms(g.n, g.row_ptr, g.col_idx, 12)
    rev = series.reverse_entries(g.n, g.row_ptr, g.col_idx)
    full = T + T[rev]
    for tau in (1, 3, 5, 9, 11):
        S, _ = series.series_entries(g.n, g.row_ptr, g.col_idx, tau)
        tail = r - S
        for ell in range(0, tau + 2, 2):
            b = np.array([tgtplus.even_hop_bound(t, ell, tau, lam) for t in full[:, ell]])
            assert np.all(tail <= b + 1e-12), (tau, ell)
            assert np.all(full[:, ell] >= -1e-15)  # even hop terms are sums of non-negative mode terms


def test_learned_tgt_plus_at_the_cap_is_per_source_tgt_plus():
    """Every source at the cap: no length can grow, so the result is the
    per-source TGT+ of Algorithm 4 (switch_hop, then tgt_plus_half) itself."""
    from oracle import truncation

    g = gg.tree_plus_gnp(50, 6.0, 7)
    eps = 0.05
    _, _, lam = truncation.spectrum_extremes(g.n, g.row_ptr, g.col_idx)
    cap = int(truncation.tau_entries(g.n, g.row_ptr, g.col_idx, eps / 2, lam).max())
    s, tau, tt, rounds, _ = tgtplus.tgt_plus_learned(g.n, g.row_ptr, g.col_idx, np.full(g.n, cap), cap, eps, lam,
                                                    1.0 / g.n, 10, 5, g.m)
    assert rounds == 0 and np.all(tau == cap)
    ghat = np.zeros(g.nnz)
    for i in range(g.n):
        a, b = g.row_ptr[i], g.row_ptr[i + 1]
        ti = tgtplus.switch_hop(g.n, g.row_ptr, g.col_idx, i, tau[a:b], eps, 1.0 / g.n, 10, g.m)
        assert ti == tt[i]
        gi, _, _ = tgtplus.tgt_plus_half(g.n, g.row_ptr, g.col_idx, i, tau[a:b], ti, eps, 1.0 / g.n, 10, 5, g.m)
        ghat[a:b] = gi / g.degree[i]
    assert np.array_equal(s, ghat + ghat[series.reverse_entries(g.n, g.row_ptr, g.col_idx)])


@pytest.mark.parametrize("L0", [1, 3])
def test_learned_tgt_plus_extends_short_lengths_and_meets_eps(L0):
    """Every source predicted far too short: the certificate fails, lengths
    grow (rounds >= 1) to ones the bound accepts or to the cap, and the result
    is within eps of the exact values."""
    from oracle import truncation

    g = gg.tree_plus_gnp(60, 6.0, 5)
    eps = 0.05
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    _, _, lam = truncation.spectrum_extremes(g.n, g.row_ptr, g.col_idx)
    cap = int(truncation.tau_entries(g.n, g.row_ptr, g.col_idx, eps / 2, lam).max())
    s, tau, tt, rounds, _ = tgtplus.tgt_plus_learned(g.n, g.row_ptr, g.col_idx, np.full(g.n, L0), cap, eps, lam,
                                                    1.0 / g.n, 10, 11, g.m)
    assert rounds >= 1 and tau.max() > L0 and np.all(tau % 2 == 1) and np.all(tau <= cap)
    rev = series.reverse_entries(g.n, g.row_ptr, g.col_idx)
    assert np.array_equal(tau, tau[rev])
    assert np.max(np.abs(s - r)) <= eps
