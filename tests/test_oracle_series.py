"""Pins for the truncated-series oracle (O2) and the truncation length.

The series oracle (Algorithm 2 in C) is checked against:
  * closed forms of the truncated series on K_n and C_n (from the spectra of
    their walk matrices, Eq. 4),
  * the series evaluated in exact rational arithmetic from matrix powers of P
    on tiny graphs (Eq. 2 written out, independent code path),
  * the odd-tau lower-bound and monotonicity property (proof of Thm. 3.2),
  * convergence to the exact resistance (O1) for large tau,
  * the bipartite bias of exactly 1/m per edge-transitive cycle edge, and its
    removal by the end-corrected estimator,
  * Theorem 3.2: with tau from Eq. (6) every edge is within eps.
"""
from fractions import Fraction

import numpy as np
import pytest

import graphgen as gg
from oracle import exact, series, truncation


def _entries(g, tau, **kw):
    s, q = series.series_entries(g.n, g.row_ptr, g.col_idx, tau, **kw)
    return s, q


@pytest.mark.parametrize("n", [3, 5, 8])
@pytest.mark.parametrize("tau", [0, 1, 2, 3, 7])
def test_complete_graph_closed_form(n, tau):
    g = gg.complete(n)
    s, _ = _entries(g, tau)
    mu = -1.0 / (n - 1)
    want = (2.0 / n) * (1.0 - mu ** (tau + 1))
    assert np.max(np.abs(s - want)) < 1e-14


@pytest.mark.parametrize("n", [5, 6, 9])
@pytest.mark.parametrize("tau", [1, 2, 5, 11])
def test_cycle_closed_form(n, tau):
    g = gg.cycle(n)
    s, _ = _entries(g, tau)
    k = np.arange(1, n)
    want = (n - 1) / n - np.sum(np.cos(2 * np.pi * k / n) ** (tau + 1)) / n
    assert np.max(np.abs(s - want)) < 1e-14


def _exact_rational_series(g, tau):
    """Eq. (2) term by term from exact matrix powers of P = D^-1 A."""
    n = g.n
    deg = g.degree
    P = [[Fraction(0)] * n for _ in range(n)]
    for r in range(n):
        for c in g.col_idx[g.row_ptr[r]:g.row_ptr[r + 1]]:
            P[r][int(c)] = Fraction(1, int(deg[r]))
    Pl = [[Fraction(int(r == c)) for c in range(n)] for r in range(n)]
    acc = {}
    edges = [tuple(map(int, e)) for e in g.edges()]
    for e in edges:
        acc[e] = Fraction(0)
    for _ in range(tau + 1):
        for (i, j) in edges:
            di, dj = int(deg[i]), int(deg[j])
            acc[(i, j)] += Pl[i][i] / di + Pl[j][j] / dj - Pl[i][j] / dj - Pl[j][i] / di
        Pl = [[sum(Pl[r][x] * P[x][c] for x in range(n)) for c in range(n)] for r in range(n)]
    return acc


@pytest.mark.parametrize("maker", [lambda: gg.lollipop(4, 2), lambda: gg.petersen(),
                                   lambda: gg.tree_plus_gnp(7, 3.0, 1)])
@pytest.mark.parametrize("tau", [0, 3, 6])
def test_matches_exact_rational_series(maker, tau):
    g = maker()
    s, _ = _entries(g, tau)
    want = _exact_rational_series(g, tau)
    k = exact.entry_of_edges(g.n, g.row_ptr, g.col_idx, np.array(list(want.keys())))
    got = s[k]
    ref = np.array([float(v) for v in want.values()])
    assert np.max(np.abs(got - ref)) < 1e-14


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_odd_tau_lower_bound_and_monotone(seed):
    g = gg.tree_plus_gnp(120, 5.0, seed)
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    prev = None
    for tau in range(1, 30, 2):
        s, _ = _entries(g, tau)
        assert np.all(s <= r + 1e-13)
        if prev is not None:
            assert np.all(s >= prev - 1e-13)
        prev = s


def test_large_tau_converges_to_exact():
    g = gg.tree_plus_gnp(150, 8.0, 4)
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    s, _ = _entries(g, 301)
    assert np.max(np.abs(s - r)) < 1e-11


@pytest.mark.parametrize("n", [8, 12])
def test_bipartite_bias_and_end_correction(n):
    """Even cycle: the lambda = -1 mode never decays; the odd-tau series
    converges to r - 1/m. Half of the first omitted term cancels it."""
    g = gg.cycle(n)
    r = (n - 1) / n
    s, _ = _entries(g, 401)
    assert np.max(np.abs(s - (r - 1.0 / g.m))) < 1e-12
    s_hat, _ = _entries(g, 401, end_corrected=True)
    assert np.max(np.abs(s_hat - r)) < 1e-12


def test_end_corrected_grid_lower_bound_and_tail_bound():
    g = gg.perturbed_grid(8, 9, 0.05, 3)
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    lam_plus, lam_minus, _ = truncation.spectrum_extremes(g.n, g.row_ptr, g.col_idx)
    assert abs(lam_minus + 1.0) < 1e-10  # bipartite
    for tau in (5, 15, 41):
        s_hat, q = _entries(g, tau, end_corrected=True)
        tail = r - s_hat
        assert np.all(tail >= -1e-13)
        bound = series.tail_bound(q, 1.0, lam_plus, end_corrected=True)
        assert np.all(tail <= bound + 1e-13)


@pytest.mark.parametrize("seed", [0, 1])
def test_plain_tail_bound(seed):
    g = gg.tree_plus_gnp(200, 6.0, seed)
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    _, _, lam_star = truncation.spectrum_extremes(g.n, g.row_ptr, g.col_idx)
    for tau in (1, 3, 9):
        s, q = _entries(g, tau)
        tail = r - s
        assert np.all(q >= -1e-15)
        assert np.all(tail <= series.tail_bound(q, lam_star, 0.0, False) + 1e-13)


@pytest.mark.parametrize("eps", [1e-2, 1e-3])
@pytest.mark.parametrize("seed", [0, 1])
def test_theorem_3_2_eps_guarantee(eps, seed):
    g = gg.tree_plus_gnp(300, 8.0, seed)
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    _, _, lam = truncation.spectrum_extremes(g.n, g.row_ptr, g.col_idx)
    tau = truncation.tau_entries(g.n, g.row_ptr, g.col_idx, eps, lam)
    s, _ = _entries(g, tau)
    assert np.max(np.abs(s - r)) <= eps
    # per-edge lengths: both directions of an edge agree, all odd
    rev = series.reverse_entries(g.n, g.row_ptr, g.col_idx)
    assert np.array_equal(tau, tau[rev]) and np.all(tau % 2 == 1)


def test_per_entry_lengths_match_global_runs():
    """Truncation is per edge: an entry with length t holds exactly the value a
    run with the one global length t gives it (both halves at the same t),
    whatever the lengths of the other edges of its endpoints."""
    g = gg.tree_plus_gnp(60, 4.0, 6)
    rev = series.reverse_entries(g.n, g.row_ptr, g.col_idx)
    rng = np.random.default_rng(6)
    tau = 2 * rng.integers(0, 5, g.nnz) + 1
    tau = np.where(np.arange(g.nnz) < rev, tau, tau[rev])  # one length per undirected edge
    s_mix, q_mix = _entries(g, tau)
    for t in np.unique(tau):
        s_t, q_t = _entries(g, int(t))
        sel = tau == t
        assert np.max(np.abs(s_mix[sel] - s_t[sel])) < 1e-15
        assert np.max(np.abs(q_mix[sel] - q_t[sel])) < 1e-15


def test_tail_bounds_are_tight_at_large_tau():
    """For odd tau the tail is sum_k c_k lambda_k^(tau+1) / (1 - lambda_k) and the
    observed pair q = sum_k c_k (1 + lambda_k) lambda_k^(tau+1) (c_k >= 0, proof
    of Theorem 3.2). As tau grows the modes of largest |lambda_k| dominate both,
    so tail / bound tends to 1 on an edge those modes reach: the plain bound
    q / (1 - lambda_star^2) and, on a bipartite graph (lambda = -1 cancelled,
    lambda_plus the slowest mode left), the end-corrected q / (2 (1 - lambda_plus))
    are asymptotically exact, not merely valid."""
    g = gg.tree_plus_gnp(200, 6.0, 0)
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    lam_plus, _, lam_star = truncation.spectrum_extremes(g.n, g.row_ptr, g.col_idx)
    s, q = _entries(g, 41)
    ratio = (r - s) / series.tail_bound(q, lam_star, lam_plus, False)
    assert 0.95 <= np.max(ratio) <= 1.0 + 1e-6
    h = gg.perturbed_grid(8, 9, 0.05, 3)
    r = exact.exact_dense(h.n, h.row_ptr, h.col_idx)
    lam_plus, _, _ = truncation.spectrum_extremes(h.n, h.row_ptr, h.col_idx)
    s_hat, q = _entries(h, 101, end_corrected=True)
    ratio = (r - s_hat) / series.tail_bound(q, 1.0, lam_plus, True)
    assert 0.95 <= np.max(ratio) <= 1.0 + 1e-6


def test_tau_is_smallest_odd_meeting_the_bound():
    """Eq. (6) inverted: tau is the least odd t >= 1 whose a-priori tail bound
    X_e lam^(t+1) / (1 - lam^2) is <= eps (proof of Thm. 3.2)."""
    rng = np.random.default_rng(0)
    d_i = rng.integers(1, 500, 2000)
    d_j = rng.integers(1, 500, 2000)
    keep = (d_i > 1) | (d_j > 1)
    d_i, d_j = d_i[keep], d_j[keep]
    for eps in (1e-2, 1e-3, 5e-5):
        for lam in (0.05, 0.43, 0.6, 0.93):
            tau = truncation.odd_ceil(truncation.f_edge(d_i, d_j, eps, lam))
            x = 1.0 / d_i + 1.0 / d_j - 2.0 / (d_i * d_j)
            def bound(t, xx):
                return xx * lam ** (t + 1) / (1 - lam * lam)
            assert np.all(bound(tau, x) <= eps * (1 + 1e-12))
            lower = tau - 2
            ok = lower >= 1
            assert np.all(bound(lower[ok], x[ok]) > eps * (1 - 1e-12))


@pytest.mark.parametrize("n", [5, 8, 13])
def test_spectrum_cycle(n):
    g = gg.cycle(n)
    lp, lm, ls = truncation.spectrum_extremes(g.n, g.row_ptr, g.col_idx)
    assert abs(lp - np.cos(2 * np.pi / n)) < 1e-12
    assert abs(lm - np.cos(2 * np.pi * (n // 2) / n)) < 1e-12


def test_spectrum_named():
    lp, lm, _ = truncation.spectrum_extremes(*_csr(gg.complete(9)))
    assert abs(lp + 1 / 8) < 1e-12 and abs(lm + 1 / 8) < 1e-12
    lp, lm, ls = truncation.spectrum_extremes(*_csr(gg.petersen()))
    assert abs(lp - 1 / 3) < 1e-12 and abs(lm + 2 / 3) < 1e-12
    assert abs(ls - 2 / 3) < 1e-12  # lambda_star is the larger modulus, here the negative end
    _, _, ls = truncation.spectrum_extremes(*_csr(gg.cycle(9)))
    assert abs(ls - np.cos(np.pi / 9)) < 1e-12  # odd cycle: |cos(2 pi 4 / 9)| > cos(2 pi / 9)
    lp, lm, _ = truncation.spectrum_extremes(*_csr(gg.hypercube(4)))
    assert abs(lp - 0.5) < 1e-12 and abs(lm + 1.0) < 1e-12


def test_spectrum_sparse_path_matches_dense():
    g = gg.tree_plus_gnp(1500, 8.0, 9)
    dense = truncation.spectrum_extremes(*_csr(g), dense_max=5000)
    sparse = truncation.spectrum_extremes(*_csr(g), dense_max=10)
    assert np.allclose(dense, sparse, atol=1e-9)


def _csr(g):
    return g.n, g.row_ptr, g.col_idx
