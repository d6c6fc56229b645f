"""Pins for CalTau with omega eigenpairs (Algorithm 1, Eq. 6-8, Theorem 3.2).

  * the eigenpairs reproduce the terms of Eq. 2 (matrix powers of P), the
    exact resistance and X_e (Lemma 3.1 and the identities of Theorem 3.2's
    proof);
  * with omega = 2, CalTau is Eq. 6 with lambda_star (Algorithm 1's start);
  * with omega = n the bound Delta_t + lambda_n^(t+1) / (1 - lambda_n^2)
    (X_e - Upsilon) equals the exact tail after t hops, and for fewer
    eigenpairs it bounds the tail after every odd tau >= t;
  * Theorem 3.2: the series truncated at CalTau's lengths is within eps of the
    exact value, and CalTau is never longer than Eq. 6;
  * a bottleneck graph, where lambda_2 is close to 1 and the third eigenvalue
    is small, needs orders of magnitude fewer hops with omega = 3.
CPU only.
"""
import numpy as np
import pytest

import graphgen as gg
from oracle import exact, series, truncation


def _csr(g):
    return g.n, g.row_ptr, g.col_idx


def _P(g):
    P = np.zeros((g.n, g.n))
    for r in range(g.n):
        nb = g.col_idx[g.row_ptr[r]:g.row_ptr[r + 1]]
        P[r, nb] = 1.0 / len(nb)
    return P


def _c(g, F):
    rows = g.entry_rows()
    return (F[:, rows] - F[:, g.col_idx]) ** 2  # c_k per entry, k = 1 .. omega


@pytest.mark.parametrize("maker", [lambda: gg.lollipop(5, 3), lambda: gg.petersen(), lambda: gg.tree_plus_gnp(30, 4.0, 2),
                                   lambda: gg.barbell(4, 2)])
def test_eigenpairs_reproduce_the_series_terms(maker):
    g = maker()
    lam, F = truncation.eigenpairs_by_modulus(*_csr(g), g.n)
    assert lam[0] == 1.0 and np.all(np.abs(F[0] - 1.0) == 0.0)
    assert np.all(np.diff(np.abs(lam)) <= 1e-12)  # sorted by modulus
    two_m = 2.0 * g.m
    c = _c(g, F)
    rows, cols = g.entry_rows(), g.col_idx
    d = g.degree.astype(np.float64)
    P = _P(g)
    Pl = np.eye(g.n)
    for ell in range(6):
        # Eq. 2's hop-ell term of every edge from matrix powers of P
        term = Pl[rows, rows] / d[rows] + Pl[cols, cols] / d[cols] - Pl[rows, cols] / d[cols] - Pl[cols, rows] / d[rows]
        assert np.max(np.abs((lam ** ell) @ c / two_m - term)) < 1e-13
        Pl = Pl @ P
    x_e = 1 / d[rows] + 1 / d[cols] - 2 / (d[rows] * d[cols])
    assert np.max(np.abs((1 + lam[1:]) @ c[1:] / two_m - x_e)) < 1e-13
    r = exact.exact_dense(*_csr(g))
    assert np.max(np.abs((1 / (1 - lam[1:])) @ c[1:] / two_m - r)) < 1e-12


@pytest.mark.parametrize("maker", [lambda: gg.tree_plus_gnp(200, 6.0, 1), lambda: gg.barabasi_albert(300, 3, 2),
                                   lambda: gg.lollipop(8, 3)])
@pytest.mark.parametrize("eps", [1e-2, 1e-4])
def test_omega_two_is_eq6(maker, eps):
    g = maker()
    _, _, lam_star = truncation.spectrum_extremes(*_csr(g))
    lam, F = truncation.eigenpairs_by_modulus(*_csr(g), 2)
    assert abs(abs(lam[1]) - lam_star) < 1e-12
    assert np.array_equal(truncation.caltau(*_csr(g), eps, lam, F),
                          truncation.tau_entries(*_csr(g), eps, lam_star))


@pytest.mark.parametrize("maker", [lambda: gg.tree_plus_gnp(40, 4.0, 3), lambda: gg.petersen(), lambda: gg.lollipop(6, 2)])
def test_bound_is_the_exact_tail_with_every_eigenpair(maker):
    """omega = n leaves only the last mode to the lambda_omega term, which it
    then describes exactly: the bound equals r - s_t."""
    g = maker()
    r = exact.exact_dense(*_csr(g))
    lam, F = truncation.eigenpairs_by_modulus(*_csr(g), g.n)
    d = g.degree.astype(np.float64)
    rows, cols = g.entry_rows(), g.col_idx
    x_e = 1 / d[rows] + 1 / d[cols] - 2 / (d[rows] * d[cols])
    lw = abs(lam[-1])
    for t in (1, 3, 5, 9):
        ups, delta = truncation.upsilon_delta(*_csr(g), lam, F, t)
        s, _ = series.series_entries(*_csr(g), t)
        bound = delta + lw ** (t + 1) / (1 - lw * lw) * (x_e - ups)
        assert np.max(np.abs((r - s) - bound)) < 1e-12


@pytest.mark.parametrize("omega", [3, 5, 9, 16])
def test_bound_holds_for_every_odd_tau_from_t(omega):
    g = gg.tree_plus_gnp(60, 5.0, 4)
    r = exact.exact_dense(*_csr(g))
    lam, F = truncation.eigenpairs_by_modulus(*_csr(g), omega)
    d = g.degree.astype(np.float64)
    rows, cols = g.entry_rows(), g.col_idx
    x_e = 1 / d[rows] + 1 / d[cols] - 2 / (d[rows] * d[cols])
    lw = abs(lam[-1])
    tails = {tau: r - series.series_entries(*_csr(g), tau)[0] for tau in range(1, 16, 2)}
    for t in range(1, 16, 2):
        ups, delta = truncation.upsilon_delta(*_csr(g), lam, F, t)
        for tau in range(t, 16, 2):
            bound = delta + lw ** (tau + 1) / (1 - lw * lw) * (x_e - ups)
            assert np.all(tails[tau] <= bound + 1e-13)


@pytest.mark.parametrize("maker", [lambda: gg.tree_plus_gnp(300, 8.0, 0), lambda: gg.barabasi_albert(400, 4, 1),
                                   lambda: gg.petersen(), lambda: gg.lollipop(8, 3), lambda: gg.barbell(12, 1),
                                   lambda: gg.gnp_lcc(200, 5.0, 2)])
@pytest.mark.parametrize("eps", [1e-2, 1e-3])
def test_theorem_3_2_with_caltau(maker, eps):
    g = maker()
    r = exact.exact_dense(*_csr(g))
    _, _, lam_star = truncation.spectrum_extremes(*_csr(g))
    eq6 = truncation.tau_entries(*_csr(g), eps, lam_star)
    rev = series.reverse_entries(*_csr(g))
    for omega in (3, 8, 32, g.n):
        lam, F = truncation.eigenpairs_by_modulus(*_csr(g), omega)
        tau = truncation.caltau(*_csr(g), eps, lam, F)
        assert np.all(tau % 2 == 1) and np.all(tau <= eq6) and np.array_equal(tau, tau[rev])
        s, _ = series.series_entries(*_csr(g), tau)
        assert np.max(np.abs(s - r)) <= eps


def _caltau_brute(g, eps, omega):
    """Algorithm 1 by direct search: the omega remainder weight from the whole
    spectrum, sum_{k >= omega} c_k (1 + lambda_k) / 2m (not X_e - Upsilon), and
    each candidate length found by trying tau = 0, 1, 2, ... (not Eq. 6's
    logarithm)."""
    lam, F = truncation.eigenpairs_by_modulus(*_csr(g), g.n)
    c = _c(g, F)
    two_m = 2.0 * g.m
    lw = abs(lam[omega - 1])
    rest = (1 + lam[omega - 1:]) @ c[omega - 1:] / two_m

    def least_tau(delta, weight, lam_a):
        # least integer tau >= -1 with delta + lam_a^(tau+1) / (1 - lam_a^2) * weight <= eps
        for tau in range(-1, 100_000):
            if delta + lam_a ** (tau + 1) / (1 - lam_a * lam_a) * weight <= eps:
                return tau
        raise AssertionError("no length found")

    x_e = (1 + lam[1:]) @ c[1:] / two_m
    out = np.empty(g.nnz, dtype=np.int64)
    for k in range(g.nnz):
        tau0 = least_tau(0.0, x_e[k], abs(lam[1]))
        tau0 = max(tau0 + (tau0 % 2 == 0), 1)
        t = 1
        while t < tau0:
            delta = (lam[1:omega - 1] ** (t + 1) / (1 - lam[1:omega - 1])) @ c[1:omega - 1, k] / two_m
            if delta > eps:
                f = np.inf
            elif rest[k] <= 1e-15 or lw == 0.0:
                f = -np.inf
            else:
                f = least_tau(delta, rest[k], lw)
            if t > f:
                break
            t += 2
        out[k] = min(t, tau0)
    return out


@pytest.mark.parametrize("maker", [lambda: gg.tree_plus_gnp(60, 4.0, 5), lambda: gg.lollipop(8, 3),
                                   lambda: gg.barbell(6, 1)])
@pytest.mark.parametrize("omega", [3, 8])
def test_caltau_matches_a_direct_search(maker, omega):
    g = maker()
    for eps in (1e-2, 1e-3):
        lam, F = truncation.eigenpairs_by_modulus(*_csr(g), omega)
        assert np.array_equal(truncation.caltau(*_csr(g), eps, lam, F), _caltau_brute(g, eps, omega))


def test_bottleneck_needs_far_fewer_hops():
    """Two K_12 joined by one edge: lambda_2 = 0.987 (the bottleneck), every
    other modulus <= 0.17. Eq. 6 with lambda_2 asks ~490 hops of every edge;
    CalTau with omega = 3 handles the slow mode exactly and most edges need a
    handful."""
    g = gg.barbell(12, 1)
    eps = 1e-2
    _, _, lam_star = truncation.spectrum_extremes(*_csr(g))
    eq6 = truncation.tau_entries(*_csr(g), eps, lam_star)
    lam, F = truncation.eigenpairs_by_modulus(*_csr(g), 3)
    tau = truncation.caltau(*_csr(g), eps, lam, F)
    assert eq6.mean() > 400 and tau.mean() < 10 and np.median(tau) <= 5
    s, _ = series.series_entries(*_csr(g), tau)
    assert np.max(np.abs(s - exact.exact_dense(*_csr(g)))) <= eps


def test_arpack_path_matches_dense():
    g = gg.tree_plus_gnp(1200, 8.0, 9)
    lam_d, F_d = truncation.eigenpairs_by_modulus(*_csr(g), 8)
    lam_s, F_s = truncation.eigenpairs_by_modulus(*_csr(g), 8, dense_max=10)
    assert np.allclose(lam_d, lam_s, atol=1e-10)
    assert np.allclose(_c(g, F_d), _c(g, F_s), atol=1e-8)  # the sign of a vector is free; c_k is not
    for eps in (1e-2, 1e-3):
        assert np.array_equal(truncation.caltau(*_csr(g), eps, lam_d, F_d),
                              truncation.caltau(*_csr(g), eps, lam_s, F_s))


def _caltau_brute_subset(g, eps, used):
    """The remainder form by direct search: the modes `used` (positions in the
    whole spectrum sorted by modulus, 1 = lambda_2) taken exactly, r = the
    largest modulus of every other nontrivial mode, the remainder weight
    sum_{k not used} c_k (1 + lambda_k) / 2m straight from the spectrum, and
    each candidate length found by trying tau = -1, 0, 1, ..."""
    lam, F = truncation.eigenpairs_by_modulus(*_csr(g), g.n)
    c = _c(g, F)
    two_m = 2.0 * g.m
    rest = [k for k in range(1, g.n) if k not in used]
    r = float(np.max(np.abs(lam[rest]))) if rest else 0.0
    rest_w = (1 + lam[rest]) @ c[rest] / two_m
    lam_top = float(np.max(np.abs(lam[1:])))
    x_e = (1 + lam[1:]) @ c[1:] / two_m
    u = np.asarray(used)

    def least_tau(delta, weight, lam_a):
        for tau in range(-1, 100_000):
            if delta + lam_a ** (tau + 1) / (1 - lam_a * lam_a) * weight <= eps:
                return tau
        raise AssertionError("no length found")

    out = np.empty(g.nnz, dtype=np.int64)
    for k in range(g.nnz):
        tau0 = least_tau(0.0, x_e[k], lam_top)
        tau0 = max(tau0 + (tau0 % 2 == 0), 1)
        t = 1
        while t < tau0:
            delta = (lam[u] ** (t + 1) / (1 - lam[u])) @ c[u, k] / two_m
            if delta > eps:
                f = np.inf
            elif rest_w[k] <= 1e-15 or r == 0.0:
                f = -np.inf
            else:
                f = least_tau(delta, rest_w[k], r)
            if t > f:
                break
            t += 2
        out[k] = min(t, tau0)
    return out, lam, F, r


@pytest.mark.parametrize("maker", [lambda: gg.tree_plus_gnp(60, 4.0, 5), lambda: gg.lollipop(8, 3),
                                   lambda: gg.barbell(6, 1)])
@pytest.mark.parametrize("used", [[1, 2], [1, 3, 4], [2], [1, 2, 3, 5, 8]])
def test_remainder_form_matches_a_direct_search(maker, used):
    """Any set of exact modes with r bounding the others: the leading mode left
    out, a gap in the set, the paper's contiguous set."""
    g = maker()
    for eps in (1e-2, 1e-3):
        want, lam, F, r = _caltau_brute_subset(g, eps, used)
        sel = [0] + used
        got = truncation.caltau(*_csr(g), eps, lam[sel], F[sel], lam_rest=r)
        assert np.array_equal(got, want)


def test_remainder_form_with_the_paper_set_is_the_paper_form():
    g = gg.lollipop(8, 3)
    lam, F = truncation.eigenpairs_by_modulus(*_csr(g), 6)
    for eps in (1e-2, 1e-4):
        assert np.array_equal(truncation.caltau(*_csr(g), eps, lam[:5], F[:5], lam_rest=abs(lam[5])),
                              truncation.caltau(*_csr(g), eps, lam, F))


def test_remainder_form_with_one_copy_of_a_repeated_eigenvalue():
    """Two K_12 joined by an edge: -1/11 has a 20-fold eigenspace. A
    single-vector Krylov method sees one vector of it; with that one vector
    taken exactly (with the two modes above it) and r = 1/11 for the rest,
    Theorem 3.2 still holds, and
    still needs far fewer hops than Eq. 6."""
    g = gg.barbell(12, 1)
    lam, F = truncation.eigenpairs_by_modulus(*_csr(g), g.n)
    copies = np.flatnonzero(np.abs(lam + 1.0 / 11.0) < 1e-9)
    assert copies.size >= 18
    sel = [0, 1, 2, int(copies[0])]  # 1, 0.987, -0.161 and one copy of -1/11
    rest = np.setdiff1d(np.arange(1, g.n), sel)
    r = float(np.max(np.abs(lam[rest])))
    assert abs(r - 1.0 / 11.0) < 1e-9
    ex = exact.exact_dense(*_csr(g))
    _, _, lam_star = truncation.spectrum_extremes(*_csr(g))
    for eps in (1e-2, 1e-3):
        tau = truncation.caltau(*_csr(g), eps, lam[sel], F[sel], lam_rest=r)
        s, _ = series.series_entries(*_csr(g), tau)
        assert np.max(np.abs(s - ex)) <= eps
        assert tau.mean() < 0.05 * truncation.tau_entries(*_csr(g), eps, lam_star).mean()
