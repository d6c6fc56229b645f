"""Pins for the meet-in-the-middle form of the series (oracle/meet.py).

  * it equals Algorithm 2's series (the C traversal of oracle/series.py, one
    propagation per source) at per-entry lengths, on graphs with odd and even
    lengths;
  * on K_n it equals the closed form t_l = 2 (-1/(n-1))^l / (n-1), whose sum
    tends to the resistance 2/n;
  * the hop terms equal the matrix-power terms of Eq. 2, every even term is
    non-negative, and at a long length the sum is within Theorem 3.2's tail of
    the exact resistance.
CPU only."""
import numpy as np
import pytest

import graphgen as gg
from oracle import exact, meet, series, truncation


def _csr(g):
    return g.n, g.row_ptr, g.col_idx


@pytest.mark.parametrize("maker", [lambda: gg.lollipop(7, 4), lambda: gg.petersen(), lambda: gg.tree_plus_gnp(120, 5.0, 3),
                                   lambda: gg.barbell(5, 2), lambda: gg.grid(5, 6)])
def test_equals_algorithm_2_at_per_entry_lengths(maker):
    g = maker()
    rng = np.random.default_rng(g.n)
    tau = rng.integers(0, 14, size=g.nnz)
    tau = np.maximum(tau, tau[series.reverse_entries(*_csr(g))])  # one length per edge
    got = meet.series_meet(*_csr(g), tau)
    want, _ = series.series_entries(*_csr(g), tau)
    assert np.max(np.abs(got - want)) < 1e-13


@pytest.mark.parametrize("n", [4, 7, 12])
def test_complete_graph_closed_form(n):
    g = gg.complete(n)
    T = meet.hop_terms_meet(*_csr(g), 9)
    ell = np.arange(10)[:, None]
    want = 2.0 * (-1.0 / (n - 1)) ** ell / (n - 1)
    assert np.max(np.abs(T - want)) < 1e-15
    s = meet.series_meet(*_csr(g), 60)
    assert np.max(np.abs(s - 2.0 / n)) < 1e-15


def test_terms_equal_matrix_powers_and_even_terms_are_non_negative():
    g = gg.tree_plus_gnp(60, 4.0, 8)
    T = meet.hop_terms_meet(*_csr(g), 11)
    d = g.degree.astype(np.float64)
    rows, cols = g.entry_rows(), g.col_idx
    P = np.zeros((g.n, g.n))
    P[rows, cols] = 1.0 / d[rows]
    Pl = np.eye(g.n)
    for ell in range(12):
        term = Pl[rows, rows] / d[rows] + Pl[cols, cols] / d[cols] - Pl[rows, cols] / d[cols] - Pl[cols, rows] / d[rows]
        assert np.max(np.abs(T[ell] - term)) < 1e-14
        Pl = Pl @ P
    assert np.all(T[0::2] >= 0.0)
    assert np.any(T[1::2] < 0.0)  # odd terms carry no sign


def test_long_length_reaches_the_resistance():
    g = gg.lollipop(8, 3)
    _, _, lam = truncation.spectrum_extremes(*_csr(g))
    tau = truncation.tau_entries(*_csr(g), 1e-6, lam)
    s = meet.series_meet(*_csr(g), tau)
    assert np.max(np.abs(s - exact.exact_dense(*_csr(g)))) <= 1e-6
