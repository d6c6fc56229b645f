"""Randomised pins of the oracle (CPU only; skipped where hypothesis is absent):
properties the paper and the mathematics fix, on graphs drawn by hypothesis.

  * exact spanning centrality by the grounded Laplacian equals Kirchhoff's
    matrix-tree theorem (exact rationals) and sums to n - 1 (Foster);
  * the truncated series of Eq. 2 at odd lengths is a non-decreasing lower
    bound of the exact value, and the end-corrected estimator lies between it
    and the exact value (proof of Theorem 3.2: every omitted term pair is >= 0);
  * on a bipartite graph the end-corrected series at odd tau stays a lower
    bound while the plain one carries the -1/m deficit of the lambda = -1 mode;
  * the power-law tail estimate is invariant under scaling the pair sums'
    common factor out of both (it is linear in C) and grows as they decay slower.
"""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import graphgen as gg  # noqa: E402
from oracle import exact, learned, series  # noqa: E402


def _csr(g):
    return g.n, g.row_ptr, g.col_idx


graphs = st.builds(lambda n, d, seed: gg.tree_plus_gnp(n, d, seed),
                   st.integers(min_value=4, max_value=9), st.floats(min_value=2.0, max_value=3.5),
                   st.integers(min_value=0, max_value=10_000))


@settings(max_examples=25, deadline=None)
@given(graphs)
def test_dense_equals_matrix_tree_and_foster(g):
    r = exact.exact_dense(*_csr(g))
    mt = exact.matrix_tree(*_csr(g))
    rows = g.entry_rows()
    for k in range(g.nnz):
        i, j = int(rows[k]), int(g.col_idx[k])
        assert abs(r[k] - float(mt[(min(i, j), max(i, j))])) < 1e-12
    assert abs(0.5 * r.sum() - (g.n - 1)) < 1e-10


@settings(max_examples=25, deadline=None)
@given(st.integers(min_value=6, max_value=40), st.integers(min_value=0, max_value=10_000))
def test_odd_series_rises_to_the_exact_value(n, seed):
    g = gg.tree_plus_gnp(n, 4.0, seed)
    r = exact.exact_dense(*_csr(g))
    prev = np.zeros(g.nnz)
    for tau in (1, 3, 5, 9):
        s, q = series.series_entries(*_csr(g), tau)
        e, _ = series.series_entries(*_csr(g), tau, end_corrected=True)
        assert np.all(s >= prev - 1e-12) and np.all(s <= r + 1e-12)
        assert np.all(e >= s - 1e-12) and np.all(e <= r + 1e-12)
        assert np.all(q >= -1e-12)  # the omitted pair t_{tau+1} + t_{tau+2} is non-negative
        prev = s


@settings(max_examples=10, deadline=None)
@given(st.integers(min_value=3, max_value=6), st.integers(min_value=3, max_value=7),
       st.integers(min_value=0, max_value=1000))
def test_bipartite_end_correction_and_deficit(rows, cols, seed):
    g = gg.perturbed_grid(rows, cols, 0.1, seed)
    r = exact.exact_dense(*_csr(g))
    s, _ = series.series_entries(*_csr(g), 401)
    e, _ = series.series_entries(*_csr(g), 401, end_corrected=True)
    assert np.all(e <= r + 1e-12)
    # the plain series keeps the lambda = -1 mode's deficit: Foster's sum falls short by 1 (1/m per edge)
    assert abs(0.5 * s.sum() - (g.n - 2)) < 1e-6
    assert abs(0.5 * e.sum() - (g.n - 1)) < 1e-6


@settings(max_examples=50, deadline=None)
@given(st.floats(min_value=1.1, max_value=4.0), st.integers(min_value=3, max_value=2001).filter(lambda t: t % 2),
       st.floats(min_value=1e-6, max_value=1e3))
def test_tail_estimate_is_linear_in_the_scale_and_slower_decay_means_more_tail(p, tau, C):
    def est(c, pw):
        return learned.tail_estimate(np.array([c * (tau - 1.0) ** -pw]), np.array([c * (tau + 1.0) ** -pw]), tau)[0]

    a, b = est(C, p), est(2.0 * C, p)
    assert np.isfinite(a) and abs(b - 2.0 * a) <= 1e-9 * abs(b)
    # at the same q(tau), a slower decay (smaller p) leaves more tail
    q = C * (tau + 1.0) ** -p
    slow = learned.tail_estimate(np.array([q * ((tau + 1.0) / (tau - 1.0)) ** (p - 0.05)]), np.array([q]), tau)[0]
    fast = learned.tail_estimate(np.array([q * ((tau + 1.0) / (tau - 1.0)) ** (p + 0.05)]), np.array([q]), tau)[0]
    assert slow >= fast
