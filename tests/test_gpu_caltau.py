"""GPU parity of CalTau with omega eigenpairs (Algorithm 1, Eq. 6-8) through
the C ABI against the oracle.

Tolerances:
  * lengths are integers decided in FP64 on both sides, but the sums of Eq. 7
    and Eq. 8 run in other orders (a warp tree here, BLAS there), so an edge
    whose Eq. 6 argument lies within rounding of an integer may land on the
    next odd length. Every GPU length lies between the oracle's at eps (1 +
    1e-9) and at eps (1 - 1e-9) (CalTau is monotone in eps), and at least 99%
    equal the oracle's at eps;
  * Ritz values against the dense spectrum: 1e-8 (the residual tolerance of
    the pairs taken); c_k = (f_k[i] - f_k[j])^2 against the dense vectors of a
    simple eigenvalue: 1e-5 relative to max c_k (a Ritz vector's error is at
    most its residual, <= 1e-8, over the gap to the rest of the spectrum,
    Davis-Kahan; gaps here are above 1e-3; a numpy model of the two runs,
    over six start vectors, stays below 1.3e-7);
  * the series at the CalTau lengths: 1e-12 (FP64 blocks), and within eps of
    the exact value (Theorem 3.2).

The file is named so that pytest collects it after the other GPU suites.
"""
import numpy as np
import pytest

import graphgen as gg
from oracle import exact, series, truncation

pytestmark = pytest.mark.gpu

GRAPHS = [lambda: gg.barbell(12, 1), lambda: gg.lollipop(30, 12), lambda: gg.tree_plus_gnp(600, 6.0, 1),
          lambda: gg.barabasi_albert(800, 3, 2)]


def _csr(g):
    return g.n, g.row_ptr, g.col_idx


def _bracketed(got, g, eps, lam, F, lam_rest=None):
    lo = truncation.caltau(*_csr(g), eps * (1 + 1e-9), lam, F, lam_rest=lam_rest)
    hi = truncation.caltau(*_csr(g), eps * (1 - 1e-9), lam, F, lam_rest=lam_rest)
    want = truncation.caltau(*_csr(g), eps, lam, F, lam_rest=lam_rest)
    assert np.all((lo <= got) & (got <= hi)), np.flatnonzero((got < lo) | (got > hi))[:10]
    assert np.mean(got == want) >= 0.99
    return want


@pytest.mark.parametrize("maker", GRAPHS)
@pytest.mark.parametrize("omega", [3, 16])
def test_caltau_kernel_matches_the_oracle_on_the_same_pairs(cuda_lib, maker, omega):
    from paper_2305_16086_gb300 import Graph

    g = maker()
    lam, F = truncation.eigenpairs_by_modulus(*_csr(g), omega)
    with Graph(g.row_ptr, g.col_idx) as G:
        for eps in (1e-2, 1e-3):
            # the paper's form: modes 2 .. omega-1 exact, |lambda_omega| for the rest
            tau, ell = G.caltau(eps, lam[:omega - 1], F[:omega - 1], lam_rest=abs(lam[omega - 1]))
            _bracketed(tau, g, eps, lam, F)
            assert ell == tau.max() and np.array_equal(tau, tau[series.reverse_entries(*_csr(g))])


def test_caltau_kernel_with_a_gap_and_one_copy(cuda_lib):
    """The remainder form: one copy of the 20-fold -1/11 of two joined K_12."""
    from paper_2305_16086_gb300 import Graph

    g = gg.barbell(12, 1)
    lam, F = truncation.eigenpairs_by_modulus(*_csr(g), g.n)
    copies = np.flatnonzero(np.abs(lam + 1.0 / 11.0) < 1e-9)
    sel = [0, 1, 2, int(copies[0])]
    with Graph(g.row_ptr, g.col_idx) as G:
        for eps in (1e-2, 1e-3):
            tau, _ = G.caltau(eps, lam[sel], F[sel], lam_rest=1.0 / 11.0)
            _bracketed(tau, g, eps, lam[sel], F[sel], lam_rest=1.0 / 11.0)


@pytest.mark.parametrize("maker", GRAPHS)
def test_eigenpairs_against_the_dense_spectrum(cuda_lib, maker):
    from paper_2305_16086_gb300 import Graph

    g = maker()
    lam_all, F_all = truncation.eigenpairs_by_modulus(*_csr(g), g.n)
    with Graph(g.row_ptr, g.col_idx) as G:
        lam, F, rep = G.eigenpairs(omega=16)
    used = rep["used"]
    assert 2 <= used <= 16 and lam[0] == 1.0 and np.all(F[0] == 1.0)
    assert np.all(lam[used:] == 0.0) and np.all(F[used:] == 0.0)
    assert np.all(np.diff(np.abs(lam[1:used])) <= 1e-12)  # by decreasing modulus
    rows, cols = g.entry_rows(), g.col_idx
    taken = []
    for k in range(1, used):
        gap = np.abs(lam_all[1:] - lam[k])
        q = 1 + int(np.argmin(gap))
        assert gap[q - 1] < 1e-8, (k, lam[k])
        taken.append(q)
        mult = np.sum(np.abs(lam_all[1:] - lam_all[q]) < 1e-9)
        if mult == 1:  # a simple eigenvalue: the vector is fixed up to sign
            c_gpu = (F[k, rows] - F[k, cols]) ** 2
            c_ref = (F_all[q, rows] - F_all[q, cols]) ** 2
            assert np.max(np.abs(c_gpu - c_ref)) < 1e-5 * max(c_ref.max(), 1e-30)
    # r bounds every nontrivial mode not taken (one copy per taken value removed)
    rest = np.setdiff1d(np.arange(1, g.n), taken)
    assert rep["lambda_rest"] >= np.max(np.abs(lam_all[rest])) - 1e-9
    assert rep["lambda_rest"] <= np.max(np.abs(lam_all[rest])) + 1e-5
    assert rep["rest_converged"] == 1


@pytest.mark.parametrize("maker", GRAPHS)
def test_caltau_policy_meets_theorem_3_2(cuda_lib, maker):
    """Device eigenpairs -> device CalTau -> sc_all_edges with SC_ELL_CALTAU:
    the oracle's remainder form on the same pairs gives the same lengths, the
    series at those lengths matches, every edge is within eps of the exact
    value, and no length exceeds Eq. 6's."""
    from paper_2305_16086_gb300 import Graph

    g = maker()
    r = exact.exact_dense(*_csr(g))
    _, _, lam_star = truncation.spectrum_extremes(*_csr(g))
    with Graph(g.row_ptr, g.col_idx) as G:
        lam, F, rep = G.eigenpairs(omega=16)
        used = rep["used"]
        for eps in (1e-2, 1e-3):
            tau, ell = G.caltau(eps)
            _bracketed(tau, g, eps, lam[:used], F[:used], lam_rest=rep["lambda_rest"])
            assert np.all(tau <= truncation.tau_entries(*_csr(g), eps, lam_star + 1e-5))  # r carries residual margins
            s, _, rp = G.all_edges(eps=eps, policy="caltau", precision="fp64")
            ref, _ = series.series_entries(*_csr(g), tau)
            assert np.max(np.abs(s - ref)) < 1e-12
            assert np.max(np.abs(s - r)) <= eps
            assert rp["ell_global"] == ell


def test_bottleneck_lengths_drop(cuda_lib):
    from paper_2305_16086_gb300 import Graph

    g = gg.barbell(12, 1)
    with Graph(g.row_ptr, g.col_idx) as G:
        G.eigenpairs(omega=8)
        tau, _ = G.caltau(1e-2)
        G.estimate_lambda()
        _, _, pe = G.truncation_length(1e-2)
    assert pe.mean() > 400 and tau.mean() < 10


def test_caltau_errors(cuda_lib):
    from paper_2305_16086_gb300 import Graph, ScError

    g = gg.cycle(8)  # bipartite
    with Graph(g.row_ptr, g.col_idx) as G:
        with pytest.raises(ScError, match="SC_ERR_UNSUPPORTED"):
            G.eigenpairs(omega=4)
    g = gg.lollipop(8, 3)
    with Graph(g.row_ptr, g.col_idx) as G:
        with pytest.raises(ScError, match="SC_ERR_INVALID_ARG"):
            G.caltau(1e-2)  # no pairs yet
        with pytest.raises(ScError, match="SC_ERR_INVALID_ARG"):
            G.all_edges(eps=1e-2, policy="caltau")  # no lengths yet
        G.eigenpairs(omega=4)
        G.caltau(1e-2)
        with pytest.raises(ScError, match="SC_ERR_INVALID_ARG"):
            G.all_edges(eps=1e-3, policy="caltau")  # lengths of another eps
        with pytest.raises(ScError, match="SC_ERR_INVALID_ARG"):
            G.eigenpairs(omega=1)
        lam, F = truncation.eigenpairs_by_modulus(*_csr(g), 3)
        with pytest.raises(ScError, match="SC_ERR_INVALID_ARG"):
            G.caltau(1e-2, lam, F, lam_rest=1.0)


@pytest.mark.slow
def test_planted_partition_sampled_within_eps(cuda_lib):
    """16 communities of 2,500 nodes (15 eigenvalues near 1): the device pairs
    take the slow modes exactly, every sampled edge is within eps of the CG
    value, and the lengths are a fraction of Eq. 6's."""
    from paper_2305_16086_gb300 import Graph

    g = gg.planted_partition(16, 2500, 10.0, 0.3, 7)
    rng = np.random.default_rng(7)
    e = g.edges()
    pick = e[rng.choice(e.shape[0], size=300, replace=False)]
    k = exact.entry_of_edges(g.n, g.row_ptr, g.col_idx, pick)
    r = exact.exact_cg(g.n, g.row_ptr, g.col_idx, pick)
    with Graph(g.row_ptr, g.col_idx) as G:
        lam, _, rep = G.eigenpairs(omega=32)
        assert rep["used"] >= 16 and np.all(lam[1:16] > 0.9)
        tau, _ = G.caltau(1e-3)
        s, _, _ = G.all_edges(eps=1e-3, policy="caltau", precision="fp32")
        G.estimate_lambda()
        _, _, pe = G.truncation_length(1e-3)
    assert np.max(np.abs(s[k] - r)) <= 1e-3
    assert tau.mean() < 0.2 * pe.mean()
