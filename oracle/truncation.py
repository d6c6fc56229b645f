"""Eigenvalue bound and truncation lengths (oracle for Eq. 5-6, Algorithm 1's initial length).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the timed
CPU baseline; the CUDA path never imports it.

Spectrum (Lemma 3.1): the eigenvalues of N = D^{1/2} P D^{-1/2} =
D^{-1/2} A D^{-1/2} are those of P; lambda_1 = 1. With them sorted by
absolute value, the paper's lambda_2 is the second largest in absolute value,

    lambda_star = max(|lambda_plus|, |lambda_minus|),

lambda_plus the largest eigenvalue below 1 and lambda_minus the smallest.

Truncation length (Eq. 6 with omega = 2, Upsilon = Delta_t = 0, i.e. the
initial length of Algorithm 1):

    f(e_ij, eps) = ceil( log( X_e / (eps (1 - lambda_star^2)) ) / log(1/lambda_star) - 1 ),
    X_e = 1/d_i + 1/d_j - 2/(d_i d_j),

and tau_ij is the smallest odd integer >= f (Eq. 5), at least 1. The per
source length of Algorithm 2's per-source length is tau_p(i) = max_j tau_ij; the global length
is max over all edges.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["spectrum_extremes", "f_edge", "odd_ceil", "tau_entries", "tau_per_source",
           "peng_tau"]


def _normalized_adjacency(n, row_ptr, col_idx):
    import scipy.sparse as sp

    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    deg = np.diff(row_ptr).astype(np.float64)
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    cols = np.asarray(col_idx, dtype=np.int64)
    vals = 1.0 / np.sqrt(deg[rows] * deg[cols])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n)), deg


def spectrum_extremes(n, row_ptr, col_idx, dense_max: int = 3000, tol: float = 1e-12):
    """(lambda_plus, lambda_minus, lambda_star) of N.

    Dense symmetric eigensolver for n <= dense_max, else ARPACK Lanczos
    (scipy eigsh) on N with the top eigenvector sqrt(d)/sqrt(2m) deflated.
    """
    nmat, deg = _normalized_adjacency(n, row_ptr, col_idx)
    if n <= dense_max:
        w = np.linalg.eigvalsh(nmat.toarray())  # ascending
        lam_minus = float(w[0])
        lam_plus = float(w[-2])
    else:
        import scipy.sparse.linalg as spla

        phi = np.sqrt(deg)
        phi /= np.linalg.norm(phi)

        def mv(x):
            y = nmat @ x
            return y - phi * (phi @ y)

        op = spla.LinearOperator((n, n), matvec=mv, dtype=np.float64)
        v0 = np.ones(n) - phi * phi.sum()
        lam_plus = float(spla.eigsh(op, k=1, which="LA", tol=tol, v0=v0, ncv=64,
                                    return_eigenvectors=False)[0])
        lam_minus = float(spla.eigsh(op, k=1, which="SA", tol=tol, v0=v0, ncv=64,
                                     return_eigenvectors=False)[0])
    lam_star = max(abs(lam_plus), abs(lam_minus))
    return lam_plus, lam_minus, lam_star


def f_edge(d_i, d_j, eps: float, lam: float):
    """Eq. (6) with omega = 2 and Upsilon = Delta_t = 0 (real-valued argument
    of the ceiling is returned as an integer array)."""
    d_i = np.asarray(d_i, dtype=np.float64)
    d_j = np.asarray(d_j, dtype=np.float64)
    x_e = 1.0 / d_i + 1.0 / d_j - 2.0 / (d_i * d_j)
    if lam <= 0.0:
        return np.zeros_like(x_e, dtype=np.int64)
    if lam >= 1.0:
        raise ValueError("lambda_star >= 1: the series does not converge (bipartite or disconnected)")
    with np.errstate(divide="ignore"):
        val = np.log(x_e / (eps * (1.0 - lam * lam))) / math.log(1.0 / lam) - 1.0
    # x_e == 0 (both endpoints of degree 1: a single-edge component) needs no terms
    val = np.where(x_e > 0.0, val, -np.inf)
    return np.ceil(val)


def odd_ceil(f):
    """Smallest odd integer >= f, and at least 1 (Eq. 5)."""
    f = np.asarray(f, dtype=np.float64)
    t = np.maximum(np.ceil(f), 1.0).astype(np.int64)
    return np.where(t % 2 == 0, t + 1, t)


def tau_entries(n, row_ptr, col_idx, eps: float, lam_star: float):
    """tau_ij for every CSR entry (same value in both directions)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    deg = np.diff(row_ptr)
    rows = np.repeat(np.arange(n), deg)
    cols = np.asarray(col_idx, dtype=np.int64)
    return odd_ceil(f_edge(deg[rows], deg[cols], eps, lam_star))


def tau_per_source(n, row_ptr, tau_k):
    """Algorithm 2's per-source length: tau_p(i) = max over the entries of row i."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    out = np.zeros(n, dtype=np.int64)
    deg = np.diff(row_ptr)
    rows = np.repeat(np.arange(n), deg)
    np.maximum.at(out, rows, np.asarray(tau_k, dtype=np.int64))
    return out


def peng_tau(eps: float, lam: float):
    """Eq. (3): Peng et al.'s global truncation length (reported for contrast)."""
    return int(math.ceil(math.log(4.0 / (eps - eps * lam)) / math.log(1.0 / lam) - 1.0))
