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

With omega > 2 eigenpairs (Algorithm 1, CalTau): eigenvalues of N sorted by
modulus, lambda_1 = 1 first, with f_k = sqrt(2m) D^{-1/2} phi_k (Lemma 3.1,
Theorem 3.2; f_1 = 1). For an edge e = (i, j) let c_k = (f_k[i] - f_k[j])^2.
Then (proof of Theorem 3.2) the terms of Eq. 2 are
t_l(e) = (1/2m) sum_k c_k lambda_k^l, X_e = (1/2m) sum_{k>=2} c_k (1 + lambda_k),
and for odd t <= tau the tail after tau is at most

    Delta_t + lambda_omega^(tau+1) / (1 - lambda_omega^2) * (X_e - Upsilon),

Upsilon = Eq. 7, Delta_t = Eq. 8 (sums over k = 2 .. omega-1). Eq. 6 with
Upsilon and Delta_t gives the least tau for which this is <= eps. CalTau
starts from Eq. 6 with lambda_2 alone, then walks t = 1, 3, 5, ... while t <=
Eq. 6(Delta_t) and returns the first t above it. Reading taken: the result is
min(t, the starting length), both of which meet Theorem 3.2; with omega = 2
this is the starting length, i.e. Eq. 6 with lambda_star.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["spectrum_extremes", "f_edge", "odd_ceil", "tau_entries", "tau_per_source",
           "peng_tau", "eigenpairs_by_modulus", "upsilon_delta", "caltau"]


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


def eigenpairs_by_modulus(n, row_ptr, col_idx, omega: int, dense_max: int = 3000):
    """The omega eigenvalues of N of largest modulus, lambda_1 = 1 first (ties in
    modulus: the larger value first), and f_k = sqrt(2m) D^{-1/2} phi_k as the
    rows of F (omega x n), f_1 = 1. Dense symmetric solver for n <= dense_max,
    else ARPACK (largest magnitude)."""
    nmat, deg = _normalized_adjacency(n, row_ptr, col_idx)
    omega = int(min(omega, n))
    if n <= dense_max:
        w, vec = np.linalg.eigh(nmat.toarray())
    else:
        import scipy.sparse.linalg as spla

        w, vec = spla.eigsh(nmat, k=omega, which="LM", tol=1e-12, ncv=max(2 * omega + 1, 64))
    order = np.lexsort((-w, -np.abs(w)))[:omega]
    lam = w[order]
    F = np.sqrt(deg.sum()) * (vec[:, order] / np.sqrt(deg)[:, None]).T
    F[0] = 1.0
    lam[0] = 1.0
    return lam, F


def _entry_terms(n, row_ptr, col_idx):
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    deg = np.diff(row_ptr).astype(np.float64)
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    cols = np.asarray(col_idx, dtype=np.int64)
    return deg, rows, cols


def upsilon_delta(n, row_ptr, col_idx, lam, F, t: int):
    """Eq. 7 and Eq. 8 per CSR entry for the eigenpairs k = 2 .. omega-1."""
    deg, rows, cols = _entry_terms(n, row_ptr, col_idx)
    two_m = deg.sum()
    mid = np.asarray(lam[1:len(lam) - 1], dtype=np.float64)
    c = (F[1:len(lam) - 1][:, rows] - F[1:len(lam) - 1][:, cols]) ** 2
    ups = ((1.0 + mid) @ c) / two_m
    delta = ((mid ** (t + 1) / (1.0 - mid)) @ c) / two_m
    return ups, delta


def _eq6(num, budget, lam_w):
    """Ceiling argument of Eq. 6 for remainder weight num = X_e - Upsilon and error
    budget eps - Delta_t: -inf when nothing remains, +inf when the budget is spent."""
    out = np.empty(num.shape)
    none_left = (num <= 0.0) | (lam_w == 0.0)  # the omega remainder term is zero
    spent = (budget < 0.0) | (~none_left & (budget == 0.0))  # Delta_t alone exceeds eps
    ok = ~none_left & ~spent
    out[none_left & ~spent] = -np.inf
    out[spent] = np.inf
    out[ok] = np.ceil(np.log(num[ok] / (budget[ok] * (1.0 - lam_w * lam_w))) / math.log(1.0 / lam_w) - 1.0)
    return out


def caltau(n, row_ptr, col_idx, eps: float, lam, F, lam_rest=None):
    """Algorithm 1 (CalTau) for every CSR entry with the omega = len(lam)
    eigenpairs of eigenpairs_by_modulus (lambda_1 = 1 first).

    lam_rest None: the paper's form, modes 2 .. omega-1 taken exactly and
    |lambda_omega| bounding the modulus of every mode after them.
    lam_rest = r: every given pair 2 .. omega is taken exactly and r bounds the
    modulus of every nontrivial mode that is not given. The proof of Theorem
    3.2 needs no more than that (each left-out term c_k lambda_k^(t+1) /
    (1 - lambda_k) is at most r^(t+1) / (1 - r^2) c_k (1 + lambda_k)), so the
    given pairs need not be the leading ones nor all copies of a repeated
    eigenvalue; this is the paper's form with r in the last place."""
    lam = np.asarray(lam, dtype=np.float64)
    if lam_rest is not None:
        lam = np.append(lam, float(lam_rest))
        F = np.vstack([np.asarray(F, dtype=np.float64), np.zeros((1, n))])
    omega = lam.size
    if omega < 2:
        raise ValueError("CalTau needs lambda_2")
    lam_top = float(np.max(np.abs(lam[1:])))  # lambda_star: the largest nontrivial modulus
    if lam_top >= 1.0:
        raise ValueError("|lambda_2| >= 1: the series does not converge (bipartite or disconnected)")
    deg, rows, cols = _entry_terms(n, row_ptr, col_idx)
    tau0 = odd_ceil(f_edge(deg[rows], deg[cols], eps, lam_top))  # Eq. 6 with lambda_star alone
    if omega == 2:
        return tau0
    d_i, d_j = deg[rows], deg[cols]
    x_e = 1.0 / d_i + 1.0 / d_j - 2.0 / (d_i * d_j)
    lam_w = abs(lam[omega - 1])
    ups, _ = upsilon_delta(n, row_ptr, col_idx, lam, F, 1)
    mid = lam[1:omega - 1]
    c = (F[1:omega - 1][:, rows] - F[1:omega - 1][:, cols]) ** 2
    two_m = deg.sum()
    out = tau0.copy()
    t = 1
    active = t < tau0
    while active.any():
        idx = np.flatnonzero(active)
        delta = ((mid ** (t + 1) / (1.0 - mid)) @ c[:, idx]) / two_m  # Eq. 8 at this t
        f = _eq6(x_e[idx] - ups[idx], eps - delta, lam_w)
        stop = t > f  # Eq. 6 with Delta_t no longer reaches t: t meets Theorem 3.2
        out[idx[stop]] = t
        active[idx[stop]] = False
        t += 2
        active &= t < tau0  # from here on the starting length is the shorter one
    return out
