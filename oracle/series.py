"""Truncated random-walk series for spanning centrality (oracle O2).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the timed
CPU baseline; the CUDA path never imports it.

The series (Eq. 2) truncated at hop tau:

    s_tau(e_ij) = sum_{l=0}^{tau} p_l(i,i)/d_i + p_l(j,j)/d_j - p_l(i,j)/d_j - p_l(j,i)/d_i,

split into the two half sums of Eq. (9),

    g_tau(v_i, v_j) = sum_{l=0}^{tau} (p_l(v_i,v_i) - p_l(v_j,v_i)) / d(v_i),
    s_tau(e_ij)     = g_tau(v_i, v_j) + g_tau(v_j, v_i)     (Algorithm 2's final combine).

``half_sums`` runs Algorithm 2 in C (oracle.c) for chosen sources and returns
g, plus the hop tau+1 and tau+2 half terms. Both halves of an edge use the
same tau (one truncation length per edge).

Estimators assembled from the half sums:

* plain:          S_tau(e) = g(i,j) + g(j,i)
* end-corrected:  S_tau(e) + t_{tau+1}(e) / 2, where t_l(e) is the full hop-l
                  term of Eq. (2). For odd tau the series tail is
                  sum_k c_k lambda_k^{tau+1} / (1 - lambda_k) with c_k >= 0
                  (proof of Theorem 3.2); adding half of the first omitted
                  term cancels the non-decaying lambda = -1 mode of a
                  bipartite graph exactly and leaves every other mode's tail
                  a non-negative multiple (1+lambda)/2 of its old value.

A-posteriori tail bounds (from the same expansion, q = t_{tau+1} + t_{tau+2}):

* plain:          0 <= s - S_tau <= q / (1 - lambda_star^2)
* end-corrected:  0 <= s - S_hat <= q / (2 (1 - lambda_plus))
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native

__all__ = ["reverse_entries", "half_sums", "series_entries", "tail_bound", "sources_for_pairs"]


def reverse_entries(n, row_ptr, col_idx):
    """rev[k] = index of the CSR entry (j -> i) for entry k = (i -> j)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    cols = np.asarray(col_idx, dtype=np.int64)
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    keys = rows * n + cols
    rev = np.searchsorted(keys, cols * n + rows)
    if np.any(rev >= keys.size) or np.any(keys[np.minimum(rev, keys.size - 1)] != cols * n + rows):
        raise ValueError("CSR is not symmetric")
    return rev


def half_sums(n, row_ptr, col_idx, tau_entries, sources=None, extra_steps: int = 2,
              threads: int = 0):
    """Algorithm 2 in FP64 for ``sources`` (default: every node).

    tau_entries: int per CSR entry (or a scalar for one global length).
    Returns (g, t1, t2), float64 arrays over all CSR entries; entries of rows
    that were not computed hold NaN.
    """
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    nnz = ci.size
    tau = np.broadcast_to(np.asarray(tau_entries, dtype=np.int32), (nnz,))
    tau = np.ascontiguousarray(tau)
    if sources is None:
        src = np.arange(n, dtype=np.int32)
    else:
        src = np.ascontiguousarray(np.unique(np.asarray(sources, dtype=np.int64)), dtype=np.int32)
    g = np.full(nnz, np.nan)
    t1 = np.full(nnz, np.nan)
    t2 = np.full(nnz, np.nan)
    L = _native.lib()
    rc = L.oracle_series(n, _native.ptr(rp, ctypes.c_int32), _native.ptr(ci, ctypes.c_int32),
                         _native.ptr(tau, ctypes.c_int32), int(extra_steps), src.size,
                         _native.ptr(src, ctypes.c_int32), _native.ptr(g, ctypes.c_double),
                         _native.ptr(t1, ctypes.c_double), _native.ptr(t2, ctypes.c_double),
                         threads or _native.default_threads())
    if rc != 0:
        raise RuntimeError("oracle_series failed")
    return g, t1, t2


def series_entries(n, row_ptr, col_idx, tau_entries, sources=None, end_corrected: bool = False,
                   threads: int = 0):
    """Per CSR entry estimate S_tau (or the end-corrected S_hat) and the
    observed pair q = t_{tau+1} + t_{tau+2}; both directions of an edge hold
    the same value. Rows outside ``sources`` (and their partners) are NaN."""
    g, t1, t2 = half_sums(n, row_ptr, col_idx, tau_entries, sources, 2, threads)
    rev = reverse_entries(n, row_ptr, col_idx)
    s = g + g[rev]
    tf1 = t1 + t1[rev]
    tf2 = t2 + t2[rev]
    if end_corrected:
        s = s + 0.5 * tf1
    return s, tf1 + tf2


def tail_bound(q, lam_star: float, lam_plus: float, end_corrected: bool):
    """A-posteriori bound on the remaining tail from the observed pair q."""
    q = np.asarray(q, dtype=np.float64)
    if end_corrected:
        return q / (2.0 * (1.0 - lam_plus))
    return q / (1.0 - lam_star * lam_star)


def sources_for_pairs(pairs):
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    return np.unique(pairs.ravel())
