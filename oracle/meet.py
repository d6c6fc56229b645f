"""Meet-in-the-middle form of the truncated series (Eq. 2): the deterministic
counterpart of the collision view that MonteCarlo-C takes of an l-hop
transition probability (Section 2.3), and the oracle for a traversal that
stops at half the length.

TEST INFRASTRUCTURE ONLY: imported by the tests; the CUDA path never imports it.

For l = a + b steps, the Chapman-Kolmogorov equation and reversibility of the
walk (d_z P^b[z, y] = d_y P^b[y, z]) give

    P^l[x, y] / d_y = sum_z P^a[x, z] P^b[y, z] / d_z,

the D^-1 inner product of the a-step distribution r_a(x) = e_x^T P^a and the
b-step distribution r_b(y). The hop-l term of Eq. 2 for the edge (i, j),
t_l = P^l[i,i]/d_i + P^l[j,j]/d_j - P^l[i,j]/d_j - P^l[j,i]/d_i, is then

    t_l = <u_a, u_b>_{D^-1},   u_h = r_h(i) - r_h(j),   a = floor(l/2), b = l - a,

so S_tau = sum_{l <= tau} t_l needs the distributions of ceil(tau/2) steps
from both endpoints only, and every even term t_{2k} = |u_k|^2_{D^-1} is
non-negative. Dense matrices: small graphs only.
"""
from __future__ import annotations

import numpy as np

__all__ = ["walk_distributions", "hop_terms_meet", "series_meet"]


def _transition(n, row_ptr, col_idx):
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    deg = np.diff(row_ptr).astype(np.float64)
    P = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    P[rows, np.asarray(col_idx, dtype=np.int64)] = 1.0 / deg[rows]
    return P, deg


def walk_distributions(n, row_ptr, col_idx, steps: int):
    """[r_0, ..., r_steps]: r_h[x] = e_x^T P^h, the distribution of a walk of h
    steps from x (row x of P^h), by repeated products with P."""
    P, _ = _transition(n, row_ptr, col_idx)
    R = [np.eye(n)]
    for _ in range(steps):
        R.append(R[-1] @ P)
    return R


def hop_terms_meet(n, row_ptr, col_idx, hops: int):
    """t_l per CSR entry for l = 0..hops (rows: l), each as <u_a, u_b>_{D^-1}."""
    _, deg = _transition(n, row_ptr, col_idx)
    rows = np.repeat(np.arange(n), np.diff(np.asarray(row_ptr, dtype=np.int64)))
    cols = np.asarray(col_idx, dtype=np.int64)
    R = walk_distributions(n, row_ptr, col_idx, (hops + 1) // 2)
    U = [Rh[rows] - Rh[cols] for Rh in R]  # u_h per entry (nnz x n)
    out = np.empty((hops + 1, rows.size))
    for ell in range(hops + 1):
        a = ell // 2
        b = ell - a
        out[ell] = np.sum(U[a] * U[b] / deg[None, :], axis=1)
    return out


def series_meet(n, row_ptr, col_idx, tau_entries):
    """S_tau per CSR entry (tau per entry, or one tau) from the half-length
    distributions: the sum of t_l for l = 0..tau."""
    nnz = len(col_idx)
    tau = np.broadcast_to(np.asarray(tau_entries, dtype=np.int64), (nnz,))
    T = hop_terms_meet(n, row_ptr, col_idx, int(tau.max()))
    ell = np.arange(T.shape[0])[:, None]
    return np.sum(np.where(ell <= tau[None, :], T, 0.0), axis=0)
