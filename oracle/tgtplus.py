"""TGT+ pieces (oracle O3): CalChi, walk counts, the walk estimator, the switch rule.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the timed
CPU baseline; the CUDA path never imports it.

Notation: p = p_{tt}(., v_i), the column of the source v_i after tt hops (tt
is the switch length written tau-tilde in Section 4); L = tau_ij - tt is the
walk length for the entry (i -> j).

* Lemma 4.3: for a walk W of length L >= 1 from v,
      LB(v, L) = min_{N(v)} p + (L - 1) min_V p
      UB(v, L) = max_{N(v)} p / 2 + max_V p / 2 + (L - 1) rho / 2,
  rho = max over edges (x, y) of p(x) + p(y) (Eq. 16).
* Eq. 17: chi = UB(v_i, L) + UB(v_j, L) - LB(v_i, L) - LB(v_j, L); with
  gamma = 0, Eq. 15: chi = 2 L (max_V p - min_V p).
* Alg. 3 (CalChi): C = the gamma nodes of largest p (ties: smaller id first);
  rho_hat from the edges inside C, else p(c_1) + p(c_gamma). Reading taken
  here: rho_hat = max(largest p(c_a) + p(c_b) over edges inside C,
  p(c_1) + p(c_gamma)). An edge with one end outside C sums to at most
  p(c_1) + p(c_gamma), so this is always an upper bound of rho; Algorithm 3 as
  printed keeps only the first term when an edge exists inside C, which can be
  below rho (``calchi(..., literal=True)`` computes that version).
* Eq. 13: R = ceil(8 chi^2 log(2m/delta) / (d_i^2 eps^2)), at least 1.
* Eq. 11: X = (sum_{t=1..L} p(W_i[t]) - sum_{t=1..L} p(W_j[t])) / d_i, walks
  W_i from v_i and W_j from v_j; positions 1..L, the start excluded.
* Eq. 14: switch to walks after hop l when
  sum_{x: p_l(x, v_i) != 0} d(x) > sum_j R(e_ij, tau_ij - l);
  ``switch_hop`` tests it per source from l = 0, as Algorithm 4 prints it.

Random numbers: walk w of entry k takes its step t (t = 1..L) from word
(t-1) mod 4 of Philox4x32-10 with counter (k, w, side * 2^31 + (t-1) div 4,
0x57414C4B) and key (seed mod 2^32, seed div 2^32); side 0 is the walk from
v_i, side 1 the walk from v_j; the neighbour is N(cur)[floor(u d / 2^32)].
"""
from __future__ import annotations

import math

import numpy as np

from .philox import philox4x32_10, uniform_index

WALK_TAG = 0x57414C4B


def _nbrs(row_ptr, col_idx, v):
    return col_idx[row_ptr[v]:row_ptr[v + 1]]


def top_candidates(p, gamma):
    """Algorithm 3's candidate set: the gamma largest entries of p, ties by smaller node id."""
    order = np.lexsort((np.arange(p.size), -p))
    return order[:gamma]


def rho_hat(row_ptr, col_idx, p, gamma, literal=False):
    """Upper bound of rho (Eq. 16) from the candidate set C (Algorithm 3)."""
    C = top_candidates(p, gamma)
    best = -np.inf
    cset = set(C.tolist())
    for a in C.tolist():
        for b in _nbrs(row_ptr, col_idx, a).tolist():
            if b in cset and a < b:
                best = max(best, p[a] + p[b])
    two = p[C[0]] + p[C[-1]]
    if literal:
        return best if best > -np.inf else two
    return max(best, two)


def rho_exact(row_ptr, col_idx, p):
    """Eq. 16 by brute force over every edge."""
    n = p.size
    rows = np.repeat(np.arange(n), np.diff(np.asarray(row_ptr, dtype=np.int64)))
    return float(np.max(p[rows] + p[np.asarray(col_idx)]))


def lemma43(row_ptr, col_idx, p, v, L, rho):
    """(LB(v, L), UB(v, L)) of Lemma 4.3."""
    nb = p[_nbrs(row_ptr, col_idx, v)]
    lb = nb.min() + (L - 1) * p.min()
    ub = nb.max() / 2.0 + p.max() / 2.0 + (L - 1) * rho / 2.0
    return lb, ub


def calchi(row_ptr, col_idx, p, i, j, L, gamma, literal=False):
    """Alg. 3 for the entry (i -> j) with walk length L."""
    if gamma == 0:
        return 2.0 * L * (p.max() - p.min())  # Eq. 15
    rho = rho_hat(row_ptr, col_idx, p, gamma, literal)
    lb_i, ub_i = lemma43(row_ptr, col_idx, p, i, L, rho)
    lb_j, ub_j = lemma43(row_ptr, col_idx, p, j, L, rho)
    return ub_i + ub_j - lb_i - lb_j  # Eq. 17


def walk_count(chi, d_i, m, delta, eps):
    """Eq. 13, rounded up, at least one walk pair."""
    r = 8.0 * chi * chi * math.log(2.0 * m / delta) / (d_i * d_i * eps * eps)
    return max(1, int(math.ceil(r)))


def walk_sums(row_ptr, col_idx, p, start, L, k, R, side, seed):
    """sum_{t=1..L} p(W[t]) for the R walks of entry k on one side (vector of R)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col_idx = np.asarray(col_idx, dtype=np.int64)
    w = np.arange(R, dtype=np.uint64).astype(np.uint32)
    cur = np.full(R, start, dtype=np.int64)
    total = np.zeros(R)
    k0 = np.uint32(seed & 0xFFFFFFFF)
    k1 = np.uint32((seed >> 32) & 0xFFFFFFFF)
    words = None
    for t in range(1, L + 1):
        q, r = divmod(t - 1, 4)
        if r == 0:
            words = philox4x32_10(np.uint32(k), w, np.uint32((side << 31) | q), np.uint32(WALK_TAG), k0, k1)
        deg = row_ptr[cur + 1] - row_ptr[cur]
        idx = uniform_index(words[r], deg)
        cur = col_idx[row_ptr[cur] + idx]
        total += p[cur]
    return total


def walk_estimate(row_ptr, col_idx, p, i, j, L, k, R, seed):
    """Mean of X (Eq. 11) over R walk pairs, times d_i (unscaled by 1/d_i)."""
    si = walk_sums(row_ptr, col_idx, p, i, L, k, R, 0, seed)
    sj = walk_sums(row_ptr, col_idx, p, j, L, k, R, 1, seed)
    return float(np.mean(si - sj))


def frontier_volume(row_ptr, p):
    """Left side of Eq. 14: sum of d(x) over nodes with p(x) != 0."""
    deg = np.diff(np.asarray(row_ptr, dtype=np.int64))
    return int(deg[p != 0].sum())


def source_column(n, row_ptr, col_idx, i, hops):
    """p_hops(., v_i) = P^hops e_i by repeated push hops (Algorithm 2's hop)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    deg = np.diff(row_ptr)
    p = np.zeros(n)
    p[i] = 1.0
    for _ in range(hops):
        q = np.zeros(n)
        for v in np.flatnonzero(p > 0):
            nb = col_idx[row_ptr[v]:row_ptr[v + 1]]
            q[nb] += p[v] / deg[nb]
        p = q
    return p


def switch_hop(n, row_ptr, col_idx, i, tau_row, eps, delta, gamma, m):
    """Algorithm 4's switch length for source v_i, Eq. 14 tested per source as
    printed: from l = 0 (p_0 = e_i), while the frontier volume of p_l(., v_i) is
    at most sum_j R(e_ij, tau_ij - l) over the neighbours with tau_ij - l > 0
    (chi from Alg. 3 on p_l, R from Eq. 13), take one more hop; the l at which
    it first exceeds it is tau-tilde. Once every tau_ij <= l the right side is
    empty, so tau-tilde <= max_j tau_ij."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    nbr = col_idx[row_ptr[i]:row_ptr[i + 1]]
    d_i = len(nbr)
    deg = np.diff(row_ptr)
    p = np.zeros(n)
    p[i] = 1.0
    ell = 0
    while True:
        rhs = 0
        for t, j in enumerate(nbr):
            L = int(tau_row[t]) - ell
            if L > 0:
                rhs += walk_count(calchi(row_ptr, col_idx, p, i, int(j), L, gamma), d_i, m, delta, eps)
        if frontier_volume(row_ptr, p) > rhs:
            return ell
        q = np.zeros(n)
        for v in np.flatnonzero(p > 0):
            nb = col_idx[row_ptr[v]:row_ptr[v + 1]]
            q[nb] += p[v] / deg[nb]
        p = q
        ell += 1


def tgt_plus_half(n, row_ptr, col_idx, i, tau_row, tt, eps, delta, gamma, seed, m):
    """Algorithm 4 for source v_i with the switch length tt given.

    tau_row: tau_ij for the entries of row i. Returns (g_hat unscaled per entry
    of row i, R per entry, chi per entry): g_hat = sum_{l <= min(tau_ij, tt)}
    (p_l(i,i) - p_l(j,i)) plus, where tau_ij > tt, the walk mean of Eq. 11 times
    d_i (the combine divides by d_i).
    """
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    nbr = col_idx[row_ptr[i]:row_ptr[i + 1]]
    k0 = row_ptr[i]
    d_i = len(nbr)
    g = np.ones(d_i)  # hop 0
    p = np.zeros(n)
    p[i] = 1.0
    deg = np.diff(row_ptr)
    for l in range(1, tt + 1):
        q = np.zeros(n)
        for v in np.flatnonzero(p > 0):
            nb = col_idx[row_ptr[v]:row_ptr[v + 1]]
            q[nb] += p[v] / deg[nb]
        p = q
        for t, j in enumerate(nbr):
            if l <= tau_row[t]:
                g[t] += p[i] - p[j]
    R = np.zeros(d_i, dtype=np.int64)
    chi = np.zeros(d_i)
    for t, j in enumerate(nbr):
        L = int(tau_row[t]) - tt
        if L <= 0:
            continue
        chi[t] = calchi(row_ptr, col_idx, p, i, j, L, gamma)
        R[t] = walk_count(chi[t], d_i, m, delta, eps)
        g[t] += walk_estimate(row_ptr, col_idx, p, i, j, L, k0 + t, int(R[t]), seed)
    return g, R, chi
