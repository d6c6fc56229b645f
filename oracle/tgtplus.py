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


# ---------------------------------------------------------------------------
# TGT+ at per-source lengths (the learned length; not in the paper) with the
# truncation certified after the run.
#
# For odd tau and even l <= tau + 1 the tail of Eq. 2 past tau is at most
# lam*^(tau + 1 - l) / (1 - lam*) t_l(e). The expansion in the proof of
# Theorem 3.2 writes the tail as sum_k c_k lam_k^(tau+1) / (1 - lam_k) with
# c_k >= 0, and the hop-l term as t_l(e) = sum_k c_k lam_k^l, whose terms are
# all >= 0 for even l. Each tail term then splits as c_k lam_k^l (>= 0) times
# lam_k^(tau+1-l), an even power at most lam*^(tau+1-l), over 1 - lam_k >= 1 - lam*.
# The bound needs one hop term, and only one the traversal has already reached,
# so TGT+ can certify a length its walks run past.
# ---------------------------------------------------------------------------

def even_hop_bound(t_l, ell, tau, lam_star):
    """lam*^(tau + 1 - ell) / (1 - lam*) * t_l: the power by repeated
    multiplication (tau odd, ell even, ell <= tau + 1)."""
    f = 1.0
    for _ in range(tau + 1 - ell):
        f *= lam_star
    return f / (1.0 - lam_star) * t_l


def tgt_plus_learned(n, row_ptr, col_idx, L_src, cap, eps, lam_star, delta, gamma, seed, m, depth_cap=16,
                     max_rounds=64):
    """TGT+ (Algorithm 4, the switch of Eq. 14 per source as printed) at the
    per-source lengths L_src (odd, at most cap = Eq. 6's length at eps / 2).
    tau_e = min(L_i, L_j) for both halves of an edge. After the run each edge
    is certified with eps / 2 for the truncation (Algorithm 4's split: the
    walks take the other eps / 2) by ``even_hop_bound`` at
    l* = the largest even hop <= min(tt_i, tt_j, tau_e + 1, depth_cap) (tt =
    the source's switch hop: its traversal reached it); an edge that fails
    takes the least odd tau > tau_e the same bound accepts (at most cap), and
    both endpoints run again. Returns (s_hat per entry, tau per entry, tt per
    source (its last run), rounds with an extension, (smallest, largest) tt
    over every run)."""
    from . import series

    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col_idx = np.asarray(col_idx)
    deg = np.diff(row_ptr)
    rows = np.repeat(np.arange(n), deg)
    rev = series.reverse_entries(n, row_ptr, col_idx)
    L_src = np.asarray(L_src, dtype=np.int64)
    tau = np.minimum(L_src[rows], L_src[col_idx])
    half = np.zeros(col_idx.size)           # g_hat(v_i, v_j) / d_i per entry
    even = np.zeros((col_idx.size, depth_cap // 2 + 1))  # (p_l(i,i) - p_l(j,i)) / d_i at even l
    tt = np.zeros(n, dtype=np.int64)
    need = list(range(n))
    rounds = 0
    seen = [None, None]
    for _ in range(max_rounds + 1):
        for i in need:
            a, b = row_ptr[i], row_ptr[i + 1]
            t_i = switch_hop(n, row_ptr, col_idx, i, tau[a:b], eps, delta, gamma, m)
            seen = [t_i if seen[0] is None else min(seen[0], t_i), t_i if seen[1] is None else max(seen[1], t_i)]
            g_i, _, _ = tgt_plus_half(n, row_ptr, col_idx, i, tau[a:b], t_i, eps, delta, gamma, seed, m)
            half[a:b] = g_i / deg[i]
            tt[i] = t_i
            nbr = col_idx[a:b]
            for ell in range(0, min(t_i, depth_cap) + 1, 2):
                p = source_column(n, row_ptr, col_idx, i, ell)
                even[a:b, ell // 2] = (p[i] - p[nbr]) / deg[i]
        redo = set()
        for k in range(col_idx.size):
            i, j = int(rows[k]), int(col_idx[k])
            if i > j:
                continue
            kr = int(rev[k])
            te = int(tau[k])
            d = min(int(tt[i]), int(tt[j]), te + 1, depth_cap)
            ell = d - (d % 2)
            t_l = even[k, ell // 2] + even[kr, ell // 2]
            if te < cap and even_hop_bound(t_l, ell, te, lam_star) > 0.5 * eps:
                t_new = te + 2
                while t_new < cap and even_hop_bound(t_l, ell, t_new, lam_star) > 0.5 * eps:
                    t_new += 2
                tau[k] = tau[kr] = min(t_new, cap)
                redo.update((i, j))
        if not redo:
            break
        rounds += 1
        need = sorted(redo)
    return half + half[rev], tau, tt, rounds, tuple(seen)
