"""Learned per-source truncation length (oracle for the MLP step).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the timed
CPU baseline; the CUDA path never imports it.

The paper truncates every edge at the a-priori length of Eq. (6). A source
usually needs far fewer hops: for odd tau the tail of the series is
sum_k c_k lambda_k^{tau+1} / (1 - lambda_k) with c_k >= 0 (proof of Theorem
3.2), and writing each term as c_k (1 + lambda_k) lambda_k^{tau-1} *
lambda_k^2 / (1 - lambda_k^2) gives the a-posteriori bound

    tail(tau) <= lambda*^2 / (1 - lambda*^2) * (t_{tau-1}(e) + t_tau(e)),

with t_l(e) the full hop-l term of Eq. (2): it uses only hops already
traversed. An edge is certified at the least odd tau where the bound is at
most eps. The label of source i is the largest certified length over its
edges; a small MLP predicts it from six per-source features.

Features (in this order; all local and independent of the graph's size, so
that a model trained on a smaller graph of a family serves a larger one):
  0  log d_i
  1  log min_{j in N(i)} d_j
  2  local clustering c_i = triangles(i) / (d_i (d_i - 1) / 2) (0 for d_i < 2)
  3  log((sum_{j in N(i)} d_j / d_i) / (2m / n))  (mean neighbour degree over the mean degree)
  4  p_2(i, i) = (1/d_i) sum_{j in N(i)} 1/d_j
  5  p_3(i, i) = (1/d_i) sum over triangles (i, j, k) of 1/(d_j d_k)

Network: inputs standardised with the training set's mean and standard
deviation, then 6 -> 32 -> 32 -> 1 with ReLU after the two hidden layers; the
output is log L. Loss: mean over sources of (y - log L*)^2 / 2. Optimiser:
Adam (Kingma and Ba, ICLR 2015) with bias correction. Prediction: the
smallest odd integer >= exp(y) - 1/4, clipped to [1, cap]: the labels are
odd, and a prediction at most 1/4 above one takes it (a prediction below the
label costs its source a rerun, one above it wasted hops).

Flat parameter layout (float32, 1313 entries): W1[32][6], b1[32], W2[32][32],
b2[32], W3[32], b3[1].

Bipartite graphs (lambda* = 1) have neither the bound above nor an a-priori
length, and need the end-corrected estimator S_hat = S_tau + t_{tau+1}/2.
Its remainder past odd tau is sum_k c_k lambda_k^(tau+1) (1 + lambda_k) /
(2 (1 - lambda_k)) >= 0 (the same mode expansion; the lambda = -1 mode drops
out), which for the slow modes is about the sum of the pair sums
q(tau) = t_{tau+1} + t_{tau+2}, q(tau + 2), ... On a lattice these decay like
a power of the hop (diffusion), so the pair sums are fitted by C x^-p through
q(tau - 2) at x = tau - 1 and q(tau) at x = tau + 1, and the fit is summed
past tau as an integral at half a unit of x per hop:

    p   = ln(q(tau - 2) / q(tau)) / ln((tau + 1) / (tau - 1)),
    est = C tau^(1-p) / (2 (p - 1)) = q(tau) (tau + 1) ((tau + 1)/tau)^(p-1) / (2 (p - 1)).

This is an estimate, not a bound (``tail_estimate``). A bipartite graph's
labels are the least odd tau in [3, cap] whose estimate is at most eps
(``estimated_lengths``); ``learned_bipartite`` is the extension loop of the
learned policy with this acceptance. Where it differs from a geometric
extrapolation of the same ratio: a geometric fit assumes the ratio
q(tau)/q(tau-2) stays fixed, and on a power-law tail C x^-p it falls short by
the factor (p - 1)/p (one half on a 2-D lattice); the power-law fit is
exact there and overshoots a geometric tail (parity unpinned against the
paper: the paper has no bipartite rule; pinned by closed forms and brute
force below).
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _native, series

H = 32
NF = 6
NPARAM = H * NF + H + H * H + H + H + 1


def features(n, row_ptr, col_idx):
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col_idx = np.asarray(col_idx, dtype=np.int64)
    deg = np.diff(row_ptr).astype(np.float64)
    mean_deg = deg.sum() / n
    F = np.zeros((n, NF))
    for i in range(n):
        nb = col_idx[row_ptr[i]:row_ptr[i + 1]]
        d = deg[i]
        tri = 0
        cyc = 0.0
        s = set(nb.tolist())
        for j in nb:
            for y in col_idx[row_ptr[j]:row_ptr[j + 1]]:
                if y in s:  # the walk i -> j -> y -> i
                    tri += 1
                    cyc += 1.0 / (deg[j] * deg[y])
        tri //= 2  # each triangle at i is seen from both of its other corners
        F[i, 0] = math.log(d)
        F[i, 1] = math.log(deg[nb].min())
        F[i, 2] = tri / (d * (d - 1) / 2.0) if d >= 2 else 0.0
        F[i, 3] = math.log(deg[nb].sum() / d / mean_deg)
        F[i, 4] = np.sum(1.0 / deg[nb]) / d
        F[i, 5] = cyc / d
    return F


def hop_terms(n, row_ptr, col_idx, L, sources=None, threads=0):
    """T[k, l] = (p_l(i,i) - p_l(j,i)) / d_i for l = 0..L and every entry k of
    the requested sources' rows (other rows NaN)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    src = np.arange(n, dtype=np.int32) if sources is None else np.ascontiguousarray(np.unique(sources), dtype=np.int32)
    deg = np.diff(rp.astype(np.int64))
    off = np.zeros(src.size + 1, dtype=np.int64)
    np.cumsum(deg[src], out=off[1:])
    out = np.empty(int(off[-1]) * (L + 1))
    lib = _native.lib()
    rc = lib.oracle_series_terms(n, _native.ptr(rp, ctypes.c_int32), _native.ptr(ci, ctypes.c_int32), L, src.size,
                                 _native.ptr(src, ctypes.c_int32), _native.ptr(off, ctypes.c_int64),
                                 _native.ptr(out, ctypes.c_double), threads or _native.default_threads())
    if rc != 0:
        raise RuntimeError("oracle_series_terms failed")
    T = np.full((ci.size, L + 1), np.nan)
    out = out.reshape(-1, L + 1)
    for t, i in enumerate(src):
        T[rp[i]:rp[i + 1]] = out[off[t]:off[t + 1]]
    return T


def certified_lengths(n, row_ptr, col_idx, eps, lam_star, cap):
    """Least odd tau <= cap per entry whose a-posteriori bound is <= eps (else cap)."""
    T = hop_terms(n, row_ptr, col_idx, cap)
    rev = series.reverse_entries(n, row_ptr, col_idx)
    full = T + T[rev]  # t_l(e), l = 0..cap
    factor = lam_star * lam_star / (1.0 - lam_star * lam_star)
    tau = np.full(full.shape[0], cap, dtype=np.int64)
    done = np.zeros(full.shape[0], dtype=bool)
    for t in range(1, cap + 1, 2):
        ok = (~done) & (factor * (full[:, t - 1] + full[:, t]) <= eps)
        tau[ok] = t
        done |= ok
    return tau


def source_labels(n, row_ptr, tau_entries):
    out = np.zeros(n, dtype=np.int64)
    rows = np.repeat(np.arange(n), np.diff(np.asarray(row_ptr, dtype=np.int64)))
    np.maximum.at(out, rows, tau_entries)
    return out


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    o = 0

    def take(shape):
        nonlocal o
        size = int(np.prod(shape))
        v = theta[o:o + size].reshape(shape)
        o += size
        return v

    W1 = take((H, NF))
    b1 = take((H,))
    W2 = take((H, H))
    b2 = take((H,))
    W3 = take((H,))
    b3 = take((1,))
    return W1, b1, W2, b2, W3, b3


def forward(theta, X):
    """X: standardised features (N, 6). Returns (y (N,), cache)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3 + b3[0]
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(theta, X, target):
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    N = X.shape[0]
    r = y - target
    loss = 0.5 * np.mean(r * r)
    dy = r / N
    gW3 = h2.T @ dy
    gb3 = np.array([dy.sum()])
    dh2 = np.outer(dy, W3) * (z2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (z1 > 0)
    gW1 = dh1.T @ X
    gb1 = dh1.sum(axis=0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, gb3])
    return loss, grad


def adam_step(theta, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step t (1-based); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def standardise(F):
    """Mean and population standard deviation per feature. A spread at
    rounding level (below 1e-9 max(|mean|, 1)) marks a constant feature, such
    as the clustering over a lattice; it gets scale 1."""
    mu = F.mean(axis=0)
    sd = F.std(axis=0)
    sd = np.where(sd > 1e-9 * np.maximum(np.abs(mu), 1.0), sd, 1.0)
    return mu, sd


def predict_lengths(theta, F, mu, sd, cap):
    y, _ = forward(theta, (F - mu) / sd)
    with np.errstate(over="ignore"):
        e = np.ceil(np.exp(y) - 0.25)
    L = np.clip(np.nan_to_num(e, nan=1.0, posinf=float(cap)), 1, cap).astype(np.int64)
    return np.where(L % 2 == 0, np.minimum(L + 1, cap if cap % 2 == 1 else cap + 1), L)


# ---------------------------------------------------------------------------
# bipartite graphs: the tail estimate and the learned policy's loop with it
# ---------------------------------------------------------------------------

def tail_estimate(q_prev, q, tau):
    """Power-law tail estimate from the pair sums q(tau - 2) and q(tau) (see the
    module notes): 0 where q <= 0; +inf where tau < 3, q(tau - 2) <= 0 or the
    fitted exponent p <= 1 (no decay fast enough to sum)."""
    q_prev = np.asarray(q_prev, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    tau = np.broadcast_to(np.asarray(tau, dtype=np.float64), q.shape)
    out = np.full(q.shape, np.inf)
    ok = (tau >= 3) & (q_prev > 0) & (q > 0)
    x = tau[ok]
    p = np.log(q_prev[ok] / q[ok]) / np.log((x + 1.0) / (x - 1.0))
    est = np.full(x.shape, np.inf)
    dec = p > 1.0
    pd, xd = p[dec], x[dec]
    est[dec] = q[ok][dec] * (xd + 1.0) * np.exp((pd - 1.0) * np.log((xd + 1.0) / xd)) / (2.0 * (pd - 1.0))
    out[ok] = est
    out[q <= 0] = 0.0
    return out


def estimated_lengths(n, row_ptr, col_idx, eps, cap):
    """Least odd tau in [3, cap] per entry whose tail estimate is <= eps (else cap)."""
    T = hop_terms(n, row_ptr, col_idx, cap + 2)
    rev = series.reverse_entries(n, row_ptr, col_idx)
    full = T + T[rev]  # t_l(e), l = 0..cap+2
    tau = np.full(full.shape[0], cap, dtype=np.int64)
    done = np.zeros(full.shape[0], dtype=bool)
    for t in range(3, cap + 1, 2):
        est = tail_estimate(full[:, t - 1] + full[:, t], full[:, t + 1] + full[:, t + 2], t)
        ok = (~done) & (est <= eps)
        tau[ok] = t
        done |= ok
    return tau


def learned_bipartite(n, row_ptr, col_idx, L_src, cap, eps):
    """The learned policy on a bipartite graph: tau_e = min(L_i, L_j); each
    round evaluates the tail estimate of every edge at its tau from the
    end-corrected series at tau and tau - 2, and an edge whose estimate exceeds
    eps below the cap takes tau <- min(2 tau + 1, cap); until none does.
    Returns (s_hat per entry, tau per entry, rounds)."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    L_src = np.asarray(L_src, dtype=np.int64)
    rows = np.repeat(np.arange(n), np.diff(rp))
    cols = np.asarray(col_idx, dtype=np.int64)
    tau = np.minimum(L_src[rows], L_src[cols])
    rounds = 0
    while True:
        s, q = series.series_entries(n, row_ptr, col_idx, tau, end_corrected=True)
        _, q_prev = series.series_entries(n, row_ptr, col_idx, np.maximum(tau - 2, 0), end_corrected=True)
        est = tail_estimate(q_prev, q, tau)
        fail = (est > eps) & (tau < cap)
        if not fail.any():
            return s, tau, rounds
        tau = np.where(fail, np.minimum(2 * tau + 1, cap), tau)
        rounds += 1
