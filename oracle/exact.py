"""Exact spanning centrality, the target the method approximates (oracle O1).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the timed
CPU baseline; the CUDA path never imports it.

For a connected undirected graph the spanning centrality of an edge equals its
effective resistance (Section 2.3, the matrix form R = B L^+ B^T; the per-pair
formula L^+[i,i] + L^+[j,j] - 2 L^+[i,j] of Section 6):

    s(e_ij) = r(i, j) = (e_i - e_j)^T L^+ (e_i - e_j).

Routines, by graph size:

* ``kirchhoff_bruteforce``  Definition 2.1 itself: enumerate every
  (n-1)-edge subset, keep the spanning trees, count the trees containing each
  edge. Exact rationals, tiny graphs only.
* ``matrix_tree``           Kirchhoff's matrix-tree theorem with exact integer
  (Bareiss) determinants: s(e) = 1 - T(G - e) / T(G). Exact rationals, n <= 40.
* ``exact_dense``           r(i, j) from the inverse of the grounded Laplacian
  (node n-1 deleted; its potential is pinned to 0, which leaves every
  difference e_i - e_j unchanged). FP64, n up to a few thousand.
* ``exact_sparse_lu``       the same grounded system solved by a sparse LU
  factorisation per sampled pair: for low-fill graphs such as grids.
* ``exact_cg``              Jacobi-preconditioned FP64 CG per sampled pair (C,
  OpenMP over pairs, eight pairs side by side per thread): for expander-like
  graphs.

Library pseudo-inverses are not used anywhere.
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np

from . import _native

__all__ = ["kirchhoff_bruteforce", "matrix_tree", "exact_dense", "exact_sparse_lu",
           "exact_cg", "foster_sum", "entry_of_edges"]


def _edge_list(n, row_ptr, col_idx):
    deg = np.diff(np.asarray(row_ptr, dtype=np.int64))
    rows = np.repeat(np.arange(n), deg)
    cols = np.asarray(col_idx, dtype=np.int64)
    keep = rows < cols
    return list(zip(rows[keep].tolist(), cols[keep].tolist()))


def kirchhoff_bruteforce(n, row_ptr, col_idx):
    """Definition 2.1: fraction of spanning trees containing each edge.

    Returns {(u, v): Fraction} for u < v. Enumerates C(m, n-1) subsets, so keep
    C(m, n-1) to a few hundred thousand.
    """
    edges = _edge_list(n, row_ptr, col_idx)
    count = {e: 0 for e in edges}
    total = 0
    for subset in itertools.combinations(range(len(edges)), n - 1):
        parent = list(range(n))

        def find(a):
            while parent[a] != a:
                parent[a] = parent[parent[a]]
                a = parent[a]
            return a

        acyclic = True
        for t in subset:
            a, b = edges[t]
            ra, rb = find(a), find(b)
            if ra == rb:
                acyclic = False
                break
            parent[ra] = rb
        if not acyclic:
            continue  # n-1 acyclic edges on n nodes always span
        total += 1
        for t in subset:
            count[edges[t]] += 1
    if total == 0:
        raise ValueError("graph is disconnected")
    return {e: Fraction(c, total) for e, c in count.items()}


def _bareiss_det(mat):
    """Exact integer determinant by fraction-free (Bareiss) elimination."""
    a = [list(map(int, row)) for row in mat]
    size = len(a)
    if size == 0:
        return 1
    sign = 1
    prev = 1
    for k in range(size - 1):
        if a[k][k] == 0:
            swap = next((r for r in range(k + 1, size) if a[r][k] != 0), None)
            if swap is None:
                return 0
            a[k], a[swap] = a[swap], a[k]
            sign = -sign
        for i in range(k + 1, size):
            for j in range(k + 1, size):
                a[i][j] = (a[i][j] * a[k][k] - a[i][k] * a[k][j]) // prev
        prev = a[k][k]
    return sign * a[-1][-1]


def _spanning_tree_count(n, edges):
    lap = [[0] * n for _ in range(n)]
    for u, v in edges:
        lap[u][u] += 1
        lap[v][v] += 1
        lap[u][v] -= 1
        lap[v][u] -= 1
    reduced = [row[:-1] for row in lap[:-1]]
    return _bareiss_det(reduced)


def matrix_tree(n, row_ptr, col_idx):
    """Kirchhoff's matrix-tree theorem: s(e) = 1 - T(G - e) / T(G), exactly.

    Returns {(u, v): Fraction} for u < v.
    """
    edges = _edge_list(n, row_ptr, col_idx)
    total = _spanning_tree_count(n, edges)
    if total == 0:
        raise ValueError("graph is disconnected")
    out = {}
    for t, e in enumerate(edges):
        rest = edges[:t] + edges[t + 1:]
        out[e] = 1 - Fraction(_spanning_tree_count(n, rest), total)
    return out


def _grounded_laplacian_dense(n, row_ptr, col_idx):
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    deg = np.diff(row_ptr)
    rows = np.repeat(np.arange(n), deg)
    lap = np.zeros((n, n), dtype=np.float64)
    lap[rows, np.asarray(col_idx, dtype=np.int64)] = -1.0
    lap[np.arange(n), np.arange(n)] = deg
    return lap[:-1, :-1]


def exact_dense(n, row_ptr, col_idx):
    """Effective resistance of every CSR entry (FP64), from the inverse of the
    grounded Laplacian obtained by a Cholesky factorisation.

    Raises numpy.linalg.LinAlgError if the graph is disconnected (the grounded
    Laplacian is then singular).
    """
    import scipy.linalg as sla

    lg = _grounded_laplacian_dense(n, row_ptr, col_idx)
    cf = sla.cho_factor(lg, lower=True, check_finite=False)
    inv_g = sla.cho_solve(cf, np.eye(n - 1), check_finite=False)
    m = np.zeros((n, n), dtype=np.float64)
    m[:-1, :-1] = inv_g
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    cols = np.asarray(col_idx, dtype=np.int64)
    dg = np.diag(m)
    return dg[rows] + dg[cols] - 2.0 * m[rows, cols]


def _grounded_csc(n, row_ptr, col_idx):
    import scipy.sparse as sp

    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    deg = np.diff(row_ptr)
    rows = np.repeat(np.arange(n), deg)
    cols = np.asarray(col_idx, dtype=np.int64)
    lap = sp.csr_matrix((-np.ones(cols.size), (rows, cols)), shape=(n, n))
    lap = lap + sp.diags(deg.astype(np.float64))
    grounded = lap[:-1, :-1]  # node n-1 deleted
    return grounded.tocsc()


def _lu_solve_pairs(n, row_ptr, col_idx, pairs, chunk: int = 64):
    import scipy.sparse.linalg as spla

    lu = spla.splu(_grounded_csc(n, row_ptr, col_idx))
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    out = np.empty(pairs.shape[0])
    for s in range(0, pairs.shape[0], chunk):
        pp = pairs[s:s + chunk]
        cols = np.arange(pp.shape[0])
        b = np.zeros((n, pp.shape[0]))
        b[pp[:, 0], cols] += 1.0
        b[pp[:, 1], cols] -= 1.0
        x = np.zeros((n, pp.shape[0]))
        x[:-1] = lu.solve(b[:-1])
        out[s:s + chunk] = x[pp[:, 0], cols] - x[pp[:, 1], cols]
    return out


def exact_sparse_lu(n, row_ptr, col_idx, pairs, processes: int = 1):
    """Effective resistance of each (u, v) in ``pairs`` from a sparse LU
    factorisation of the grounded Laplacian (node n-1 deleted). With
    ``processes`` > 1 the pairs are split over that many worker processes
    (started with spawn), each factorising the matrix once."""
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    if processes <= 1 or pairs.shape[0] < 2 * processes:
        return _lu_solve_pairs(n, row_ptr, col_idx, pairs)
    import concurrent.futures as cf
    import multiprocessing as mp
    import os

    parts = np.array_split(pairs, processes)
    rp = np.asarray(row_ptr)
    ci = np.asarray(col_idx)
    # one BLAS / OpenMP thread per worker: the workers share the cores
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        with cf.ProcessPoolExecutor(max_workers=processes, mp_context=mp.get_context("spawn")) as ex:
            res = list(ex.map(_lu_solve_pairs, [n] * processes, [rp] * processes, [ci] * processes, parts))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return np.concatenate(res)


def exact_cg(n, row_ptr, col_idx, pairs, rtol: float = 1e-12, max_iter: int = 100_000,
             threads: int = 0, return_iters: bool = False, blocked: bool | None = None):
    """Effective resistance of each (u, v) in ``pairs`` by Jacobi-preconditioned
    FP64 CG (one independent solve per pair, OpenMP over pairs). ``blocked``
    runs eight solves side by side per thread, which gives the same values bit
    for bit; None picks it when a vector outgrows a core's cache (n > 1M),
    where one pass over the CSR then serves eight solves."""
    if blocked is None:
        blocked = n > 1_000_000
    L = _native.lib()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    u = np.ascontiguousarray(pairs[:, 0], dtype=np.int32)
    v = np.ascontiguousarray(pairs[:, 1], dtype=np.int32)
    out = np.empty(pairs.shape[0], dtype=np.float64)
    its = np.empty(pairs.shape[0], dtype=np.int32)
    import ctypes
    fn = L.oracle_cg_block if blocked else L.oracle_cg
    rc = fn(n, _native.ptr(rp, ctypes.c_int32), _native.ptr(ci, ctypes.c_int32),
                     pairs.shape[0], _native.ptr(u, ctypes.c_int32), _native.ptr(v, ctypes.c_int32),
                     rtol, max_iter, _native.ptr(out, ctypes.c_double),
                     _native.ptr(its, ctypes.c_int32), threads or _native.default_threads())
    if rc != 0:
        raise RuntimeError("oracle_cg failed (bad argument or out of memory)")
    if np.any(its < 0):
        raise RuntimeError("oracle_cg: some solves did not converge")
    return (out, its) if return_iters else out


def foster_sum(n, row_ptr, col_idx, r_entries):
    """Sum over undirected edges of r(e), from per-CSR-entry values (each edge
    appears twice). Foster's theorem fixes it at n - 1 for a connected graph."""
    return 0.5 * float(np.sum(r_entries))


def entry_of_edges(n, row_ptr, col_idx, pairs):
    """CSR entry index of each directed pair (u -> v); -1 if absent."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    cols = np.asarray(col_idx, dtype=np.int64)
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    keys = rows * n + cols
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    want = pairs[:, 0] * n + pairs[:, 1]
    pos = np.searchsorted(keys, want)
    pos = np.minimum(pos, keys.size - 1)
    return np.where(keys[pos] == want, pos, -1)


def reference_values(n, row_ptr, col_idx, dense_max: int = 5000, sample: int = 200, seed: int = 0,
                     low_fill: bool = False, threads: int = 0):
    """Exact resistances for checking a graph: every CSR entry by the dense
    grounded-Laplacian inverse when n <= dense_max, else `sample` uniformly
    drawn edges (seeded), by sparse LU for low-fill graphs (lattices) or by CG.
    Returns (entry indices, values)."""
    if n <= dense_max:
        return np.arange(len(col_idx), dtype=np.int64), exact_dense(n, row_ptr, col_idx)
    rp = np.asarray(row_ptr, dtype=np.int64)
    rows = np.repeat(np.arange(n), np.diff(rp))
    cols = np.asarray(col_idx, dtype=np.int64)
    keep = np.flatnonzero(rows < cols)
    rng = np.random.default_rng(seed)
    pick_k = np.sort(rng.choice(keep, size=min(sample, keep.size), replace=False))
    pairs = np.stack([rows[pick_k], cols[pick_k]], axis=1)
    if low_fill:
        vals = exact_sparse_lu(n, row_ptr, col_idx, pairs)
    else:
        vals = exact_cg(n, row_ptr, col_idx, pairs, threads=threads)
    return pick_k, vals
