"""Pins for the exact oracle (O1): SC = effective resistance.

Every check compares the oracle against something other than itself:
Definition 2.1 by brute-force enumeration, Kirchhoff's matrix-tree theorem in
exact integers, closed forms of named graphs, Foster's theorem, and golden
fractions written by tests/golden/make_golden.py (which calls only the
exact enumeration).
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import graphgen as gg
from oracle import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense_by_edge(g):
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    e = g.edges()
    k = exact.entry_of_edges(g.n, g.row_ptr, g.col_idx, e)
    return {(int(a), int(b)): float(r[kk]) for (a, b), kk in zip(e, k)}


SMALL = [gg.cycle(5), gg.complete(5), gg.complete_bipartite(2, 3), gg.barbell(3, 2),
         gg.lollipop(4, 2), gg.grid(2, 3), gg.petersen()]


@pytest.mark.parametrize("g", SMALL[:6], ids=lambda g: g.name)
def test_kirchhoff_matches_matrix_tree_and_dense(g):
    brute = exact.kirchhoff_bruteforce(g.n, g.row_ptr, g.col_idx)
    mt = exact.matrix_tree(g.n, g.row_ptr, g.col_idx)
    dense = _dense_by_edge(g)
    assert brute == mt
    for e, val in brute.items():
        assert abs(float(val) - dense[e]) < 1e-13


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_matrix_tree_matches_dense_on_random_graphs(seed):
    g = gg.tree_plus_gnp(14, 4.0, seed)
    mt = exact.matrix_tree(g.n, g.row_ptr, g.col_idx)
    dense = _dense_by_edge(g)
    for e, val in mt.items():
        assert abs(float(val) - dense[e]) < 1e-12


def test_golden_fractions():
    """Exact SC values stored as fractions (Definition 2.1 by enumeration)."""
    with open(os.path.join(GOLDEN, "sc_exact_small.json")) as fh:
        data = json.load(fh)
    for case in data["cases"]:
        n = case["n"]
        g = gg.from_edges(n, [e[0] for e in case["edges"]], [e[1] for e in case["edges"]])
        dense = _dense_by_edge(g)
        for (u, v), frac in zip(case["edges_sorted"], case["sc"]):
            assert abs(dense[(u, v)] - float(Fraction(frac))) < 1e-13
        assert sum(Fraction(f) for f in case["sc"]) == n - 1  # Foster, exactly


@pytest.mark.parametrize("n", [3, 4, 7, 10])
def test_cycle_closed_form(n):
    vals = _dense_by_edge(gg.cycle(n)).values()
    assert max(abs(v - (n - 1) / n) for v in vals) < 1e-13


@pytest.mark.parametrize("n", [2, 3, 6, 12])
def test_complete_closed_form(n):
    vals = _dense_by_edge(gg.complete(n)).values()
    assert max(abs(v - 2.0 / n) for v in vals) < 1e-13


@pytest.mark.parametrize("a,b", [(1, 4), (2, 3), (3, 5)])
def test_complete_bipartite_closed_form(a, b):
    vals = _dense_by_edge(gg.complete_bipartite(a, b)).values()
    want = (a + b - 1) / (a * b)
    assert max(abs(v - want) for v in vals) < 1e-13


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5])
def test_hypercube_closed_form(d):
    vals = _dense_by_edge(gg.hypercube(d)).values()
    want = (2 ** d - 1) / (d * 2 ** (d - 1))
    assert max(abs(v - want) for v in vals) < 1e-13


def test_edge_transitive_petersen():
    g = gg.petersen()
    vals = _dense_by_edge(g).values()
    assert max(abs(v - (g.n - 1) / g.m) for v in vals) < 1e-13


@pytest.mark.parametrize("seed", [0, 3])
def test_tree_edges_are_one(seed):
    g = gg.random_tree(60, seed)
    vals = _dense_by_edge(g).values()
    assert max(abs(v - 1.0) for v in vals) < 1e-12


def test_bridges_are_one():
    g = gg.barbell(5, 3)  # the 3 path edges are bridges
    d = _dense_by_edge(g)
    bridges = [(4, 10), (10, 11), (5, 11)]
    for u, v in bridges:
        key = (min(u, v), max(u, v))
        assert abs(d[key] - 1.0) < 1e-12
    g = gg.lollipop(5, 4)
    d = _dense_by_edge(g)
    for t in range(4, 8):
        assert abs(d[(t, t + 1)] - 1.0) < 1e-12


@pytest.mark.parametrize("seed", [0, 1])
def test_foster_random(seed):
    g = gg.tree_plus_gnp(400, 8.0, seed)
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    assert abs(exact.foster_sum(g.n, g.row_ptr, g.col_idx, r) - (g.n - 1)) < 1e-9
    # both directions of each edge carry the same value, all in (0, 1]
    assert np.all(r > 0) and np.all(r <= 1 + 1e-12)


def test_disconnected_rejected():
    g = gg.from_edges(6, [0, 1, 3, 4], [1, 2, 4, 5])
    with pytest.raises(Exception):
        exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    with pytest.raises(ValueError):
        exact.kirchhoff_bruteforce(g.n, g.row_ptr, g.col_idx)


@pytest.mark.parametrize("maker", [lambda: gg.tree_plus_gnp(300, 6.0, 5),
                                   lambda: gg.perturbed_grid(12, 15, 0.05, 7),
                                   lambda: gg.barabasi_albert(300, 3, 2)])
def test_cg_and_sparse_lu_match_dense(maker):
    g = maker()
    r = exact.exact_dense(g.n, g.row_ptr, g.col_idx)
    rng = np.random.default_rng(0)
    e = g.edges()
    pick = e[rng.choice(e.shape[0], size=min(40, e.shape[0]), replace=False)]
    k = exact.entry_of_edges(g.n, g.row_ptr, g.col_idx, pick)
    cg = exact.exact_cg(g.n, g.row_ptr, g.col_idx, pick)
    lu = exact.exact_sparse_lu(g.n, g.row_ptr, g.col_idx, pick)
    assert np.max(np.abs(cg - r[k])) < 1e-10
    assert np.max(np.abs(lu - r[k])) < 1e-10
    # CG also takes non-adjacent pairs: r is a metric (triangle inequality)
    a, b, c = 0, g.n // 2, g.n - 1
    rab, rbc, rac = exact.exact_cg(g.n, g.row_ptr, g.col_idx, [(a, b), (b, c), (a, c)])
    assert rac <= rab + rbc + 1e-12


@pytest.mark.parametrize("g", [gg.barabasi_albert(3000, 4, 9), gg.perturbed_grid(30, 41, 0.05, 3),
                               gg.rmat(12)], ids=lambda g: g.name)
def test_blocked_cg_matches_dense_and_single_solves(g):
    """The blocked CG (eight solves side by side per thread) against the dense
    grounded-Laplacian values to 1e-10, and against one solve per pair bit for
    bit, on pair counts that leave a partial group of eight."""
    rng = np.random.default_rng(1)
    e = g.edges()
    pick = e[rng.choice(e.shape[0], size=29, replace=False)]
    blocked, it_b = exact.exact_cg(g.n, g.row_ptr, g.col_idx, pick, blocked=True, return_iters=True)
    single, it_s = exact.exact_cg(g.n, g.row_ptr, g.col_idx, pick, blocked=False, return_iters=True)
    dense = exact.exact_dense(g.n, g.row_ptr, g.col_idx)[exact.entry_of_edges(g.n, g.row_ptr, g.col_idx, pick)]
    assert np.max(np.abs(blocked - dense)) < 1e-10
    assert np.array_equal(blocked, single) and np.array_equal(it_b, it_s)


def test_sparse_lu_worker_processes_give_the_single_process_values():
    g = gg.perturbed_grid(20, 23, 0.05, 4)
    rng = np.random.default_rng(2)
    e = g.edges()
    pick = e[rng.choice(e.shape[0], size=37, replace=False)]
    one = exact.exact_sparse_lu(g.n, g.row_ptr, g.col_idx, pick)
    two = exact.exact_sparse_lu(g.n, g.row_ptr, g.col_idx, pick, processes=3)
    assert np.array_equal(one, two)


def test_reference_values_dense_and_sampled_agree():
    g = gg.barabasi_albert(600, 3, 4)
    k_all, dense = exact.reference_values(g.n, g.row_ptr, g.col_idx)
    assert k_all.size == g.nnz
    k, cg = exact.reference_values(g.n, g.row_ptr, g.col_idx, dense_max=100, sample=50, seed=3)
    assert k.size == 50 and np.all(g.entry_rows()[k] < g.col_idx[k])
    assert np.max(np.abs(cg - dense[k])) < 1e-10
    grid = gg.perturbed_grid(15, 16, 0.05, 2)
    kg, lu = exact.reference_values(grid.n, grid.row_ptr, grid.col_idx, dense_max=10, sample=30, seed=1, low_fill=True)
    assert np.max(np.abs(lu - exact.exact_dense(grid.n, grid.row_ptr, grid.col_idx)[kg])) < 1e-10
