"""The seeded input generators (shared by the oracle tests, the GPU tests and
the bench): every graph is a valid symmetric CSR of a simple connected graph,
the same seed gives the same graph, and the recipes have the documented sizes
and structure. CPU only."""
import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import connected_components

import graphgen as gg


def _check_csr(g):
    rp, ci = g.row_ptr, g.col_idx
    assert rp.dtype == np.int32 and ci.dtype == np.int32
    assert rp[0] == 0 and rp[-1] == ci.size and np.all(np.diff(rp) >= 1)  # no isolated node
    rows = np.repeat(np.arange(g.n), np.diff(rp))
    assert np.all(ci != rows)  # no self-loop
    for r in range(0, g.n, max(1, g.n // 200)):  # sorted, duplicate-free rows (sampled)
        seg = ci[rp[r]:rp[r + 1]]
        assert np.all(np.diff(seg) > 0)
    a = csr_matrix((np.ones(ci.size), ci, rp), shape=(g.n, g.n))
    assert (a != a.T).nnz == 0  # symmetric
    assert connected_components(a, directed=False)[0] == 1


@pytest.mark.parametrize("make", [
    lambda: gg.tree_plus_gnp(500, 10.0, 3),
    lambda: gg.planted_partition(6, 150, 8.0, 0.4, 2),
    lambda: gg.barabasi_albert(3000, 5, 2),
    lambda: gg.perturbed_grid(30, 40, 0.05, 1),
    lambda: gg.gnp_lcc(2000, 8.0, 4),
    lambda: gg.rmat(12, 16, seed=5),
    lambda: gg.random_tree(300, 9),
])
def test_valid_connected_symmetric_csr_and_deterministic(make):
    g1, g2 = make(), make()
    _check_csr(g1)
    assert np.array_equal(g1.row_ptr, g2.row_ptr) and np.array_equal(g1.col_idx, g2.col_idx)


def test_documented_sizes():
    assert gg.tree_plus_gnp(2000, 10.0, 0).m == 10_083
    ba = gg.barabasi_albert(20_000, 10, 1)
    assert ba.m == 10 * (20_000 - 11) + 10 and int(np.diff(ba.row_ptr).min()) == 10
    grid = gg.perturbed_grid(40, 50, 0.05, 2)
    full = 40 * 49 + 39 * 50
    assert grid.m == full - int(round(0.05 * full))
    assert grid.meta["bipartite"]


def test_tree_is_a_tree_and_grid_rows_are_banded():
    t = gg.random_tree(500, 3)
    assert t.m == t.n - 1
    g = gg.perturbed_grid(20, 30, 0.05, 4)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    assert int(np.max(np.abs(g.col_idx - rows))) == 30  # row-major ids: bandwidth = cols


def test_batch_recipe_cycles_families_and_sizes():
    gs = gg.batch_graphs(9, 200, 2000, base_seed=40)
    assert len(gs) == 9
    for i, g in enumerate(gs):
        _check_csr(g)
        assert bool(g.meta.get("bipartite")) == (i % 3 == 2)  # lattices every third graph
        assert 100 <= g.n <= 2100


def test_planted_partition_communities_and_slow_modes():
    """Nodes c*size .. (c+1)*size - 1 form community c; about d_in of a node's
    neighbours are inside and d_out outside; k - 1 eigenvalues of N lie near 1
    and the k-th below them is far lower (the bottleneck the recipe is for)."""
    k, size, d_in, d_out = 5, 200, 10.0, 0.3
    g = gg.planted_partition(k, size, d_in, d_out, 3)
    assert g.n == k * size
    rows = g.entry_rows()
    inside = (rows // size) == (g.col_idx // size)
    assert abs(inside.sum() / g.n - d_in) < 0.6 and abs((~inside).sum() / g.n - d_out) < 0.15
    d = g.degree.astype(np.float64)
    nmat = np.zeros((g.n, g.n))
    nmat[rows, g.col_idx] = 1.0 / np.sqrt(d[rows] * d[g.col_idx])
    ev = np.sort(np.linalg.eigvalsh(nmat))[::-1]
    assert abs(ev[0] - 1.0) < 1e-12 and np.all(ev[1:k] > 0.9) and ev[k] < 0.75
    h = gg.planted_partition(k, size, d_in, d_out, 3)
    assert np.array_equal(g.row_ptr, h.row_ptr) and np.array_equal(g.col_idx, h.col_idx)
