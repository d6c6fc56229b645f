"""GPU parity of the meet-in-the-middle series (sc_series_meet) through the C
ABI: the same S_tau as Algorithm 2's series (oracle/series.py, the C
traversal) and as oracle/meet.py, to 1e-12 (FP64 on both sides, summation
orders differ: each hop term is a sum of at most 2m products of magnitude <= 1),
at per-edge lengths with odd, even and zero values, on bipartite and
non-bipartite graphs; and the same values as sc_all_edges at a fixed length.
The file is named so that pytest collects it after the other GPU suites.
"""
import numpy as np
import pytest

import graphgen as gg
from oracle import meet, series

pytestmark = pytest.mark.gpu


def _csr(g):
    return g.n, g.row_ptr, g.col_idx


@pytest.mark.parametrize("maker", [lambda: gg.lollipop(7, 4), lambda: gg.petersen(), lambda: gg.tree_plus_gnp(300, 5.0, 3),
                                   lambda: gg.barbell(5, 2), lambda: gg.grid(6, 7), lambda: gg.barabasi_albert(500, 3, 1)])
def test_equals_the_series_at_per_edge_lengths(cuda_lib, maker):
    from paper_2305_16086_gb300 import Graph

    g = maker()
    rng = np.random.default_rng(g.n)
    tau = rng.integers(0, 16, size=g.nnz)
    tau = np.maximum(tau, tau[series.reverse_entries(*_csr(g))]).astype(np.int32)
    with Graph(g.row_ptr, g.col_idx) as G:
        s = G.series_meet(tau)
    want, _ = series.series_entries(*_csr(g), tau)
    assert np.max(np.abs(s - want)) < 1e-12
    assert np.max(np.abs(s - meet.series_meet(*_csr(g), tau))) < 1e-12


def test_equals_all_edges_at_a_fixed_length(cuda_lib):
    from paper_2305_16086_gb300 import Graph

    g = gg.tree_plus_gnp(2000, 10.0, 0)
    with Graph(g.row_ptr, g.col_idx) as G:
        s1, _, _ = G.all_edges(policy="fixed", ell_fixed=13, precision="fp64")
        s2 = G.series_meet(13)
    assert np.max(np.abs(s1 - s2)) < 1e-12


def test_rejects_lengths_that_differ_between_directions(cuda_lib):
    from paper_2305_16086_gb300 import Graph, ScError

    g = gg.lollipop(6, 2)
    tau = np.full(g.nnz, 5, dtype=np.int32)
    tau[0] = 7
    with Graph(g.row_ptr, g.col_idx) as G:
        with pytest.raises(ScError, match="SC_ERR_INVALID_ARG"):
            G.series_meet(tau)
        with pytest.raises(ScError, match="SC_ERR_INVALID_ARG"):
            G.series_meet(np.full(g.nnz, -1, dtype=np.int32))
