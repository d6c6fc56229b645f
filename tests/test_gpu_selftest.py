"""Failure detection on the GPU without a fault: the library's bounded device
waits (an mbarrier phase that nothing completes, a device flag that nothing
sets) give up after their limit and report SC_ERR_TIMEOUT through a status
word; the CUDA context stays usable, so a traversal right after still matches
the oracle."""
import time

import numpy as np
import pytest

import graphgen as gg
from oracle import series

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("limit_us", [1000, 20000])
def test_bounded_waits_give_up_and_report(cuda_lib, limit_us):
    from paper_2305_16086_gb300 import Graph, binding

    t0 = time.perf_counter()
    st, detail = binding.selftest_bounded_waits(limit_us)
    dt = time.perf_counter() - t0
    assert binding.STATUS_NAMES[st] == "SC_ERR_TIMEOUT", detail
    assert "gave up" in detail
    assert dt >= 2 * limit_us * 1e-6  # two waits in a row, each at least the limit
    g = gg.barabasi_albert(400, 3, 5)
    with Graph(g.row_ptr, g.col_idx) as G:
        s, _, rep = G.all_edges(policy="fixed", ell_fixed=7, precision="fp64")
    ref, _ = series.series_entries(g.n, g.row_ptr, g.col_idx, 7)
    assert np.max(np.abs(s - ref)) < 1e-12
