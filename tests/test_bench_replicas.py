"""The N > 1 path of bench.py (independent replicas, no data-path exchange):
its max-over-ranks timing and whole-job value, run as two gloo ranks on the
CPU; and the reference arm leaves ranks other than 0 without work."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench.dist_setup()
        ms = 100.0 + 50.0 * rank  # the second replica is slower
        slowest = bench.max_over_ranks(dist, ms, "cpu")
        q.put((r, w, slowest, bench.replica_value(w, 1000, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for r, (rank, w, slowest, value) in enumerate(got):
        assert rank == r and w == world
        assert slowest == 150.0
        assert value == pytest.approx(2 * 1000 / 0.150)


def test_single_process_needs_no_group():
    import bench

    assert bench.max_over_ranks(None, 12.5, "cpu") == 12.5
    assert bench.replica_value(1, 2_000, 1000.0) == pytest.approx(2_000.0)


def test_reference_arm_other_ranks_do_nothing():
    import bench

    class Args:
        workload = "ba_200k"

    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(Args(), 2, 1) is None
    assert buf.getvalue() == ""


def test_arguments_default_and_tgt_plus_mode():
    import bench

    a = bench.parse_args([])
    assert (a.gpus, a.mode, a.policy, a.workload, a.impl) == (1, "tgt", "learned", "ba_200k", "ours")
    assert a.warmup >= 3
    a = bench.parse_args(["--mode", "tgt_plus", "--policy", "global"])
    assert (a.mode, a.policy) == ("tgt_plus", "global")
    a = bench.parse_args(["--mode", "tgt_plus"])  # TGT+ at learned lengths (the composite path)
    assert (a.mode, a.policy) == ("tgt_plus", "learned")
    a = bench.parse_args(["--workload", "rmat_22"])  # the R-MAT workload's own configuration
    assert (a.mode, a.policy, a.precision) == ("tgt_plus", "learned", "bf16")
    a = bench.parse_args(["--workload", "rmat_22", "--explicit-config", "--mode", "tgt", "--policy", "global"])
    assert (a.mode, a.policy, a.precision) == ("tgt", "global", "fp32")
    a = bench.parse_args(["--workload", "lattice_1000"])  # learned lengths by the tail estimate, eps = 1e-2
    assert (a.eps, a.mode, a.policy, a.estimator, a.precision, a.ell_cap) == (
        1e-2, "tgt", "learned", "end_corrected", "fp32", 1023)
    a = bench.parse_args(["--workload", "lattice_1000", "--explicit-config", "--policy", "fixed", "--ell", "105"])
    assert (a.eps, a.policy, a.ell, a.estimator) == (1e-3, "fixed", 105, "plain")


def test_timed_passes_split_only_the_warmups():
    import time as _time

    import bench

    calls = {"sync": 0, "barrier": 0, "passes": 0}

    def run_pass(mark):
        calls["passes"] += 1
        _time.sleep(0.002)
        mark("a")
        _time.sleep(0.001)
        mark("b")

    def sync():
        calls["sync"] += 1

    def barrier():
        calls["barrier"] += 1

    times, phases = bench.timed_passes(run_pass, 2, 3, sync, barrier)
    assert calls["passes"] == 5 and calls["barrier"] == 5
    assert calls["sync"] == 2 * 3 + 3  # warm-ups: two marks + the end; timed: the end only
    assert len(times) == 3 and all(t >= 3.0 for t in times)
    assert list(phases) == ["a", "b"] and phases["a"] >= 2.0 and phases["b"] >= 1.0
