"""bench.py's main path run on the CPU with the CUDA pieces replaced by fakes:
the JSON line carries every key the benchmark contract asks for, in both
modes, so that a mistake in the benchmark's own code shows up here rather
than on the GPU. The numbers are the fakes' and mean nothing. CPU only."""
import io
import json
import sys
from contextlib import redirect_stdout

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import graphgen as gg  # noqa: E402


class _Event:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        pass

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return 25.0


def _kc(kw):
    t = 1.0 if kw.get("time_kernels") else 0.0
    return {name: {"ms": t * (20.0 if name == "dense_hop" else 2.0), "launches": 4, "bytes": 4.0e8}
            for name in ("dense_hop", "mask_hop", "sparse_hop", "ball_hop", "last_hop", "switch_test", "walks")}


def _report(kw):
    return {"kernel_classes": _kc(kw), "tt_min": 4, "tt_max": 5, "walks": 10, "walk_steps": 40, "switch_tests": 2, "switch_ms": 1.0,
            "walk_ms": 0.5, "hop_ms": 20.0 if kw.get("time_kernels") else 0.0, "hop_bytes": 4.0e8,
            "hop_launches": 4, "launches": 12, "foster_sum": 0.0, "ell_global": 7, "block_width": 64,
            "rows_split": 1, "slices": 1, "blocks": 3, "windowed": 0, "source_hops": 700, "extension_rounds": 0,
            "edges_extended": 0, "max_tail_bound": 1e-4, "uncertified": 0}


class _FakeGraph:
    calls = []

    def __init__(self, row_ptr, col_idx, stream=None, **kw):
        self.n = len(row_ptr) - 1
        self.nnz = len(col_idx)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def close(self):
        pass

    def info(self):
        return {"n": self.n, "nnz": self.nnz, "bipartite": 0}

    def estimate_lambda(self, **kw):
        return {"lambda_star": 0.43, "lambda_plus": 0.43, "lambda_minus": -0.3, "converged": 1, "iterations": 40,
                "residual_plus": 1e-5, "residual_minus": 1e-5}

    def eigenpairs(self, omega=128, **kw):
        return np.zeros(omega), None, {"used": 5, "lambda_rest": 0.6}

    def caltau(self, eps, **kw):
        self.tau = np.full(self.nnz, 7, dtype=np.int32)
        return self.tau, 7

    def truncation_length(self, eps, lam=None):
        return 301, np.full(self.n, 301, dtype=np.int32), np.full(self.nnz, 301, dtype=np.int32)

    def all_edges(self, out=None, **kw):
        _FakeGraph.calls.append(kw)
        rep = _report(kw)
        rep["foster_sum"] = float(self.n - 1)
        return out, None, rep


class _Clock:
    def __init__(self, dev):
        pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def summary(self):
        return {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}


@pytest.fixture
def fake_cuda(monkeypatch):
    import bench
    import paper_2305_16086_gb300 as pkg
    from paper_2305_16086_gb300 import binding

    real_empty = torch.empty
    monkeypatch.setattr(torch.cuda, "set_device", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "current_device", lambda *a, **k: 0)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda.nvtx, "range_push", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda.nvtx, "range_pop", lambda *a, **k: None)
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self, *a, **k: self)
    monkeypatch.setattr(torch, "empty", lambda *a, device=None, **k: real_empty(*a, **k) if not a or a[0] < (1 << 20)
                        else real_empty(16, dtype=k.get("dtype")))
    monkeypatch.setattr(pkg, "Graph", _FakeGraph)
    monkeypatch.setattr(binding, "mlp_load", lambda *a, **k: None)
    monkeypatch.setattr(bench, "train_model", lambda *a, **k: np.zeros(binding.MLP_MODEL_FLOATS, np.float32))
    monkeypatch.setattr(bench, "ClockSampler", _Clock)
    monkeypatch.setattr(bench, "cpu_baseline", lambda g, ell, target_s=10.0: {
        "value": 1.0, "unit": "edges/s", "cores": 1, "kind": "oracle", "sample": "fake"})
    monkeypatch.setitem(bench.WORKLOADS, "ba_200k", dict(desc="tiny stand-in", make=lambda g: gg.barabasi_albert(300, 3, 1)))
    _FakeGraph.calls = []
    return bench


def _run(bench, argv):
    buf = io.StringIO()
    old = sys.argv
    sys.argv = ["bench.py"] + argv
    try:
        with redirect_stdout(buf):
            bench.main()
    finally:
        sys.argv = old
    lines = [l for l in buf.getvalue().splitlines() if l.strip()]
    assert len(lines) == 1
    return json.loads(lines[0])


CONTRACT = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches"}


def test_default_line_has_every_contract_key(fake_cuda):
    d = _run(fake_cuda, ["--steps", "2", "--warmup", "3"])
    assert CONTRACT <= set(d)
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert set(d["roofline"]) >= {"bound", "achieved", "peak", "unit", "frac", "traffic"}
    assert d["roofline"]["frac"] == pytest.approx(d["roofline"]["achieved"] / d["roofline"]["peak"])
    assert d["roofline"]["kernel_class"] == "dense_hop" and set(d["kernel_classes"]) == {
        "dense_hop", "mask_hop", "sparse_hop", "ball_hop", "last_hop", "switch_test", "walks"}
    assert set(d["cpu_baseline"]) >= {"value", "unit", "cores", "kind", "sample"} and d["cpu_baseline"]["kind"] == "oracle"
    assert set(d["e2e"]) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert list(d["e2e"]["phases_ms_of_a_warmup_pass"]) == ["create_validate", "lanczos", "model_load", "all_edges_d2h"]
    assert d["value"] == pytest.approx(fake_cuda.replica_value(1, gg.barabasi_albert(300, 3, 1).m, d["ms_per_step"]))
    assert d["config"]["mode"] == "tgt" and d["tgt_plus"] is None and d["learned"] is not None
    assert d["gpu_launches"] == 2 * 12
    # the CPU baseline leg's exact check (real oracle CG on the stand-in graph; the fake s_hat is arbitrary)
    assert d["accuracy"]["sampled_edges"] == gg.barabasi_albert(300, 3, 1).m
    assert d["max_abs_err"] == d["accuracy"]["max_abs_err"] and d["mean_abs_err"] <= d["max_abs_err"]
    assert d["config"]["lambda_converged"] is True
    json.dumps(d)


def test_tgt_plus_mode_line(fake_cuda):
    d = _run(fake_cuda, ["--mode", "tgt_plus", "--policy", "global", "--steps", "1", "--warmup", "3", "--no-e2e"])
    assert d["config"]["mode"] == "tgt_plus" and d["learned"] is None
    assert d["tgt_plus"]["switch_after_hops"] == [4, 5] and d["tgt_plus"]["walk_pairs"] == 10
    timed = [kw for kw in _FakeGraph.calls if kw.get("time_kernels")]
    assert timed and all(kw["mode"] == "tgt_plus" for kw in timed)
    arms = [kw for kw in _FakeGraph.calls if kw.get("precision") == "fp64"]
    assert arms and all(kw["mode"] == "tgt" for kw in arms)  # the comparison arms stay TGT


def test_reference_arm_line(monkeypatch):
    """The reference arm times the oracle itself (real, on a tiny stand-in graph)."""
    import bench

    monkeypatch.setitem(bench.WORKLOADS, "ba_200k", dict(desc="tiny stand-in", make=lambda g: gg.barabasi_albert(300, 3, 1)))
    d = _run(bench, ["--impl", "reference", "--steps", "2", "--warmup", "1", "--ref-step-seconds", "0.05"])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "edges/s"
    assert {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "cpu_baseline",
            "e2e", "config"} <= set(d)
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    # ms_per_step is the measured sample time; the full-job extrapolation is a key of its own
    assert d["ms_per_step"] > 0 and d["full_job_ms_extrapolated"] > 0
    g = gg.barabasi_albert(300, 3, 1)
    assert {"workload", "n", "m", "eps", "mode", "policy", "estimator", "precision", "ell_global"} <= set(d["config"])
    assert (d["config"]["n"], d["config"]["m"]) == (g.n, g.m)


def test_caltau_arm_section(fake_cuda, monkeypatch):
    monkeypatch.setattr(gg, "workload", lambda name, **kw: gg.planted_partition(4, 60, 8.0, 0.3, 1))
    d = _run(fake_cuda, ["--steps", "1", "--warmup", "3", "--no-e2e", "--no-arms", "--caltau-arm",
                         "--caltau-omega", "9"])
    c = d["caltau"]
    assert c["omega"] == 9 and c["pairs_taken"] == 5 and c["mean_length"] == 7 and c["eq6"]["mean_length"] == 301
    assert c["source_hops"] == 7 * 240 and c["eq6"]["source_hops"] == 301 * 240 and c["value"] > 0
    d = _run(fake_cuda, ["--steps", "1", "--warmup", "3", "--no-e2e", "--no-arms"])
    assert d["caltau"] is None


@pytest.mark.parametrize("need,cap", [(67, 1023), (1, 1023), (1023, 1023), (5, 7)])
def test_empirical_length_is_the_least_odd_length_within_eps(monkeypatch, need, cap):
    """The lattice's global judge: bisection over odd lengths with a series
    that grows with the length (errors fall below eps from `need` on) returns
    `need`, and None when even the cap is not within eps."""
    import bench
    from paper_2305_16086_gb300 import binding

    r = np.array([1.0, 2.0])
    calls = []

    def fake_some_edges(G, entries, **kw):
        ell = kw["ell_fixed"]
        calls.append(ell)
        err = 0.5 if ell < need else 0.0  # monotone in the length, like the end-corrected series
        return r - err, {}

    monkeypatch.setattr(binding, "some_edges", fake_some_edges)
    ref = {"k": np.array([0, 1]), "r": r}
    got = bench.empirical_length(None, ref, 1e-2, cap, dict(eps=1e-2))
    assert got == need and all(c % 2 == 1 for c in calls)
    assert len(calls) <= 12  # a bisection, not a scan
    monkeypatch.setattr(binding, "some_edges", lambda G, e, **kw: (r - 1.0, {}))
    assert bench.empirical_length(None, ref, 1e-2, cap, dict(eps=1e-2)) is None


def test_errors_at_uses_the_sampled_entries():
    import bench

    ref = {"k": np.array([2, 0]), "r": np.array([0.5, 0.25])}
    e = bench.errors_at(ref, np.array([0.2, 9.0, 0.45]))
    assert e["sampled_edges"] == 2
    assert e["max_abs_err"] == pytest.approx(0.05) and e["mean_abs_err"] == pytest.approx(0.05)
