"""Host-side checks of the C ABI (no GPU): the library loads, exports every
function include/sc.h declares, and the ctypes structures have the C layout."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2305_16086_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sc.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sc_[a-z_0-9]+)\s*\(", text)))


def test_library_loads_and_exports_every_declared_symbol():
    lib = binding.load()
    declared = _declared_functions()
    assert declared, "no declarations parsed"
    for name in declared:
        assert hasattr(lib, name), f"libsc.so does not export {name}"
    assert sorted(binding.EXPORTS) == declared
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (sc_\w+)", out))
    assert set(declared) <= exported


def test_abi_version_and_status_strings():
    lib = binding.load()
    assert lib.sc_abi_version() == 1
    for code in range(15):
        assert lib.sc_status_string(code)
    assert lib.sc_status_string(3) == b"adjacency is not symmetric"


def test_options_default():
    o = binding.Options()
    binding.load().sc_options_default(ctypes.byref(o))
    assert o.eps == 1e-3 and o.mode == 0 and o.precision == 1 and o.ell_policy == 0 and o.gamma == 10
    assert o.bf16_from_hop == 0 and o.flags == 0 and o.switch_rule == 0 and o.ell_cap == 0


def test_binding_marshals_every_option():
    """The binding writes what the header defines (host logic only, no GPU)."""
    o = binding.Graph.options(eps=2e-3, mode="tgt_plus", precision="bf16", policy="fixed", ell_fixed=9,
                              estimator="end_corrected", block_width=64, rows_split=-1, heavy_threshold=99,
                              max_slices=3, record_tail=True, time_kernels=True, seed=7, delta=0.5, gamma=4,
                              switch="paper", windows=True, bf16_from_hop=5, ell_cap=1023,
                              sparse_hops=True, full_topgamma_scan=True)
    assert (o.eps, o.mode, o.precision, o.ell_policy, o.ell_fixed, o.estimator) == (2e-3, 1, 2, 2, 9, 1)
    assert (o.block_width, o.rows_split, o.heavy_threshold, o.max_slices) == (64, -1, 99, 3)
    assert o.flags == (binding.SC_OPT_RECORD_TAIL | binding.SC_OPT_TIME_KERNELS | binding.SC_OPT_WINDOWS_FORCE |
                       binding.SC_OPT_SPARSE_HOPS | binding.SC_OPT_FULL_TOPGAMMA_SCAN)
    assert (o.seed, o.delta, o.gamma, o.switch_rule, o.bf16_from_hop, o.ell_cap) == (7, 0.5, 4, 1, 5, 1023)
    t = binding.MlpTrainOpts(300, 1e-2, 0.0, 0.0, 0.0, binding.PREC["fp32"], 1e-3, 4095, 0)
    assert (t.epochs, t.precision, t.eps, t.ell_cap) == (300, 1, 1e-3, 4095)
    assert binding.Graph.options(windows=False).flags == binding.SC_OPT_WINDOWS_OFF
    assert binding.Graph.options().flags == 0


LAYOUT_C = r"""
#include <stdio.h>
#include <stddef.h>
#include "sc.h"
#define F(T, f) printf("%s.%s %zu\n", #T, #f, offsetof(T, f));
int main(void) {
  printf("sc_graph_info %zu\nsc_lambda %zu\nsc_lambda_opts %zu\nsc_options %zu\nsc_report %zu\n",
         sizeof(sc_graph_info), sizeof(sc_lambda), sizeof(sc_lambda_opts), sizeof(sc_options), sizeof(sc_report));
  printf("sc_eig_opts %zu\nsc_eig_report %zu\n", sizeof(sc_eig_opts), sizeof(sc_eig_report));
  printf("sc_mlp_train_opts %zu\n", sizeof(sc_mlp_train_opts));
  F(sc_mlp_train_opts, eps) F(sc_mlp_train_opts, ell_cap) F(sc_options, ell_cap) F(sc_report, uncertified)
  F(sc_eig_opts, tol) F(sc_eig_opts, rest_tol) F(sc_eig_opts, rest_max_iter) F(sc_eig_opts, seed)
  F(sc_eig_report, rest_converged) F(sc_eig_report, max_residual) F(sc_eig_report, lambda_rest)
  F(sc_options, seed) F(sc_options, delta) F(sc_options, gamma) F(sc_options, flags) F(sc_options, bf16_from_hop)
  F(sc_report, algorithmic_bytes) F(sc_report, walks) F(sc_report, edges_extended) F(sc_report, total_ms)
  F(sc_report, hop_ms) F(sc_report, hop_launches) F(sc_report, hop_bytes) F(sc_report, tt_min) F(sc_report, tt_max) F(sc_report, switch_ms) F(sc_report, walk_ms) F(sc_report, source_hops) F(sc_report, extension_rounds) F(sc_report, windowed) F(sc_report, walk_steps) F(sc_report, walk_device_ms)
  F(sc_report, kc_ms) F(sc_report, kc_launches) F(sc_report, kc_bytes)
  F(sc_lambda, iterations) F(sc_graph_info, diameter_lb) F(sc_lambda_opts, seed)
  return 0;
}
"""


def test_struct_layouts_match_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(LAYOUT_C)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    c = dict(line.split() for line in lines if line.strip())
    py = {"sc_graph_info": binding.GraphInfo, "sc_lambda": binding.Lambda, "sc_lambda_opts": binding.LambdaOpts,
          "sc_options": binding.Options, "sc_report": binding.Report, "sc_eig_opts": binding.EigOpts,
          "sc_eig_report": binding.EigReport, "sc_mlp_train_opts": binding.MlpTrainOpts}
    for name, cls in py.items():
        assert int(c[name]) == ctypes.sizeof(cls), name
    for key, val in c.items():
        if "." in key:
            sname, field = key.split(".")
            assert getattr(py[sname], field).offset == int(val), key


CONSTS_C = r"""
#include <stdio.h>
#include "sc.h"
#define P(x) printf("%s %lld\n", #x, (long long)(x));
int main(void) {
  P(SC_OK) P(SC_ERR_INVALID_ARG) P(SC_ERR_BAD_CSR) P(SC_ERR_NOT_SYMMETRIC) P(SC_ERR_SELF_LOOP)
  P(SC_ERR_DUPLICATE_EDGE) P(SC_ERR_ISOLATED_NODE) P(SC_ERR_DISCONNECTED) P(SC_ERR_BIPARTITE)
  P(SC_ERR_LAMBDA_NOT_CONVERGED) P(SC_ERR_BOUND_UNMET) P(SC_ERR_TIMEOUT) P(SC_ERR_OOM) P(SC_ERR_CUDA)
  P(SC_ERR_UNSUPPORTED)
  P(SC_PTRS_HOST) P(SC_PTRS_DEVICE) P(SC_FLAG_REJECT_BIPARTITE)
  P(SC_ELL_GLOBAL) P(SC_ELL_PER_EDGE) P(SC_ELL_FIXED) P(SC_ELL_LEARNED) P(SC_ELL_CALTAU) P(SC_OMEGA_MAX)
  P(SC_PREC_FP64) P(SC_PREC_FP32) P(SC_PREC_BF16) P(SC_EST_PLAIN) P(SC_EST_END_CORRECTED)
  P(SC_MODE_TGT) P(SC_MODE_TGT_PLUS) P(SC_SWITCH_COST) P(SC_SWITCH_PAPER) P(SC_SWITCH_PER_SOURCE)
  P(SC_OUT_DEVICE) P(SC_OPT_RECORD_TAIL) P(SC_OPT_TIME_KERNELS) P(SC_OPT_WINDOWS_OFF) P(SC_OPT_WINDOWS_FORCE)
  P(SC_OPT_SPARSE_HOPS) P(SC_OPT_FULL_TOPGAMMA_SCAN) P(SC_KC_DENSE_HOP) P(SC_KC_MASK_HOP) P(SC_KC_SPARSE_HOP) P(SC_KC_BALL_HOP) P(SC_KC_LAST_HOP)
  P(SC_KC_SWITCH_TEST) P(SC_KC_WALKS) P(SC_KC_COUNT)
  P(SC_MLP_PARAMS) P(SC_MLP_FEATURES) P(SC_MLP_MODEL_FLOATS)
  return 0;
}
"""


def test_header_constants_match_binding(tmp_path):
    """Every status, flag and enum value the binding mirrors equals the header's."""
    src = tmp_path / "consts.c"
    src.write_text(CONSTS_C)
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    c = {k: int(v) for k, v in (line.split() for line in out if line.strip())}
    for code, name in binding.STATUS_NAMES.items():
        assert c[name] == code, name
    assert len(binding.STATUS_NAMES) == sum(1 for k in c if k == "SC_OK" or k.startswith("SC_ERR_"))
    assert (c["SC_PTRS_HOST"], c["SC_PTRS_DEVICE"], c["SC_FLAG_REJECT_BIPARTITE"]) == (
        binding.SC_PTRS_HOST, binding.SC_PTRS_DEVICE, binding.SC_FLAG_REJECT_BIPARTITE)
    for table, prefix in ((binding.ELL, "SC_ELL_"), (binding.PREC, "SC_PREC_"), (binding.EST, "SC_EST_"),
                          (binding.MODE, "SC_MODE_")):
        assert {k.upper(): v for k, v in table.items()} == {k[len(prefix):]: v for k, v in c.items()
                                                            if k.startswith(prefix)}, prefix
    assert (c["SC_SWITCH_COST"], c["SC_SWITCH_PAPER"], c["SC_SWITCH_PER_SOURCE"]) == (0, 1, 2)  # switch="cost" / "paper" / "per_source"
    assert binding.Graph.options(switch="per_source").switch_rule == 2
    for name in ("SC_OUT_DEVICE", "SC_OPT_RECORD_TAIL", "SC_OPT_TIME_KERNELS", "SC_OPT_WINDOWS_OFF",
                 "SC_OPT_WINDOWS_FORCE", "SC_OPT_SPARSE_HOPS", "SC_OPT_FULL_TOPGAMMA_SCAN"):
        assert c[name] == getattr(binding, name), name
    assert c["SC_KC_COUNT"] == len(binding.KC_NAMES)
    for i, name in enumerate(binding.KC_NAMES):
        assert c["SC_KC_" + name.upper()] == i, name
    assert c["SC_OMEGA_MAX"] == binding.OMEGA_MAX
    assert (c["SC_MLP_PARAMS"], c["SC_MLP_FEATURES"], c["SC_MLP_MODEL_FLOATS"]) == (
        binding.MLP_PARAMS, binding.MLP_FEATURES, binding.MLP_MODEL_FLOATS)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError, match="libsc.so not found"):
        binding.load(str(tmp_path / "libsc.so"))


def test_selftest_rejects_a_limit_out_of_range():
    """Argument checks come before any CUDA call, so they run without a GPU."""
    for bad in (0, 1000001):
        st, detail = binding.selftest_bounded_waits(bad)
        assert binding.STATUS_NAMES[st] == "SC_ERR_INVALID_ARG" and "limit_us" in detail


def test_tridiag_eig_rejects_bad_arguments():
    lib = binding.load()
    theta = (ctypes.c_double * 2)()
    a = (ctypes.c_double * 2)(1.0, 2.0)
    assert binding.STATUS_NAMES[lib.sc_tridiag_eig(0, a, a, theta, None)] == "SC_ERR_INVALID_ARG"
    assert binding.STATUS_NAMES[lib.sc_tridiag_eig(2, a, None, theta, None)] == "SC_ERR_INVALID_ARG"
    assert binding.STATUS_NAMES[lib.sc_tridiag_eig(2, None, a, theta, None)] == "SC_ERR_INVALID_ARG"
