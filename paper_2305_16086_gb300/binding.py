"""ctypes binding of libsc (include/sc.h): argument marshalling only.

Every computation happens inside libsc.so's CUDA kernels. PyTorch is used
only to hold device memory and to name the CUDA stream. If libsc.so is
missing or fails to load, ``load()`` raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsc.so")

# ---- constants mirrored from sc.h -------------------------------------------
SC_OK = 0
STATUS_NAMES = {
    0: "SC_OK", 1: "SC_ERR_INVALID_ARG", 2: "SC_ERR_BAD_CSR", 3: "SC_ERR_NOT_SYMMETRIC",
    4: "SC_ERR_SELF_LOOP", 5: "SC_ERR_DUPLICATE_EDGE", 6: "SC_ERR_ISOLATED_NODE",
    7: "SC_ERR_DISCONNECTED", 8: "SC_ERR_BIPARTITE", 9: "SC_ERR_LAMBDA_NOT_CONVERGED",
    10: "SC_ERR_BOUND_UNMET", 11: "SC_ERR_TIMEOUT", 12: "SC_ERR_OOM", 13: "SC_ERR_CUDA",
    14: "SC_ERR_UNSUPPORTED",
}
SC_PTRS_HOST, SC_PTRS_DEVICE, SC_FLAG_REJECT_BIPARTITE = 0, 1, 2
ELL = {"global": 0, "per_edge": 1, "fixed": 2, "learned": 3, "caltau": 4}
PREC = {"fp64": 0, "fp32": 1, "bf16": 2}
EST = {"plain": 0, "end_corrected": 1}
MODE = {"tgt": 0, "tgt_plus": 1}
SC_OUT_DEVICE, SC_OPT_RECORD_TAIL, SC_OPT_TIME_KERNELS = 1, 2, 4
SC_OPT_WINDOWS_OFF, SC_OPT_WINDOWS_FORCE, SC_OPT_SPARSE_HOPS, SC_OPT_FULL_TOPGAMMA_SCAN = 8, 16, 32, 64
KC_NAMES = ["dense_hop", "mask_hop", "sparse_hop", "ball_hop", "last_hop", "switch_test", "walks"]  # SC_KC_* order

# every symbol include/sc.h declares
EXPORTS = [
    "sc_graph_create", "sc_graph_get_info", "sc_graph_destroy", "sc_estimate_lambda",
    "sc_truncation_length", "sc_options_default", "sc_all_edges", "sc_status_string",
    "sc_last_error_detail", "sc_abi_version", "sc_all_edges_noalloc", "sc_source_features",
    "sc_certified_lengths", "sc_mlp_train", "sc_mlp_load", "sc_mlp_predict", "sc_mlp_loss_grad",
    "sc_batch_all_edges", "sc_selftest_bounded_waits", "sc_eigenpairs", "sc_caltau", "sc_tridiag_eig",
    "sc_series_meet", "sc_some_edges", "sc_graph_set_lambda", "sc_estimated_lengths",
]
OMEGA_MAX = 257
MLP_PARAMS, MLP_FEATURES = 1313, 6
MLP_MODEL_FLOATS = MLP_PARAMS + 2 * MLP_FEATURES


class GraphInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("m", ctypes.c_int64),
                ("min_degree", ctypes.c_int32), ("max_degree", ctypes.c_int32),
                ("bipartite", ctypes.c_int32), ("diameter_lb", ctypes.c_int32)]


class Lambda(ctypes.Structure):
    _fields_ = [("lambda_plus", ctypes.c_double), ("lambda_minus", ctypes.c_double),
                ("lambda_star", ctypes.c_double), ("residual_plus", ctypes.c_double),
                ("residual_minus", ctypes.c_double), ("iterations", ctypes.c_int32),
                ("converged", ctypes.c_int32)]


class LambdaOpts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("tol", ctypes.c_double), ("seed", ctypes.c_uint64)]


class Options(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("mode", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("ell_policy", ctypes.c_int32), ("ell_fixed", ctypes.c_int32),
                ("estimator", ctypes.c_int32), ("block_width", ctypes.c_int32),
                ("rows_split", ctypes.c_int32), ("heavy_threshold", ctypes.c_int32),
                ("max_slices", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("delta", ctypes.c_double), ("gamma", ctypes.c_int32),
                ("switch_rule", ctypes.c_int32), ("bf16_from_hop", ctypes.c_int32),
                ("ell_cap", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class Report(ctypes.Structure):
    _fields_ = [("ell_global", ctypes.c_int32), ("ell_min_source", ctypes.c_int32),
                ("ell_max_source", ctypes.c_int32), ("block_width", ctypes.c_int32),
                ("rows_split", ctypes.c_int32), ("slices", ctypes.c_int32),
                ("blocks", ctypes.c_int64), ("launches", ctypes.c_int64), ("hops", ctypes.c_int64),
                ("algorithmic_bytes", ctypes.c_double), ("foster_sum", ctypes.c_double),
                ("max_tail_bound", ctypes.c_double), ("lambda_star", ctypes.c_double),
                ("propagate_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("hop_ms", ctypes.c_double), ("hop_launches", ctypes.c_int64), ("hop_bytes", ctypes.c_double),
                ("walks", ctypes.c_int64), ("edges_extended", ctypes.c_int32),
                ("tt_min", ctypes.c_int32), ("tt_max", ctypes.c_int32),
                ("switch_tests", ctypes.c_int32), ("switch_ms", ctypes.c_double), ("walk_ms", ctypes.c_double),
                ("source_hops", ctypes.c_int64), ("extension_rounds", ctypes.c_int32), ("windowed", ctypes.c_int32),
                ("walk_steps", ctypes.c_int64), ("walk_device_ms", ctypes.c_double),
                ("kc_ms", ctypes.c_double * 7), ("kc_launches", ctypes.c_int64 * 7),
                ("kc_bytes", ctypes.c_double * 7), ("uncertified", ctypes.c_int32),
                ("reserved_r", ctypes.c_int32)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        for name in ("kc_ms", "kc_launches", "kc_bytes"):
            d[name] = list(d[name])
        d["kernel_classes"] = {KC_NAMES[c]: {"ms": d["kc_ms"][c], "launches": d["kc_launches"][c],
                                             "bytes": d["kc_bytes"][c]} for c in range(len(KC_NAMES))}
        return d


class EigOpts(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("tol", ctypes.c_double),
                ("rest_tol", ctypes.c_double), ("rest_max_iter", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


class EigReport(ctypes.Structure):
    _fields_ = [("used", ctypes.c_int32), ("iterations", ctypes.c_int32), ("rest_iterations", ctypes.c_int32),
                ("rest_converged", ctypes.c_int32), ("max_residual", ctypes.c_double),
                ("rest_residual", ctypes.c_double), ("lambda_rest", ctypes.c_double)]


class MlpTrainOpts(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("adam_eps", ctypes.c_float), ("precision", ctypes.c_int32),
                ("eps", ctypes.c_double), ("ell_cap", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ScError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{where}: {self.name}: {detail}")


_lib = None


def load(path: str = LIB_PATH):
    """Load libsc.so and declare its C signatures. Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libsc.so not found at {path}: build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(path)
    vp, i32, i64, u32, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double
    i32p = ctypes.POINTER(ctypes.c_int32)
    f64p = ctypes.POINTER(ctypes.c_double)
    L.sc_graph_create.argtypes = [ctypes.POINTER(vp), i32, i64, vp, vp, u32, vp]
    L.sc_graph_create.restype = ctypes.c_int
    L.sc_graph_get_info.argtypes = [vp, ctypes.POINTER(GraphInfo)]
    L.sc_graph_get_info.restype = ctypes.c_int
    L.sc_graph_destroy.argtypes = [vp]
    L.sc_graph_destroy.restype = None
    L.sc_estimate_lambda.argtypes = [vp, ctypes.POINTER(LambdaOpts), ctypes.POINTER(Lambda)]
    L.sc_estimate_lambda.restype = ctypes.c_int
    L.sc_truncation_length.argtypes = [vp, f64, ctypes.POINTER(Lambda), i32p, i32p, i32p]
    L.sc_truncation_length.restype = ctypes.c_int
    L.sc_options_default.argtypes = [ctypes.POINTER(Options)]
    L.sc_options_default.restype = None
    L.sc_all_edges.argtypes = [vp, ctypes.POINTER(Options), vp, vp, ctypes.POINTER(Report)]
    L.sc_all_edges.restype = ctypes.c_int
    L.sc_batch_all_edges.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(Options), ctypes.POINTER(i32),
                                     ctypes.POINTER(vp), ctypes.POINTER(Report)]
    L.sc_batch_all_edges.restype = ctypes.c_int
    L.sc_status_string.argtypes = [ctypes.c_int]
    L.sc_status_string.restype = ctypes.c_char_p
    L.sc_last_error_detail.argtypes = []
    L.sc_last_error_detail.restype = ctypes.c_char_p
    L.sc_abi_version.argtypes = []
    L.sc_abi_version.restype = ctypes.c_int32
    L.sc_all_edges_noalloc.argtypes = [i32, i64, vp, vp, i32, vp, vp]
    L.sc_all_edges_noalloc.restype = ctypes.c_int
    f32p = ctypes.POINTER(ctypes.c_float)
    L.sc_source_features.argtypes = [vp, f32p]
    L.sc_source_features.restype = ctypes.c_int
    L.sc_certified_lengths.argtypes = [vp, f64, i32, i32p, i32p, i32p]
    L.sc_certified_lengths.restype = ctypes.c_int
    L.sc_estimated_lengths.argtypes = [vp, f64, i32, i32, i32p, i32p]
    L.sc_estimated_lengths.restype = ctypes.c_int
    L.sc_mlp_train.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(MlpTrainOpts), f32p, f32p, f32p]
    L.sc_mlp_train.restype = ctypes.c_int
    L.sc_mlp_load.argtypes = [vp, f32p]
    L.sc_mlp_load.restype = ctypes.c_int
    L.sc_mlp_predict.argtypes = [vp, i32, i32p]
    L.sc_mlp_predict.restype = ctypes.c_int
    L.sc_mlp_loss_grad.argtypes = [f32p, f32p, f32p, i32, f32p, f32p, vp]
    L.sc_mlp_loss_grad.restype = ctypes.c_int
    L.sc_eigenpairs.argtypes = [vp, ctypes.POINTER(EigOpts), f64p, f64p, ctypes.POINTER(EigReport)]
    L.sc_eigenpairs.restype = ctypes.c_int
    L.sc_caltau.argtypes = [vp, f64, i32, f64p, f64p, f64, i32p, i32p]
    L.sc_caltau.restype = ctypes.c_int
    L.sc_graph_set_lambda.argtypes = [vp, ctypes.POINTER(Lambda)]
    L.sc_graph_set_lambda.restype = ctypes.c_int
    L.sc_some_edges.argtypes = [vp, ctypes.POINTER(Options), i64, ctypes.POINTER(ctypes.c_int64), vp,
                                ctypes.POINTER(Report)]
    L.sc_some_edges.restype = ctypes.c_int
    L.sc_series_meet.argtypes = [vp, i32p, f64p]
    L.sc_series_meet.restype = ctypes.c_int
    L.sc_tridiag_eig.argtypes = [i32, f64p, f64p, f64p, f64p]
    L.sc_tridiag_eig.restype = ctypes.c_int
    L.sc_selftest_bounded_waits.argtypes = [ctypes.c_uint32]
    L.sc_selftest_bounded_waits.restype = ctypes.c_int
    _lib = L
    return L


def _check(status: int, where: str):
    if status != SC_OK:
        detail = load().sc_last_error_detail().decode(errors="replace")
        raise ScError(status, where, detail)


def _torch():
    import torch

    return torch


def _stream_handle(stream):
    if stream is None:
        torch = _torch()
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr_and_flag(arr):
    """(pointer, is_device, keepalive) for a numpy array or torch tensor of int32."""
    try:
        torch = _torch()
        if isinstance(arr, torch.Tensor):
            t = arr.contiguous().to(torch.int32)
            return ctypes.c_void_p(t.data_ptr()), t.is_cuda, t
    except ImportError:
        pass
    a = np.ascontiguousarray(arr, dtype=np.int32)
    return ctypes.c_void_p(a.ctypes.data), False, a


class Graph:
    """A validated graph resident on the GPU (wraps ``sc_graph``)."""

    def __init__(self, row_ptr, col_idx, stream=None, reject_bipartite: bool = False):
        L = load()
        rp, rp_dev, keep_rp = _ptr_and_flag(row_ptr)
        ci, ci_dev, keep_ci = _ptr_and_flag(col_idx)
        if rp_dev != ci_dev:
            raise ValueError("row_ptr and col_idx must both be host or both be device arrays")
        n = int(keep_rp.shape[0]) - 1
        nnz = int(keep_ci.shape[0])
        flags = (SC_PTRS_DEVICE if rp_dev else SC_PTRS_HOST) | (SC_FLAG_REJECT_BIPARTITE if reject_bipartite else 0)
        self._stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        _check(L.sc_graph_create(ctypes.byref(h), n, nnz, rp, ci, flags, self._stream), "sc_graph_create")
        self._h = h
        self.n, self.nnz = n, nnz

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().sc_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def info(self) -> dict:
        out = GraphInfo()
        _check(load().sc_graph_get_info(self._h, ctypes.byref(out)), "sc_graph_get_info")
        return {name: getattr(out, name) for name, _ in GraphInfo._fields_}

    def estimate_lambda(self, max_iter: int = 0, tol: float = 0.0, seed: int = 0x1a2b3c4d,
                        allow_unconverged: bool = False) -> dict:
        opts = LambdaOpts(max_iter, tol, seed)
        out = Lambda()
        st = load().sc_estimate_lambda(self._h, ctypes.byref(opts), ctypes.byref(out))
        if not (allow_unconverged and st == 9):
            _check(st, "sc_estimate_lambda")
        return {name: getattr(out, name) for name, _ in Lambda._fields_}

    def set_lambda(self, lambda_plus: float, lambda_minus: float, lambda_star: float):
        """sc_graph_set_lambda: use the caller's eigenvalue bound (residuals 0)."""
        lam = Lambda(lambda_plus, lambda_minus, lambda_star, 0.0, 0.0, 0, 1)
        _check(load().sc_graph_set_lambda(self._h, ctypes.byref(lam)), "sc_graph_set_lambda")

    def eigenpairs(self, omega: int = 128, max_iter: int = 0, tol: float = 0.0, rest_tol: float = 0.0,
                   rest_max_iter: int = 0, seed: int = 0x1a2b3c4d, allow_unconverged: bool = False):
        """sc_eigenpairs: (lam float64[omega], F float64[omega, n], report dict); lam[0] = 1, F[0] = 1,
        the pairs taken exactly in rows 1 .. used - 1, zeros after them."""
        opts = EigOpts(omega, max_iter, tol, rest_tol, rest_max_iter, 0, seed)
        lam = np.zeros(omega, dtype=np.float64)
        F = np.zeros((omega, self.n), dtype=np.float64)
        rep = EigReport()
        st = load().sc_eigenpairs(self._h, ctypes.byref(opts), _f64p(lam), _f64p(F), ctypes.byref(rep))
        if not (allow_unconverged and st == 9):
            _check(st, "sc_eigenpairs")
        return lam, F, {name: getattr(rep, name) for name, _ in EigReport._fields_}

    def caltau(self, eps: float, lam=None, F=None, lam_rest: float = 0.0):
        """sc_caltau: (tau int32[nnz], longest length). lam / F None: the pairs of the last eigenpairs()."""
        tau = np.empty(self.nnz, dtype=np.int32)
        ell = ctypes.c_int32()
        if lam is None:
            st = load().sc_caltau(self._h, eps, 0, None, None, 0.0, _i32p(tau), ctypes.byref(ell))
        else:
            lam = np.ascontiguousarray(lam, dtype=np.float64)
            F = np.ascontiguousarray(F, dtype=np.float64)
            if F.shape != (lam.size, self.n):
                raise ValueError(f"F must be {lam.size} x {self.n}")
            st = load().sc_caltau(self._h, eps, lam.size, _f64p(lam), _f64p(F), float(lam_rest), _i32p(tau),
                                  ctypes.byref(ell))
        _check(st, "sc_caltau")
        return tau, int(ell.value)

    def series_meet(self, tau):
        """sc_series_meet: S_tau per CSR entry (host float64[nnz]) at the lengths tau (int32[nnz] or one int)."""
        t = np.ascontiguousarray(np.broadcast_to(np.asarray(tau, dtype=np.int32), (self.nnz,)))
        out = np.empty(self.nnz, dtype=np.float64)
        _check(load().sc_series_meet(self._h, _i32p(t), _f64p(out)), "sc_series_meet")
        return out

    def truncation_length(self, eps: float, lam: dict | None = None):
        """(ell_global, per_source int32[n], per_entry int32[nnz]) on the host."""
        ell = ctypes.c_int32()
        ps = np.empty(self.n, dtype=np.int32)
        pe = np.empty(self.nnz, dtype=np.int32)
        lp = None
        if lam is not None:
            lp = ctypes.byref(Lambda(*[lam[name] for name, _ in Lambda._fields_]))
        _check(load().sc_truncation_length(
            self._h, eps, lp, ctypes.byref(ell), ps.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            pe.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "sc_truncation_length")
        return int(ell.value), ps, pe

    @staticmethod
    def options(eps=1e-3, mode="tgt", precision="fp32", policy="global", ell_fixed=0,
                estimator="plain", block_width=0, rows_split=0, heavy_threshold=0, max_slices=0,
                record_tail=False, time_kernels=False, seed=None, delta=0.0, gamma=None,
                switch="cost", windows=None, bf16_from_hop=0, sparse_hops=False,
                full_topgamma_scan=False, ell_cap=0) -> Options:
        o = Options()
        load().sc_options_default(ctypes.byref(o))
        o.eps = eps
        o.mode = MODE[mode]
        o.precision = PREC[precision]
        o.ell_policy = ELL[policy]
        o.ell_fixed = ell_fixed
        o.estimator = EST[estimator]
        o.block_width = block_width
        o.rows_split = rows_split
        o.heavy_threshold = heavy_threshold
        o.max_slices = max_slices
        o.flags = (SC_OPT_RECORD_TAIL if record_tail else 0) | (SC_OPT_TIME_KERNELS if time_kernels else 0)
        if windows is not None:  # None: automatic; True / False: force on / off
            o.flags |= SC_OPT_WINDOWS_FORCE if windows else SC_OPT_WINDOWS_OFF
        if sparse_hops:
            o.flags |= SC_OPT_SPARSE_HOPS
        if full_topgamma_scan:
            o.flags |= SC_OPT_FULL_TOPGAMMA_SCAN
        if seed is not None:
            o.seed = seed
        o.delta = delta
        if gamma is not None:
            o.gamma = gamma
        o.switch_rule = {"cost": 0, "paper": 1, "per_source": 2}[switch]
        o.bf16_from_hop = bf16_from_hop
        o.ell_cap = ell_cap
        return o

    def all_edges(self, out=None, tail_bound=None, **kw):
        """Run sc_all_edges. ``out``/``tail_bound``: torch CUDA float64 tensors
        of nnz entries (device output) or None (host numpy output).
        Returns (s_hat, tail_bound or None, report dict)."""
        o = self.options(**kw)
        rep = Report()
        if out is not None and not getattr(out, "is_cuda", False):
            # caller-provided host buffer (e.g. a pinned torch tensor)
            tb = ctypes.c_void_p(tail_bound.data_ptr()) if tail_bound is not None else None
            _check(load().sc_all_edges(self._h, ctypes.byref(o), ctypes.c_void_p(out.data_ptr()), tb,
                                       ctypes.byref(rep)), "sc_all_edges")
            return out, tail_bound, rep.as_dict()
        if out is not None:
            o.flags |= SC_OUT_DEVICE
            tb = ctypes.c_void_p(tail_bound.data_ptr()) if tail_bound is not None else None
            _check(load().sc_all_edges(self._h, ctypes.byref(o), ctypes.c_void_p(out.data_ptr()), tb,
                                       ctypes.byref(rep)), "sc_all_edges")
            return out, tail_bound, rep.as_dict()
        s = np.empty(self.nnz, dtype=np.float64)
        b = np.empty(self.nnz, dtype=np.float64) if kw.get("record_tail") or kw.get("estimator") == "end_corrected" else None
        _check(load().sc_all_edges(self._h, ctypes.byref(o), ctypes.c_void_p(s.ctypes.data),
                                   ctypes.c_void_p(b.ctypes.data) if b is not None else None,
                                   ctypes.byref(rep)), "sc_all_edges")
        return s, b, rep.as_dict()


def some_edges(graph, entries, out=None, **kw):
    """sc_some_edges: s_hat at the listed CSR entries (int64 indices) only.
    ``out``: a torch CUDA float64 tensor of len(entries) values (device output)
    or None (host numpy output). Returns (values, report dict)."""
    ent = np.ascontiguousarray(entries, dtype=np.int64)
    o = Graph.options(**kw)
    rep = Report()
    if out is not None:
        o.flags |= SC_OUT_DEVICE
        dst = ctypes.c_void_p(out.data_ptr())
        res = out
    else:
        res = np.empty(ent.size, dtype=np.float64)
        dst = ctypes.c_void_p(res.ctypes.data)
    _check(load().sc_some_edges(graph._h, ctypes.byref(o), ent.size,
                                ent.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), dst, ctypes.byref(rep)),
           "sc_some_edges")
    return res, rep.as_dict()


def batch_all_edges(graphs, ell_per_graph=None, outs=None, **kw):
    """sc_batch_all_edges over a list of Graph objects. ``ell_per_graph``:
    None or one length per graph (0 keeps the policy). ``outs``: None (host
    numpy outputs) or one torch CUDA float64 tensor per graph. Returns
    (list of s_hat, list of report dicts)."""
    count = len(graphs)
    o = Graph.options(**kw)
    hs = (ctypes.c_void_p * count)(*[g._h.value for g in graphs])
    if outs is None:
        res = [np.empty(g.nnz, dtype=np.float64) for g in graphs]
        ptrs = (ctypes.c_void_p * count)(*[r.ctypes.data for r in res])
    else:
        res = list(outs)
        o.flags |= SC_OUT_DEVICE
        ptrs = (ctypes.c_void_p * count)(*[r.data_ptr() for r in res])
    ells = None
    if ell_per_graph is not None:
        ells = (ctypes.c_int32 * count)(*[int(x) for x in ell_per_graph])
    reps = (Report * count)()
    _check(load().sc_batch_all_edges(ctypes.cast(hs, ctypes.POINTER(ctypes.c_void_p)), count, ctypes.byref(o),
                                     ells, ctypes.cast(ptrs, ctypes.POINTER(ctypes.c_void_p)), reps),
           "sc_batch_all_edges")
    return res, [r.as_dict() for r in reps]


def _noalloc_args(row_ptr, col_idx, out):
    """Checks the tensors sc_all_edges_noalloc receives as raw pointers, since the
    library trusts n, nnz and the output length: 1-D contiguous int32 CSR arrays
    and a float64 output of at least nnz entries, all on one CUDA device.
    Raises ValueError / TypeError before anything reaches the library."""
    torch = _torch()
    for name, t in (("row_ptr", row_ptr), ("col_idx", col_idx), ("out", out)):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
        if t.dim() != 1:
            raise ValueError(f"{name} must be 1-D")
    if row_ptr.dtype != torch.int32 or col_idx.dtype != torch.int32:
        raise TypeError("row_ptr and col_idx must be int32")
    if out.dtype != torch.float64:
        raise TypeError("out must be float64")
    for name, t in (("row_ptr", row_ptr), ("col_idx", col_idx), ("out", out)):
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    n = int(row_ptr.numel()) - 1
    nnz = int(col_idx.numel())
    if n < 2 or nnz < 2:
        raise ValueError("need row_ptr with at least 3 entries (n >= 2) and at least 2 CSR entries")
    if out.numel() < nnz:
        raise ValueError(f"out holds {out.numel()} values, fewer than nnz = {nnz}")
    for name, t in (("row_ptr", row_ptr), ("col_idx", col_idx), ("out", out)):
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
    if not (row_ptr.device == col_idx.device == out.device):
        raise ValueError("row_ptr, col_idx and out must be on the same CUDA device")
    return n, nnz


def all_edges_noalloc(row_ptr, col_idx, ell: int, out, stream=None):
    """sc_all_edges_noalloc on torch CUDA tensors (int32 CSR, float64 output of
    nnz entries): the traversal for callers that cannot allocate device memory.
    Works in the library's fixed 64 MiB device array; see include/sc.h.
    The tensors are checked here (dtype, contiguity, sizes, one device) and the
    call runs with their device current."""
    n, nnz = _noalloc_args(row_ptr, col_idx, out)
    torch = _torch()
    with torch.cuda.device(row_ptr.device):
        _check(load().sc_all_edges_noalloc(n, nnz, ctypes.c_void_p(row_ptr.data_ptr()),
                                           ctypes.c_void_p(col_idx.data_ptr()), int(ell),
                                           ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
               "sc_all_edges_noalloc")
    return out


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _f64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def tridiag_eig(alpha, beta):
    """sc_tridiag_eig (host only): eigenvalues ascending and eigenvectors as columns."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    k = a.size
    if b.size != max(k - 1, 0):
        raise ValueError("beta must hold k - 1 values")
    theta = np.empty(k, dtype=np.float64)
    Z = np.empty((k, k), dtype=np.float64)  # row q = eigenvector q (the C column q)
    _check(load().sc_tridiag_eig(k, _f64p(a), _f64p(b) if k > 1 else None, _f64p(theta), _f64p(Z)), "sc_tridiag_eig")
    return theta, Z.T.copy()


def _i32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def source_features(graph) -> np.ndarray:
    out = np.empty((graph.n, MLP_FEATURES), dtype=np.float32)
    _check(load().sc_source_features(graph._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
           "sc_source_features")
    return out


def certified_lengths(graph, eps: float, precision: str = "fp64"):
    """(per_entry int32[nnz], per_source int32[n], cap)"""
    pe = np.empty(graph.nnz, dtype=np.int32)
    ps = np.empty(graph.n, dtype=np.int32)
    cap = ctypes.c_int32()
    _check(load().sc_certified_lengths(graph._h, eps, PREC[precision], _i32p(pe), _i32p(ps), ctypes.byref(cap)),
           "sc_certified_lengths")
    return pe, ps, int(cap.value)


def estimated_lengths(graph, eps: float, cap: int, precision: str = "fp64"):
    """Bipartite graph: (per_entry int32[nnz], per_source int32[n]) from the tail estimate."""
    pe = np.empty(graph.nnz, dtype=np.int32)
    ps = np.empty(graph.n, dtype=np.int32)
    _check(load().sc_estimated_lengths(graph._h, eps, PREC[precision], cap, _i32p(pe), _i32p(ps)),
           "sc_estimated_lengths")
    return pe, ps


def mlp_train(graphs, init_params, epochs=300, lr=1e-2, eps=1e-3, precision="fp32", ell_cap=0):
    """Train on the GPU. Returns (model float32[MLP_MODEL_FLOATS], loss curve float32[epochs]).
    ell_cap: the label cap of bipartite training graphs (sc_estimated_lengths)."""
    hs = (ctypes.c_void_p * len(graphs))(*[g._h.value for g in graphs])
    opts = MlpTrainOpts(epochs, lr, 0.0, 0.0, 0.0, PREC[precision], eps, ell_cap, 0)
    p, pp = _f32(init_params)
    model = np.empty(MLP_MODEL_FLOATS, dtype=np.float32)
    curve = np.empty(epochs, dtype=np.float32)
    _check(load().sc_mlp_train(hs, len(graphs), ctypes.byref(opts), pp,
                               model.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                               curve.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "sc_mlp_train")
    return model, curve


def mlp_load(graph, model):
    m, mp = _f32(model)
    _check(load().sc_mlp_load(graph._h, mp), "sc_mlp_load")


def mlp_predict(graph, cap: int) -> np.ndarray:
    out = np.empty(graph.n, dtype=np.int32)
    _check(load().sc_mlp_predict(graph._h, cap, _i32p(out)), "sc_mlp_predict")
    return out


def mlp_loss_grad(model, features, targets):
    m, mp = _f32(model)
    f, fp = _f32(features)
    t, tp = _f32(targets)
    loss = ctypes.c_float()
    grad = np.empty(MLP_PARAMS, dtype=np.float32)
    _check(load().sc_mlp_loss_grad(mp, fp, tp, t.size, ctypes.byref(loss),
                                   grad.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _stream_handle(None)),
           "sc_mlp_loss_grad")
    return float(loss.value), grad


def selftest_bounded_waits(limit_us: int = 2000) -> tuple[int, str]:
    """Runs the library's bounded-wait self-test (a wait that nothing
    completes, limited to limit_us); returns (status, detail). SC_ERR_TIMEOUT
    is the expected status: both waits gave up and said so."""
    L = load()
    st = int(L.sc_selftest_bounded_waits(int(limit_us)))
    return st, L.sc_last_error_detail().decode(errors="replace")
