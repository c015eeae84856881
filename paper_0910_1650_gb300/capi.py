"""Thin Python binding of libapgb.so (ctypes).

Argument marshalling only: every step runs in the CUDA library.  Tensors are
torch CUDA tensors (torch provides device memory and streams); the functions
carry the names of the C entry points in ``include/apgb.h``.  If the library
is missing or a call fails, an exception is raised -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libapgb.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "apgb.h")

AP_OK = 0
AP_NOT_CONVERGED = 1
AP_NO_EXEMPLARS = 2
AP_PREC_FP32, AP_PREC_BF16 = 0, 1
AP_PREF_MEDIAN, AP_PREF_SCALAR, AP_PREF_VECTOR = 0, 1, 2
AP_FLAG_TIME_SWEEP = 1
AP_FLAG_NO_GRAPH = 2
AP_FLAG_PAP_CARRY_R = 4
AP_FLAG_S_CHECKED = 8
AP_FLAG_COLD = 16
AP_LANDMARK_UNIFORM, AP_LANDMARK_SCORE, AP_LANDMARK_GIVEN = 0, 1, 2
AP_ERR_TOO_LARGE = -7
AP_ERR_CAPACITY = -8
AP_ERR_TIMEOUT = -4
AP_NOALLOC_MAX_N = 65536


class ApParams(C.Structure):
    _fields_ = [("damping", C.c_float), ("max_iter", C.c_int32), ("conv_iter", C.c_int32),
                ("check_every", C.c_int32), ("flags", C.c_int32)]


class ApResult(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("n_exemplars", C.c_int32),
                ("status", C.c_int32), ("dpsim", C.c_double), ("expref", C.c_double),
                ("netsim", C.c_double), ("sweep_ms", C.c_double),
                ("sweep_launches", C.c_int32), ("pad", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class ApSweepConfig(C.Structure):
    _fields_ = [("cluster", C.c_int32), ("ept", C.c_int32), ("stages", C.c_int32),
                ("threads", C.c_int32), ("clusters", C.c_int32), ("smem_bytes", C.c_int32),
                ("ms_per_iter", C.c_float), ("pad", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class PapResult(C.Structure):
    _fields_ = [("k", C.c_int32), ("sub_iters_max", C.c_int32), ("sub_iters_sum", C.c_int64),
                ("sub_not_converged", C.c_int32), ("pad", C.c_int32), ("sub_ms", C.c_double),
                ("merge_ms", C.c_double), ("final_ms", C.c_double), ("exemplars_ms", C.c_double),
                ("final", ApResult)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("pad", "final")}
        d["final"] = self.final.as_dict()
        return d


class LapResult(C.Structure):
    _fields_ = [("n_landmarks", C.c_int32), ("n_exemplars", C.c_int32), ("pref", C.c_float),
                ("pad", C.c_int32), ("dpsim", C.c_double), ("expref", C.c_double),
                ("netsim", C.c_double), ("select_ms", C.c_double), ("landmark_ms", C.c_double),
                ("assign_ms", C.c_double), ("netsim_ms", C.c_double), ("landmark", ApResult)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("pad", "landmark")}
        d["landmark"] = self.landmark.as_dict()
        return d


AP_LAP_MAX_LEVELS = 8


class LapFullResult(C.Structure):
    _fields_ = [("levels", C.c_int32), ("n_exemplars", C.c_int32), ("pref", C.c_float),
                ("base_case", C.c_int32), ("unassigned", C.c_int32 * AP_LAP_MAX_LEVELS),
                ("exemplars_at", C.c_int32 * (AP_LAP_MAX_LEVELS + 1)), ("ms", C.c_float),
                ("dpsim", C.c_double), ("expref", C.c_double), ("netsim", C.c_double),
                ("refine_rounds", C.c_int32), ("refine_removed", C.c_int32),
                ("refine_moved", C.c_int32), ("pad2", C.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "pad2"}
        d["unassigned"] = list(self.unassigned)[:max(self.levels, 1)]
        d["exemplars_at"] = list(self.exemplars_at)[:self.levels + self.base_case]
        return d


class LapRefineResult(C.Structure):
    _fields_ = [("rounds", C.c_int32), ("removed", C.c_int32), ("moved", C.c_int32),
                ("n_exemplars", C.c_int32), ("dpsim", C.c_double), ("expref", C.c_double),
                ("netsim", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AplResult(C.Structure):
    _fields_ = [("used_warm", C.c_int32), ("warm_iters", C.c_int32), ("cold_iters", C.c_int32),
                ("pad", C.c_int32), ("warm_netsim", C.c_double), ("cold_netsim", C.c_double),
                ("features_ms", C.c_double), ("forward_ms", C.c_double), ("warm_ms", C.c_double),
                ("cold_ms", C.c_double), ("result", ApResult)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("pad", "result")}
        d["result"] = self.result.as_dict()
        return d


class ApgbError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        super().__init__(f"{fn} failed: {status} ({status_string(status)})")


_lib = None
_P = C.c_void_p
_I64 = C.c_int64
_SZ = C.c_size_t

_SIGNATURES = {
    "ap_similarity_workspace_size": (_SZ, [_I64, _I64]),
    "ap_similarity": (C.c_int32, [_P, _I64, _I64, _I64, _P, _I64, C.c_int32, C.c_int32, _P,
                                  C.c_double, C.c_uint64, _P, _P, _SZ, _P]),
    "ap_similarity_batched_workspace_size": (_SZ, [_P, C.c_int32, _I64]),
    "ap_similarity_batched": (C.c_int32, [_P, _P, _P, C.c_int32, _I64, _I64, _P, _P, _P,
                                          C.c_int32, C.c_int32, _P, _P, _P, _SZ, _P]),
    "ap_preference_median_workspace_size": (_SZ, [_I64]),
    "ap_preference_median": (C.c_int32, [_P, _I64, _I64, _P, _P, _SZ, _P]),
    "ap_iterate_workspace_size": (_SZ, [_I64, _I64]),
    "ap_iterate": (C.c_int32, [_P, _P, _P, _I64, _I64, C.POINTER(ApParams), _P,
                               C.POINTER(ApResult), _P, _SZ, _P]),
    "ap_iterate_batched_workspace_size": (_SZ, [_P, _P, C.c_int32]),
    "ap_iterate_batched": (C.c_int32, [_P, _P, _P, _P, _P, _P, C.c_int32, C.POINTER(ApParams), _P,
                                       _P, _P, _SZ, _P]),
    "pap_run_workspace_size": (_SZ, [_I64, _I64, C.c_int32, _P]),
    "pap_run": (C.c_int32, [_P, _I64, _I64, C.c_int32, _P, C.POINTER(ApParams), _P, _P, _P,
                            C.POINTER(PapResult), _P, _SZ, _P]),
    "lap_run_workspace_size": (_SZ, [_I64, _I64, _I64]),
    "lap_run": (C.c_int32, [_P, _I64, _I64, _I64, _I64, C.c_int32, _P, _P, C.c_uint64, C.c_int32,
                            C.POINTER(ApParams), _P, _P, C.POINTER(LapResult), _P, _SZ, _P]),
    "lap_assign_workspace_size": (_SZ, [_I64, _I64, _I64]),
    "lap_assign": (C.c_int32, [_P, _I64, _I64, _I64, _P, _I64, _P, _P, _P, _SZ, _P]),
    "lap_refine_workspace_size": (_SZ, [_I64, _I64, _I64]),
    "lap_refine": (C.c_int32, [_P, _I64, _I64, _I64, _P, _I64, C.c_float, C.c_int32, _P, _P,
                               C.POINTER(LapRefineResult), _P, _SZ, _P]),
    "lap_run_full_workspace_size": (_SZ, [_I64, _I64, _I64, _I64, C.c_int32]),
    "lap_run_full": (C.c_int32, [_P, _I64, _I64, _I64, _I64, _I64, C.c_uint64, C.c_int32,
                                 C.POINTER(ApParams), C.c_int32, C.c_int32, _P, _P,
                                 C.POINTER(LapFullResult),
                                 _P, _SZ, _P]),
    "apl_param_count": (C.c_int64, []),
    "apl_features_workspace_size": (_SZ, [_I64]),
    "apl_features": (C.c_int32, [_P, _I64, _I64, C.c_float, _P, _P, _SZ, _P]),
    "apl_targets": (C.c_int32, [_P, _P, _P, _I64, _I64, C.c_float, _P, _P]),
    "apl_workspace_size": (_SZ, [_I64]),
    "apl_sync_bf16": (C.c_int32, [_P, _P, _P]),
    "apl_forward": (C.c_int32, [_P, _P, _P, _I64, _P, _P, _SZ, _P]),
    "apl_train_step": (C.c_int32, [_P, _P, _P, _P, C.c_int64, C.c_float, _P, _P, _I64, _P, _P,
                                   _P, _SZ, _P]),
    "apl_warm_start": (C.c_int32, [_P, _I64, C.c_float, _P, _P, _I64, _P]),
    "apl_warm_start_batched_workspace_size": (_SZ, [_P, C.c_int32]),
    "apl_warm_start_batched": (C.c_int32, [_P, _P, _P, _P, _P, _P, C.c_int32, _P, _P, _P, _P, _P,
                                           _SZ, _P]),
    "apl_set_standardisation": (C.c_int32, [_P, _P, _I64, _P]),
    "apl_judge": (C.c_int32, [_P, _P, C.c_int32, C.c_double, _P]),
    "apl_ap_run_workspace_size": (_SZ, [_I64, _I64]),
    "apl_ap_run": (C.c_int32, [_P, _I64, _I64, _P, _P, C.c_float, C.POINTER(ApParams), C.c_int32,
                               _P, _P, _P, C.POINTER(AplResult), _P, _SZ, _P]),
    "ap_shard_workspace_size": (_SZ, [_I64, _I64, _I64, _I64]),
    "ap_shard_begin": (C.c_int32, [_P, _P, _P, _I64, _I64, _I64, _I64, C.POINTER(ApParams), _P, _P,
                                   _SZ, _P]),
    "ap_shard_sweep": (C.c_int32, [_P, _P, _P, _I64, _I64, _I64, _I64, C.POINTER(ApParams), _P, _P,
                                   _P, _SZ, _P]),
    "ap_shard_finish": (C.c_int32, [_P, _P, _P, _I64, _I64, _I64, _I64, C.POINTER(ApParams), _P, _P,
                                    _P, C.POINTER(ApResult), _P, _SZ, _P]),
    "ap_sweep_get_config": (C.c_int32, [_I64, C.POINTER(ApSweepConfig)]),
    "ap_sweep_set_config": (C.c_int32, [_I64, C.POINTER(ApSweepConfig)]),
    "ap_sweep_plan": (C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int32, _P, C.c_int32, _P,
                                  C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "ap_sweep_classes": (C.c_int32, [_P, C.c_int32, _P]),
    "ap_sweep_autotune_workspace_size": (_SZ, [_I64, _I64]),
    "ap_sweep_autotune": (C.c_int32, [_P, _P, _P, _I64, _I64, C.c_float, C.c_int32,
                                      C.POINTER(ApSweepConfig), _P, _SZ, _P]),
    "ap_exemplars_workspace_size": (_SZ, [_I64]),
    "ap_exemplars": (C.c_int32, [_P, _P, _P, _I64, _I64, _P, C.POINTER(ApResult), _P, _SZ, _P]),
    "ap_exemplars_noalloc": (C.c_int32, [_P, _P, _P, _I64, _I64, _P, C.POINTER(ApResult), _P]),
    "ap_status_string": (C.c_char_p, [C.c_int32]),
    "ap_version": (C.c_int32, []),
    "ap_kernel_launches": (C.c_uint64, []),
    "ap_wait_selftest": (C.c_int32, [C.c_uint32, _P]),
}


def header_functions():
    """Names of every function declared in include/apgb.h."""
    with open(HEADER) as f:
        text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    return sorted(set(re.findall(r"\b(ap[a-z_0-9]*)\s*\(", text)))


def lib():
    """The loaded library (loads it on first use; raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                               "(the CUDA library is required; there is no CPU path)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().ap_status_string(int(s)).decode()


def kernel_launches() -> int:
    return int(lib().ap_kernel_launches())


def _check(fn, status, ok=(AP_OK, AP_NOT_CONVERGED, AP_NO_EXEMPLARS)):
    if status not in ok:
        raise ApgbError(fn, status)
    return status


def _dev_f32(t, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32):
        raise TypeError(f"{name} must be a float32 CUDA tensor")
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError(f"{name} must be 2-D with unit column stride")
    return t


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def workspace(nbytes: int, device) -> torch.Tensor:
    """Caller-owned scratch for one call (torch allocation, 256-B aligned)."""
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def padded_ld(n: int) -> int:
    """Leading dimension used for library-allocated N x N matrices (x32)."""
    return (n + 31) // 32 * 32


def empty_square(n: int, device, fill=None) -> torch.Tensor:
    """N x N float32 view with a 32-padded leading dimension."""
    ld = padded_ld(n)
    base = torch.empty((n, ld), dtype=torch.float32, device=device)
    if fill is not None:
        base.fill_(fill)
    return base[:, :n]


# ---------------------------------------------------------------------------

def ap_similarity(X, S=None, precision="fp32", pref="median", noise_rel=0.0, seed=0,
                  stream=None):
    """S (n x n) from features X (n x d); returns (S, preference used)."""
    _dev_f32(X, "X")
    n, d = X.shape
    if S is None:
        S = empty_square(n, X.device)
    _dev_f32(S, "S")
    prec = {"fp32": AP_PREC_FP32, "bf16": AP_PREC_BF16}[precision]
    keep = None
    if isinstance(pref, str):
        mode, pptr = AP_PREF_MEDIAN, None
    elif isinstance(pref, torch.Tensor):
        keep = pref.to(device=X.device, dtype=torch.float32).contiguous()
        mode, pptr = AP_PREF_VECTOR, C.c_void_p(keep.data_ptr())
    else:
        keep = (C.c_float * 1)(float(pref))
        mode, pptr = AP_PREF_SCALAR, C.cast(keep, C.c_void_p)
    ws = workspace(lib().ap_similarity_workspace_size(n, d), X.device)
    out = C.c_float(0.0)
    st = lib().ap_similarity(C.c_void_p(X.data_ptr()), n, d, X.stride(0),
                             C.c_void_p(S.data_ptr()), S.stride(0), prec, mode, pptr,
                             float(noise_rel), int(seed) & 0xFFFFFFFFFFFFFFFF,
                             C.cast(C.pointer(out), C.c_void_p), C.c_void_p(ws.data_ptr()),
                             ws.numel(), _stream(stream))
    _check("ap_similarity", st, ok=(AP_OK,))
    return S, float(out.value)


def ap_similarity_batched_workspace_bytes(n, d):
    """Workspace bytes ap_similarity_batched needs for problems of sizes n, dimension d."""
    na = _i64_array(n)
    return int(lib().ap_similarity_batched_workspace_size(C.cast(na, C.c_void_p), len(n), int(d)))


def ap_similarity_batched_workspace(n, d, device):
    """A workspace for ap_similarity_batched on problems of sizes n, dimension d."""
    return workspace(ap_similarity_batched_workspace_bytes(n, d), device)


def ap_similarity_batched(X, xoff, n, S, soff, lds, precision="bf16", pref="median", ws=None,
                          stream=None):
    """ap_similarity for several problems in one call.  X: float32 CUDA
    tensor (rows of every problem, same d; 2-D), problem b's rows start at
    element offset xoff[b]; S: 1-D float32 CUDA arena, problem b's n[b] x n[b]
    matrix at element offset soff[b] with leading dimension lds[b].  ws: a
    uint8 CUDA workspace of at least the size the library asks for (allocated
    here when omitted).  Returns the list of preferences."""
    _dev_f32(X, "X")
    if not (S.is_cuda and S.dtype == torch.float32 and S.is_contiguous()):
        raise TypeError("S must be a contiguous float32 CUDA tensor")
    d, ldx = X.shape[1], X.stride(0)
    count = len(n)
    prec = {"fp32": AP_PREC_FP32, "bf16": AP_PREC_BF16}[precision]
    if isinstance(pref, str):
        mode, pptr, keep = AP_PREF_MEDIAN, None, None
    else:
        keep = (C.c_float * 1)(float(pref))
        mode, pptr = AP_PREF_SCALAR, C.cast(keep, C.c_void_p)
    xo, na, so, la = _i64_array(xoff), _i64_array(n), _i64_array(soff), _i64_array(lds)
    out = (C.c_float * count)()
    if ws is None:
        ws = ap_similarity_batched_workspace(n, d, X.device)
    st = lib().ap_similarity_batched(_ptr(X), C.cast(xo, C.c_void_p), C.cast(na, C.c_void_p), count,
                                     d, ldx, _ptr(S), C.cast(so, C.c_void_p), C.cast(la, C.c_void_p),
                                     prec, mode, pptr, C.cast(out, C.c_void_p), _ptr(ws), ws.numel(),
                                     _stream(stream))
    _check("ap_similarity_batched", st, ok=(AP_OK,))
    return [float(v) for v in out]


def ap_preference_median(S, stream=None):
    """Exact median of the off-diagonal entries of S (float)."""
    _dev_f32(S, "S")
    n = S.shape[0]
    ws = workspace(lib().ap_preference_median_workspace_size(n), S.device)
    out = C.c_float(0.0)
    st = lib().ap_preference_median(C.c_void_p(S.data_ptr()), n, S.stride(0),
                                    C.cast(C.pointer(out), C.c_void_p),
                                    C.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream))
    _check("ap_preference_median", st, ok=(AP_OK,))
    return float(out.value)


def ap_iterate(S, R=None, A=None, damping=0.5, max_iter=200, conv_iter=15, check_every=0,
               time_sweep=False, decisions=True, graph=True, s_checked=False, cold=False,
               stream=None):
    """Runs Algorithm 1 in place on (R, A) (zeros when omitted).  ``graph``:
    enqueue each chunk of iterations as one CUDA graph (ignored with
    ``time_sweep``); ``s_checked``: S is known finite (skip the library's
    NaN/Inf pass); ``cold``: start from R = A = 0 whatever R and A hold (they
    are not read).  Returns (R, A, result dict, decisions int32 tensor or None)."""
    _dev_f32(S, "S")
    n = S.shape[0]
    if R is None:
        R = empty_square(n, S.device, 0.0)
    if A is None:
        A = empty_square(n, S.device, 0.0)
    _dev_f32(R, "R")
    _dev_f32(A, "A")
    if not (R.stride(0) == A.stride(0) == S.stride(0)):
        raise ValueError("S, R and A must share one leading dimension")
    dec = torch.empty(n, dtype=torch.int32, device=S.device) if decisions else None
    p = ApParams(float(damping), int(max_iter), int(conv_iter), int(check_every),
                 (AP_FLAG_TIME_SWEEP if time_sweep else 0) | (0 if graph else AP_FLAG_NO_GRAPH)
                 | (AP_FLAG_S_CHECKED if s_checked else 0) | (AP_FLAG_COLD if cold else 0))
    res = ApResult()
    ws = workspace(lib().ap_iterate_workspace_size(n, S.stride(0)), S.device)
    st = lib().ap_iterate(C.c_void_p(S.data_ptr()), C.c_void_p(R.data_ptr()),
                          C.c_void_p(A.data_ptr()), n, S.stride(0), C.byref(p),
                          C.c_void_p(dec.data_ptr()) if dec is not None else None,
                          C.byref(res), C.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream))
    _check("ap_iterate", st)
    return R, A, res.as_dict(), dec


def _i64_array(v):
    v = [int(x) for x in v]
    return (C.c_int64 * len(v))(*v)


def ap_iterate_batched_workspace(n, ld, device):
    """A workspace for ap_iterate_batched on problems of sizes n, ld."""
    n_a, ld_a = _i64_array(n), _i64_array(ld)
    return workspace(lib().ap_iterate_batched_workspace_size(C.cast(n_a, C.c_void_p),
                                                             C.cast(ld_a, C.c_void_p), len(n)), device)


def ap_iterate_batched(S, R, A, offsets, n, ld, damping=0.5, max_iter=200, conv_iter=15,
                       check_every=0, decisions=False, ws=None, cold=False, stream=None):
    """Algorithm 1 on several problems stored in 1-D float32 arenas (CUDA
    tensors).  Problem b: n[b] x n[b] at element offset offsets[b], leading
    dimension ld[b].  Returns (list of result dicts, decisions or None)."""
    for t, nm in ((S, "S"), (R, "R"), (A, "A")):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise TypeError(f"{nm} must be a contiguous float32 CUDA tensor")
    count = len(n)
    off_a, n_a, ld_a = _i64_array(offsets), _i64_array(n), _i64_array(ld)
    dec = torch.empty(sum(int(x) for x in n), dtype=torch.int32, device=S.device) if decisions else None
    p = ApParams(float(damping), int(max_iter), int(conv_iter), int(check_every),
                 AP_FLAG_COLD if cold else 0)
    out = (ApResult * count)()
    if ws is None:
        ws = ap_iterate_batched_workspace(n, ld, S.device)
    st = lib().ap_iterate_batched(C.c_void_p(S.data_ptr()), C.c_void_p(R.data_ptr()),
                                  C.c_void_p(A.data_ptr()), C.cast(off_a, C.c_void_p),
                                  C.cast(n_a, C.c_void_p), C.cast(ld_a, C.c_void_p), count,
                                  C.byref(p), C.c_void_p(dec.data_ptr()) if dec is not None else None,
                                  C.cast(out, C.c_void_p), C.c_void_p(ws.data_ptr()), ws.numel(),
                                  _stream(stream))
    _check("ap_iterate_batched", st)
    return [o.as_dict() for o in out], dec


def pap_run(S, k, part_offsets=None, damping=0.5, max_iter=200, conv_iter=15, check_every=0,
            R=None, A=None, carry_r=False, stream=None):
    """Algorithm 2 on S (n x n).  Returns (R, A, idx, result dict)."""
    _dev_f32(S, "S")
    n = S.shape[0]
    R = empty_square(n, S.device) if R is None else R
    A = empty_square(n, S.device) if A is None else A
    idx = torch.empty(n, dtype=torch.int32, device=S.device)
    part = _i64_array(part_offsets) if part_offsets is not None else None
    partp = C.cast(part, C.c_void_p) if part is not None else None
    p = ApParams(float(damping), int(max_iter), int(conv_iter), int(check_every),
                 AP_FLAG_PAP_CARRY_R if carry_r else 0)
    res = PapResult()
    ws = workspace(lib().pap_run_workspace_size(n, S.stride(0), int(k), partp), S.device)
    st = lib().pap_run(C.c_void_p(S.data_ptr()), n, S.stride(0), int(k), partp, C.byref(p),
                       C.c_void_p(R.data_ptr()), C.c_void_p(A.data_ptr()),
                       C.c_void_p(idx.data_ptr()), C.byref(res), C.c_void_p(ws.data_ptr()),
                       ws.numel(), _stream(stream))
    _check("pap_run", st)
    return R, A, idx, res.as_dict()


def lap_run(X, n_landmarks, mode="uniform", score=None, landmarks=None, seed=0, precision="fp32",
            damping=0.5, max_iter=200, conv_iter=15, check_every=0, stream=None):
    """Algorithm 3 Steps 1-2 on features X (n x d).  Returns (idx, landmarks,
    result dict)."""
    _dev_f32(X, "X")
    n, d = X.shape
    L = int(n_landmarks)
    m = {"uniform": AP_LANDMARK_UNIFORM, "score": AP_LANDMARK_SCORE, "given": AP_LANDMARK_GIVEN}[mode]
    sc = None
    if m == AP_LANDMARK_SCORE:
        sc = score.to(device=X.device, dtype=torch.float32).contiguous()
    lm_in = None
    if m == AP_LANDMARK_GIVEN:
        lm_in = landmarks.to(device=X.device, dtype=torch.int32).contiguous()
    idx = torch.empty(n, dtype=torch.int32, device=X.device)
    lm = torch.empty(L, dtype=torch.int32, device=X.device)
    p = ApParams(float(damping), int(max_iter), int(conv_iter), int(check_every), 0)
    res = LapResult()
    ws = workspace(lib().lap_run_workspace_size(n, d, L), X.device)
    prec = {"fp32": AP_PREC_FP32, "bf16": AP_PREC_BF16}[precision]
    st = lib().lap_run(C.c_void_p(X.data_ptr()), n, d, X.stride(0), L, m,
                       C.c_void_p(sc.data_ptr()) if sc is not None else None,
                       C.c_void_p(lm_in.data_ptr()) if lm_in is not None else None,
                       int(seed) & 0xFFFFFFFFFFFFFFFF, prec, C.byref(p),
                       C.c_void_p(idx.data_ptr()), C.c_void_p(lm.data_ptr()), C.byref(res),
                       C.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream))
    _check("lap_run", st)
    return idx, lm, res.as_dict()


def lap_assign(X, centres, best=False, stream=None):
    """Algorithm 3 Step 2 alone: every point's nearest centre (point indices
    ``centres``).  Returns idx (int32, n) and, with ``best``, the maximum
    score 2 x.e - |e|^2 of every point on the centred bf16 features."""
    _dev_f32(X, "X")
    n, d = X.shape
    cen = centres.to(device=X.device, dtype=torch.int32).contiguous()
    c = cen.numel()
    idx = torch.empty(n, dtype=torch.int32, device=X.device)
    bst = torch.empty(n, dtype=torch.float32, device=X.device) if best else None
    ws = workspace(lib().lap_assign_workspace_size(n, d, c), X.device)
    st = lib().lap_assign(_ptr(X), n, d, X.stride(0), _ptr(cen), c, _ptr(idx), _ptr(bst), _ptr(ws),
                          ws.numel(), _stream(stream))
    _check("lap_assign", st)
    return (idx, bst) if best else idx


def lap_refine(X, centres, pref, rounds=8, stream=None):
    """Algorithm 3 Step 4 alone on the centre set ``centres`` (point
    indices): returns (refined centres, ascending; idx; result dict)."""
    _dev_f32(X, "X")
    n, d = X.shape
    cen = centres.to(device=X.device, dtype=torch.int32).contiguous()
    c = cen.numel()
    cout = torch.empty(c, dtype=torch.int32, device=X.device)
    idx = torch.empty(n, dtype=torch.int32, device=X.device)
    res = LapRefineResult()
    ws = workspace(lib().lap_refine_workspace_size(n, d, c), X.device)
    st = lib().lap_refine(_ptr(X), n, d, X.stride(0), _ptr(cen), c, float(pref), int(rounds), _ptr(cout),
                          _ptr(idx), C.byref(res), _ptr(ws), ws.numel(), _stream(stream))
    _check("lap_refine", st)
    return cout[:res.n_exemplars], idx, res.as_dict()


def lap_run_full(X, n_landmarks, m0, seed=0, precision="fp32", damping=0.5, max_iter=200,
                 conv_iter=15, max_levels=AP_LAP_MAX_LEVELS, refine_rounds=0, check_every=0,
                 stream=None):
    """Algorithm 3 Steps 1-4 on features X (n x d); ``refine_rounds`` > 0
    refines the merged centres in Step 4.  Returns (idx, level_of, result
    dict)."""
    _dev_f32(X, "X")
    n, d = X.shape
    idx = torch.empty(n, dtype=torch.int32, device=X.device)
    level_of = torch.empty(n, dtype=torch.int32, device=X.device)
    p = ApParams(float(damping), int(max_iter), int(conv_iter), int(check_every), 0)
    res = LapFullResult()
    ws = workspace(lib().lap_run_full_workspace_size(n, d, int(n_landmarks), int(m0), int(max_levels)),
                   X.device)
    prec = {"fp32": AP_PREC_FP32, "bf16": AP_PREC_BF16}[precision]
    st = lib().lap_run_full(_ptr(X), n, d, X.stride(0), int(n_landmarks), int(m0),
                            int(seed) & 0xFFFFFFFFFFFFFFFF, prec, C.byref(p), int(max_levels),
                            int(refine_rounds), _ptr(idx),
                            _ptr(level_of), C.byref(res), _ptr(ws), ws.numel(), _stream(stream))
    _check("lap_run_full", st)
    return idx, level_of, res.as_dict()


def ap_sweep_get_config(n):
    c = ApSweepConfig()
    _check("ap_sweep_get_config", lib().ap_sweep_get_config(int(n), C.byref(c)), ok=(AP_OK,))
    return c.as_dict()


def ap_sweep_set_config(n, cluster=None, ept=None, stages=None):
    """Pins (cluster, ept, stages) for n; with no arguments, unpins."""
    if cluster is None:
        st = lib().ap_sweep_set_config(int(n), None)
    else:
        c = ApSweepConfig(int(cluster), int(ept), int(stages), 0, 0, 0, 0.0, 0)
        st = lib().ap_sweep_set_config(int(n), C.byref(c))
    _check("ap_sweep_set_config", st, ok=(AP_OK,))


def ap_sweep_plan(n, cluster, resident):
    """The sweep's work list for problems of sizes n, all running, with clusters
    of `cluster` CTAs of which `resident` fit at once (host only).  Returns
    (units as a list of (problem, slot, first, count, stride), ubeg list)."""
    n_a = _i64_array(n)
    cap = int(resident) + len(n)
    units = (C.c_int32 * (5 * cap))()
    ubeg = (C.c_int32 * (int(resident) + 1))()
    nu, nc = C.c_int32(0), C.c_int32(0)
    _check("ap_sweep_plan", lib().ap_sweep_plan(C.cast(n_a, C.c_void_p), len(n), int(cluster),
                                                int(resident), C.cast(units, C.c_void_p), cap,
                                                C.cast(ubeg, C.c_void_p), C.byref(nu), C.byref(nc)),
           ok=(AP_OK,))
    us = [tuple(units[5 * u:5 * u + 5]) for u in range(nu.value)]
    return us, list(ubeg[:nc.value + 1])


def ap_sweep_classes(n):
    """The size class of every problem of a batch (host only)."""
    n_a = _i64_array(n)
    out = (C.c_int32 * len(n))()
    k = lib().ap_sweep_classes(C.cast(n_a, C.c_void_p), len(n), C.cast(out, C.c_void_p))
    _check("ap_sweep_classes", min(k, 0), ok=(AP_OK,))
    return list(out)


def ap_sweep_autotune(S, R=None, A=None, damping=0.9, iters=5, stream=None):
    """Times every admissible sweep configuration on S (R, A are scratch),
    pins the fastest for this n and returns it."""
    _dev_f32(S, "S")
    n = S.shape[0]
    R = empty_square(n, S.device, 0.0) if R is None else R
    A = empty_square(n, S.device, 0.0) if A is None else A
    ws = workspace(lib().ap_sweep_autotune_workspace_size(n, S.stride(0)), S.device)
    best = ApSweepConfig()
    st = lib().ap_sweep_autotune(C.c_void_p(S.data_ptr()), C.c_void_p(R.data_ptr()),
                                 C.c_void_p(A.data_ptr()), n, S.stride(0), float(damping),
                                 int(iters), C.byref(best), C.c_void_p(ws.data_ptr()),
                                 ws.numel(), _stream(stream))
    _check("ap_sweep_autotune", st, ok=(AP_OK,))
    return best.as_dict()


def ap_exemplars(S, R, A, stream=None):
    """Labels idx (int32, -1 without exemplars) and dpsim/expref/netsim."""
    for t, nm in ((S, "S"), (R, "R"), (A, "A")):
        _dev_f32(t, nm)
    n = S.shape[0]
    idx = torch.empty(n, dtype=torch.int32, device=S.device)
    res = ApResult()
    ws = workspace(lib().ap_exemplars_workspace_size(n), S.device)
    st = lib().ap_exemplars(C.c_void_p(S.data_ptr()), C.c_void_p(R.data_ptr()),
                            C.c_void_p(A.data_ptr()), n, S.stride(0),
                            C.c_void_p(idx.data_ptr()), C.byref(res),
                            C.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream))
    _check("ap_exemplars", st)
    return idx, res.as_dict()


def ap_exemplars_noalloc(S, R, A, idx=None, stream=None):
    """ap_exemplars without a workspace: the library's built-in scratch array
    is used instead (n <= AP_NOALLOC_MAX_N), so no device memory is
    allocated by the call.  ``idx`` (int32, n) may be passed preallocated."""
    for t, nm in ((S, "S"), (R, "R"), (A, "A")):
        _dev_f32(t, nm)
    n = S.shape[0]
    if idx is None:
        idx = torch.empty(n, dtype=torch.int32, device=S.device)
    res = ApResult()
    st = lib().ap_exemplars_noalloc(C.c_void_p(S.data_ptr()), C.c_void_p(R.data_ptr()),
                                    C.c_void_p(A.data_ptr()), n, S.stride(0),
                                    C.c_void_p(idx.data_ptr()), C.byref(res), _stream(stream))
    _check("ap_exemplars_noalloc", st)
    return idx, res.as_dict()


# ---- learned warm start ----------------------------------------------------------

def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def apl_param_count():
    return int(lib().apl_param_count())


APL_IN = 25


def apl_features(S, scale, stream=None):
    """The APL_IN per-point features of S (n x 25 float32)."""
    _dev_f32(S, "S")
    n = S.shape[0]
    F = torch.empty((n, APL_IN), dtype=torch.float32, device=S.device)
    ws = workspace(lib().apl_features_workspace_size(n), S.device)
    _check("apl_features", lib().apl_features(_ptr(S), n, S.stride(0), float(scale), _ptr(F),
                                              _ptr(ws), ws.numel(), _stream(stream)), ok=(AP_OK,))
    return F


def apl_targets(R, A, decisions, scale, stream=None):
    n = R.shape[0]
    T = torch.empty((n, 3), dtype=torch.float32, device=R.device)
    _check("apl_targets", lib().apl_targets(_ptr(R), _ptr(A), _ptr(decisions), n, R.stride(0),
                                            float(scale), _ptr(T), _stream(stream)), ok=(AP_OK,))
    return T


def apl_sync_bf16(P, P16, stream=None):
    _check("apl_sync_bf16", lib().apl_sync_bf16(_ptr(P), _ptr(P16), _stream(stream)), ok=(AP_OK,))


def apl_forward(P, P16, F, stream=None):
    rows = F.shape[0]
    Y = torch.empty((rows, 3), dtype=torch.float32, device=F.device)
    ws = workspace(lib().apl_workspace_size(rows), F.device)
    _check("apl_forward", lib().apl_forward(_ptr(P), _ptr(P16), _ptr(F), rows, _ptr(Y),
                                            _ptr(ws), ws.numel(), _stream(stream)), ok=(AP_OK,))
    return Y


def apl_train_step(P, P16, M, V, step, lr, F, T, ws=None, want_grad=False, stream=None):
    """One Adam step in place on (P, P16, M, V).  Returns (loss tensor, grad or None)."""
    rows = F.shape[0]
    if ws is None:
        ws = workspace(lib().apl_workspace_size(rows), F.device)
    loss = torch.empty(1, dtype=torch.float32, device=F.device)
    grad = torch.empty(apl_param_count(), dtype=torch.float32, device=F.device) if want_grad else None
    _check("apl_train_step", lib().apl_train_step(_ptr(P), _ptr(P16), _ptr(M), _ptr(V), int(step),
                                                  float(lr), _ptr(F), _ptr(T), rows, _ptr(loss),
                                                  _ptr(grad), _ptr(ws), ws.numel(),
                                                  _stream(stream)), ok=(AP_OK,))
    return loss, grad


def apl_warm_start(Y, scale, R, A, stream=None):
    n = Y.shape[0]
    _check("apl_warm_start", lib().apl_warm_start(_ptr(Y), n, float(scale), _ptr(R), _ptr(A),
                                                  R.stride(0), _stream(stream)), ok=(AP_OK,))


def apl_ap_run(S, P, P16, scale, damping=0.9, max_iter=1000, conv_iter=15, judge=True,
               check_every=0, stream=None):
    """Warm-started Algorithm 1 (judged by the cold start).  Returns
    (R, A, idx, result dict)."""
    _dev_f32(S, "S")
    n = S.shape[0]
    R = empty_square(n, S.device)
    A = empty_square(n, S.device)
    idx = torch.empty(n, dtype=torch.int32, device=S.device)
    p = ApParams(float(damping), int(max_iter), int(conv_iter), int(check_every), 0)
    res = AplResult()
    ws = workspace(lib().apl_ap_run_workspace_size(n, S.stride(0)), S.device)
    st = lib().apl_ap_run(_ptr(S), n, S.stride(0), _ptr(P), _ptr(P16), float(scale), C.byref(p),
                          1 if judge else 0, _ptr(R), _ptr(A), _ptr(idx), C.byref(res), _ptr(ws),
                          ws.numel(), _stream(stream))
    _check("apl_ap_run", st)
    return R, A, idx, res.as_dict()


def ap_wait_selftest(spin_limit=1 << 16, stream=None):
    """Status of the library's bounded-wait self-test (AP_ERR_TIMEOUT expected)."""
    return int(lib().ap_wait_selftest(int(spin_limit), _stream(stream)))


def apl_warm_start_batched_workspace(n, device):
    """A workspace for apl_warm_start_batched on problems of sizes n."""
    return workspace(lib().apl_warm_start_batched_workspace_size(_i64_array(n), len(n)), device)


def apl_warm_start_batched(S, R, A, offsets, n, ld, scale, P, P16, Y=None, ws=None, stream=None):
    """Features, forward pass and column-constant warm start of every problem
    of 1-D arenas (S, R, A) in one call; ``scale`` one float per problem."""
    count = len(n)
    sc = (C.c_float * count)(*[float(x) for x in scale])
    if ws is None:
        ws = apl_warm_start_batched_workspace(n, S.device)
    _check("apl_warm_start_batched",
           lib().apl_warm_start_batched(_ptr(S), _ptr(R), _ptr(A), _i64_array(offsets), _i64_array(n),
                                        _i64_array(ld), count, sc, _ptr(P), _ptr(P16), _ptr(Y),
                                        _ptr(ws), ws.numel(), _stream(stream)))
    return R, A


def apl_set_standardisation(P, F, stream=None):
    """Writes the input standardisation of features F (rows x 25) into P."""
    _check("apl_set_standardisation",
           lib().apl_set_standardisation(_ptr(P), _ptr(F.contiguous()), F.shape[0], _stream(stream)))


def apl_judge(cold_netsim, warm_netsim, tol=0.005):
    """Per problem: True when the warm net similarity is within ``tol`` of the
    cold one (the library's judge)."""
    count = len(cold_netsim)
    c = (C.c_double * count)(*[float(x) for x in cold_netsim])
    w = (C.c_double * count)(*[float(x) for x in warm_netsim])
    out = (C.c_int32 * count)()
    k = lib().apl_judge(c, w, count, float(tol), out)
    if k < 0:
        raise ApgbError("apl_judge", k)
    return [bool(x) for x in out]
