"""Python binding of the GB300 library for exhaustive Gaussian-copula
higher-order information (arXiv 2501.03381).

The binding only marshals arguments: every step of the computation runs in
the CUDA library ``_lib/libthoi.so`` (C ABI in ``include/thoi.h``).  There is
no CPU fallback; if the library cannot be loaded the functions raise.  PyTorch
provides device memory and the current CUDA stream.

Module-level functions carry the C names (``thoi_create``, ``thoi_measures``,
...).  ``Context`` wraps them for convenience, and ``MeasureSum`` is a
``torch.autograd.Function`` whose backward is the library's adjoint.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "_lib", "libthoi.so")
_HEADER = os.path.join(os.path.dirname(_PKG), "include", "thoi.h")
_lock = threading.Lock()
_lib = None

MEASURES = ("H", "TC", "DTC", "O", "S")
THOI_F32_FIX64, THOI_F64 = 0, 1
THOI_RED_NONE, THOI_RED_PER_ORDER = 0, 1
THOI_DTYPE_F32, THOI_DTYPE_F64 = 0, 1
THOI_SIGMA32_TENSORCORE, THOI_SIGMA32_FROM_F64 = 0, 1
RECORDS_MODES = ("auto", "fused", "stored")  # thoi_records_mode
GROUP_OBJECTIVES = ("mean", "cohen_d")  # thoi_group_objective
STATUS = {0: "THOI_OK", 1: "THOI_ERR_INVALID_ARG", 2: "THOI_ERR_NONFINITE_INPUT",
          3: "THOI_ERR_TOO_LARGE", 4: "THOI_ERR_NOT_PD", 5: "THOI_ERR_OOM", 6: "THOI_ERR_CUDA",
          7: "THOI_ERR_TIMEOUT", 8: "THOI_ERR_CANCELLED", 9: "THOI_ERR_WORKSPACE"}


class ThoiError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        self.name = STATUS.get(code, str(code))
        super().__init__(f"{what}: {self.name} ({_status_string(code)})")


class thoi_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("pivot_tau", ctypes.c_float),
                ("trace_tau", ctypes.c_float), ("bias_correct", ctypes.c_int32),
                ("top_m", ctypes.c_int32), ("out_f64", ctypes.c_int32),
                ("sigma32_source", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("flag_capacity", ctypes.c_uint64), ("profile", ctypes.c_int32),
                ("records_mode", ctypes.c_int32)]


class thoi_stats(ctypes.Structure):
    _fields_ = [("nplets", ctypes.c_uint64), ("n_refactored", ctypes.c_uint64),
                ("n_not_pd", ctypes.c_uint64), ("launches", ctypes.c_int32),
                ("nplet_launches", ctypes.c_int32), ("nplet_ms", ctypes.c_double),
                ("refactor_ms", ctypes.c_double), ("merge_ms", ctypes.c_double),
                ("reduce_ms", ctypes.c_double), ("fused_retries", ctypes.c_int32),
                ("pad2", ctypes.c_int32), ("n_candidates", ctypes.c_uint64)]


RECORD_DTYPE = np.dtype([("k", "<i4"), ("top_count", "<i4"), ("count", "<u8"),
                         ("count_neg_O", "<u8"), ("n_refactored", "<u8"), ("n_not_pd", "<u8"),
                         ("min", "<f8", (5,)), ("max", "<f8", (5,)), ("mean", "<f8", (5,)),
                         ("argmin", "<u8", (5,)), ("argmax", "<u8", (5,))])
TOP_DTYPE = np.dtype([("value", "<f8"), ("id", "<u8")])
assert RECORD_DTYPE.itemsize == 240 and TOP_DTYPE.itemsize == 16


def library_path() -> str:
    return _LIB_PATH


def load(build_if_missing: bool = True):
    """Load libthoi.so (building it with nvcc if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            if not build_if_missing:
                raise OSError(f"{_LIB_PATH} not built")
            from . import _build
            _build.build()
        lib = ctypes.CDLL(_LIB_PATH)
        vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        sig = {
            "thoi_default_options": (None, [ctypes.POINTER(thoi_options)]),
            "thoi_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "thoi_create": (ctypes.c_int, [ctypes.POINTER(vp), vp, i64, i64, i64, i32,
                                           ctypes.POINTER(thoi_options), vp]),
            "thoi_create_from_cov": (ctypes.c_int, [ctypes.POINTER(vp), vp, i64, i64,
                                                    ctypes.POINTER(thoi_options), vp]),
            "thoi_get_cov": (ctypes.c_int, [vp, vp, vp, vp]),
            "thoi_get_ranks": (ctypes.c_int, [vp, vp, vp]),
            "thoi_n": (i64, [vp]),
            "thoi_count": (u64, [i64, vp, i32]),
            "thoi_unrank": (ctypes.c_int, [i64, vp, i32, u64, vp, vp]),
            "thoi_unrank_device": (ctypes.c_int, [i64, vp, i32, vp, i64, i32, vp, vp]),
            "thoi_records_bytes": (ctypes.c_size_t, [i32, i32]),
            "thoi_measures": (ctypes.c_int, [vp, vp, i32, u64, u64, i32, vp, ctypes.c_size_t,
                                             ctypes.POINTER(thoi_stats), vp]),
            "thoi_measures_grad": (ctypes.c_int, [vp, vp, i32, i32, vp,
                                                  ctypes.POINTER(thoi_stats), vp]),
            "thoi_batch_measures": (ctypes.c_int, [vp, i32, i32, i32, vp, ctypes.c_size_t,
                                                   ctypes.POINTER(thoi_stats), vp]),
            "thoi_autotune": (ctypes.c_int, [vp, i32, i32, ctypes.c_char_p, vp]),
            "thoi_set_cancel": (ctypes.c_int, [vp, i32]),
            "thoi_order_record_noalloc": (ctypes.c_int, [vp, i64, i32, i32, vp, vp, vp]),
            "thoi_partition": (ctypes.c_int, [i64, vp, i32, i32, vp]),
            "thoi_greedy": (ctypes.c_int, [vp, i32, i32, i32, i32, i32, vp, vp,
                                           ctypes.POINTER(thoi_stats), vp]),
            "thoi_merge_records": (ctypes.c_int, [vp, i32, i32, i32, vp]),
            "thoi_anneal": (ctypes.c_int, [vp, i32, i32, i32, i32, ctypes.c_double,
                                           ctypes.c_double, i32, i32, i32, u64, vp, vp, vp, vp,
                                           ctypes.POINTER(thoi_stats), vp]),
            "thoi_group_measures": (ctypes.c_int, [vp, i32, vp, i32, u64, u64, i32, i32, i32,
                                                   vp, ctypes.c_size_t,
                                                   ctypes.POINTER(thoi_stats), vp]),
            "thoi_group_greedy": (ctypes.c_int, [vp, i32, i32, i32, i32, i32, i32, i32, vp, vp,
                                                 ctypes.POINTER(thoi_stats), vp]),
            "thoi_group_anneal": (ctypes.c_int, [vp, i32, i32, i32, i32, i32, ctypes.c_double,
                                                 ctypes.c_double, i32, i32, i32, i32, u64, vp,
                                                 vp, vp, vp, ctypes.POINTER(thoi_stats), vp]),
            "thoi_fma_peak": (ctypes.c_int, [i32, i32, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double), vp]),
            "thoi_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def header_symbols() -> list:
    """Entry points declared in include/thoi.h."""
    with open(_HEADER) as fh:
        txt = fh.read()
    return sorted(set(re.findall(r"^\s*[\w\s\*]*?\b(thoi_\w+)\s*\(", txt, flags=re.M)))


def _status_string(code: int) -> str:
    try:
        return load().thoi_status_string(code).decode()
    except Exception:
        return STATUS.get(code, "?")


def _check(code: int, what: str):
    if code != 0:
        raise ThoiError(code, what)


def _stream_ptr(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _orders_arr(orders) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(list(orders), dtype=np.int32))


def _ptr(x):
    """Raw pointer of a torch tensor or numpy array."""
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(x.data_ptr())


def make_options(precision: str | int = "f32_fix64", pivot_tau: float | None = None,
                 trace_tau: float | None = None, bias_correct: bool = False,
                 top_m: int | None = None, out_f64: bool | None = None,
                 sigma32_source: str | int = "from_f64", autotune: bool = True,
                 flag_capacity: int = 0, profile: bool = False,
                 records_mode: str | int = "auto") -> thoi_options:
    o = thoi_options()
    load().thoi_default_options(ctypes.byref(o))
    if isinstance(precision, str):
        precision = {"f32_fix64": THOI_F32_FIX64, "f64": THOI_F64}[precision]
    o.precision = precision
    if pivot_tau is not None:
        o.pivot_tau = pivot_tau
    if trace_tau is not None:
        o.trace_tau = trace_tau
    o.bias_correct = int(bool(bias_correct))
    if top_m is not None:
        o.top_m = top_m
    if out_f64 is not None:
        o.out_f64 = int(bool(out_f64))
    if isinstance(sigma32_source, str):
        sigma32_source = {"tensorcore": THOI_SIGMA32_TENSORCORE,
                          "from_f64": THOI_SIGMA32_FROM_F64}[sigma32_source]
    o.sigma32_source = sigma32_source
    o.autotune = int(bool(autotune))
    o.flag_capacity = flag_capacity
    o.profile = int(bool(profile))
    o.records_mode = (records_mode if isinstance(records_mode, int)
                      else RECORDS_MODES.index(records_mode))
    return o


# --------------------------------------------------------------------- C-named wrappers
def thoi_count(N: int, orders) -> int:
    o = _orders_arr(orders)
    return int(load().thoi_count(N, _ptr(o), len(o)))


def thoi_partition(N: int, orders, R: int) -> np.ndarray:
    """R + 1 id bounds splitting the request into ranges of equal work."""
    o = _orders_arr(orders)
    b = np.zeros(R + 1, dtype=np.uint64)
    _check(load().thoi_partition(N, _ptr(o), len(o), R, _ptr(b)), "thoi_partition")
    return b


def thoi_merge_records(blocks, n_orders: int, top_m: int) -> np.ndarray:
    """Merge per-order record blocks of disjoint id ranges (host bytes, one
    block per range, each thoi_records_bytes(n_orders, top_m) long)."""
    per = thoi_records_bytes(n_orders, top_m)
    raw = np.ascontiguousarray(np.concatenate([np.asarray(b).view(np.uint8).ravel()
                                               for b in blocks]))
    R = len(blocks)
    if raw.nbytes != R * per:
        raise ValueError("record blocks have the wrong size")
    out = np.zeros(per, dtype=np.uint8)
    _check(load().thoi_merge_records(_ptr(raw), R, n_orders, top_m, _ptr(out)),
           "thoi_merge_records")
    return out


def thoi_unrank(N: int, orders, gid: int):
    o = _orders_arr(orders)
    idx = np.zeros(64, dtype=np.int32)
    k = ctypes.c_int32()
    _check(load().thoi_unrank(N, _ptr(o), len(o), gid, _ptr(idx), ctypes.byref(k)), "thoi_unrank")
    return idx[:k.value].copy()


def thoi_unrank_device(N: int, orders, ids, kmax: int | None = None, stream=None):
    """Subsets of global ids computed by the device unranking (int8 rows, -1 padded)."""
    import torch
    o = _orders_arr(orders)
    kmax = int(kmax or max(o))
    ids_t = torch.as_tensor(np.asarray(ids, dtype=np.int64), device="cuda")
    out = torch.empty((len(ids_t), kmax), dtype=torch.int8, device="cuda")
    _check(load().thoi_unrank_device(N, _ptr(o), len(o), _ptr(ids_t), len(ids_t), kmax, _ptr(out),
                                     _stream_ptr(stream)), "thoi_unrank_device")
    return out


def thoi_records_bytes(n_orders: int, top_m: int) -> int:
    return int(load().thoi_records_bytes(n_orders, top_m))


def thoi_create(X, options: thoi_options | None = None, stream=None):
    """Create a context from a T x N sample matrix (torch tensor on the GPU or
    the host, or a numpy array), float32 or float64, row-major."""
    import torch
    if isinstance(X, np.ndarray):
        if X.dtype not in (np.float32, np.float64):
            X = X.astype(np.float64)
        X = np.ascontiguousarray(X)
        dtype = THOI_DTYPE_F64 if X.dtype == np.float64 else THOI_DTYPE_F32
        T, N = X.shape
        ld = X.strides[0] // X.itemsize
        keep = X
    else:
        if X.dtype not in (torch.float32, torch.float64):
            X = X.double()
        if X.stride(1) != 1:
            X = X.contiguous()
        dtype = THOI_DTYPE_F64 if X.dtype == torch.float64 else THOI_DTYPE_F32
        T, N = X.shape
        ld = X.stride(0)
        keep = X
    h = ctypes.c_void_p()
    opt = options if options is not None else make_options()
    _check(load().thoi_create(ctypes.byref(h), _ptr(keep), T, N, ld, dtype, ctypes.byref(opt),
                              _stream_ptr(stream)), "thoi_create")
    return h


def thoi_create_from_cov(Sigma, T_for_bias: int = 0, options: thoi_options | None = None,
                         stream=None):
    import torch
    if isinstance(Sigma, np.ndarray):
        S = np.ascontiguousarray(Sigma, dtype=np.float64)
    else:
        S = Sigma.detach().to(torch.float64).contiguous()
    h = ctypes.c_void_p()
    opt = options if options is not None else make_options()
    _check(load().thoi_create_from_cov(ctypes.byref(h), _ptr(S), S.shape[0], T_for_bias,
                                       ctypes.byref(opt), _stream_ptr(stream)),
           "thoi_create_from_cov")
    return h


def thoi_destroy(h):
    if h:
        load().thoi_destroy(h)


def thoi_n(h) -> int:
    return int(load().thoi_n(h))


def thoi_get_cov(h, stream=None):
    N = thoi_n(h)
    S64 = np.empty((N, N))
    S32 = np.empty((N, N), dtype=np.float32)
    _check(load().thoi_get_cov(h, _ptr(S64), _ptr(S32), _stream_ptr(stream)), "thoi_get_cov")
    return S64, S32


def thoi_get_ranks(h, T: int, stream=None):
    N = thoi_n(h)
    R = np.empty((T, N), dtype=np.int32)
    _check(load().thoi_get_ranks(h, _ptr(R), _stream_ptr(stream)), "thoi_get_ranks")
    return R


def thoi_measures(h, orders, id_begin: int = 0, id_end: int | None = None, kind: int = 0,
                  out=None, out_f64: bool = False, top_m: int = 256, stream=None):
    """Per-nplet SoA (kind 0: returns a 5 x n CUDA tensor) or per-order
    records (kind 1: returns (records, top_hi, top_lo) numpy arrays).
    `out` may be given (device tensor for kind 0; device tensor or host
    numpy uint8 buffer for kind 1)."""
    import torch
    o = _orders_arr(orders)
    N = thoi_n(h)
    total = thoi_count(N, o)
    end = total if id_end is None else int(id_end)
    st = thoi_stats()
    if kind == THOI_RED_NONE:
        n = end - id_begin
        if out is None:
            out = torch.empty((5, max(n, 0)), dtype=torch.float64 if out_f64 else torch.float32,
                              device="cuda")
        nbytes = out.numel() * out.element_size()
        _check(load().thoi_measures(h, _ptr(o), len(o), id_begin, end, kind, _ptr(out), nbytes,
                                    ctypes.byref(st), _stream_ptr(stream)), "thoi_measures")
        return out, st
    nbytes = thoi_records_bytes(len(o), top_m)
    if out is None:
        out = np.zeros(nbytes, dtype=np.uint8)
    n_out = out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size()
    _check(load().thoi_measures(h, _ptr(o), len(o), id_begin, end, kind, _ptr(out), n_out,
                                ctypes.byref(st), _stream_ptr(stream)), "thoi_measures")
    return parse_records(out, len(o), top_m), st


def parse_records(buf, n_orders: int, top_m: int):
    """(records, top_hi, top_lo) from a record buffer (numpy or torch)."""
    if not isinstance(buf, np.ndarray):
        buf = buf.detach().cpu().numpy()
    raw = np.ascontiguousarray(buf).view(np.uint8)
    nb = n_orders * RECORD_DTYPE.itemsize
    recs = raw[:nb].view(RECORD_DTYPE)
    tops = raw[nb:nb + n_orders * 2 * top_m * TOP_DTYPE.itemsize].view(TOP_DTYPE)
    tops = tops.reshape(n_orders, 2, top_m) if top_m > 0 else tops.reshape(n_orders, 2, 0)
    return recs.copy(), tops[:, 0].copy(), tops[:, 1].copy()


def thoi_measures_grad(h, orders, measure: str = "O", out=None, stream=None):
    import torch
    o = _orders_arr(orders)
    N = thoi_n(h)
    if out is None:
        out = torch.empty((N, N), dtype=torch.float32, device="cuda")
    st = thoi_stats()
    _check(load().thoi_measures_grad(h, _ptr(o), len(o), MEASURES.index(measure), _ptr(out),
                                     ctypes.byref(st), _stream_ptr(stream)), "thoi_measures_grad")
    return out, st


def thoi_batch_measures(handles, kmin: int, kmax: int, top_m: int = 256, out=None, stream=None):
    D = len(handles)
    arr = (ctypes.c_void_p * D)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    per = thoi_records_bytes(kmax - kmin + 1, top_m)
    if out is None:
        out = np.zeros(per * D, dtype=np.uint8)
    n_out = out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size()
    st = thoi_stats()
    _check(load().thoi_batch_measures(ctypes.cast(arr, ctypes.c_void_p), D, kmin, kmax, _ptr(out),
                                      n_out, ctypes.byref(st), _stream_ptr(stream)),
           "thoi_batch_measures")
    if not isinstance(out, np.ndarray):
        out = out.detach().cpu().numpy()
    res = [parse_records(out[d * per:(d + 1) * per], kmax - kmin + 1, top_m) for d in range(D)]
    return res, st


def thoi_greedy(h, k0: int, k1: int, kappa: int, measure: str = "O", maximize: bool = True,
                stream=None):
    """Greedy search from the exhaustive top-kappa of order k0 up to order k1.
    Returns (masks uint64[k1-k0+1, kappa], values float64[k1-k0+1, kappa],
    stats); row k-k0 holds the selected sets of order k, best first."""
    L = k1 - k0 + 1
    masks = np.zeros((L, kappa), dtype=np.uint64)
    values = np.zeros((L, kappa), dtype=np.float64)
    st = thoi_stats()
    _check(load().thoi_greedy(h, k0, k1, kappa, MEASURES.index(measure), int(bool(maximize)),
                              _ptr(masks), _ptr(values), ctypes.byref(st), _stream_ptr(stream)),
           "thoi_greedy")
    return masks, values, st


def thoi_anneal(h, k_lo: int, k_hi: int, n_chains: int, iters: int, T0: float, alpha: float,
                measure: str = "O", maximize: bool = True, seed: int = 0, stream=None,
                patience: int = 0):
    """Simulated annealing chains on the device (patience > 0: a chain also
    stops after `patience` steps without a better set).  Returns
    (final_masks, final_values, best_masks, best_values, stats), n_chains
    entries each."""
    fm = np.zeros(n_chains, dtype=np.uint64)
    fv = np.zeros(n_chains, dtype=np.float64)
    bm = np.zeros(n_chains, dtype=np.uint64)
    bv = np.zeros(n_chains, dtype=np.float64)
    st = thoi_stats()
    _check(load().thoi_anneal(h, k_lo, k_hi, n_chains, iters, T0, alpha, patience,
                              MEASURES.index(measure), int(bool(maximize)), seed & ((1 << 64) - 1), _ptr(fm), _ptr(fv),
                              _ptr(bm), _ptr(bv), ctypes.byref(st), _stream_ptr(stream)),
           "thoi_anneal")
    return fm, fv, bm, bv, st


def _handles(handles):
    hs = [getattr(h, "h", h) for h in handles]
    return (ctypes.c_void_p * len(hs))(*hs), len(hs)


def _objective(objective) -> int:
    return objective if isinstance(objective, int) else GROUP_OBJECTIVES.index(objective)


def thoi_group_measures(handles, orders, measure: str = "O", objective="mean",
                        id_begin: int = 0, id_end: int | None = None, kind: int = 0, out=None,
                        top_m: int = 256, stream=None):
    """Group objective of one measure over the datasets of `handles` (raw
    handles or Contexts, the same N).  kind 0: a float64 CUDA tensor with the
    objective of every nplet in [id_begin, id_end); kind 1: per-order records
    (records, top_hi, top_lo) with top_m = the first context's."""
    import torch
    arr, D = _handles(handles)
    o = _orders_arr(orders)
    N = thoi_n(arr[0])
    end = thoi_count(N, o) if id_end is None else int(id_end)
    st = thoi_stats()
    if kind == THOI_RED_NONE:
        if out is None:
            out = torch.empty(max(end - id_begin, 0), dtype=torch.float64, device="cuda")
        nbytes = out.numel() * out.element_size()
    else:
        if out is None:
            out = np.zeros(thoi_records_bytes(len(o), top_m), dtype=np.uint8)
        nbytes = out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size()
    _check(load().thoi_group_measures(arr, D, _ptr(o), len(o), id_begin, end,
                                      MEASURES.index(measure), _objective(objective), kind,
                                      _ptr(out), nbytes, ctypes.byref(st), _stream_ptr(stream)),
           "thoi_group_measures")
    if kind == THOI_RED_NONE:
        return out, st
    return parse_records(out, len(o), top_m), st


def thoi_group_greedy(handles, k0: int, k1: int, kappa: int, measure: str = "O",
                      objective="mean", maximize: bool = True, stream=None):
    """Greedy search on a group objective; outputs as thoi_greedy."""
    arr, D = _handles(handles)
    L = k1 - k0 + 1
    masks = np.zeros((L, kappa), dtype=np.uint64)
    values = np.zeros((L, kappa), dtype=np.float64)
    st = thoi_stats()
    _check(load().thoi_group_greedy(arr, D, k0, k1, kappa, MEASURES.index(measure),
                                    _objective(objective), int(bool(maximize)), _ptr(masks),
                                    _ptr(values), ctypes.byref(st), _stream_ptr(stream)),
           "thoi_group_greedy")
    return masks, values, st


def thoi_group_anneal(handles, k_lo: int, k_hi: int, n_chains: int, iters: int, T0: float,
                      alpha: float, measure: str = "O", objective="mean", maximize: bool = True,
                      seed: int = 0, stream=None, patience: int = 0):
    """Simulated annealing on a group objective; outputs as thoi_anneal."""
    arr, D = _handles(handles)
    fm = np.zeros(n_chains, dtype=np.uint64)
    fv = np.zeros(n_chains, dtype=np.float64)
    bm = np.zeros(n_chains, dtype=np.uint64)
    bv = np.zeros(n_chains, dtype=np.float64)
    st = thoi_stats()
    _check(load().thoi_group_anneal(arr, D, k_lo, k_hi, n_chains, iters, T0, alpha, patience,
                                    MEASURES.index(measure), _objective(objective),
                                    int(bool(maximize)), seed & ((1 << 64) - 1), _ptr(fm),
                                    _ptr(fv), _ptr(bm), _ptr(bv), ctypes.byref(st),
                                    _stream_ptr(stream)), "thoi_group_anneal")
    return fm, fv, bm, bv, st


def thoi_autotune(h, kmin: int, kmax: int, cache_path: str | None = None, stream=None):
    _check(load().thoi_autotune(h, kmin, kmax, cache_path.encode() if cache_path else None,
                                _stream_ptr(stream)), "thoi_autotune")


def thoi_fma_peak(fp64: bool = False, iters: int | None = None, stream=None):
    """Measured FFMA (fp64=False) or DFMA (fp64=True) peak of the current
    device in TFLOP/s, and the timed launch's milliseconds."""
    iters = iters or (50 if fp64 else 2000)
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().thoi_fma_peak(int(bool(fp64)), iters, ctypes.byref(t), ctypes.byref(ms),
                                _stream_ptr(stream)), "thoi_fma_peak")
    return t.value, ms.value


def thoi_set_cancel(h, flag: bool):
    _check(load().thoi_set_cancel(h, int(bool(flag))), "thoi_set_cancel")


def thoi_order_record_noalloc(Sigma, k: int, top_m: int = 0, rec_out=None, top_out=None,
                              stream=None):
    """Per-order record of order k from a device covariance, allocating no
    device memory inside the library (for callers that cannot call
    cudaMalloc/cudaFree).  Sigma, rec_out and top_out are CUDA tensors on one
    device (uint8 buffers of at least 240 and 2*top_m*16 bytes when given);
    the call runs with that device current, on `stream` or its current
    stream.  Calls that overlap on the GPU share one scratch array and must
    be serialised."""
    import torch
    S = Sigma if Sigma.dtype == torch.float64 else Sigma.double()
    S = S.contiguous()
    if not S.is_cuda:
        raise ValueError("Sigma must be a CUDA tensor")
    N = S.shape[0]
    with torch.cuda.device(S.device):
        if rec_out is None:
            rec_out = torch.zeros(RECORD_DTYPE.itemsize, dtype=torch.uint8, device=S.device)
        if top_out is None and top_m > 0:
            top_out = torch.zeros(2 * top_m * TOP_DTYPE.itemsize, dtype=torch.uint8,
                                  device=S.device)
        need = [(rec_out, RECORD_DTYPE.itemsize, "rec_out")]
        if top_m > 0:
            need.append((top_out, 2 * top_m * TOP_DTYPE.itemsize, "top_out"))
        for buf, nbytes, name in need:
            if not torch.is_tensor(buf) or buf.device != S.device or not buf.is_contiguous():
                raise ValueError(f"{name} must be a contiguous tensor on {S.device}")
            if buf.numel() * buf.element_size() < nbytes:
                raise ValueError(f"{name} holds fewer than {nbytes} bytes")
        _check(load().thoi_order_record_noalloc(_ptr(S), N, k, top_m, _ptr(rec_out),
                                                _ptr(top_out) if top_m > 0 else None,
                                                _stream_ptr(stream)),
               "thoi_order_record_noalloc")
    rec = rec_out.cpu().numpy().view(np.uint8)[:RECORD_DTYPE.itemsize].view(RECORD_DTYPE)[0].copy()
    tops = (top_out.cpu().numpy().view(np.uint8)[:2 * top_m * TOP_DTYPE.itemsize]
            .view(TOP_DTYPE).reshape(2, top_m).copy() if top_m > 0
            else np.zeros((2, 0), dtype=TOP_DTYPE))
    return rec, tops[0], tops[1]


# --------------------------------------------------------------------- convenience
class Context:
    """Owns one library context (covariance, tables, workspace)."""

    def __init__(self, X=None, *, Sigma=None, T_for_bias: int = 0, stream=None, **options):
        self.opt = make_options(**options)
        if (X is None) == (Sigma is None):
            raise ValueError("give exactly one of X or Sigma")
        if X is not None:
            self.T = X.shape[0]
            self.h = thoi_create(X, self.opt, stream)
        else:
            self.T = T_for_bias
            self.h = thoi_create_from_cov(Sigma, T_for_bias, self.opt, stream)
        self.N = thoi_n(self.h)

    def close(self):
        if getattr(self, "h", None):
            thoi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def cov(self):
        return thoi_get_cov(self.h)

    def ranks(self):
        return thoi_get_ranks(self.h, self.T)

    def measures(self, orders, id_begin=0, id_end=None, reduction="none", out=None, stream=None):
        kind = THOI_RED_PER_ORDER if reduction == "per_order" else THOI_RED_NONE
        return thoi_measures(self.h, orders, id_begin, id_end, kind, out,
                             out_f64=bool(self.opt.out_f64) if self.opt.out_f64 >= 0
                             else self.opt.precision == THOI_F64,
                             top_m=self.opt.top_m, stream=stream)

    def anneal(self, k_lo, k_hi, n_chains, iters, T0, alpha, measure="O", maximize=True, seed=0,
               stream=None, patience=0):
        fm, fv, bm, bv, _ = thoi_anneal(self.h, k_lo, k_hi, n_chains, iters, T0, alpha, measure,
                                        maximize, seed, stream, patience)
        return fm, fv, bm, bv

    def greedy(self, k0, k1, kappa, measure="O", maximize=True, stream=None):
        masks, values, _ = thoi_greedy(self.h, k0, k1, kappa, measure, maximize, stream)
        return masks, values

    def grad(self, orders, measure="O", out=None, stream=None):
        return thoi_measures_grad(self.h, orders, measure, out, stream)


def measures(X, orders, reduction: str = "none", stream=None, **options):
    """One call over a T x N sample matrix (a tensor on the device, or a host
    array): a context is created, evaluated and freed.  Returns what
    Context.measures returns: (SoA tensor, stats) for reduction "none",
    ((records, top_hi, top_lo), stats) for "per_order"."""
    with Context(X, stream=stream, **options) as c:
        return c.measures(orders, reduction=reduction, stream=stream)


def measure_sum(Sigma, orders, measure: str = "O", T_for_bias: int = 0):
    """L = sum over every nplet of the listed orders of one measure, as a
    differentiable function of the covariance Sigma (MeasureSum)."""
    if MeasureSum is None:
        raise RuntimeError("measure_sum needs torch")
    return MeasureSum.apply(Sigma, orders, measure, T_for_bias)


def _measure_total(recs, measure: str) -> float:
    m = MEASURES.index(measure)
    return float(sum(float(r["mean"][m]) * (int(r["count"]) - int(r["n_not_pd"])) for r in recs))


try:
    import torch as _torch

    class MeasureSum(_torch.autograd.Function):
        """L = sum over every nplet of the listed orders of one measure, as a
        differentiable function of the covariance Sigma (N x N CUDA tensor).
        Forward: per-order reductions; backward: the library's adjoint."""

        @staticmethod
        def forward(fctx, Sigma, orders, measure="O", T_for_bias=0):
            c = Context(Sigma=Sigma, T_for_bias=T_for_bias, top_m=0)
            (recs, _, _), _ = c.measures(orders, reduction="per_order")
            fctx.thoi = c
            fctx.orders = list(orders)
            fctx.measure = measure
            return _torch.tensor(_measure_total(recs, measure), dtype=Sigma.dtype,
                                 device=Sigma.device)

        @staticmethod
        def backward(fctx, g):
            G, _ = fctx.thoi.grad(fctx.orders, fctx.measure)
            fctx.thoi.close()
            return g * G.to(g.dtype), None, None, None
except Exception:  # torch missing: the ctypes functions still work with numpy
    MeasureSum = None
