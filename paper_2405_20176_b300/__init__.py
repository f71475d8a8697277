"""Python binding of libsnaps, the sm_103a CUDA hot path of SNAPS population
outlier detection (Gowanlock et al., arXiv 2405.20176).

The functions below carry the C ABI's names (include/snaps.h) and only
marshal arguments: every step of the computation runs in the CUDA library.
There is no CPU fallback -- importing works anywhere, but the first call that
needs the library raises if ``libsnaps.so`` is missing, and the library itself
reports an error when no CUDA device is present.

Arrays may be torch tensors (host or CUDA) or NumPy arrays; outputs are
written in place.  ``stream`` defaults to torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsnaps.so")

SNAPS_OK, SNAPS_EINVAL, SNAPS_ENOMEM, SNAPS_EBUSY, SNAPS_EAGAIN, SNAPS_ETIMEOUT, SNAPS_ECUDA, \
    SNAPS_ECANCELED = range(8)
STATUS_NAMES = ["SNAPS_OK", "SNAPS_EINVAL", "SNAPS_ENOMEM", "SNAPS_EBUSY", "SNAPS_EAGAIN",
                "SNAPS_ETIMEOUT", "SNAPS_ECUDA", "SNAPS_ECANCELED"]
SNAPS_MAX_FEATURES = 15
SNAPS_MAX_K = 32
SNAPS_N_SCORES = 4
SNAPS_SCORE_EPS_COUNT, SNAPS_SCORE_EPS_MEAN, SNAPS_SCORE_KNN_INDEG, SNAPS_SCORE_KNN_MEAN = range(4)
SNAPS_NORM_MINMAX = 0x1
SNAPS_NAN_TO_MEAN = 0x2
SNAPS_FP32 = 0
SNAPS_TC_F16 = 1
SNAPS_TC_BF16 = 2
SNAPS_TC_TF32 = 3
SNAPS_INDEX_GRID = 0x100
SNAPS_INDEX_NONE = 0x200
SNAPS_GRID_AUTO_N = 65536
SNAPS_TC_MIN_FILL = 128
SNAPS_TC_NEVER = 257
SNAPS_STATIC_MAX_N = 32768
SNAPS_STATIC_MAX_MASKS = 32768
SNAPS_PHASE_INDEX, SNAPS_PHASE_JOIN_TREE, SNAPS_PHASE_JOIN_LANE, SNAPS_PHASE_NORM, SNAPS_PHASE_TOP, \
    SNAPS_PHASE_JOIN_TC, SNAPS_PHASE_ORDER, SNAPS_PHASE_GRID, SNAPS_PHASE_SELECT = range(9)
SNAPS_N_PHASES = 9
SNAPS_SELECT_MAX_GRID = 64
SNAPS_TUNE_CELLS = 3
SNAPS_TUNE_MAX_N = 65536
SNAPS_SELECTIVITY_MAX_SAMPLE = 65536
SNAPS_SELECTIVITY_MAX_BINS = 4096
PHASE_NAMES = ["index", "join_tree", "join_lane", "norm", "top", "join_tc", "order", "grid", "select"]


class SnapsError(RuntimeError):
    def __init__(self, status: int, func: str, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{func}: {name}: {msg}")


class snaps_request(ctypes.Structure):
    _fields_ = [("pop", ctypes.c_void_p), ("masks", ctypes.c_void_p), ("n_masks", ctypes.c_int),
                ("k", ctypes.c_int), ("eps", ctypes.c_void_p), ("precision", ctypes.c_uint32),
                ("scores", ctypes.c_void_p), ("norm", ctypes.c_void_p), ("top", ctypes.c_void_p),
                ("top_n", ctypes.c_int)]


class snaps_tune_entry(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("grid", ctypes.c_int), ("cell_mult", ctypes.c_float),
                ("ms_brute", ctypes.c_double), ("ms_grid", ctypes.c_double * 3)]


class snaps_tc_tune(ctypes.Structure):
    _fields_ = [("min_fill", ctypes.c_int), ("ms_block", ctypes.c_double), ("ms_lone", ctypes.c_double)]


class snaps_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("queue_us", ctypes.c_double),
                ("latency_us", ctypes.c_double), ("objects_x_subspaces", ctypes.c_int64)]


_lib = None


def lib():
    """Load libsnaps.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2405_20176_b300.build` (nvcc, sm_103a)")
        L = ctypes.CDLL(LIB_PATH)
        p, i32, i64, u32, sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint32,
                                ctypes.c_size_t)
        sig = {
            "snaps_version": ([], ctypes.c_char_p),
            "snaps_last_error": ([], ctypes.c_char_p),
            "snaps_create": ([i32, sz, p], i32),
            "snaps_destroy": ([p], i32),
            "snaps_mem_info": ([p, p, p], i32),
            "snaps_index": ([p, p, i64, i32, u32, p, p], i32),
            "snaps_release": ([p], i32),
            "snaps_pop_shape": ([p, p, p], i32),
            "snaps_pop_features": ([p, p, p], i32),
            "snaps_knn_selfjoin": ([p, p, i32, i32, p, p, p], i32),
            "snaps_eps_selfjoin": ([p, p, i32, p, p, p, p], i32),
            "snaps_scores": ([p, p, i32, i32, p, u32, p, p, p, i32, p], i32),
            "snaps_submit": ([p, ctypes.POINTER(snaps_request), ctypes.POINTER(ctypes.c_uint64)], i32),
            "snaps_poll": ([p, ctypes.c_uint64, i64, ctypes.POINTER(snaps_result)], i32),
            "snaps_cancel": ([p, ctypes.c_uint64], i32),
            "snaps_set_slots": ([p, i32], i32),
            "snaps_trace": ([p, i32], i32),
            "snaps_set_wait_limit": ([p, u32], i32),
            "snaps_serving_stats": ([p, p, p], i32),
            "snaps_trace_steps": ([p, p, p], i32),
            "snaps_calibrate_alu": ([i32, p], i32),
            "snaps_scores_static": ([i32, p, i64, i32, u32, p, i32, i32, p, p, p, i32, p], i32),
            "snaps_trace_read": ([p, p, p], i32),
            "snaps_select": ([p, p, i32, p, p, i32, p, i32, i32, p, p, p, p, p], i32),
            "snaps_eps_selectivity": ([p, p, i32, p, i32, i32, i32, p, p, p], i32),
            "snaps_autotune": ([p, i32, p, p], i32),
            "snaps_autotune_clear": ([p], i32),
            "snaps_autotune_set": ([p, i64, i32, p], i32),
            "snaps_autotune_tc": ([p, i32, u32, p, p], i32),
            "snaps_set_tc_min_fill": ([p, i32], i32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(status: int, func: str):
    if status != SNAPS_OK:
        msg = lib().snaps_last_error().decode(errors="replace")
        raise SnapsError(status, func, msg)


def _ptr(a):
    """Raw pointer of a torch tensor / NumPy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else getattr(stream, "cuda_stream", stream)
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover - torch missing
        pass
    return None


def _masks(masks) -> np.ndarray:
    m = np.ascontiguousarray(np.asarray(masks, dtype=np.uint16).ravel())
    if m.size == 0:
        raise ValueError("at least one mask is required")
    return m


def _eps(eps, n_masks):
    if eps is None:
        return None
    e = np.ascontiguousarray(np.asarray(eps, dtype=np.float32).ravel())
    if e.size != n_masks:
        raise ValueError("eps needs one radius per mask")
    return e


# ---- thin wrappers with the C names -------------------------------------------------------

def snaps_version() -> str:
    return lib().snaps_version().decode()


def snaps_last_error() -> str:
    return lib().snaps_last_error().decode(errors="replace")


def snaps_create(device: int = 0, hbm_budget_bytes: int = 0) -> int:
    out = ctypes.c_void_p()
    _check(lib().snaps_create(device, hbm_budget_bytes, ctypes.byref(out)), "snaps_create")
    return out.value


def snaps_destroy(ctx: int) -> None:
    _check(lib().snaps_destroy(ctx), "snaps_destroy")


def snaps_mem_info(ctx: int):
    held, budget = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().snaps_mem_info(ctx, ctypes.byref(held), ctypes.byref(budget)), "snaps_mem_info")
    return held.value, budget.value


def snaps_index(ctx: int, feat, flags: int = SNAPS_NORM_MINMAX, stream=None) -> int:
    """Index an (n, f) float32 population (host or device)."""
    if len(feat.shape) != 2:
        raise ValueError("feat must be 2-D (n, f)")
    n, f = int(feat.shape[0]), int(feat.shape[1])
    out = ctypes.c_void_p()
    _check(lib().snaps_index(ctx, _ptr(feat), n, f, flags, _stream(stream), ctypes.byref(out)),
           "snaps_index")
    return out.value


def snaps_release(pop: int) -> None:
    _check(lib().snaps_release(pop), "snaps_release")


def snaps_pop_shape(pop: int):
    n, f = ctypes.c_int64(), ctypes.c_int()
    _check(lib().snaps_pop_shape(pop, ctypes.byref(n), ctypes.byref(f)), "snaps_pop_shape")
    return n.value, f.value


def snaps_pop_features(pop: int, out, stream=None) -> None:
    _check(lib().snaps_pop_features(pop, _ptr(out), _stream(stream)), "snaps_pop_features")


def snaps_knn_selfjoin(pop: int, masks, k: int, idx, dist=None, stream=None) -> None:
    m = _masks(masks)
    _check(lib().snaps_knn_selfjoin(pop, m.ctypes.data, m.size, k, _ptr(idx), _ptr(dist),
                                    _stream(stream)), "snaps_knn_selfjoin")


def snaps_eps_selfjoin(pop: int, masks, eps=None, count=None, mean_dist=None, stream=None) -> None:
    m = _masks(masks)
    e = _eps(eps, m.size)
    _check(lib().snaps_eps_selfjoin(pop, m.ctypes.data, m.size, None if e is None else e.ctypes.data,
                                    _ptr(count), _ptr(mean_dist), _stream(stream)),
           "snaps_eps_selfjoin")


def snaps_scores(pop: int, masks, k: int, eps=None, precision: int = SNAPS_FP32, scores=None,
                 norm=None, top=None, top_n: int = 100, stream=None) -> None:
    m = _masks(masks)
    e = _eps(eps, m.size)
    _check(lib().snaps_scores(pop, m.ctypes.data, m.size, k, None if e is None else e.ctypes.data,
                              precision, _ptr(scores), _ptr(norm), _ptr(top),
                              top_n if top is not None else 0, _stream(stream)), "snaps_scores")


def snaps_select(pop: int, masks, eps_min=None, eps_max=None, n_eps: int = 0, k_grid=None,
                 top_n: int = 1, stream=None):
    """Parameter selection (Sec. 3.5.2 Eq. 2-3, Sec. 3.6.2) through the C ABI.
    eps_min / eps_max: per-subspace grid ends (None skips the eps grid); k_grid:
    ascending k values (None skips it).  Returns (u_eps, eps_select, u_k,
    k_select) as NumPy arrays shaped (m, 2, 2, n_eps), (m, 2), (m, 2, 2, n_k),
    (m, 2); the skipped halves are None."""
    m = _masks(masks)
    want_eps = eps_min is not None
    want_k = k_grid is not None
    emin = np.ascontiguousarray(np.broadcast_to(np.asarray(eps_min, dtype=np.float32), m.shape)) \
        if want_eps else None
    emax = np.ascontiguousarray(np.broadcast_to(np.asarray(eps_max, dtype=np.float32), m.shape)) \
        if want_eps else None
    kg = np.ascontiguousarray(np.asarray(k_grid, dtype=np.int32)) if want_k else None
    n_k = int(kg.size) if want_k else 0
    u_eps = np.zeros((m.size, 2, 2, n_eps), dtype=np.float32) if want_eps else None
    e_sel = np.zeros((m.size, 2), dtype=np.int32) if want_eps else None
    u_k = np.zeros((m.size, 2, 2, n_k), dtype=np.float32) if want_k else None
    k_sel = np.zeros((m.size, 2), dtype=np.int32) if want_k else None
    _check(lib().snaps_select(pop, m.ctypes.data, m.size, _ptr(emin), _ptr(emax), n_eps if want_eps else 0,
                              _ptr(kg), n_k, top_n, _ptr(u_eps), _ptr(e_sel), _ptr(u_k), _ptr(k_sel),
                              _stream(stream)), "snaps_select")
    return u_eps, e_sel, u_k, k_sel


def snaps_eps_selectivity(pop: int, masks, targets, n_sample: int = 1024, n_bins: int = 4096, stream=None):
    """Radii at which the sampled mean neighbour count reaches each target
    (Sec. 3.5.3) through the C ABI.  targets: mean neighbours per object.
    Returns (eps, eps_mean) as NumPy arrays shaped (m, len(targets)), (m,)."""
    m = _masks(masks)
    t = np.ascontiguousarray(np.atleast_1d(np.asarray(targets, dtype=np.float64)))
    eps = np.zeros((m.size, t.size), dtype=np.float32)
    mean = np.zeros(m.size, dtype=np.float32)
    _check(lib().snaps_eps_selectivity(pop, m.ctypes.data, m.size, t.ctypes.data, t.size, n_sample, n_bins,
                                       eps.ctypes.data, mean.ctypes.data, _stream(stream)),
           "snaps_eps_selectivity")
    return eps, mean


def snaps_eps_range(pop: int, n: int, masks, s_min: float = 0.001, s_max: float = 0.15, n_sample: int = 1024,
                    n_bins: int = 4096, stream=None):
    """The eps grid ends of Sec. 3.5.3: the radii of selectivities s_min n and
    s_max n.  Returns (eps_min, eps_max), each shaped (m,)."""
    eps, _ = snaps_eps_selectivity(pop, masks, [s_min * n, s_max * n], n_sample, n_bins, stream)
    return eps[:, 0].copy(), eps[:, 1].copy()


def snaps_autotune(pop: int, k: int, stream=None):
    """Time the index routes for subspaces of 2-4 features on this population
    and record the fastest in its context.  Returns one dict per dimension."""
    out = (snaps_tune_entry * 3)()
    _check(lib().snaps_autotune(pop, k, out, _stream(stream)), "snaps_autotune")
    return [{"d": e.d, "grid": bool(e.grid), "cell_mult": e.cell_mult, "ms_brute": e.ms_brute,
             "ms_grid": list(e.ms_grid)} for e in out]


def snaps_autotune_set(ctx: int, n: int, k: int, d: int, grid: bool, cell_mult: float) -> None:
    """Record an index choice for populations of n's size class without timing it."""
    e = snaps_tune_entry(d=d, grid=1 if grid else 0, cell_mult=cell_mult)
    _check(lib().snaps_autotune_set(ctx, n, k, ctypes.byref(e)), "snaps_autotune_set")


def snaps_autotune_clear(ctx: int) -> None:
    _check(lib().snaps_autotune_clear(ctx), "snaps_autotune_clear")


def snaps_autotune_tc(pop: int, k: int, precision: int = SNAPS_TC_F16, stream=None) -> dict:
    """Time one tensor-core block against subspaces joined on their own and
    record the block's minimum fill for this population's size class."""
    out = snaps_tc_tune()
    _check(lib().snaps_autotune_tc(pop, k, precision, ctypes.byref(out), _stream(stream)), "snaps_autotune_tc")
    return {"min_fill": out.min_fill, "ms_block": out.ms_block, "ms_lone": out.ms_lone}


def snaps_set_tc_min_fill(ctx: int, fill: int) -> None:
    """Fewest subspaces a tensor-core block carries on this context (0: tuned or built-in)."""
    _check(lib().snaps_set_tc_min_fill(ctx, fill), "snaps_set_tc_min_fill")


def snaps_scores_static(device: int, feat, masks, k: int, eps=None, flags: int = SNAPS_NORM_MINMAX,
                        scores=None, top=None, top_n: int = 100, stream=None) -> None:
    """Allocation-free scoring: ``feat`` (n, f), ``scores`` and ``top`` are
    device arrays owned by the caller; the library uses only its fixed static
    working array."""
    if len(feat.shape) != 2:
        raise ValueError("feat must be 2-D (n, f)")
    m = _masks(masks)
    e = _eps(eps, m.size)
    _check(lib().snaps_scores_static(device, _ptr(feat), int(feat.shape[0]), int(feat.shape[1]),
                                     flags, m.ctypes.data, m.size, k,
                                     None if e is None else e.ctypes.data, _ptr(scores), _ptr(top),
                                     top_n if top is not None else 0, _stream(stream)),
           "snaps_scores_static")


def snaps_set_slots(ctx: int, slots: int) -> None:
    _check(lib().snaps_set_slots(ctx, slots), "snaps_set_slots")


def snaps_calibrate_alu(device: int = 0) -> float:
    """Measured FP32 (add, compare) pairs per second on `device`."""
    v = ctypes.c_double()
    _check(lib().snaps_calibrate_alu(device, ctypes.byref(v)), "snaps_calibrate_alu")
    return v.value


def snaps_serving_stats(ctx: int):
    """(launches that served two or more requests, requests they served)."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().snaps_serving_stats(ctx, ctypes.byref(a), ctypes.byref(b)), "snaps_serving_stats")
    return a.value, b.value


def snaps_set_wait_limit(ctx: int, spins: int = 0) -> None:
    """Tries after which a tensor-core pipeline wait gives up (0 = the default)."""
    _check(lib().snaps_set_wait_limit(ctx, int(spins)), "snaps_set_wait_limit")


def snaps_trace(ctx: int, enable: bool = True) -> None:
    _check(lib().snaps_trace(ctx, 1 if enable else 0), "snaps_trace")


def snaps_trace_steps(ctx: int):
    """(steps loaded, all steps) of the subspace-batched join since tracing was enabled."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().snaps_trace_steps(ctx, ctypes.byref(a), ctypes.byref(b)), "snaps_trace_steps")
    return a.value, b.value


def snaps_trace_read(ctx: int):
    """{phase name: (ms, launches)} since tracing was enabled or last read."""
    ms = (ctypes.c_double * SNAPS_N_PHASES)()
    cnt = (ctypes.c_int64 * SNAPS_N_PHASES)()
    _check(lib().snaps_trace_read(ctx, ms, cnt), "snaps_trace_read")
    return {PHASE_NAMES[p]: (ms[p], cnt[p]) for p in range(SNAPS_N_PHASES)}


class Request:
    """A submitted request: keeps its mask / eps arrays and outputs alive."""

    def __init__(self, ticket, keep):
        self.ticket = ticket
        self._keep = keep


def snaps_submit(ctx: int, pop: int, masks, k: int, eps=None, precision: int = SNAPS_FP32,
                 scores=None, norm=None, top=None, top_n: int = 100) -> Request:
    m = _masks(masks)
    e = _eps(eps, m.size)
    req = snaps_request(pop, m.ctypes.data, m.size, k, None if e is None else e.ctypes.data,
                        precision, _ptr(scores), _ptr(norm), _ptr(top),
                        top_n if top is not None else 0)
    t = ctypes.c_uint64()
    _check(lib().snaps_submit(ctx, ctypes.byref(req), ctypes.byref(t)), "snaps_submit")
    return Request(t.value, (m, e, scores, norm, top))


def snaps_poll(ctx: int, request, timeout_us: int = -1):
    """Returns a snaps_result once the request finished, or None (EAGAIN)."""
    ticket = request.ticket if isinstance(request, Request) else int(request)
    res = snaps_result()
    st = lib().snaps_poll(ctx, ticket, timeout_us, ctypes.byref(res))
    if st == SNAPS_EAGAIN:
        return None
    _check(st, "snaps_poll")
    return res


def snaps_cancel(ctx: int, request) -> None:
    ticket = request.ticket if isinstance(request, Request) else int(request)
    _check(lib().snaps_cancel(ctx, ticket), "snaps_cancel")


def header_symbols() -> list[str]:
    """Names of the functions include/snaps.h declares."""
    import re
    path = os.path.join(os.path.dirname(_HERE), "include", "snaps.h")
    with open(path) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:snaps_status|const char \*)\s*(snaps_\w+)\s*\(", text,
                                 flags=re.M)))
