"""ctypes binding of libsj (include/simjoin.h): argument marshalling only.

Every function here has the name of the C entry point it wraps and does no
arithmetic of the join: points go to the library as a pointer (a CUDA tensor's
device pointer, or host memory of a numpy array / CPU tensor), results come
back as the library's device pages, copied out by ``sj_result_copy``.

The library must have been built (``paper_2209_11287_gb300.build.build()``);
loading fails loudly otherwise — there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import build as _build

SJ_OK = 0
SJ_ERR_ARG = -1
SJ_ERR_OOM = -2
SJ_ERR_RESULT_OVERFLOW = -3
SJ_ERR_TIMEOUT = -4
SJ_ERR_CUDA = -5
SJ_ERR_UNSUPPORTED = -6

SJ_NO_INDEX = -1  # sj_options.indexed_dims: no index, every pair evaluated

SJ_KERNEL_AUTO = 0
SJ_KERNEL_FP64_FMA = 1
SJ_KERNEL_FP64_DMMA = 2
SJ_KERNEL_FILTER_F32 = 3
SJ_KERNEL_FILTER_BF16X3 = 4
SJ_KERNEL_FILTER_BF16X2 = 5
SJ_KERNEL_FILTER_FP16X2 = 6

KERNELS = {
    "auto": SJ_KERNEL_AUTO,
    "fp64_fma": SJ_KERNEL_FP64_FMA,
    "fp64_dmma": SJ_KERNEL_FP64_DMMA,
    "filter_f32": SJ_KERNEL_FILTER_F32,
    "filter_bf16x3": SJ_KERNEL_FILTER_BF16X3,
    "filter_bf16x2": SJ_KERNEL_FILTER_BF16X2,
    "filter_fp16x2": SJ_KERNEL_FILTER_FP16X2,
}


class SimJoinError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"libsj status {status}: {message}")
        self.status = status


class sj_options(ctypes.Structure):
    _fields_ = [
        ("kernel", ctypes.c_int32),
        ("emit_distances", ctypes.c_int32),
        ("indexed_dims", ctypes.c_int32),
        ("symmetric", ctypes.c_int32),
        ("queries_per_item", ctypes.c_int32),
        ("graph", ctypes.c_int32),
        ("page_pairs", ctypes.c_int64),
        ("max_pairs_hint", ctypes.c_int64),
        ("tune_cache", ctypes.c_char_p),
        ("short_circuit", ctypes.c_int32),
    ]


class sj_result(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_int64),
        ("page_pairs", ctypes.c_int64),
        ("n_pages", ctypes.c_int32),
        ("has_distances", ctypes.c_int32),
        ("pair_pages", ctypes.POINTER(ctypes.c_void_p)),
        ("dist_pages", ctypes.POINTER(ctypes.c_void_p)),
        ("n_candidates", ctypes.c_int64),
        ("n_evaluated", ctypes.c_int64),
        ("n_rechecked", ctypes.c_int64),
        ("reruns", ctypes.c_int32),
        ("kernel", ctypes.c_int32),
        ("ms_tile", ctypes.c_double),
        ("internal", ctypes.c_void_p),
    ]


class sj_filter_dump(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("dp", ctypes.c_int32),
        ("kernel", ctypes.c_int32),
        ("c1", ctypes.c_double),
        ("pbound", ctypes.c_double),
        ("e2", ctypes.c_double),
        ("records", ctypes.c_int64),
        ("count", ctypes.c_int64),
        ("prune_r2", ctypes.c_double),
    ]


_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


def library_path() -> str:
    """The library to load: SJ_LIBRARY when set (the bounds-checking build in
    its test), else the regular build."""
    return os.environ.get("SJ_LIBRARY") or _build.LIB


def load():
    """Load libsj (declares the C signatures).  Raises if it was not built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libsj is not built ({path} missing); run paper_2209_11287_gb300.build.build()")
        lib = ctypes.CDLL(path)
        lib.sj_default_options.argtypes = [ctypes.POINTER(sj_options)]
        lib.sj_default_options.restype = None
        lib.sj_build_index.argtypes = [_vp, _i64, _i32, ctypes.c_double, ctypes.POINTER(sj_options), _vp,
                                       ctypes.POINTER(_vp)]
        lib.sj_build_index.restype = ctypes.c_int
        lib.sj_destroy.argtypes = [_vp]
        lib.sj_destroy.restype = None
        lib.sj_index_info.argtypes = [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i32),
                                      ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
        lib.sj_index_info.restype = ctypes.c_int
        lib.sj_self_join.argtypes = [_vp, ctypes.POINTER(sj_result)]
        lib.sj_self_join.restype = ctypes.c_int
        lib.sj_result_copy.argtypes = [ctypes.POINTER(sj_result), _vp, _vp]
        lib.sj_result_copy.restype = ctypes.c_int
        lib.sj_result_free.argtypes = [ctypes.POINTER(sj_result)]
        lib.sj_result_free.restype = None
        lib.sj_join.argtypes = [_vp, _i64, _i32, ctypes.c_double, ctypes.POINTER(sj_options), _vp,
                                ctypes.POINTER(sj_result)]
        lib.sj_join.restype = ctypes.c_int
        lib.sj_join_batch.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(_i64), ctypes.POINTER(_i32),
                                      ctypes.POINTER(ctypes.c_double), _i32, ctypes.POINTER(sj_options), _vp,
                                      ctypes.POINTER(sj_result)]
        lib.sj_join_batch.restype = ctypes.c_int
        lib.sj_error_string.argtypes = [ctypes.c_int]
        lib.sj_error_string.restype = ctypes.c_char_p
        lib.sj_last_error_message.argtypes = []
        lib.sj_last_error_message.restype = ctypes.c_char_p
        lib.sj_version.argtypes = []
        lib.sj_version.restype = ctypes.c_char_p
        lib.sj_kernel_launches.argtypes = []
        lib.sj_kernel_launches.restype = ctypes.c_int64
        lib.sj_self_join_noalloc.argtypes = [_vp, _i64, _i32, ctypes.c_double, _vp, _i64, ctypes.POINTER(_i64), _vp]
        lib.sj_self_join_noalloc.restype = ctypes.c_int
        lib.sj_results_free.argtypes = [ctypes.POINTER(sj_result), _i32]
        lib.sj_results_free.restype = None
        lib.sj_selftest_bounded_wait.argtypes = [_vp]
        lib.sj_selftest_bounded_wait.restype = ctypes.c_int
        lib.sj_autotune.argtypes = [_vp, _i64, _i32, ctypes.c_double, ctypes.POINTER(sj_options), _vp, _i32,
                                    ctypes.c_char_p, ctypes.POINTER(sj_options), ctypes.POINTER(ctypes.c_double)]
        lib.sj_autotune.restype = ctypes.c_int
        lib.sj_autotune_batch.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(_i64), ctypes.POINTER(_i32),
                                          ctypes.POINTER(ctypes.c_double), _i32, ctypes.POINTER(sj_options), _vp,
                                          _i32, ctypes.c_char_p, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                          ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                          ctypes.POINTER(ctypes.c_double)]
        lib.sj_autotune_batch.restype = ctypes.c_int
        lib.sj_tune_lookup.argtypes = [ctypes.c_char_p, _i32, _i32, _i64, ctypes.POINTER(_i32),
                                       ctypes.POINTER(_i32), ctypes.POINTER(_i32)]
        lib.sj_tune_lookup.restype = ctypes.c_int
        lib.sj_self_join_to_host.argtypes = [_vp, _vp, _i64, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i32)]
        lib.sj_self_join_to_host.restype = ctypes.c_int
        lib.sj_debug_filter_dump.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _i64, ctypes.POINTER(sj_filter_dump)]
        lib.sj_debug_filter_dump.restype = ctypes.c_int
        lib.sj_index_perm.argtypes = [_vp, _vp]
        lib.sj_index_perm.restype = ctypes.c_int
        lib.sj_debug_fail_allocations.argtypes = [_i64]
        lib.sj_debug_fail_allocations.restype = None
        lib.sj_debug_live_allocations.argtypes = []
        lib.sj_debug_live_allocations.restype = ctypes.c_int64
        lib.sj_index_item_work.argtypes = [_vp, _vp]
        lib.sj_index_item_work.restype = ctypes.c_int
        lib.sj_shard_bounds.argtypes = [_vp, _i64, _i32, _vp]
        lib.sj_shard_bounds.restype = ctypes.c_int
        lib.sj_self_join_range.argtypes = [_vp, _i64, _i64, ctypes.POINTER(sj_result)]
        lib.sj_self_join_range.restype = ctypes.c_int
        lib.sj_dbscan.argtypes = [ctypes.POINTER(sj_result), _i64, _i32, _vp, ctypes.POINTER(_i64)]
        lib.sj_dbscan.restype = ctypes.c_int
        lib.sj_sqdist_tile.argtypes = [_vp, _i64, _vp, _i64, _i32, _vp, _vp]
        lib.sj_sqdist_tile.restype = ctypes.c_int
        lib.sj_knn_from_join.argtypes = [ctypes.POINTER(sj_result), _i64, _i32, _vp, _vp, _vp]
        lib.sj_knn_from_join.restype = ctypes.c_int
        lib.sj_set_tracing.argtypes = [_i32]
        lib.sj_set_tracing.restype = None
        lib.sj_index_phase_ms.argtypes = [_vp, _vp, _vp]
        lib.sj_index_phase_ms.restype = ctypes.c_int
        _lib = lib
        return lib


def header_symbols() -> list[str]:
    """Entry points declared in include/simjoin.h."""
    src = open(os.path.join(_build.INCLUDE, "simjoin.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sj_[a-z_0-9]+)\s*\(", src)))


def _check(status: int):
    if status != SJ_OK:
        lib = load()
        raise SimJoinError(status, f"{lib.sj_error_string(status).decode()}: {lib.sj_last_error_message().decode()}")


# ---- argument marshalling helpers ---------------------------------------------

def _points_ptr(points):
    """(pointer, n, d, keepalive) of a 2-D float64 C-contiguous array or tensor."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(points, torch.Tensor):
        if points.dtype != torch.float64 or points.dim() != 2:
            raise ValueError("points must be a 2-D float64 tensor")
        points = points.contiguous()
        return points.data_ptr(), points.shape[0], points.shape[1], points
    a = np.ascontiguousarray(points, dtype=np.float64)
    if a.ndim != 2:
        raise ValueError("points must be an n x d array")
    return a.ctypes.data, a.shape[0], a.shape[1], a


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:  # pragma: no cover
            pass
        return 0
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# ---- entry points --------------------------------------------------------------

def sj_default_options(**overrides) -> sj_options:
    o = sj_options()
    load().sj_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "tune_cache":
            o.tune_cache = None if v is None else os.fsencode(v)
            continue
        if k == "kernel" and isinstance(v, str):
            v = KERNELS[v]
        setattr(o, k, int(v))
    return o


def sj_build_index(points, eps: float, options: sj_options | None = None, stream=None):
    """Build the grid index; returns an opaque handle (int).  ``points``: n x d
    float64, a CUDA tensor (used in place) or host memory (copied)."""
    ptr, n, d, keep = _points_ptr(points)
    h = ctypes.c_void_p()
    _check(load().sj_build_index(ptr, n, d, float(eps), ctypes.byref(options) if options is not None else None,
                                 _stream_ptr(stream), ctypes.byref(h)))
    del keep
    return h.value


def sj_destroy(handle) -> None:
    if handle:
        load().sj_destroy(handle)


def sj_index_info(handle) -> dict:
    c, it, e, f = _i64(), _i64(), _i64(), _i64()
    m = _i32()
    _check(load().sj_index_info(handle, ctypes.byref(c), ctypes.byref(it), ctypes.byref(m), ctypes.byref(e),
                                ctypes.byref(f)))
    return {"n_cells": c.value, "n_items": it.value, "m": m.value, "n_candidates": e.value, "n_evaluated": f.value}


def sj_self_join(handle) -> sj_result:
    r = sj_result()
    _check(load().sj_self_join(handle, ctypes.byref(r)))
    return r


def sj_self_join_to_host(handle, pairs_out, device_pairs: int):
    """Join in rounds into ``pairs_out`` (host int32 array or CPU tensor of
    shape (capacity, 2); pinned memory overlaps the copies) through device
    buffers of ``device_pairs`` pairs.  Returns (count, rounds); raises on
    overflow (the exception's status is SJ_ERR_RESULT_OVERFLOW)."""
    if hasattr(pairs_out, "data_ptr"):
        if str(pairs_out.dtype) != "torch.int32" or not pairs_out.is_contiguous() or pairs_out.is_cuda:
            raise ValueError("pairs_out must be a contiguous int32 CPU tensor")
        ptr, cap = pairs_out.data_ptr(), pairs_out.numel() // 2
    else:
        if pairs_out.dtype != np.int32 or not pairs_out.flags.c_contiguous:
            raise ValueError("pairs_out must be a contiguous int32 array")
        ptr, cap = pairs_out.ctypes.data, pairs_out.size // 2
    cnt, rounds = _i64(0), _i32(0)
    _check(load().sj_self_join_to_host(handle, ptr, cap, int(device_pairs), ctypes.byref(cnt), ctypes.byref(rounds)))
    return int(cnt.value), int(rounds.value)


def sj_result_copy(result: sj_result, pairs_out=None, dist_out=None):
    """Copy pairs (count x 2 int32) and distances (count float64) into the given
    outputs (CUDA tensors, CPU tensors or numpy arrays), allocating host numpy
    arrays when an output is None.  Returns (pairs, dists or None)."""
    cnt = int(result.count)
    if pairs_out is None:
        pairs_out = np.empty((cnt, 2), dtype=np.int32)
    if dist_out is None and result.has_distances:
        dist_out = np.empty(cnt, dtype=np.float64)

    def ptr(a, dtype_np, torch_dtype_name):
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            if str(a.dtype) != f"torch.{torch_dtype_name}" or not a.is_contiguous() or a.numel() < (2 * cnt if torch_dtype_name == "int32" else cnt):
                raise ValueError("output tensor has the wrong dtype, layout or size")
            return a.data_ptr()
        if a.dtype != dtype_np or not a.flags.c_contiguous or a.size < (2 * cnt if dtype_np == np.int32 else cnt):
            raise ValueError("output array has the wrong dtype, layout or size")
        return a.ctypes.data

    _check(load().sj_result_copy(ctypes.byref(result), ptr(pairs_out, np.int32, "int32"),
                                 ptr(dist_out, np.float64, "float64") if result.has_distances else None))
    return pairs_out, (dist_out if result.has_distances else None)


def sj_result_free(result: sj_result) -> None:
    load().sj_result_free(ctypes.byref(result))


def sj_join(points, eps: float, options: sj_options | None = None, stream=None) -> sj_result:
    ptr, n, d, keep = _points_ptr(points)
    r = sj_result()
    _check(load().sj_join(ptr, n, d, float(eps), ctypes.byref(options) if options is not None else None,
                          _stream_ptr(stream), ctypes.byref(r)))
    del keep
    return r


class BatchInputs:
    """The argument arrays of sj_join_batch (instance pointers, sizes,
    dimensions, eps), marshalled once for joins repeated on the same inputs."""

    def __init__(self, points_list, eps_list):
        count = len(points_list)
        if len(eps_list) != count:
            raise ValueError("one eps per instance")
        self.count = count
        self.ptrs = (_vp * count)()
        self.ns = (_i64 * count)()
        self.ds = (_i32 * count)()
        self.es = (ctypes.c_double * count)()
        self._keep = []
        for k, (p, e) in enumerate(zip(points_list, eps_list)):
            ptr, n, d, kp = _points_ptr(p)
            self._keep.append(kp)
            self.ptrs[k], self.ns[k], self.ds[k], self.es[k] = ptr, n, d, float(e)


def sj_join_batch_raw(inputs: BatchInputs, options: sj_options | None = None, stream=None):
    """sj_join_batch on prepared inputs; returns the ctypes array of results
    (release with sj_results_free)."""
    res = (sj_result * inputs.count)()
    _check(load().sj_join_batch(inputs.ptrs, inputs.ns, inputs.ds, inputs.es, inputs.count,
                                ctypes.byref(options) if options is not None else None, _stream_ptr(stream), res))
    return res


def sj_results_free(results) -> None:
    load().sj_results_free(results, len(results))


def results_table(results) -> np.ndarray:
    """The scalar fields of an array of sj_result (count, n_candidates,
    n_evaluated, n_rechecked, reruns, kernel, ms_tile) as a numpy record view."""
    names = ["count", "n_candidates", "n_evaluated", "n_rechecked", "reruns", "kernel", "ms_tile"]
    fmts = {"count": "<i8", "n_candidates": "<i8", "n_evaluated": "<i8", "n_rechecked": "<i8", "reruns": "<i4",
            "kernel": "<i4", "ms_tile": "<f8"}
    dt = np.dtype({"names": names, "formats": [fmts[n] for n in names],
                   "offsets": [getattr(sj_result, n).offset for n in names], "itemsize": ctypes.sizeof(sj_result)})
    return np.frombuffer(results, dtype=dt)


def sj_join_batch(points_list, eps_list, options: sj_options | None = None, stream=None) -> list:
    return list(sj_join_batch_raw(BatchInputs(points_list, eps_list), options, stream))


def sj_self_join_noalloc(points, eps: float, pairs_out, stream=None) -> int:
    """The allocation-free self-join for callers that cannot allocate while
    they run: ``points`` an n x d float64 CUDA tensor (n <= 32768, d <= 8),
    ``pairs_out`` a preallocated CUDA int32 tensor of shape (capacity, 2).
    Returns the pair count (raises on overflow, with the count in the
    message)."""
    ptr, n, d, keep = _points_ptr(points)
    if not hasattr(pairs_out, "data_ptr") or str(pairs_out.dtype) != "torch.int32" or not pairs_out.is_contiguous():
        raise ValueError("pairs_out must be a contiguous int32 CUDA tensor of shape (capacity, 2)")
    cnt = _i64(0)
    _check(load().sj_self_join_noalloc(ptr, n, d, float(eps), pairs_out.data_ptr(), pairs_out.numel() // 2,
                                       ctypes.byref(cnt), _stream_ptr(stream)))
    del keep
    return int(cnt.value)


def sj_autotune(points, eps: float, base: sj_options | None = None, stream=None, reps: int = 0,
                cache_path=None):
    """Times the candidate configurations of a single join on ``points``
    and returns (best options, median ms of the whole path); the winner is
    appended to ``cache_path`` when given."""
    ptr, n, d, keep = _points_ptr(points)
    best = sj_options()
    ms = ctypes.c_double(0.0)
    _check(load().sj_autotune(ptr, n, d, float(eps), ctypes.byref(base) if base is not None else None,
                              _stream_ptr(stream), int(reps), None if cache_path is None else os.fsencode(cache_path),
                              ctypes.byref(best), ctypes.byref(ms)))
    del keep
    return best, float(ms.value)


def sj_autotune_batch(inputs: "BatchInputs", base: sj_options | None = None, stream=None, reps: int = 0,
                      cache_path=None) -> list:
    """Tunes a batched join per group of padded dimension; returns one dict
    per group (dp, kernel, qpi, ms), the winners also appended to
    ``cache_path`` when given."""
    mg = 64
    ng = _i32(0)
    gdp, gk, gq = (_i32 * mg)(), (_i32 * mg)(), (_i32 * mg)()
    gms = (ctypes.c_double * mg)()
    _check(load().sj_autotune_batch(inputs.ptrs, inputs.ns, inputs.ds, inputs.es, inputs.count,
                                    ctypes.byref(base) if base is not None else None, _stream_ptr(stream), int(reps),
                                    None if cache_path is None else os.fsencode(cache_path), mg, ctypes.byref(ng),
                                    gdp, gk, gq, gms))
    return [{"dp": gdp[i], "kernel": gk[i], "qpi": gq[i], "ms": gms[i]} for i in range(ng.value)]


def sj_tune_lookup(path, batch: int, d: int, n: int = 0):
    """The tuning-cache entry a join would use (no GPU needed): a dict with
    kernel, qpi and m, or None when no entry matches."""
    k, q, m = _i32(0), _i32(0), _i32(0)
    r = load().sj_tune_lookup(os.fsencode(path), int(batch), int(d), int(n), ctypes.byref(k), ctypes.byref(q),
                              ctypes.byref(m))
    if r < 0:
        _check(r)
    return {"kernel": k.value, "qpi": q.value, "m": m.value} if r == 1 else None


def sj_selftest_bounded_wait(stream=None) -> int:
    """Runs the library's bounded-wait self-test; returns its status
    (SJ_ERR_TIMEOUT when the wait gave up as designed)."""
    return int(load().sj_selftest_bounded_wait(_stream_ptr(stream)))


def sj_error_string(status: int) -> str:
    return load().sj_error_string(int(status)).decode()


def sj_last_error_message() -> str:
    return load().sj_last_error_message().decode()


def sj_version() -> str:
    return load().sj_version().decode()


def sj_kernel_launches() -> int:
    return int(load().sj_kernel_launches())


# ---- convenience ------------------------------------------------------------------

def self_join(points, eps: float, kernel="auto", emit_distances=False, symmetric=True, indexed_dims=0,
              max_pairs_hint=0, queries_per_item=0, tune_cache=None, short_circuit=0, stream=None):
    """Build, join and copy out in one call: returns (pairs int32 n x 2 numpy,
    distances or None, stats dict: the index's sizes (n_evaluated: the
    scheduled pair evaluations), count, n_rechecked, reruns, kernel and
    n_performed, the evaluations the tile kernel performed)."""
    opt = sj_default_options(kernel=kernel, emit_distances=int(emit_distances), symmetric=int(symmetric),
                             indexed_dims=indexed_dims, max_pairs_hint=max_pairs_hint,
                             queries_per_item=queries_per_item, tune_cache=tune_cache,
                             short_circuit=int(short_circuit))
    h = sj_build_index(points, eps, opt, stream)
    try:
        info = sj_index_info(h)
        r = sj_self_join(h)
        try:
            pairs, dists = sj_result_copy(r)
            stats = dict(info, count=int(r.count), n_rechecked=int(r.n_rechecked), reruns=int(r.reruns),
                         kernel=int(r.kernel), n_performed=int(r.n_evaluated))
        finally:
            sj_result_free(r)
    finally:
        sj_destroy(h)
    return pairs, dists, stats


def join_batch(points_list, eps_list, kernel="auto", emit_distances=False, symmetric=True, page_pairs=0,
               max_pairs_hint=0, indexed_dims=0, queries_per_item=0, graph=0, tune_cache=None, stream=None):
    """Batched self-joins in one call: returns one (pairs, distances or None,
    stats) per instance, the results already copied to the host and freed."""
    opt = sj_default_options(kernel=kernel, emit_distances=int(emit_distances), symmetric=int(symmetric),
                             page_pairs=page_pairs, max_pairs_hint=max_pairs_hint, indexed_dims=indexed_dims,
                             queries_per_item=queries_per_item, graph=int(graph), tune_cache=tune_cache)
    res = sj_join_batch(points_list, eps_list, opt, stream)
    out = []
    try:
        for r in res:
            pairs, dists = sj_result_copy(r)
            out.append((pairs, dists, dict(count=int(r.count), n_candidates=int(r.n_candidates),
                                           n_evaluated=int(r.n_evaluated), reruns=int(r.reruns),
                                           kernel=int(r.kernel), ms_tile=float(r.ms_tile))))
    finally:
        for r in res:
            sj_result_free(r)
    return out


def pairs_to_keys(pairs: np.ndarray) -> np.ndarray:
    """Sorted 64-bit keys (i << 32) | j of an (i, j) int32 pair array."""
    p = np.asarray(pairs).astype(np.int64)
    return np.sort((p[:, 0] << 32) | p[:, 1])


def sj_debug_filter_dump(handle, capacity: int):
    """The filter's own value for every evaluated pair of a built index
    (test aid): returns (info, records, arrays) with records an (m, 4) int64
    array of (query position, candidate position, float32 bits of a, pruned)
    in cell order (m = min(info.records, capacity); pruned = 1 marks a pair
    the FP32 filter's bounding-box prune decided out without evaluating it,
    with no value of a) and arrays a dict of the index's perm, y (n x dp
    float32), h, thr_out, thr_in in cell order."""
    lib = load()
    info = sj_filter_dump()
    # sizes first (no arrays, no records: nothing runs), then the dump
    _check(lib.sj_debug_filter_dump(handle, None, None, None, None, None, None, 0, ctypes.byref(info)))
    nn, dp = int(info.n), int(info.dp)
    perm = np.empty(nn, dtype=np.int32)
    y = np.empty((nn, dp), dtype=np.float32)
    h = np.empty(nn, dtype=np.float32)
    to = np.empty(nn, dtype=np.float32)
    ti = np.empty(nn, dtype=np.float32)
    rec = np.empty((max(int(capacity), 1), 4), dtype=np.int32)
    _check(lib.sj_debug_filter_dump(handle, perm.ctypes.data, y.ctypes.data, h.ctypes.data, to.ctypes.data,
                                    ti.ctypes.data, rec.ctypes.data, int(capacity), ctypes.byref(info)))
    m = min(int(info.records), int(capacity))
    return info, rec[:m, :4].astype(np.int64), {"perm": perm, "y": y, "h": h, "thr_out": to, "thr_in": ti}


def sj_index_perm(handle, n: int) -> np.ndarray:
    """The cell order of a built index: input index of each sorted position."""
    out = np.empty(int(n), dtype=np.int32)
    _check(load().sj_index_perm(handle, out.ctypes.data))
    return out


def sj_debug_fail_allocations(after: int) -> None:
    """Test aid: the next ``after`` device allocations succeed, later ones fail
    with SJ_ERR_OOM; a negative value switches the injection off."""
    load().sj_debug_fail_allocations(int(after))


def sj_debug_live_allocations() -> int:
    """Test aid: device blocks the library holds at the moment."""
    return int(load().sj_debug_live_allocations())


def sj_index_item_work(handle) -> np.ndarray:
    """Pair evaluations of each work item of a built index (int64)."""
    n_items = sj_index_info(handle)["n_items"]
    out = np.zeros(n_items, dtype=np.int64)
    _check(load().sj_index_item_work(handle, out.ctypes.data))
    return out


def sj_shard_bounds(item_work, n_shards: int) -> np.ndarray:
    """Contiguous item ranges of about equal work (host only): bounds[k] ..
    bounds[k + 1] is shard k."""
    w = np.ascontiguousarray(item_work, dtype=np.int64)
    out = np.zeros(int(n_shards) + 1, dtype=np.int64)
    _check(load().sj_shard_bounds(w.ctypes.data, w.size, int(n_shards), out.ctypes.data))
    return out


def sj_self_join_range(handle, item_begin: int, item_end: int) -> sj_result:
    """sj_self_join over work items [item_begin, item_end)."""
    r = sj_result()
    _check(load().sj_self_join_range(handle, int(item_begin), int(item_end), ctypes.byref(r)))
    return r


def sj_set_tracing(on: bool) -> None:
    """Record the build phases of later sj_build_index calls."""
    load().sj_set_tracing(int(bool(on)))


def sj_index_phase_ms(handle):
    """(device ms, host ms) of the four build phases of a traced index:
    extent + grid, sort, packing, runs + items (-1 where not traced)."""
    dev = np.zeros(4)
    host = np.zeros(4)
    _check(load().sj_index_phase_ms(handle, dev.ctypes.data, host.ctypes.data))
    return dev, host


def sj_dbscan(result: sj_result, n: int, min_pts: int):
    """DBSCAN labels (n int32 numpy, -1 for noise) and the cluster count from
    a single join's result over n points."""
    labels = np.empty(int(n), dtype=np.int32)
    k = _i64(0)
    _check(load().sj_dbscan(ctypes.byref(result), int(n), int(min_pts), labels.ctypes.data, ctypes.byref(k)))
    return labels, int(k.value)


def sj_sqdist_tile(a, b, out=None, stream=None):
    """All squared distances between the rows of two float64 CUDA tensors
    (m x d, nb x d) in the decision rule's arithmetic; returns the m x nb
    float64 CUDA tensor."""
    import torch
    if a.dtype != torch.float64 or b.dtype != torch.float64 or not a.is_cuda or not b.is_cuda:
        raise ValueError("a and b must be float64 CUDA tensors")
    a, b = a.contiguous(), b.contiguous()
    if out is None:
        out = torch.empty((a.shape[0], b.shape[0]), dtype=torch.float64, device=a.device)
    _check(load().sj_sqdist_tile(a.data_ptr(), a.shape[0], b.data_ptr(), b.shape[0], a.shape[1], out.data_ptr(),
                                 _stream_ptr(stream)))
    return out


def sj_knn_from_join(result: sj_result, n: int, k: int):
    """(indices n x k int32, distances n x k float64, found n int32) of every
    point's k nearest other eps-neighbours from a result with distances."""
    idx = np.empty((int(n), int(k)), dtype=np.int32)
    dist = np.empty((int(n), int(k)), dtype=np.float64)
    found = np.empty(int(n), dtype=np.int32)
    _check(load().sj_knn_from_join(ctypes.byref(result), int(n), int(k), idx.ctypes.data, dist.ctypes.data,
                                   found.ctypes.data))
    return idx, dist, found
