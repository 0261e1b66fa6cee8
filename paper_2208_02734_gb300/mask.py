"""ctypes binding of libmask_gb300.so (C ABI in include/mask.h).

Argument marshalling only: every function here forwards to the C entry point
of the same name.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays;
outputs are allocated like the first array argument (CUDA tensor in ->
CUDA tensor out, otherwise numpy).  CUDA tensors are passed on torch's current
stream.  There is no fallback: if the library cannot be loaded (or built with
nvcc), every call raises.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

MASK_PENDING = 1
MASK_OK, MASK_EINVAL, MASK_ENOMEM, MASK_ECUDA, MASK_ETIMEOUT, MASK_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
MASK_FP32, MASK_BF16, MASK_FP8E4M3 = 0, 1, 2
MASK_MAX_LEVELS = 16

_STATUS = {1: "MASK_PENDING", 0: "MASK_OK", -1: "MASK_EINVAL", -2: "MASK_ENOMEM", -3: "MASK_ECUDA",
           -4: "MASK_ETIMEOUT", -5: "MASK_EUNSUPPORTED"}

EXPORTED = [
    "mask_last_error", "mask_build", "mask_build_csr", "mask_query", "mask_query_csr",
    "mask_free", "mask_index_get_info", "mask_index_export_level", "mask_index_load",
    "mask_kmeanspp", "mask_kmeans_assign", "mask_kmeans_update",
    "mask_profile_enable", "mask_profile_reset", "mask_profile_read", "mask_launch_count",
    "mask_kmeans_assign_noalloc", "mask_kmeanspp_csr", "mask_kmeans_assign_csr",
    "mask_kmeans_update_csr", "mask_server_open", "mask_server_submit", "mask_server_poll",
    "mask_server_wait", "mask_server_stats", "mask_server_close", "mask_test_bounded_wait",
    "mask_test_tc_mma_cycles",
    "mask_test_alloc_count", "mask_grouped_levels", "mask_build_grouped", "mask_descend",
    "mask_relocate", "mask_range_query", "mask_insert", "mask_merge_topk",
]


class MaskError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        super().__init__(f"{fn} -> {_STATUS.get(status, status)}: {msg}")
        self.status = status


class mask_index_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("n_levels", C.c_int32),
                ("k_per_level", C.c_int32 * MASK_MAX_LEVELS), ("iters", C.c_int32),
                ("sparse", C.c_int32), ("device_bytes", C.c_int64)]


class mask_server_info(C.Structure):
    _fields_ = [("requests_done", C.c_int64), ("requests_failed", C.c_int64),
                ("queries_done", C.c_int64), ("batches", C.c_int64),
                ("graph_launches", C.c_int64), ("graph_captures", C.c_int64),
                ("autotuned_shapes", C.c_int64), ("mean_batch_queries", C.c_double),
                ("latency_mean_ms", C.c_double), ("latency_p50_ms", C.c_double),
                ("latency_p99_ms", C.c_double), ("latency_max_ms", C.c_double),
                ("elapsed_s", C.c_double), ("peak_inflight_bytes", C.c_int64),
                ("mem_budget", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lock = threading.Lock()
_lib = None
_vp, _i32, _i64, _u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64


def library_path() -> str:
    return _build.LIB


def load(build_if_stale: bool = True):
    """Open the shared library (compiling it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_stale else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libmask_gb300.so not found at {path}")
        lib = C.CDLL(path)
        sig = {
            "mask_last_error": (C.c_char_p, []),
            "mask_build": (C.c_int, [_vp, _i64, _i32, _vp, _i32, _i32, _u64, _vp, _vp]),
            "mask_build_csr": (C.c_int, [_vp, _vp, _vp, _i64, _i32, _vp, _i32, _i32, _u64, _vp,
                                         _vp]),
            "mask_query": (C.c_int, [_vp, _vp, _i64, _i32, _vp, C.c_int, _vp, _vp, _vp]),
            "mask_query_csr": (C.c_int, [_vp, _vp, _vp, _vp, _i64, _i32, _vp, C.c_int, _vp, _vp,
                                         _vp]),
            "mask_free": (None, [_vp]),
            "mask_index_get_info": (C.c_int, [_vp, C.POINTER(mask_index_info)]),
            "mask_index_export_level": (C.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, _vp]),
            "mask_index_load": (C.c_int, [_vp, _i64, _i32, _i32, _vp, _vp, _vp, _vp, _vp]),
            "mask_kmeanspp": (C.c_int, [_vp, _i64, _i32, _i32, _u64, _i32, _vp, _vp, _vp]),
            "mask_kmeans_assign": (C.c_int, [_vp, _i64, _i32, _vp, _i32, _vp, _vp, _vp]),
            "mask_kmeans_update": (C.c_int, [_vp, _i64, _i32, _vp, _i32, _vp, _vp, _vp, _vp]),
            "mask_profile_enable": (None, [_i32]),
            "mask_profile_reset": (None, []),
            "mask_profile_read": (C.c_int32, [C.c_char_p, C.POINTER(C.c_int64),
                                              C.POINTER(C.c_double), C.POINTER(C.c_double)]),
            "mask_launch_count": (C.c_int64, []),
            "mask_test_alloc_count": (C.c_int64, []),
            "mask_grouped_levels": (C.c_int, [_i64, _i32, _i32, _vp, _vp]),
            "mask_build_grouped": (C.c_int, [_vp, _i64, _i32, _i32, _i32, _i32, _u64, _vp, _vp,
                                             _vp]),
            "mask_descend": (C.c_int, [_vp, _vp, _i64, _vp, _vp, _vp]),
            "mask_relocate": (C.c_int, [_vp, _vp, _i32, _vp, _vp, _vp, _vp]),
            "mask_range_query": (C.c_int, [_vp, _vp, _i64, C.c_float, _vp, _i64, _vp, _vp, _vp]),
            "mask_insert": (C.c_int, [_vp, _vp, _i64, _vp, _vp]),
            "mask_merge_topk": (C.c_int, [_vp, _vp, _i32, _i64, _i32, _vp, _vp, _vp, _vp]),
            "mask_test_bounded_wait": (C.c_int, [_i32, _i32, _vp]),
            "mask_test_tc_mma_cycles": (C.c_int, [_i32, _i32, _i32, _i32, _vp]),
            "mask_kmeans_assign_noalloc": (C.c_int, [_vp, _i64, _i32, _vp, _i32, _vp, _vp, _vp]),
            "mask_kmeanspp_csr": (C.c_int, [_vp, _vp, _vp, _i64, _i32, _i32, _u64, _i32, _vp,
                                            _vp, _vp]),
            "mask_kmeans_assign_csr": (C.c_int, [_vp, _vp, _vp, _i64, _i32, _vp, _i32, _vp, _vp,
                                                 _vp]),
            "mask_kmeans_update_csr": (C.c_int, [_vp, _vp, _vp, _i64, _i32, _vp, _i32, _vp, _vp,
                                                 _vp, _vp]),
            "mask_server_open": (C.c_int, [_vp, _i64, _i32, _i32, _vp]),
            "mask_server_submit": (C.c_int, [_vp, _vp, _i64, _i32, _vp, C.c_int, _vp, _vp,
                                             C.POINTER(C.c_uint64)]),
            "mask_server_poll": (C.c_int, [_vp, _u64]),
            "mask_server_wait": (C.c_int, [_vp, _u64, _i32]),
            "mask_server_stats": (C.c_int, [_vp, C.POINTER(mask_server_info), _i32]),
            "mask_server_close": (None, [_vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def mask_last_error() -> str:
    return load().mask_last_error().decode()


def _check(status: int, fn: str) -> None:
    if status != MASK_OK:
        raise MaskError(status, fn, mask_last_error())


# ------------------------------------------------------------- marshalling

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _is_cuda(x) -> bool:
    return _is_torch(x) and x.is_cuda


def _arr(x, dtype: str):
    """Contiguous array of the given dtype name; returns (obj, pointer)."""
    if x is None:
        return None, None
    if _is_torch(x):
        import torch
        td = {"float32": torch.float32, "int32": torch.int32, "int64": torch.int64,
              "float64": torch.float64}[dtype]
        x = x.to(td).contiguous()
        return x, x.data_ptr()
    x = np.ascontiguousarray(x, dtype=dtype)
    return x, x.ctypes.data


def _empty_like_kind(ref, shape, dtype: str):
    if _is_cuda(ref):
        import torch
        td = {"float32": torch.float32, "int32": torch.int32, "int64": torch.int64,
              "float64": torch.float64}[dtype]
        t = torch.empty(shape, dtype=td, device=ref.device)
        return t, t.data_ptr()
    a = np.empty(shape, dtype=dtype)
    return a, a.ctypes.data


def _stream(ref, stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    if _is_cuda(ref):
        import torch
        return torch.cuda.current_stream(ref.device).cuda_stream
    return None


def _host_i32(v):
    a = np.ascontiguousarray(v, dtype=np.int32)
    return a, a.ctypes.data


# ------------------------------------------------------------------ index

class Index:
    """Owner of a mask_index* (freed by .free() or garbage collection)."""

    def __init__(self, handle: int):
        self.handle = C.c_void_p(handle)

    def free(self) -> None:
        if self.handle and self.handle.value:
            load().mask_free(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    @property
    def info(self) -> mask_index_info:
        return mask_index_get_info(self)


def _handle(index) -> C.c_void_p:
    h = index.handle if isinstance(index, Index) else C.c_void_p(index)
    if not h or not h.value:
        raise ValueError("index is freed or NULL")
    return h


# ------------------------------------------------------------- entry points

def mask_build(points, k_per_level, iters: int, seed: int, stream=None) -> Index:
    X, px = _arr(points, "float32")
    n, d = X.shape
    kp, pk = _host_i32(k_per_level)
    out = C.c_void_p()
    _check(load().mask_build(px, n, d, pk, len(kp), iters, seed & 0xFFFFFFFFFFFFFFFF,
                             _stream(X, stream), C.byref(out)), "mask_build")
    return Index(out.value)


def mask_build_csr(row_ptr, col, val, n_cols: int, k_per_level, iters: int, seed: int,
                   stream=None) -> Index:
    rp, prp = _arr(row_ptr, "int64")
    cl, pcl = _arr(col, "int32")
    vl, pvl = _arr(val, "float32")
    kp, pk = _host_i32(k_per_level)
    out = C.c_void_p()
    _check(load().mask_build_csr(prp, pcl, pvl, len(rp) - 1, n_cols, pk, len(kp), iters,
                                 seed & 0xFFFFFFFFFFFFFFFF, _stream(vl, stream), C.byref(out)),
           "mask_build_csr")
    return Index(out.value)


def mask_query(index, queries, k: int, probes, precision: int = MASK_FP32, stream=None):
    Q, pq = _arr(queries, "float32")
    nq = Q.shape[0]
    pr, pp = _host_i32(probes)
    ids, pids = _empty_like_kind(Q, (nq, k), "int64")
    dists, pd = _empty_like_kind(Q, (nq, k), "float32")
    _check(load().mask_query(_handle(index), pq, nq, k, pp, precision, pids, pd,
                             _stream(Q, stream)), "mask_query")
    return ids, dists


def mask_query_csr(index, row_ptr, col, val, k: int, probes, precision: int = MASK_FP32,
                   stream=None):
    rp, prp = _arr(row_ptr, "int64")
    cl, pcl = _arr(col, "int32")
    vl, pvl = _arr(val, "float32")
    nq = len(rp) - 1
    pr, pp = _host_i32(probes)
    ids, pids = _empty_like_kind(vl, (nq, k), "int64")
    dists, pd = _empty_like_kind(vl, (nq, k), "float32")
    _check(load().mask_query_csr(_handle(index), prp, pcl, pvl, nq, k, pp, precision, pids, pd,
                                 _stream(vl, stream)), "mask_query_csr")
    return ids, dists


def mask_free(index) -> None:
    if isinstance(index, Index):
        index.free()
    else:
        load().mask_free(C.c_void_p(index))


def mask_index_get_info(index) -> mask_index_info:
    info = mask_index_info()
    _check(load().mask_index_get_info(_handle(index), C.byref(info)), "mask_index_get_info")
    return info


def mask_index_export_level(index, level: int, device=None, stream=None):
    """Returns dict(centroids [k x d], labels [n_below], chosen [k], objective [iters+1])."""
    info = mask_index_get_info(index)
    k = info.k_per_level[level]
    n_below = info.n if level == 0 else info.k_per_level[level - 1]
    if device is not None and str(device).startswith("cuda"):
        import torch
        ref = torch.empty(0, device=device)
    else:
        ref = None
    cen, pc = _empty_like_kind(ref, (k, info.d), "float32")
    lab, pl = _empty_like_kind(ref, (n_below,), "int32")
    chosen = np.empty(k, dtype=np.int64)
    obj = np.empty(info.iters + 1, dtype=np.float64)
    chosen[:] = -1
    obj[:] = np.nan
    _check(load().mask_index_export_level(_handle(index), level, pc, pl, chosen.ctypes.data,
                                          obj.ctypes.data, _stream(ref, stream)),
           "mask_index_export_level")
    return {"centroids": cen, "labels": lab, "chosen": chosen, "objective": obj}


def mask_index_load(points, centroids, labels, stream=None) -> Index:
    X, px = _arr(points, "float32")
    n, d = X.shape
    L = len(centroids)
    cs = [_arr(c, "float32") for c in centroids]
    ls = [_arr(lb, "int32") for lb in labels]
    kp, pk = _host_i32([c[0].shape[0] for c in cs])
    cptr = (C.c_void_p * L)(*[p for _, p in cs])
    lptr = (C.c_void_p * L)(*[p for _, p in ls])
    out = C.c_void_p()
    _check(load().mask_index_load(px, n, d, L, pk, cptr, lptr, _stream(X, stream),
                                  C.byref(out)), "mask_index_load")
    return Index(out.value)


def mask_grouped_levels(n: int, length_group: int, n_centroids: int):
    sizes = np.zeros(MASK_MAX_LEVELS, dtype=np.int64)
    L = C.c_int32()
    _check(load().mask_grouped_levels(n, length_group, n_centroids, sizes.ctypes.data,
                                      C.byref(L)), "mask_grouped_levels")
    return [int(v) for v in sizes[:L.value]]


def mask_build_grouped(points, length_group: int, n_centroids: int, iters: int, seed: int,
                       group0=None, stream=None) -> Index:
    X, px = _arr(points, "float32")
    n, d = X.shape
    g0, pg = (None, None) if group0 is None else _arr(group0, "int32")
    out = C.c_void_p()
    _check(load().mask_build_grouped(px, n, d, length_group, n_centroids, iters,
                                     seed & 0xFFFFFFFFFFFFFFFF, pg, _stream(X, stream),
                                     C.byref(out)), "mask_build_grouped")
    return Index(out.value)


def mask_descend(index, queries, probes, stream=None):
    Q, pq = _arr(queries, "float32")
    nq = Q.shape[0]
    pr, pp = _host_i32(probes)
    leaf, pl = _empty_like_kind(Q, (nq, int(pr[0])), "int32")
    _check(load().mask_descend(_handle(index), pq, nq, pp, pl, _stream(Q, stream)),
           "mask_descend")
    return leaf


def mask_relocate(index, points, n_centroids: int, group0, stream=None):
    """One relocation pass (§4.1): returns (missed, moved, new group0)."""
    X, px = _arr(points, "float32")
    g = np.array(np.asarray(group0), dtype=np.int32, copy=True)
    missed, moved = C.c_int64(0), C.c_int64(0)
    _check(load().mask_relocate(_handle(index), px, n_centroids, g.ctypes.data, C.byref(missed),
                                C.byref(moved), _stream(X, stream)), "mask_relocate")
    return int(missed.value), int(moved.value), g


def mask_range_query(index, queries, radius: float, stream=None):
    """Range search (Algorithm 3): per query, (ids, squared distances) of the
    points found within `radius`, ascending.  Sizes the output with a first
    counting call, then fills it."""
    Q, pq = _arr(queries, "float32")
    nq = Q.shape[0]
    counts = np.zeros(nq, dtype=np.int64)
    lib = load()
    st = _stream(Q, stream)
    _check(lib.mask_range_query(_handle(index), pq, nq, float(radius), counts.ctypes.data, 0,
                                None, None, st), "mask_range_query")
    total = int(counts.sum())
    ids, pids = _empty_like_kind(Q, (max(total, 1),), "int64")
    dists, pd = _empty_like_kind(Q, (max(total, 1),), "float32")
    _check(lib.mask_range_query(_handle(index), pq, nq, float(radius), counts.ctypes.data,
                                total, pids, pd, st), "mask_range_query")
    offs = np.concatenate([[0], np.cumsum(counts)])
    return [(ids[offs[q]:offs[q + 1]], dists[offs[q]:offs[q + 1]]) for q in range(nq)]


def mask_insert(index, points, stream=None):
    """Insert points (§3.3): returns the leaf cluster each new point joined."""
    X, px = _arr(points, "float32")
    n_new = X.shape[0]
    leaf, pl = _empty_like_kind(X, (n_new,), "int32")
    _check(load().mask_insert(_handle(index), px, n_new, pl, _stream(X, stream)), "mask_insert")
    return leaf


def mask_merge_topk(ids, dists, id_offset=None, stream=None):
    """Merge per-partition k-NN lists ([G x nq x k]) into the k nearest over
    all partitions (§3.4); id_offset [G] turns local ids into global ones."""
    I, pi = _arr(ids, "int64")
    D, pd = _arr(dists, "float32")
    G, nq, k = I.shape
    off, po = (None, None) if id_offset is None else _arr(id_offset, "int64")
    out_i, poi = _empty_like_kind(I, (nq, k), "int64")
    out_d, pod = _empty_like_kind(I, (nq, k), "float32")
    _check(load().mask_merge_topk(pi, pd, G, nq, k, po, poi, pod, _stream(I, stream)),
           "mask_merge_topk")
    return out_i, out_d


def mask_kmeanspp(X, k: int, seed: int, level: int = 0, stream=None):
    X, px = _arr(X, "float32")
    n, d = X.shape
    cen, pc = _empty_like_kind(X, (k, d), "float32")
    chosen = np.empty(k, dtype=np.int64)
    _check(load().mask_kmeanspp(px, n, d, k, seed & 0xFFFFFFFFFFFFFFFF, level, pc,
                                chosen.ctypes.data, _stream(X, stream)), "mask_kmeanspp")
    return cen, chosen


def mask_kmeans_assign(X, Cc, with_dist: bool = True, stream=None):
    X, px = _arr(X, "float32")
    Cc, pc = _arr(Cc, "float32")
    n, d = X.shape
    lab, pl = _empty_like_kind(X, (n,), "int32")
    dist, pd = _empty_like_kind(X, (n,), "float32") if with_dist else (None, None)
    _check(load().mask_kmeans_assign(px, n, d, pc, Cc.shape[0], pl, pd, _stream(X, stream)),
           "mask_kmeans_assign")
    return lab, dist


def _noalloc_args(X, Cc, labels_out, dist_out):
    """Checks what the C side cannot see (shapes, dtypes, layout, device) and
    raises ValueError instead of converting: a cast or a contiguous copy would
    allocate, which is what this entry point exists to avoid."""
    import torch

    def need(cond, msg):
        if not cond:
            raise ValueError("mask_kmeans_assign_noalloc: " + msg)

    arrays = {"X": X, "Cc": Cc, "labels_out": labels_out}
    if dist_out is not None:
        arrays["dist_out"] = dist_out
    for name, t in arrays.items():
        need(isinstance(t, torch.Tensor), f"{name} must be a torch tensor")
        need(t.is_cuda, f"{name} must be a CUDA tensor")
        need(t.is_contiguous(), f"{name} must be contiguous")
    need(X.dtype == torch.float32 and Cc.dtype == torch.float32, "X and Cc must be float32")
    need(X.dim() == 2 and Cc.dim() == 2, "X and Cc must be 2-D")
    need(Cc.shape[1] == X.shape[1], f"Cc has {Cc.shape[1]} columns, X has {X.shape[1]}")
    n = X.shape[0]
    need(labels_out.dtype == torch.int32, "labels_out must be int32")
    need(labels_out.numel() >= n, f"labels_out holds {labels_out.numel()} < {n} rows")
    if dist_out is not None:
        need(dist_out.dtype == torch.float32, "dist_out must be float32")
        need(dist_out.numel() >= n, f"dist_out holds {dist_out.numel()} < {n} rows")
    devs = {t.device for t in arrays.values()}
    need(len(devs) == 1, f"all tensors must be on one device, got {sorted(map(str, devs))}")


def mask_kmeans_assign_noalloc(X, Cc, labels_out, dist_out=None, stream=None):
    """Allocation-free assignment for callers that cannot let the library
    allocate: every array (inputs and the caller-provided outputs) must be a
    contiguous CUDA tensor on one device (X, Cc float32 [n x d] / [k x d];
    labels_out int32 [>= n]; dist_out float32 [>= n] or None); d a multiple of
    8; k <= 65536.  Anything else raises ValueError before the C call."""
    _noalloc_args(X, Cc, labels_out, dist_out)
    import torch
    with torch.cuda.device(X.device):
        _check(load().mask_kmeans_assign_noalloc(
            X.data_ptr(), X.shape[0], X.shape[1], Cc.data_ptr(), Cc.shape[0],
            labels_out.data_ptr(), None if dist_out is None else dist_out.data_ptr(),
            _stream(X, stream)), "mask_kmeans_assign_noalloc")
    return labels_out, dist_out


def mask_kmeans_update(X, labels, C_prev, stream=None):
    X, px = _arr(X, "float32")
    lb, pl = _arr(labels, "int32")
    Cp, pc = _arr(C_prev, "float32")
    n, d = X.shape
    k = Cp.shape[0]
    Cn, pn = _empty_like_kind(X, (k, d), "float32")
    cnt, pcnt = _empty_like_kind(X, (k,), "int64")
    _check(load().mask_kmeans_update(px, n, d, pl, k, pc, pn, pcnt, _stream(X, stream)),
           "mask_kmeans_update")
    return Cn, cnt


def _csr(row_ptr, col, val):
    rp, prp = _arr(row_ptr, "int64")
    cl, pcl = _arr(col, "int32")
    vl, pvl = _arr(val, "float32")
    return (rp, cl, vl), (prp, pcl, pvl), len(rp) - 1


def mask_kmeanspp_csr(row_ptr, col, val, n_cols: int, k: int, seed: int, level: int = 0,
                      stream=None):
    (rp, _, vl), (prp, pcl, pvl), n = _csr(row_ptr, col, val)
    cen, pc = _empty_like_kind(rp, (k, n_cols), "float32")
    chosen = np.empty(k, dtype=np.int64)
    _check(load().mask_kmeanspp_csr(prp, pcl, pvl, n, n_cols, k, seed & 0xFFFFFFFFFFFFFFFF, level,
                                    pc, chosen.ctypes.data, _stream(rp, stream)),
           "mask_kmeanspp_csr")
    return cen, chosen


def mask_kmeans_assign_csr(row_ptr, col, val, n_cols: int, Cc, with_dist: bool = True,
                           stream=None):
    (rp, _, vl), (prp, pcl, pvl), n = _csr(row_ptr, col, val)
    Cc, pc = _arr(Cc, "float32")
    lab, pl = _empty_like_kind(rp, (n,), "int32")
    dist, pd = _empty_like_kind(rp, (n,), "float32") if with_dist else (None, None)
    _check(load().mask_kmeans_assign_csr(prp, pcl, pvl, n, n_cols, pc, Cc.shape[0], pl, pd,
                                         _stream(rp, stream)), "mask_kmeans_assign_csr")
    return lab, dist


def mask_kmeans_update_csr(row_ptr, col, val, n_cols: int, labels, C_prev, stream=None):
    (rp, _, vl), (prp, pcl, pvl), n = _csr(row_ptr, col, val)
    lb, pl = _arr(labels, "int32")
    Cp, pc = _arr(C_prev, "float32")
    k = Cp.shape[0]
    Cn, pn = _empty_like_kind(rp, (k, n_cols), "float32")
    cnt, pcnt = _empty_like_kind(rp, (k,), "int64")
    _check(load().mask_kmeans_update_csr(prp, pcl, pvl, n, n_cols, pl, k, pc, pn, pcnt,
                                         _stream(rp, stream)), "mask_kmeans_update_csr")
    return Cn, cnt


# ------------------------------------------------------------------ serving

class Server:
    """Continuous-batching query service over a resident dense index (host
    queries in, host ids/dists out).  submit() returns a Ticket whose
    result() waits for the answer."""

    def __init__(self, index, mem_budget: int, max_slots: int = 4, max_batch: int = 4096):
        self._index = index          # the index must outlive the server
        self._live = {}              # ticket -> arrays the worker writes into
        out = C.c_void_p()
        _check(load().mask_server_open(_handle(index), int(mem_budget), max_slots, max_batch,
                                       C.byref(out)), "mask_server_open")
        self.handle = out

    def submit(self, queries, k: int, probes, precision: int = MASK_FP32) -> "Ticket":
        Q = np.ascontiguousarray(queries, dtype=np.float32)
        nq = Q.shape[0]
        pr, pp = _host_i32(probes)
        ids = np.empty((nq, k), dtype=np.int64)
        dists = np.empty((nq, k), dtype=np.float32)
        t = C.c_uint64()
        _check(load().mask_server_submit(self.handle, Q.ctypes.data, nq, k, pp, precision,
                                         ids.ctypes.data, dists.ctypes.data, C.byref(t)),
               "mask_server_submit")
        self._live[t.value] = (ids, dists)
        return Ticket(self, t.value, ids, dists)

    def stats(self, reset: bool = False) -> dict:
        info = mask_server_info()
        _check(load().mask_server_stats(self.handle, C.byref(info), 1 if reset else 0),
               "mask_server_stats")
        return info.as_dict()

    def close(self) -> None:
        """Finishes every queued request (their arrays are filled), then frees."""
        if self.handle and self.handle.value:
            load().mask_server_close(self.handle)
            self.handle = C.c_void_p(None)
            self._live.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ticket:
    def __init__(self, server: Server, ticket: int, ids, dists):
        self.server, self.ticket, self.ids, self.dists = server, ticket, ids, dists
        self.done = False

    def poll(self) -> bool:
        if self.done:
            return True
        st = load().mask_server_poll(self.server.handle, self.ticket)
        if st == MASK_PENDING:
            return False
        self.done = True
        self.server._live.pop(self.ticket, None)
        _check(st, "mask_server_poll")
        return True

    def result(self, timeout_ms: int = -1):
        if not self.done:
            st = load().mask_server_wait(self.server.handle, self.ticket, timeout_ms)
            if st == MASK_PENDING:
                raise TimeoutError("request still running")
            self.done = True
            self.server._live.pop(self.ticket, None)
            _check(st, "mask_server_wait")
        return self.ids, self.dists


# ------------------------------------------------------------ observability

def mask_profile_enable(on: bool = True) -> None:
    load().mask_profile_enable(1 if on else 0)


def mask_profile_reset() -> None:
    load().mask_profile_reset()


def mask_profile_read(name: str):
    """(launches, total_ms, work) for a region, or None if nothing recorded."""
    n, ms, w = C.c_int64(0), C.c_double(0.0), C.c_double(0.0)
    if not load().mask_profile_read(name.encode(), C.byref(n), C.byref(ms), C.byref(w)):
        return None
    return int(n.value), float(ms.value), float(w.value)


def mask_launch_count() -> int:
    return int(load().mask_launch_count())


def mask_test_alloc_count() -> int:
    return int(load().mask_test_alloc_count())


def mask_test_tc_mma_cycles(n: int, a_in_tmem: bool, n_acc: int, rounds: int):
    """(issue cycles, completion cycles) of rounds x 12 tcgen05 kind::f16 MMAs
    of M = 128, N = n, K = 16 on one SM (see include/mask.h)."""
    out = (C.c_int64 * 2)()
    _check(load().mask_test_tc_mma_cycles(int(n), 1 if a_in_tmem else 0, int(n_acc), int(rounds),
                                          C.cast(out, C.c_void_p)), "mask_test_tc_mma_cycles")
    return int(out[0]), int(out[1])


def mask_test_bounded_wait(flag_set: bool, limit_us: int, stream=None) -> str:
    """Run the library's bounded device wait on a flag that is set before the
    launch (flag_set) or never; returns the status name ("MASK_OK" or
    "MASK_ETIMEOUT") instead of raising for those two."""
    import torch
    if stream is None:
        st = torch.cuda.current_stream().cuda_stream
    else:
        st = stream if isinstance(stream, int) else stream.cuda_stream
    r = int(load().mask_test_bounded_wait(1 if flag_set else 0, int(limit_us), st))
    if r not in (0, -4):
        _check(r, "mask_test_bounded_wait")
    return _STATUS[r]
