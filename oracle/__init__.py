"""FP64 CPU oracle for the MASK hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
and never imports it.  The arithmetic lives in ``mask_oracle.c`` (plain C,
FP64, OpenMP over independent points/queries); this module compiles it with
gcc on first use and marshals numpy arrays through ctypes.

Functions follow the paper (Ortega et al., arXiv 2208.02734):
  seed_level / kmeanspp  -- k-means++ seeding (§3.2), readings R1-R3
  assign / update / lloyd / objective -- Lloyd's k-means (§2.4, Algorithm 1)
  build                  -- multilevel index, global form of Algorithm 1 (§3.1)
  query                  -- top-down k-NN descent (§3.3, Algorithm 2)
  bruteforce_knn         -- exact k-NN by full scan (ground truth)
  grouped_sizes / build_grouped -- Algorithm 1 as printed: random split into
                            groups of lengthGroup, nCentroids per group (§3.1)
  descend                -- the kept leaf clusters of the descent
  range_query            -- range search (§3.3, Algorithm 3)
  relocate               -- one point-relocation pass of §4.1
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mask_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_u64ref = C.POINTER(C.c_uint64)


def compile_lib(force: bool = False) -> str:
    """Compile mask_oracle.c into liboracle.so (gcc, -O2, OpenMP)."""
    stale = (not os.path.exists(_LIB)
             or os.path.getmtime(_LIB) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-std=c11", "-O2", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        try:
            subprocess.run(base[:3] + ["-fopenmp"] + base[3:], check=True,
                           capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(compile_lib())
        sig = {
            "mo_set_threads": (None, [C.c_int32]),
            "mo_max_threads": (C.c_int32, []),
            "mo_splitmix64_next": (C.c_uint64, [_u64ref]),
            "mo_uniform": (C.c_double, [_u64ref]),
            "mo_level_state": (C.c_uint64, [C.c_uint64, C.c_int32]),
            "mo_sqdist_rows": (None, [_f64p, C.c_int32, _i64p, C.c_int64, _f64p, _f64p]),
            "mo_kmeanspp": (C.c_int32, [_f64p, C.c_int64, C.c_int32, C.c_int32, _u64ref,
                                        _i64p, _f64p]),
            "mo_subsample": (C.c_int32, [C.c_int64, C.c_int64, _u64ref, _i64p]),
            "mo_seed_sample_size": (C.c_int64, [C.c_int64, C.c_int32]),
            "mo_seed_level": (C.c_int32, [_f64p, C.c_int64, C.c_int32, C.c_int32, C.c_uint64,
                                          C.c_int32, _i64p, _f64p]),
            "mo_assign": (None, [_f64p, C.c_int64, C.c_int32, _f64p, C.c_int32, _i32p, _f64p]),
            "mo_update": (C.c_int32, [_f64p, C.c_int64, C.c_int32, _i32p, C.c_int32, _f64p,
                                      _i64p]),
            "mo_objective": (C.c_double, [_f64p, C.c_int64, C.c_int32, _f64p, _i32p]),
            "mo_lloyd": (C.c_int32, [_f64p, C.c_int64, C.c_int32, C.c_int32, C.c_int32, _f64p,
                                     _i32p, _f64p]),
            "mo_build": (C.c_int32, [_f64p, C.c_int64, C.c_int32, _i32p, C.c_int32, C.c_int32,
                                     C.c_uint64, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                     C.POINTER(C.c_void_p)]),
            "mo_query": (C.c_int32, [_f64p, C.c_int64, C.c_int32, C.c_int32, _i32p,
                                     C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), _f64p,
                                     C.c_int64, C.c_int32, _i32p, _i64p, _f64p, C.c_double,
                                     _u8p]),
            "mo_bruteforce_knn": (C.c_int32, [_f64p, C.c_int64, C.c_int32, _f64p, C.c_int64,
                                              C.c_int32, _i64p, _f64p]),
            "mo_grouped_sizes": (C.c_int32, [C.c_int64, C.c_int32, C.c_int32, _i64p, C.c_int32]),
            "mo_group_state": (C.c_uint64, [C.c_uint64, C.c_int32, C.c_int64]),
            "mo_split_groups": (C.c_int32, [C.c_int64, C.c_int64, _u64ref, _i32p]),
            "mo_build_grouped": (C.c_int32, [_f64p, C.c_int64, C.c_int32, C.c_int32, C.c_int32,
                                             C.c_int32, C.c_uint64, C.c_void_p, C.c_int32,
                                             C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]),
            "mo_descend": (C.c_int32, [C.c_int64, C.c_int32, C.c_int32, _i32p,
                                       C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), _f64p,
                                       C.c_int64, _i32p, _i32p]),
            "mo_range_query": (C.c_int32, [_f64p, C.c_int64, C.c_int32, C.c_int32, _i32p,
                                           C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), _f64p,
                                           C.c_int64, C.c_double, _i64p, C.c_int64, C.c_void_p,
                                           C.c_void_p]),
            "mo_relocate": (C.c_int64, [_f64p, C.c_int64, C.c_int32, C.c_int32, _i32p,
                                        C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int32,
                                        _i32p, C.POINTER(C.c_int64)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def set_threads(t: int) -> None:
    _load().mo_set_threads(int(t))


def max_threads() -> int:
    return int(_load().mo_max_threads())


class SplitMix64:
    """SplitMix64 stream (reading R1), for pinning the generator itself."""

    def __init__(self, state: int):
        self.state = C.c_uint64(state & 0xFFFFFFFFFFFFFFFF)

    def next(self) -> int:
        return int(_load().mo_splitmix64_next(C.byref(self.state)))

    def uniform(self) -> float:
        return float(_load().mo_uniform(C.byref(self.state)))


def level_state(seed: int, level: int) -> int:
    return int(_load().mo_level_state(C.c_uint64(seed), int(level)))


def sqdist_rows(X, ids, q) -> np.ndarray:
    X = _f64(X)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    out = np.empty(len(ids))
    _load().mo_sqdist_rows(X, X.shape[1], ids, len(ids), _f64(q), out)
    return out


def kmeanspp(X, k: int, state: int):
    """k-means++ (R2) from an explicit RNG state; returns (chosen, C)."""
    X = _f64(X)
    n, d = X.shape
    chosen = np.empty(k, dtype=np.int64)
    Cc = np.empty((k, d))
    s = C.c_uint64(state)
    _check(_load().mo_kmeanspp(X, n, d, k, C.byref(s), chosen, Cc), "kmeanspp")
    return chosen, Cc


def subsample(n: int, m: int, state: int) -> np.ndarray:
    out = np.empty(m, dtype=np.int64)
    s = C.c_uint64(state)
    _check(_load().mo_subsample(n, m, C.byref(s), out), "subsample")
    return out


def seed_sample_size(n: int, k: int) -> int:
    return int(_load().mo_seed_sample_size(n, k))


def seed_level(X, k: int, seed: int, level: int):
    """Seeding of one level (R2, R3); returns (chosen indices into X, C)."""
    X = _f64(X)
    n, d = X.shape
    chosen = np.empty(k, dtype=np.int64)
    Cc = np.empty((k, d))
    _check(_load().mo_seed_level(X, n, d, k, C.c_uint64(seed), level, chosen, Cc),
           "seed_level")
    return chosen, Cc


def assign(X, Cc):
    X, Cc = _f64(X), _f64(Cc)
    labels = np.empty(X.shape[0], dtype=np.int32)
    dist = np.empty(X.shape[0])
    _load().mo_assign(X, X.shape[0], X.shape[1], Cc, Cc.shape[0], labels, dist)
    return labels, dist


def update(X, labels, Cprev):
    X = _f64(X)
    Cn = _f64(Cprev).copy()
    counts = np.empty(Cn.shape[0], dtype=np.int64)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    _check(_load().mo_update(X, X.shape[0], X.shape[1], labels, Cn.shape[0], Cn, counts),
           "update")
    return Cn, counts


def objective(X, Cc, labels) -> float:
    X, Cc = _f64(X), _f64(Cc)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    return float(_load().mo_objective(X, X.shape[0], X.shape[1], Cc, labels))


def lloyd(X, C0, iters: int):
    """Lloyd from C0; returns (C, labels, J_trace[2*iters+1])."""
    X = _f64(X)
    Cc = _f64(C0).copy()
    labels = np.empty(X.shape[0], dtype=np.int32)
    J = np.empty(2 * iters + 1)
    _check(_load().mo_lloyd(X, X.shape[0], X.shape[1], Cc.shape[0], iters, Cc, labels, J),
           "lloyd")
    return Cc, labels, J


class Index:
    """Oracle multilevel index: per level (finest first) centroids C[lv]
    (k_lv x d) and labels[lv] (the level-lv centroid of every item one level
    below), plus the seeding picks."""

    def __init__(self, X, centroids, labels, chosen=None):
        self.X = _f64(X)
        self.centroids = [_f64(c) for c in centroids]
        self.labels = [np.ascontiguousarray(lb, dtype=np.int32) for lb in labels]
        self.chosen = chosen

    @property
    def k_per_level(self):
        return [c.shape[0] for c in self.centroids]

    def query(self, Q, k: int, probes, tie_rtol: float = 1e-5):
        """k-NN descent; returns (ids, dists, sel_clear)."""
        return query(self, Q, k, probes, tie_rtol)


def build(X, k_per_level, iters: int, seed: int) -> Index:
    X = _f64(X)
    n, d = X.shape
    L = len(k_per_level)
    kp = np.ascontiguousarray(k_per_level, dtype=np.int32)
    Cs = [np.empty((int(k), d)) for k in kp]
    n_in = [n] + [int(k) for k in kp[:-1]]
    Ls = [np.empty(m, dtype=np.int32) for m in n_in]
    ch = [np.empty(int(k), dtype=np.int64) for k in kp]
    ptrs = lambda arrs: (C.c_void_p * L)(*[a.ctypes.data for a in arrs])  # noqa: E731
    _check(_load().mo_build(X, n, d, kp, L, iters, C.c_uint64(seed), ptrs(Cs), ptrs(Ls),
                            ptrs(ch)), "build")
    return Index(X, Cs, Ls, ch)


def query(index: Index, Q, k: int, probes, tie_rtol: float = 1e-5):
    Q = _f64(Q)
    nq = Q.shape[0]
    L = len(index.centroids)
    kp = np.ascontiguousarray(index.k_per_level, dtype=np.int32)
    pr = np.ascontiguousarray(probes, dtype=np.int32)
    if len(pr) != L:
        raise ValueError("one probe count per level")
    ids = np.empty((nq, k), dtype=np.int64)
    dists = np.empty((nq, k))
    clear = np.empty(nq, dtype=np.uint8)
    ptrs = lambda arrs: (C.c_void_p * L)(*[a.ctypes.data for a in arrs])  # noqa: E731
    _check(_load().mo_query(index.X, index.X.shape[0], index.X.shape[1], L, kp,
                            ptrs(index.centroids), ptrs(index.labels), Q, nq, k, pr, ids,
                            dists, tie_rtol, clear), "query")
    return ids, dists, clear.astype(bool)


def bruteforce_knn(X, Q, k: int):
    X, Q = _f64(X), _f64(Q)
    ids = np.empty((Q.shape[0], k), dtype=np.int64)
    dists = np.empty((Q.shape[0], k))
    _check(_load().mo_bruteforce_knn(X, X.shape[0], X.shape[1], Q, Q.shape[0], k, ids,
                                     dists), "bruteforce_knn")
    return ids, dists


# ------------------------------------------------ grouped build (Algorithm 1)

def grouped_sizes(n: int, length_group: int, n_centroids: int):
    """Centroids per level of the grouped build (finest first)."""
    sizes = np.empty(64, dtype=np.int64)
    L = _load().mo_grouped_sizes(n, length_group, n_centroids, sizes, 64)
    _check(0 if L >= 0 else L, "grouped_sizes")
    return [int(v) for v in sizes[:L]]


def group_state(seed: int, level: int, group: int) -> int:
    return int(_load().mo_group_state(C.c_uint64(seed), int(level), int(group)))


def split_groups(m: int, G: int, state: int) -> np.ndarray:
    """R16: the group of each of m items split at random into G groups."""
    out = np.empty(m, dtype=np.int32)
    s = C.c_uint64(state)
    _check(_load().mo_split_groups(m, G, C.byref(s), out), "split_groups")
    return out


def build_grouped(X, length_group: int, n_centroids: int, iters: int, seed: int,
                  group0=None) -> Index:
    """Algorithm 1 as printed (readings R16-R18); group0 replaces the random
    level-0 split (relocation, §4.1)."""
    X = _f64(X)
    n, d = X.shape
    sizes = grouped_sizes(n, length_group, n_centroids)
    L = len(sizes)
    if L == 0:
        raise ValueError("fewer points than lengthGroup: no level")
    Cs = [np.empty((k, d)) for k in sizes]
    n_in = [n] + sizes[:-1]
    Ls = [np.empty(m, dtype=np.int32) for m in n_in]
    ptrs = lambda arrs: (C.c_void_p * L)(*[a.ctypes.data for a in arrs])  # noqa: E731
    g0 = None if group0 is None else np.ascontiguousarray(group0, dtype=np.int32)
    _check(_load().mo_build_grouped(X, n, d, length_group, n_centroids, iters, C.c_uint64(seed),
                                    None if g0 is None else g0.ctypes.data, L, ptrs(Cs),
                                    ptrs(Ls)), "build_grouped")
    return Index(X, Cs, Ls)


def descend(index: Index, Q, probes) -> np.ndarray:
    """The kept leaf clusters of the descent, [nq x probes[0]], nearest first."""
    Q = _f64(Q)
    L = len(index.centroids)
    kp = np.ascontiguousarray(index.k_per_level, dtype=np.int32)
    pr = np.ascontiguousarray(probes, dtype=np.int32)
    out = np.empty((Q.shape[0], int(pr[0])), dtype=np.int32)
    ptrs = lambda arrs: (C.c_void_p * L)(*[a.ctypes.data for a in arrs])  # noqa: E731
    _check(_load().mo_descend(index.X.shape[0], index.X.shape[1], L, kp, ptrs(index.centroids),
                              ptrs(index.labels), Q, Q.shape[0], pr, out), "descend")
    return out


def range_query(index: Index, Q, radius: float):
    """Range search (Algorithm 3, reading R19): per query, (ids, squared
    distances) of the points found within `radius`, ascending."""
    Q = _f64(Q)
    nq = Q.shape[0]
    L = len(index.centroids)
    kp = np.ascontiguousarray(index.k_per_level, dtype=np.int32)
    counts = np.empty(nq, dtype=np.int64)
    ptrs = lambda arrs: (C.c_void_p * L)(*[a.ctypes.data for a in arrs])  # noqa: E731
    args = (index.X, index.X.shape[0], index.X.shape[1], L, kp, ptrs(index.centroids),
            ptrs(index.labels), Q, nq, float(radius) ** 2, counts)
    _check(_load().mo_range_query(*args, 0, None, None), "range_query")
    total = int(counts.sum())
    ids = np.empty(max(total, 1), dtype=np.int64)
    dists = np.empty(max(total, 1))
    _check(_load().mo_range_query(*args, total, ids.ctypes.data, dists.ctypes.data),
           "range_query")
    offs = np.concatenate([[0], np.cumsum(counts)])
    return [(ids[offs[q]:offs[q + 1]], dists[offs[q]:offs[q + 1]]) for q in range(nq)]


def relocate(index: Index, n_centroids: int, group0):
    """One relocation pass (§4.1, reading R20): returns (missed points, new
    group0, moves)."""
    L = len(index.centroids)
    kp = np.ascontiguousarray(index.k_per_level, dtype=np.int32)
    g = np.array(group0, dtype=np.int32, copy=True)
    moved = C.c_int64(0)
    ptrs = lambda arrs: (C.c_void_p * L)(*[a.ctypes.data for a in arrs])  # noqa: E731
    missed = _load().mo_relocate(index.X, index.X.shape[0], index.X.shape[1], L, kp,
                                 ptrs(index.centroids), ptrs(index.labels), n_centroids, g,
                                 C.byref(moved))
    if missed < 0:
        raise RuntimeError(f"oracle relocate failed with status {missed}")
    return int(missed), g, int(moved.value)


def point_query_error(index: Index) -> float:
    """Error rate of the exhaustive point query (§4.2): the fraction of the
    indexed points whose greedy descent does not reach their own leaf cluster."""
    leaf = descend(index, index.X, [1] * len(index.centroids))[:, 0]
    return float(np.mean(leaf != index.labels[0]))
