"""Oracle for the Euclidean distance similarity self-join — TEST INFRASTRUCTURE.

Plain, slow, obviously correct CPU statement of what the join computes
(Sec. II-A, Eq. 1: every ordered pair (a, b) of V x V with dist(a, b) <= eps,
self pairs included as the selectivity of Sec. IV-A counts them).  Only the
tests, the smoke check and the CPU-baseline leg of the benchmark use it; the
CUDA library never imports, links or calls anything here, and nothing here
imports the CUDA library.

The arithmetic lives in ``sj_oracle.c`` (binary64, every operation rounded
separately, compiled with ``-ffp-contract=off``); this module builds it with
gcc and wraps it with ctypes.  A few helpers written in numpy are here too
(grid cell counts for the canonical candidate count, eps calibration); each
states the passage it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sj_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libsj_oracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FP contraction).  Returns the path."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _configure(lib):
    """Declare the C signatures on a loaded oracle library."""
    lib.sjo_threads.argtypes = [ctypes.c_int]
    lib.sjo_threads.restype = ctypes.c_int
    lib.sjo_count.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, _i64p, ctypes.c_int]
    lib.sjo_count.restype = ctypes.c_int64
    lib.sjo_join.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, _i64p, _i64p, _f64p,
                             ctypes.c_int]
    lib.sjo_join.restype = ctypes.c_int64
    lib.sjo_rows.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, _i64p, ctypes.c_int64,
                             _i64p, _i64p, _i64p, _f64p, ctypes.c_int]
    lib.sjo_rows.restype = ctypes.c_int64
    lib.sjo_sqdist_row.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, _f64p]
    lib.sjo_sqdist_row.restype = None
    lib.sjo_sqdist_dd.argtypes = [_f64p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _f64p, _f64p]
    lib.sjo_sqdist_dd.restype = None
    lib.sjo_is_borderline.argtypes = [_f64p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                      ctypes.c_double]
    lib.sjo_is_borderline.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
        return _lib


def _pts(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.ndim != 2:
        raise ValueError("points must be an n x d array")
    return x


def _p(a, t):
    return a.ctypes.data_as(t)


def threads(n: int = 0) -> int:
    """Threads the oracle uses for a request of ``n`` (0 = all host cores)."""
    return int(_load().sjo_threads(int(n)))


def count(x, eps: float, nthreads: int = 0, lib=None):
    """Per-query neighbour counts and |R| (Sec. II-A, Eq. 1, s <= fl(eps^2))."""
    x = _pts(x)
    n, d = x.shape
    c = np.zeros(n, dtype=np.int64)
    tot = (lib or _load()).sjo_count(_p(x, _f64p), n, d, float(eps), _p(c, _i64p), int(nthreads))
    return c, int(tot)


def join(x, eps: float, with_dist: bool = False, nthreads: int = 0, lib=None):
    """The whole result set as ascending 64-bit keys (i << 32) | j, plus the
    distances sqrt(s) when ``with_dist``.  Brute force over all n^2 pairs."""
    x = _pts(x)
    n, d = x.shape
    c, tot = count(x, eps, nthreads, lib)
    keys = np.empty(tot, dtype=np.int64)
    dist = np.empty(tot, dtype=np.float64) if with_dist else None
    w = (lib or _load()).sjo_join(_p(x, _f64p), n, d, float(eps), _p(c, _i64p), _p(keys, _i64p),
                         _p(dist, _f64p) if with_dist else None, int(nthreads))
    assert w == tot
    return (keys, dist) if with_dist else keys


def rows(x, eps: float, queries, with_dist: bool = False, nthreads: int = 0):
    """Result rows of selected queries: ascending keys of every (q, j) in R for
    q in ``queries`` (in the order given), one row per query."""
    x = _pts(x)
    n, d = x.shape
    q = np.ascontiguousarray(queries, dtype=np.int64)
    if q.size and (q.min() < 0 or q.max() >= n):
        raise ValueError("query index out of range")
    rc = np.zeros(q.size, dtype=np.int64)
    lib = _load()
    lib.sjo_rows(_p(x, _f64p), n, d, float(eps), _p(q, _i64p), q.size, _p(rc, _i64p), None, None, None,
                 int(nthreads))
    start = np.zeros(q.size + 1, dtype=np.int64)
    np.cumsum(rc, out=start[1:])
    keys = np.empty(int(start[-1]), dtype=np.int64)
    dist = np.empty(int(start[-1]), dtype=np.float64) if with_dist else None
    lib.sjo_rows(_p(x, _f64p), n, d, float(eps), _p(q, _i64p), q.size, _p(rc, _i64p), _p(start, _i64p),
                 _p(keys, _i64p), _p(dist, _f64p) if with_dist else None, int(nthreads))
    return (keys, dist, rc) if with_dist else (keys, rc)


def sqdist_row(x, q: int) -> np.ndarray:
    """Squared distances from point q to all points, oracle operation order."""
    x = _pts(x)
    n, d = x.shape
    out = np.empty(n, dtype=np.float64)
    _load().sjo_sqdist_row(_p(x, _f64p), n, d, int(q), _p(out, _f64p))
    return out


def sqdist_dd(x, i: int, j: int):
    """Squared distance of (i, j) as a double-double (hi, lo), error ~2^-100."""
    x = _pts(x)
    hi = ctypes.c_double()
    lo = ctypes.c_double()
    _load().sjo_sqdist_dd(_p(x, _f64p), x.shape[1], int(i), int(j), ctypes.byref(hi), ctypes.byref(lo))
    return hi.value, lo.value


def is_borderline(x, i: int, j: int, eps: float, rel: float = 1e-9) -> bool:
    """True iff the exact distance of (i, j) lies within a relative ``rel`` of eps."""
    x = _pts(x)
    return bool(_load().sjo_is_borderline(_p(x, _f64p), x.shape[1], int(i), int(j), float(eps), float(rel)))


def keys_to_pairs(keys: np.ndarray) -> np.ndarray:
    """(i, j) columns of 64-bit pair keys."""
    keys = np.asarray(keys, dtype=np.int64)
    return np.stack([keys >> 32, keys & 0xFFFFFFFF], axis=1)


def compare_pair_sets(x, eps: float, ref_keys, got_keys, rel: float = 1e-9):
    """Compare two sorted key sets; every key present in only one of them must
    be a borderline pair (exact distance within ``rel`` of eps).  Returns
    (n_only_ref, n_only_got, n_not_borderline)."""
    ref = np.asarray(ref_keys, dtype=np.int64)
    got = np.asarray(got_keys, dtype=np.int64)
    only_ref = np.setdiff1d(ref, got, assume_unique=False)
    only_got = np.setdiff1d(got, ref, assume_unique=False)
    bad = 0
    for k in np.concatenate([only_ref, only_got]):
        if not is_borderline(x, int(k) >> 32, int(k) & 0xFFFFFFFF, eps, rel):
            bad += 1
    return int(only_ref.size), int(only_got.size), bad


# --------------------------------------------------------------------------
# Grid candidate count (Sec. III-B: the grid of cells of side eps yields, for
# each query, the points of the adjacent cells as candidates to refine).
# --------------------------------------------------------------------------

def grid_cells(x, w: float, dims=None) -> np.ndarray:
    """Integer cell coordinates floor((x_k - lo_k) * (1 / w)) over the indexed
    dims, lo_k the minimum of dim k (binary64: 1 / w rounded once, then one
    subtraction and one product per coordinate)."""
    x = _pts(x)
    if dims is None:
        dims = list(range(x.shape[1]))
    sub = x[:, dims]
    lo = sub.min(axis=0)
    inv_w = 1.0 / float(w)
    return np.floor((sub - lo) * inv_w).astype(np.int64)


def grid_candidate_count(x, w: float, dims=None) -> int:
    """Number of (query, candidate) pairs the grid produces: for every point,
    the number of points lying in the 3^m cells whose coordinates differ from
    its own by at most one in every indexed dim (self included)."""
    cells = grid_cells(x, w, dims)
    n, m = cells.shape
    uniq, cnt = np.unique(cells, axis=0, return_counts=True)
    # dictionary lookup keyed by the tuple of coordinates (shifted by one)
    table = {tuple(int(v) for v in u + 1): int(c) for u, c in zip(uniq, cnt)}
    offs = np.array(np.meshgrid(*([[-1, 0, 1]] * m), indexing="ij")).reshape(m, -1).T
    total = 0
    for u, c in zip(uniq, cnt):
        base = u + 1
        s = 0
        for o in offs:
            s += table.get(tuple(int(v) for v in base + o), 0)
        total += int(c) * s
    return int(total)


def grid_candidate_count_fast(x, w: float, dims=None) -> int:
    """The same count as grid_candidate_count, vectorised over cells with
    numpy: each cell's coordinates are shifted by each of the 3^m offsets,
    encoded as integers and looked up in the sorted list of occupied cells."""
    cells = grid_cells(x, w, dims)
    n, m = cells.shape
    uniq, cnt = np.unique(cells, axis=0, return_counts=True)
    ext = uniq.max(axis=0) + 3
    strides = np.ones(m, dtype=np.int64)
    for k in range(m - 2, -1, -1):
        strides[k] = strides[k + 1] * ext[k + 1]
    codes = (uniq + 1) @ strides
    order = np.argsort(codes)
    codes_s, cnt_s = codes[order], cnt[order]
    offs = np.array(np.meshgrid(*([[-1, 0, 1]] * m), indexing="ij")).reshape(m, -1).T
    neigh = np.zeros(uniq.shape[0], dtype=np.int64)
    for o in offs:
        c = (uniq + 1 + o) @ strides
        pos = np.searchsorted(codes_s, c)
        pos_c = np.minimum(pos, codes_s.size - 1)
        hit = codes_s[pos_c] == c
        neigh += np.where(hit, cnt_s[pos_c], 0)
    return int((cnt.astype(np.int64) * neigh).sum())


def calibrate_eps(x, target: float, n_queries: int = 2000, seed: int = 12345) -> float:
    """eps whose mean neighbour count, self excluded (the selectivity s of
    Sec. IV-A), over ``n_queries`` seeded sample queries equals ``target``:
    pool the squared distances from the sampled queries to all other points
    (oracle order) and take the sqrt of the (target * n_queries)-th smallest."""
    x = _pts(x)
    n = x.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    nq = min(n_queries, n)
    qs = rng.choice(n, size=nq, replace=False)
    k = int(round(target * nq))
    pooled = []
    for q in qs:
        r = sqdist_row(x, int(q))
        r[q] = np.inf  # self excluded
        # only the k smallest of each row can matter for the pooled k-th value
        kk = min(k, n - 1)
        pooled.append(np.partition(r, kk - 1)[:kk] if kk > 0 else r[:0])
    allv = np.concatenate(pooled)
    s = np.partition(allv, k - 1)[k - 1]
    return float(np.sqrt(s))


# --------------------------------------------------------------------------
# DBSCAN on the join's result (reuse of the self-join for density-based
# clustering, which the paper names as future work for its join, Sec. V).
# Definition followed (Ester et al. 1996, stated on the eps-neighbourhoods
# the self-join returns): a point is core iff its neighbourhood (itself
# included) holds at least min_pts points; clusters are the connected
# components of the graph whose vertices are the core points and whose edges
# are the core-core pairs of the join; a non-core point with at least one
# core neighbour is a border point and joins, of its core neighbours'
# clusters, the one with the smallest identifier; the rest is noise (-1).
# A cluster's identifier is its rank among all clusters ordered by their
# smallest core point index.
# --------------------------------------------------------------------------

def dbscan(x, eps: float, min_pts: int):
    """Labels (n int64, -1 for noise) and the number of clusters."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    x = _pts(x)
    n = x.shape[0]
    keys = join(x, eps)
    i = keys >> 32
    j = keys & 0xFFFFFFFF
    deg = np.bincount(i, minlength=n)
    core = deg >= int(min_pts)
    cc = core[i] & core[j]
    g = coo_matrix((np.ones(int(cc.sum()), dtype=np.int8), (i[cc], j[cc])), shape=(n, n))
    _, comp = connected_components(g, directed=False)
    # cluster identifier: rank of the component's smallest core index
    first = np.full(comp.max() + 1 if n else 0, n, dtype=np.int64)
    core_idx = np.nonzero(core)[0]
    np.minimum.at(first, comp[core_idx], core_idx)
    roots = np.unique(first[comp[core_idx]]) if core_idx.size else np.zeros(0, dtype=np.int64)
    rank = {int(r): k for k, r in enumerate(roots.tolist())}
    labels = np.full(n, -1, dtype=np.int64)
    for p in core_idx.tolist():
        labels[p] = rank[int(first[comp[p]])]
    # border points: the smallest cluster identifier among core neighbours
    bm = (~core[i]) & core[j]
    if bm.any():
        bi, bj = i[bm], j[bm]
        cand = labels[bj]
        best = np.full(n, np.iinfo(np.int64).max, dtype=np.int64)
        np.minimum.at(best, bi, cand)
        hit = best != np.iinfo(np.int64).max
        labels[hit] = best[hit]
    return labels, int(roots.size)
