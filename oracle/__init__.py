"""FP64 CPU oracle for the A-tSNE similarity path -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / reference leg import this package. It shares no code with
the CUDA library and the library never calls it. Each wrapper below names the
passage of the paper its C function follows (see atsne_oracle.c).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_vp = ctypes.c_void_p
_i32, _i64, _u64, _f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_num_threads.restype = ctypes.c_int
        L.oracle_set_num_threads.argtypes = [ctypes.c_int]
        L.oracle_knn_exact.argtypes = [_f32p, _i64, _i32, _vp, _i64, _i32, _i32p, _f64p]
        L.oracle_calibrate.argtypes = [_f64p, _i64, _i32, _f64, _f64, _i32, _f64p, _f64p, _f64p,
                                       _i32p]
        L.oracle_symmetrize.argtypes = [_i32p, _f64p, _i64, _i32, _i64p, _i32p, _f64p,
                                        ctypes.POINTER(_i64)]
        L.oracle_precision.argtypes = [_i32p, _i32p, _i64, _i32, _f64p, ctypes.POINTER(_f64)]
        L.oracle_splitmix64_at.restype = _u64
        L.oracle_splitmix64_at.argtypes = [_u64, _u64]
        L.oracle_forest_depth.restype = _i32
        L.oracle_forest_depth.argtypes = [_i64, _i32]
        L.oracle_forest_leaf_offsets.argtypes = [_i64, _i32, _i64p]
        L.oracle_forest_build.argtypes = [_f32p, _i64, _i32, _i32, _i32, _i32, _u64, _i32p, _f32p,
                                          _i32p, _i64p]
        L.oracle_forest_query.argtypes = [_f32p, _i64, _i32, _i32, _i32, _i32p, _f32p, _i32p,
                                          _i64p, _vp, _i64, _i32, _i32, _i32, _i32p, _f64p, _i64p]
        L.oracle_forest_query_ex.argtypes = [_f32p, _i64, _i32, _i32, _i32, _i32p, _f32p, _i32p,
                                             _i64p, _i64, _vp, _i64, _i32, _i32, _i32, _i32p, _f64p,
                                             _i64p]
        L.oracle_forest_insert.argtypes = [_f32p, _i64, _i64, _i32, _i32, _i32, _i32p, _f32p, _vp,
                                           _vp, _i32p, _i64p]
        L.oracle_forest_delete.argtypes = [_i64, _i32, _i32, _i32p, _i64p, _vp, _i64, _i32p, _i64p]
        L.oracle_kde.argtypes = [_f32p, _i64, _vp, _vp, _f64, _f64, _f64, _i32, _i32, _f64, _f64,
                                 _f64, _f64p, _f64p, _f64p, _f64p]
        L.oracle_knn_cross.argtypes = [_f32p, _i64, _f32p, _i64, _i32, _i32, _i32p, _f64p]
        L.oracle_insert.argtypes = [_f32p, _i64, _i64, _i32, _i32, _i32p, _f64p,
                                    np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")]
        L.oracle_refine.argtypes = [_f32p, _i64, _i32, _i32p, _i64, _i32, _f64, _f64, _i32, _i32p,
                                    _f64p, _f64p, _f64p, _f64p]
        L.oracle_delete.argtypes = [_f32p, _i64, _i32, _i32p, _i64, _i32, _f64, _f64, _i32, _i32p,
                                    _f64p, _f64p, _f64p, _f64p, ctypes.POINTER(_i64)]
        _lib = L
    return _lib


def num_threads() -> int:
    return lib().oracle_num_threads()


def set_num_threads(n: int) -> None:
    lib().oracle_set_num_threads(int(n))


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle %s failed (status %d)" % (what, rc))


def _queries(queries):
    if queries is None:
        return None, None, 0
    q = np.ascontiguousarray(queries, dtype=np.int32)
    return q, q.ctypes.data_as(_vp), q.shape[0]


def knn_exact(X, k, queries=None):
    """Exact kNN, Eq. 8: (idx int32 [Q,k], d2 float64 [Q,k]) sorted by (d2, idx)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    N, D = X.shape
    q, qp, S = _queries(queries)
    Q = S if q is not None else N
    idx = np.empty((Q, k), np.int32)
    d2 = np.empty((Q, k), np.float64)
    _check(lib().oracle_knn_exact(X, N, D, qp, S, k, idx, d2), "knn_exact")
    return idx, d2


def calibrate(d2, perplexity, tol=1e-10, max_iter=200):
    """Bisection on beta, Eq. 3-4: (P [R,k], beta [R], perp [R], iters [R])."""
    d2 = np.ascontiguousarray(d2, dtype=np.float64)
    R, k = d2.shape
    P = np.empty((R, k), np.float64)
    beta = np.empty(R, np.float64)
    perp = np.empty(R, np.float64)
    iters = np.empty(R, np.int32)
    _check(lib().oracle_calibrate(d2, R, k, float(perplexity), float(tol), int(max_iter), P, beta,
                                  perp, iters), "calibrate")
    return P, beta, perp, iters


def symmetrize(idx, P):
    """(P + P^T)/2N as CSR, Eq. 2 / Eq. 10: (row_ptr int64, col int32, val float64)."""
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    P = np.ascontiguousarray(P, dtype=np.float64)
    N, k = idx.shape
    row_ptr = np.empty(N + 1, np.int64)
    col = np.empty(2 * N * k, np.int32)
    val = np.empty(2 * N * k, np.float64)
    nnz = _i64(0)
    _check(lib().oracle_symmetrize(idx, P, N, k, row_ptr, col, val, ctypes.byref(nnz)),
           "symmetrize")
    return row_ptr, col[:nnz.value].copy(), val[:nnz.value].copy()


def precision(idx_a, idx_e):
    """Eq. 9: (rho_i float64 [R], rho float)."""
    idx_a = np.ascontiguousarray(idx_a, dtype=np.int32)
    idx_e = np.ascontiguousarray(idx_e, dtype=np.int32)
    R, k = idx_a.shape
    rho_i = np.empty(R, np.float64)
    mean = _f64(0.0)
    _check(lib().oracle_precision(idx_a, idx_e, R, k, rho_i, ctypes.byref(mean)), "precision")
    return rho_i, mean.value


def splitmix64_at(seed, c):
    return int(lib().oracle_splitmix64_at(seed & (2**64 - 1), c & (2**64 - 1)))


def forest_depth(N, leaf_size):
    return int(lib().oracle_forest_depth(N, leaf_size))


def forest_leaf_offsets(N, h):
    ofs = np.empty((1 << h) + 1, np.int64)
    _check(lib().oracle_forest_leaf_offsets(N, h, ofs), "forest_leaf_offsets")
    return ofs


def forest_build(X, trees, top_var_dims=5, leaf_size=1, seed=0):
    """Randomized KD-forest, Sec. 4.2. Returns a dict of the level-ordered arrays."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    N, D = X.shape
    h = forest_depth(N, leaf_size)
    n_int = (1 << h) - 1
    split_dim = np.empty((trees, max(n_int, 1)), np.int32)
    split_val = np.empty((trees, max(n_int, 1)), np.float32)
    perm = np.empty((trees, N), np.int32)
    leaf_ofs = np.empty((1 << h) + 1, np.int64)
    _check(lib().oracle_forest_build(X, N, D, trees, top_var_dims, leaf_size, seed, split_dim,
                                     split_val, perm, leaf_ofs), "forest_build")
    return dict(N=N, D=D, trees=trees, depth=h, leaf_size=leaf_size, seed=seed,
                top_var_dims=top_var_dims, split_dim=split_dim[:, :n_int],
                split_val=split_val[:, :n_int], perm=perm, leaf_ofs=leaf_ofs)


def auto_queue_cap(checks):
    """Default queue capacity: checks/2 rounded up to a power of two, in [256, 4096]."""
    q = 256
    while q < checks // 2 and q < 4096:
        q <<= 1
    return q


def forest_query(X, forest, k, checks, qcap=None, queries=None):
    """Forest search, Sec. 4.2: (idx [Q,k], d2 float64 [Q,k], evaluated [Q]).
    qcap None selects the default capacity auto_queue_cap(checks). The forest's
    leaf offsets are one array for all trees ([2^h + 1], as built) or one per
    tree ([T][2^h + 1], after points were added or removed)."""
    if qcap is None:
        qcap = auto_queue_cap(checks)
    X = np.ascontiguousarray(X, dtype=np.float32)
    N, D = X.shape
    T, h = forest["trees"], forest["depth"]
    n_int = (1 << h) - 1
    sd = np.zeros((T, max(n_int, 1)), np.int32)
    sv = np.zeros((T, max(n_int, 1)), np.float32)
    sd[:, :n_int] = forest["split_dim"]
    sv[:, :n_int] = forest["split_val"]
    q, qp, S = _queries(queries)
    Q = S if q is not None else N
    idx = np.empty((Q, k), np.int32)
    d2 = np.empty((Q, k), np.float64)
    ev = np.empty(Q, np.int64)
    ofs = np.ascontiguousarray(forest["leaf_ofs"], dtype=np.int64)
    stride = ofs.shape[1] if ofs.ndim == 2 else 0
    if ofs.shape[-1] != (1 << h) + 1 or (stride and ofs.shape[0] != T):
        raise ValueError("leaf offsets do not match the forest")
    _check(lib().oracle_forest_query_ex(X, N, D, T, h, sd, sv, np.ascontiguousarray(forest["perm"]),
                                        ofs, stride, qp, S, k, int(checks), int(qcap), idx, d2, ev),
           "forest_query")
    return idx, d2, ev


def _tree_offsets(forest):
    ofs = np.asarray(forest["leaf_ofs"], dtype=np.int64)
    if ofs.ndim == 1:
        ofs = np.broadcast_to(ofs, (forest["trees"], ofs.shape[0]))
    return np.ascontiguousarray(ofs)


def forest_insert(forest, X, n_old):
    """Sec. 5.3.1: rows n_old .. N-1 of X join every tree of `forest` (built or
    updated over the first n_old rows) by a descent to a leaf; returns the new
    forest (per-tree leaf offsets, perm [T][N])."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    N, D = X.shape
    T, h = forest["trees"], forest["depth"]
    n_int = (1 << h) - 1
    sd = np.ascontiguousarray(np.asarray(forest["split_dim"], np.int32).reshape(T, n_int))
    sv = np.ascontiguousarray(np.asarray(forest["split_val"], np.float32).reshape(T, n_int))
    if n_int == 0:
        sd, sv = np.zeros((T, 1), np.int32), np.zeros((T, 1), np.float32)
    perm_in = np.ascontiguousarray(forest["perm"], dtype=np.int32)
    ofs_in = _tree_offsets(forest)
    perm = np.empty((T, N), np.int32)
    ofs = np.empty((T, (1 << h) + 1), np.int64)
    _check(lib().oracle_forest_insert(X, int(n_old), N, D, T, h, sd, sv,
                                      perm_in.ctypes.data if n_old > 0 else None,
                                      ofs_in.ctypes.data if n_old > 0 else None, perm, ofs),
           "forest_insert")
    out = dict(forest)
    out.update(N=N, perm=perm, leaf_ofs=ofs)
    return out


def forest_delete(forest, rows):
    """Sec. 5.3.2: the listed points leave every tree; the remaining ones are
    renumbered as the corpus rows are. Returns the new forest."""
    T, h = forest["trees"], forest["depth"]
    perm_in = np.ascontiguousarray(forest["perm"], dtype=np.int32)
    N = perm_in.shape[1]
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    perm = np.empty((T, N - rows.shape[0]), np.int32)
    ofs = np.empty((T, (1 << h) + 1), np.int64)
    _check(lib().oracle_forest_delete(N, T, h, perm_in, _tree_offsets(forest),
                                      rows.ctypes.data if rows.shape[0] else None, rows.shape[0],
                                      perm, ofs), "forest_delete")
    out = dict(forest)
    out.update(N=N - rows.shape[0], perm=perm, leaf_ofs=ofs)
    return out


def refine(X, subset, k, perplexity, idx, d2, P, beta, rho, tol=1e-10, max_iter=200):
    """Exact refinement of the listed rows, Sec. 4.3 / 5.1.1; updates the arrays in place."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    N, D = X.shape
    subset = np.ascontiguousarray(subset, dtype=np.int32)
    for a, dt in ((idx, np.int32), (d2, np.float64), (P, np.float64), (beta, np.float64),
                  (rho, np.float64)):
        if a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("refine state arrays must be C-contiguous %s" % dt)
    _check(lib().oracle_refine(X, N, D, subset, subset.shape[0], k, float(perplexity), float(tol),
                               int(max_iter), idx, d2, P, beta, rho), "refine")


def kde(Y, x0, y0, pixel, width, height, h, cutoff=4.0, k=2.0, rho=None, selected=None):
    """Density view and approximation map, Eq. 12, Eq. 13, Sec. 5.2.2.
    Returns f, s, a, alpha as float64 [height][width]."""
    Y = np.ascontiguousarray(Y, dtype=np.float32)
    N = Y.shape[0]
    r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float32)
    sl = None if selected is None else np.ascontiguousarray(selected, dtype=np.uint8)
    out = [np.empty((height, width), np.float64) for _ in range(4)]
    _check(lib().oracle_kde(Y, N, None if r is None else r.ctypes.data_as(_vp),
                            None if sl is None else sl.ctypes.data_as(_vp), x0, y0, pixel, width,
                            height, h, cutoff, k, *out), "kde")
    return tuple(out)


def knn_cross(Xq, Xc, k):
    """The k nearest rows of Xc for each row of Xq (Eq. 8 across two sets)."""
    Xq = np.ascontiguousarray(Xq, dtype=np.float32)
    Xc = np.ascontiguousarray(Xc, dtype=np.float32)
    idx = np.empty((Xq.shape[0], k), np.int32)
    d2 = np.empty((Xq.shape[0], k), np.float64)
    _check(lib().oracle_knn_cross(Xq, Xq.shape[0], Xc, Xc.shape[0], Xq.shape[1], k, idx, d2),
           "knn_cross")
    return idx, d2


def delete(X, rows, k, perplexity, idx, d2, P, beta, rho, tol=1e-10, max_iter=200):
    """Deletion of the listed points, Sec. 5.3.2, on copies of the state:
    returns (X, idx, d2, P, beta, rho) over the N - R remaining points."""
    X = np.array(X, dtype=np.float32, order="C", copy=True)
    N, D = X.shape
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    st = [np.array(a, dtype=dt, order="C", copy=True)
          for a, dt in ((idx, np.int32), (d2, np.float64), (P, np.float64), (beta, np.float64),
                        (rho, np.float64))]
    n = _i64(0)
    _check(lib().oracle_delete(X, N, D, rows, rows.shape[0], k, float(perplexity), float(tol),
                               int(max_iter), *st, ctypes.byref(n)), "delete")
    n = n.value
    return (X[:n],) + tuple(a[:n] for a in st)


def insert(X, n_old, idx, d2):
    """Eq. 11 (Sec. 5.3.1) on copies of the state: rows n_old.. of X are new
    points; each of the first n_old rows takes the new points strictly closer
    than its farthest present neighbour. Returns (idx, d2, changed)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    N, D = X.shape
    idx = np.array(idx, dtype=np.int32, order="C", copy=True)
    d2 = np.array(d2, dtype=np.float64, order="C", copy=True)
    k = idx.shape[1]
    changed = np.zeros(n_old, np.uint8)
    _check(lib().oracle_insert(X, int(n_old), N, D, k, idx, d2, changed), "insert")
    return idx, d2, changed.astype(bool)
