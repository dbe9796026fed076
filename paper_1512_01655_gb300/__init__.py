"""Python binding of the sm_103a A-tSNE similarity library (include/atsne.h).

Argument marshalling only: every step runs in the library's CUDA kernels.
PyTorch supplies device memory (outputs and workspaces) and the current CUDA
stream. There is no CPU fallback: if the compiled library is missing, or no
CUDA device is present, the calls raise.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libatsne.so")

ATSNE_OK, ATSNE_EINVAL, ATSNE_ENOMEM, ATSNE_ECUDA, ATSNE_ETIMEOUT, ATSNE_EUNSUPPORTED = range(6)
KNN_EXACT, KNN_FOREST = 0, 1
FP32, BF16_RERANK, FP32_CUDA_CORES, FP8_RERANK, BF16_RERANK_APPROX = 0, 1, 2, 3, 4
(OP_KNN, OP_CALIBRATE, OP_SYMMETRIZE, OP_REFINE, OP_FOREST_BUILD, OP_FOREST_QUERY,
 OP_REFINE_BATCH, OP_KNN_CROSS, OP_KNN_CROSS_RADIUS, OP_DELETE, OP_TUNE_KNN, OP_FOREST_UPDATE) = range(12)

EXPORTED = (
    "atsne_knn_opts_default", "atsne_workspace_bytes", "atsne_knn", "atsne_calibrate_P",
    "atsne_symmetrize", "atsne_refine_subset", "atsne_knn_precision", "atsne_forest_layout",
    "atsne_forest_build", "atsne_forest_query", "atsne_check", "atsne_last_error",
    "atsne_profile_enable", "atsne_profile_reset", "atsne_profile_read", "atsne_launch_count",
    "atsne_refine_subset_noalloc", "atsne_refine_batch", "atsne_kde_map", "atsne_knn_cross",
    "atsne_knn_rows",
    "atsne_merge_neighbors", "atsne_commit_rows", "atsne_delete_rows", "atsne_tune_knn", "atsne_row_dmax",
    "atsne_tune_clear", "atsne_forest_buckets_bytes", "atsne_forest_insert", "atsne_forest_delete",
    "atsne_forest_query_buckets", "atsne_set_wait_limit",
)
REFINE_NOALLOC_MAX_ROWS, REFINE_NOALLOC_MAX_K = 2048, 128


class AtsneError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("atsne status %d: %s" % (status, message))
        self.status = status


class KnnOpts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("trees", ctypes.c_int32), ("top_var_dims", ctypes.c_int32),
                ("checks", ctypes.c_int32), ("leaf_size", ctypes.c_int32),
                ("queue_cap", ctypes.c_int32), ("rerank_k", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


class ForestLayout(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int32), ("trees", ctypes.c_int32),
                ("n_internal", ctypes.c_int64), ("off_split_dim", ctypes.c_size_t),
                ("off_split_val", ctypes.c_size_t), ("off_perm", ctypes.c_size_t),
                ("off_leaf_ofs", ctypes.c_size_t), ("off_leaf_pt", ctypes.c_size_t),
                ("bytes", ctypes.c_size_t)]


_lib = None
_vp, _i32, _i64, _f32, _sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float,
                              ctypes.c_size_t)


def lib():
    """The loaded C library (ctypes.CDLL). Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libatsne.so is not built (run __graft_entry__.build()); "
                               "there is no fallback path")
        L = ctypes.CDLL(LIB_PATH)
        L.atsne_knn_opts_default.argtypes = [ctypes.POINTER(KnnOpts)]
        L.atsne_knn_opts_default.restype = None
        L.atsne_workspace_bytes.argtypes = [_i32, _i64, _i32, _i32, _i64, ctypes.POINTER(KnnOpts)]
        L.atsne_workspace_bytes.restype = _sz
        L.atsne_knn.argtypes = [_vp, _i64, _i32, _vp, _i64, _i32, ctypes.POINTER(KnnOpts), _vp, _vp,
                                _vp, _sz, _vp]
        L.atsne_calibrate_P.argtypes = [_vp, _i64, _i32, _f32, _f32, _i32, _vp, _vp, _vp]
        L.atsne_symmetrize.argtypes = [_vp, _vp, _i64, _i32, _vp, _vp, _vp, _vp, _vp, _sz, _vp]
        L.atsne_refine_subset.argtypes = [_vp, _i64, _i32, _vp, _i64, _i32, _f32, _vp, _vp, _vp,
                                          _vp, _vp, _vp, _sz, _vp]
        L.atsne_refine_subset_noalloc.argtypes = [_vp, _i64, _i32, _vp, _i64, _i32, _f32, _vp,
                                                  _vp, _vp, _vp, _vp, _vp]
        L.atsne_refine_batch.argtypes = [_vp, _i64, _i32, _vp, _i64, _i32, _f32, _vp, _vp, _vp,
                                         _vp, _vp, _vp, _vp, _sz, _vp]
        L.atsne_knn_precision.argtypes = [_vp, _vp, _i64, _i32, _vp, _vp, _vp]
        L.atsne_knn_cross.argtypes = [_vp, _i64, _vp, _i64, _i32, _i32, ctypes.POINTER(KnnOpts),
                                      _vp, _vp, _vp, _vp, _sz, _vp]
        L.atsne_knn_rows.argtypes = [_vp, _i64, _i32, _vp, _i64, _i32, ctypes.POINTER(KnnOpts), _vp,
                                     _vp, _vp, _vp, _sz, _vp]
        L.atsne_merge_neighbors.argtypes = [_vp, _vp, _i64, _i32, _vp, _vp, _i32, _i32, _vp, _vp]
        L.atsne_commit_rows.argtypes = [_vp, _i64, _i64, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                        _vp, _vp, _vp]
        L.atsne_delete_rows.argtypes = [_vp, _i64, _vp, _i64, _i32, _i32, _f32, _vp, _vp, _vp, _vp,
                                        _vp, _vp, _sz, _vp]
        L.atsne_tune_knn.argtypes = [_vp, _i64, _i32, _vp, _i64, _i32, ctypes.POINTER(KnnOpts), _vp,
                                     _vp, _vp, _sz, _vp, ctypes.POINTER(_i32), ctypes.POINTER(_f32)]
        L.atsne_tune_clear.argtypes = []
        L.atsne_row_dmax.argtypes = [_vp, _i64, _i32, _vp, _vp]
        L.atsne_forest_buckets_bytes.argtypes = [_i64, _i32, _i32]
        L.atsne_forest_buckets_bytes.restype = _sz
        L.atsne_forest_insert.argtypes = [_vp, _i64, _i64, _i64, _i32, ctypes.POINTER(KnnOpts), _vp, _vp, _vp,
                                          _sz, ctypes.POINTER(_i32), _vp, _sz, _vp]
        L.atsne_forest_delete.argtypes = [_vp, _i64, _i64, _i64, _i32, ctypes.POINTER(KnnOpts), _vp, _vp, _vp,
                                          _sz, ctypes.POINTER(_i32), _vp, _sz, _vp]
        L.atsne_forest_query_buckets.argtypes = [_vp, _i64, _i32, _i64, _vp, _vp, _i32, _vp, _i64, _i32,
                                                 ctypes.POINTER(KnnOpts), _vp, _vp, _vp, _vp, _sz, _vp]
        L.atsne_kde_map.argtypes = [_vp, _i64, _vp, _vp, _f32, _f32, _f32, _i32, _i32, _f32, _f32,
                                    _f32, _vp, _vp, _vp, _vp, _vp]
        L.atsne_forest_layout.argtypes = [_i64, _i32, ctypes.POINTER(KnnOpts),
                                          ctypes.POINTER(ForestLayout)]
        L.atsne_forest_build.argtypes = [_vp, _i64, _i32, ctypes.POINTER(KnnOpts), _vp, _sz, _vp,
                                         _sz, _vp]
        L.atsne_forest_query.argtypes = [_vp, _i64, _i32, _vp, _vp, _i64, _i32,
                                         ctypes.POINTER(KnnOpts), _vp, _vp, _vp, _vp, _sz, _vp]
        L.atsne_check.argtypes = [_vp]
        L.atsne_set_wait_limit.argtypes = [ctypes.c_uint64]
        L.atsne_last_error.restype = ctypes.c_char_p
        L.atsne_last_error.argtypes = []
        L.atsne_launch_count.restype = ctypes.c_int64
        L.atsne_launch_count.argtypes = []
        L.atsne_profile_enable.argtypes = [_i32]
        L.atsne_profile_reset.argtypes = []
        L.atsne_profile_read.argtypes = [ctypes.c_char_p, ctypes.POINTER(_i64),
                                         ctypes.POINTER(ctypes.c_double)]
        for name in EXPORTED:
            f = getattr(L, name)
            if name not in ("atsne_knn_opts_default", "atsne_workspace_bytes",
                            "atsne_last_error", "atsne_launch_count", "atsne_forest_buckets_bytes"):
                f.restype = ctypes.c_int
        _lib = L
    return _lib


def _raise(rc):
    if rc != ATSNE_OK:
        msg = lib().atsne_last_error()
        raise AtsneError(rc, msg.decode() if msg else "")


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev(t, dtype, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError("%s must be a contiguous CUDA %s tensor" % (name, dtype))
    return t


def knn_opts(method="exact", precision="fp32", trees=4, top_var_dims=5, checks=1024, leaf_size=1,
             queue_cap=0, rerank_k=0, seed=0):
    o = KnnOpts()
    lib().atsne_knn_opts_default(ctypes.byref(o))
    o.method = {"exact": KNN_EXACT, "forest": KNN_FOREST}[method] if isinstance(method, str) else method
    o.precision = {"fp32": FP32, "bf16": BF16_RERANK, "fp32_cuda": FP32_CUDA_CORES,
                   "fp8": FP8_RERANK, "bf16_approx": BF16_RERANK_APPROX}[precision] \
        if isinstance(precision, str) else precision
    o.trees, o.top_var_dims, o.checks, o.leaf_size = trees, top_var_dims, checks, leaf_size
    o.queue_cap, o.rerank_k, o.seed = queue_cap, rerank_k, seed
    return o


def workspace_bytes(op, N, D, k, S=0, opts=None):
    return int(lib().atsne_workspace_bytes(op, N, D, k, S, ctypes.byref(opts) if opts else None))


def _workspace(nbytes, device):
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def atsne_knn(X, k, queries=None, opts=None, stream=None, **kw):
    """kNN lists (idx int32 [rows,k], d2 float32 [rows,k]) -- Eq. 8; forest: Sec. 4.2."""
    _dev(X, torch.float32, "X")
    N, D = X.shape
    o = opts or knn_opts(**kw)
    S = 0
    if queries is not None:
        _dev(queries, torch.int32, "queries")
        S = queries.shape[0]
    rows = S if queries is not None else N
    idx = torch.empty((rows, k), dtype=torch.int32, device=X.device)
    d2 = torch.empty((rows, k), dtype=torch.float32, device=X.device)
    ws = _workspace(workspace_bytes(OP_KNN, N, D, k, S, o), X.device)
    _raise(lib().atsne_knn(_p(X), N, D, _p(queries), S, k, ctypes.byref(o), _p(idx), _p(d2),
                           _p(ws), ws.numel(), _stream(stream)))
    return idx, d2


def atsne_tune_knn(X, k, queries=None, opts=None, stream=None, **kw):
    """Times the exact tensor-core kNN's column-split candidates on this problem
    and records the fastest for its shape (later calls of the shape use it);
    returns (splits, ms). Synchronises the stream."""
    _dev(X, torch.float32, "X")
    N, D = X.shape
    o = opts or knn_opts(**kw)
    S = 0
    if queries is not None:
        _dev(queries, torch.int32, "queries")
        S = queries.shape[0]
    rows = S if queries is not None else N
    idx = torch.empty((rows, k), dtype=torch.int32, device=X.device)
    d2 = torch.empty((rows, k), dtype=torch.float32, device=X.device)
    ws = _workspace(workspace_bytes(OP_TUNE_KNN, N, D, k, S, o), X.device)
    splits, ms = _i32(0), _f32(0.0)
    _raise(lib().atsne_tune_knn(_p(X), N, D, _p(queries), S, k, ctypes.byref(o), _p(idx), _p(d2),
                                _p(ws), ws.numel(), _stream(stream), ctypes.byref(splits),
                                ctypes.byref(ms)))
    return int(splits.value), float(ms.value)


def atsne_row_dmax(d2, stream=None, out=None):
    """d_i^Max of Eq. 11 per row: the largest present (finite) entry of d2,
    +inf for a row with none."""
    _dev(d2, torch.float32, "d2")
    rows, k = d2.shape
    dmax = torch.empty(rows, dtype=torch.float32, device=d2.device) if out is None else out
    _raise(lib().atsne_row_dmax(_p(d2), rows, k, _p(dmax), _stream(stream)))
    return dmax


def atsne_tune_clear():
    """Forgets every recorded split (the rule applies again)."""
    _raise(lib().atsne_tune_clear())


def atsne_calibrate_P(d2, perplexity, tol=0.0, max_iter=0, stream=None, P_out=None, beta_out=None):
    """Conditional rows P_{j|i} and beta by bisection -- Eq. 3-4 over N_i.
    P_out / beta_out: contiguous tensors to write into (else new ones)."""
    _dev(d2, torch.float32, "d2")
    rows, k = d2.shape
    P = torch.empty_like(d2) if P_out is None else P_out
    beta = torch.empty(rows, dtype=torch.float32, device=d2.device) if beta_out is None else beta_out
    _raise(lib().atsne_calibrate_P(_p(d2), rows, k, perplexity, tol, max_iter, _p(P), _p(beta),
                                   _stream(stream)))
    return P, beta


def atsne_symmetrize(idx, P_cond, stream=None, trim=True, out=None, workspace=None):
    """Joint P as CSR (row_ptr int64, col int32, val float32) -- Eq. 2 / Eq. 10.
    With trim=True col/val are cut to nnz (one device-to-host read of nnz).
    out: (row_ptr [>= N+1], col [>= 2Nk], val [>= 2Nk], nnz [1]) to write into;
    workspace: a uint8 device buffer of at least the symmetrisation's workspace."""
    _dev(idx, torch.int32, "idx")
    _dev(P_cond, torch.float32, "P_cond")
    N, k = idx.shape
    dev = idx.device
    if out is not None:
        row_ptr, col, val, nnz = out
        if row_ptr.numel() < N + 1 or col.numel() < 2 * N * k or val.numel() < 2 * N * k:
            raise ValueError("symmetrize: output buffers too small")
    else:
        row_ptr = torch.empty(N + 1, dtype=torch.int64, device=dev)
        col = torch.empty(2 * N * k, dtype=torch.int32, device=dev)
        val = torch.empty(2 * N * k, dtype=torch.float32, device=dev)
        nnz = torch.empty(1, dtype=torch.int64, device=dev)
    ws = workspace if workspace is not None else _workspace(workspace_bytes(OP_SYMMETRIZE, N, 0, k), dev)
    _raise(lib().atsne_symmetrize(_p(idx), _p(P_cond), N, k, _p(row_ptr), _p(col), _p(val),
                                  _p(nnz), _p(ws), ws.numel(), _stream(stream)))
    if trim:
        n = int(nnz.item())
        return row_ptr, col[:n], val[:n]
    return row_ptr, col, val, nnz


def atsne_refine_subset(X, subset, perplexity, idx, d2, P_cond, beta=None, rho=None, stream=None):
    """Exact refinement of the listed rows, in place -- Sec. 4.3, 5.1.1."""
    _dev(X, torch.float32, "X")
    _dev(subset, torch.int32, "subset")
    N, D = X.shape
    k = idx.shape[1]
    S = subset.shape[0]
    ws = _workspace(workspace_bytes(OP_REFINE, N, D, k, S), X.device)
    _raise(lib().atsne_refine_subset(_p(X), N, D, _p(subset), S, k, perplexity, _p(idx), _p(d2),
                                     _p(P_cond), _p(beta), _p(rho), _p(ws), ws.numel(),
                                     _stream(stream)))


def atsne_refine_batch(X, lists, perplexity, idx, d2, P_cond, beta=None, rho=None, stream=None,
                       workspace=None):
    """Refinement of many selections at once (their union, each point once) --
    Sec. 4.3, 5.1.1. `lists`: one int32 device tensor or a sequence of them
    (concatenated here). Returns a device int64 tensor holding the union's size.
    Pass a preallocated `workspace` (uint8, workspace_bytes(OP_REFINE_BATCH, N,
    D, k, total)) to record the call into a CUDA graph without allocating."""
    _dev(X, torch.float32, "X")
    if not isinstance(lists, torch.Tensor):
        lists = torch.cat([t.reshape(-1) for t in lists]) if len(lists) else \
            torch.empty(0, dtype=torch.int32, device=X.device)
    _dev(lists, torch.int32, "lists")
    N, D = X.shape
    k = idx.shape[1]
    total = lists.shape[0]
    ws = workspace if workspace is not None else \
        _workspace(workspace_bytes(OP_REFINE_BATCH, N, D, k, total), X.device)
    count = torch.zeros(1, dtype=torch.int64, device=X.device)
    _raise(lib().atsne_refine_batch(_p(X), N, D, _p(lists), total, k, perplexity, _p(idx), _p(d2),
                                    _p(P_cond), _p(beta), _p(rho), _p(count), _p(ws), ws.numel(),
                                    _stream(stream)))
    return count


def atsne_knn_rows(X, queries, k, hint_d2=None, opts=None, stream=None, **kw):
    """Exact kNN of the listed rows, with optional per-row upper bounds of the
    k-th squared distance (hint_d2 [S]) that seed the filter."""
    _dev(X, torch.float32, "X")
    _dev(queries, torch.int32, "queries")
    N, D = X.shape
    S = queries.shape[0]
    o = opts or knn_opts(**kw)
    if hint_d2 is not None:
        _dev(hint_d2, torch.float32, "hint_d2")
    idx = torch.empty((S, k), dtype=torch.int32, device=X.device)
    d2 = torch.empty((S, k), dtype=torch.float32, device=X.device)
    ws = _workspace(workspace_bytes(OP_KNN, N, D, k, S, o), X.device)
    _raise(lib().atsne_knn_rows(_p(X), N, D, _p(queries), S, k, ctypes.byref(o), _p(hint_d2),
                                _p(idx), _p(d2), _p(ws), ws.numel(), _stream(stream)))
    return idx, d2


def atsne_knn_cross(Xq, Xc, k, opts=None, stream=None, workspace=None, radius_d2=None, **kw):
    """The k nearest rows of Xc for each row of Xq (Eq. 8 across two sets);
    with radius_d2 [Nq] only those strictly inside each row's squared radius
    (the rest of the row -1 / +inf)."""
    _dev(Xq, torch.float32, "Xq")
    _dev(Xc, torch.float32, "Xc")
    Nq, D = Xq.shape
    Nc = Xc.shape[0]
    o = opts or knn_opts(**kw)
    if radius_d2 is not None:
        _dev(radius_d2, torch.float32, "radius_d2")
    idx = torch.empty((Nq, k), dtype=torch.int32, device=Xq.device)
    d2 = torch.empty((Nq, k), dtype=torch.float32, device=Xq.device)
    op = OP_KNN_CROSS if radius_d2 is None else OP_KNN_CROSS_RADIUS
    ws = workspace if workspace is not None else \
        _workspace(workspace_bytes(op, Nc, D, k, Nq, o), Xq.device)
    _raise(lib().atsne_knn_cross(_p(Xq), Nq, _p(Xc), Nc, D, k, ctypes.byref(o), _p(radius_d2),
                                 _p(idx), _p(d2), _p(ws), ws.numel(), _stream(stream)))
    return idx, d2


def atsne_merge_neighbors(idx, d2, cand_idx, cand_d2, index_offset, changed=None, stream=None):
    """Insert candidates into the first cand_idx.shape[0] rows of idx/d2 in
    place (Eq. 11, Sec. 5.3.1); returns the uint8 changed-row flags."""
    rows, kc = cand_idx.shape
    k = idx.shape[1]
    if changed is None:
        changed = torch.empty(rows, dtype=torch.uint8, device=idx.device)
    _raise(lib().atsne_merge_neighbors(_p(idx), _p(d2), rows, k, _p(cand_idx), _p(cand_d2), kc,
                                       int(index_offset), _p(changed), _stream(stream)))
    return changed


def atsne_commit_rows(rows, ti, td, tp, tb, idx, d2, P_cond, beta=None, rho=None, stream=None):
    """Write computed rows into the state (rho := 1 on them) -- Sec. 4.3."""
    S, k = ti.shape
    _raise(lib().atsne_commit_rows(_p(rows), S, idx.shape[0], k, _p(ti), _p(td), _p(tp), _p(tb),
                                   _p(idx), _p(d2), _p(P_cond), _p(beta), _p(rho), _stream(stream)))


def atsne_delete_rows(X, rows, perplexity, idx, d2, P_cond, beta=None, rho=None, N=None, stream=None,
                      workspace=None):
    """Deletion of the listed points (Sec. 5.3.2), in place over the first N
    rows (default: all): they leave every neighbourhood (an absent entry, index
    -1, per point removed; rho -= 1/k each), the remaining rows move up in order
    with every index renumbered, and their Gaussians are calibrated again.
    Returns the new number of rows."""
    _dev(X, torch.float32, "X")
    _dev(rows, torch.int32, "rows")
    N = X.shape[0] if N is None else int(N)
    D, k, R = X.shape[1], idx.shape[1], rows.shape[0]
    ws = workspace if workspace is not None else _workspace(workspace_bytes(OP_DELETE, N, D, k, 0), X.device)
    _raise(lib().atsne_delete_rows(_p(rows), R, _p(X), N, D, k, perplexity, _p(idx), _p(d2), _p(P_cond),
                                   _p(beta), _p(rho), _p(ws), ws.numel(), _stream(stream)))
    return N - R


def atsne_kde_map(Y, x0, y0, pixel, width, height, h, cutoff=4.0, lens_k=2.0, rho=None,
                  selected=None, stream=None):
    """Density view f (Eq. 12), selected share s (Eq. 13), approximation map a
    and lens alpha (Sec. 5.2.2) of a 2-D embedding Y [N][2] on a width x height
    image. Returns four float32 [height][width] device tensors."""
    _dev(Y, torch.float32, "Y")
    N = Y.shape[0]
    if rho is not None:
        _dev(rho, torch.float32, "rho")
    if selected is not None:
        selected = selected.to(torch.uint8)
    out = [torch.empty((height, width), dtype=torch.float32, device=Y.device) for _ in range(4)]
    _raise(lib().atsne_kde_map(_p(Y), N, _p(rho), _p(selected), x0, y0, pixel, width, height, h,
                               cutoff, lens_k, *[_p(t) for t in out], _stream(stream)))
    return tuple(out)


def atsne_refine_subset_noalloc(X, subset, perplexity, idx, d2, P_cond, beta=None, rho=None,
                                stream=None):
    """Refinement as atsne_refine_subset, for callers that cannot allocate: the
    library's fixed device scratch replaces the workspace (at most
    REFINE_NOALLOC_MAX_ROWS rows, k <= REFINE_NOALLOC_MAX_K). This wrapper
    allocates nothing either."""
    _dev(X, torch.float32, "X")
    _dev(subset, torch.int32, "subset")
    N, D = X.shape
    _raise(lib().atsne_refine_subset_noalloc(_p(X), N, D, _p(subset), subset.shape[0],
                                             idx.shape[1], perplexity, _p(idx), _p(d2), _p(P_cond),
                                             _p(beta), _p(rho), _stream(stream)))


def atsne_knn_precision(idx_approx, idx_exact, stream=None):
    """rho_i (float32 [rows]) and rho (Python float) -- Eq. 9."""
    _dev(idx_approx, torch.int32, "idx_approx")
    _dev(idx_exact, torch.int32, "idx_exact")
    rows, k = idx_approx.shape
    rho_i = torch.empty(rows, dtype=torch.float32, device=idx_approx.device)
    s = torch.empty(1, dtype=torch.float64, device=idx_approx.device)
    _raise(lib().atsne_knn_precision(_p(idx_approx), _p(idx_exact), rows, k, _p(rho_i), _p(s),
                                     _stream(stream)))
    return rho_i, float(s.item()) / max(rows, 1)


class Forest:
    """A randomized KD-forest held in one device buffer (layout of atsne.h)."""

    def __init__(self, buf, layout, N, D, opts):
        self.buf, self.layout, self.N, self.D, self.opts = buf, layout, N, D, opts

    def _view(self, off, count, dtype):
        esz = torch.tensor([], dtype=dtype).element_size()
        return self.buf[off:off + count * esz].view(dtype)

    def arrays(self):
        L = self.layout
        T, n_int = L.trees, L.n_internal
        return dict(
            depth=L.depth,
            split_dim=self._view(L.off_split_dim, T * n_int, torch.int32).view(T, n_int),
            split_val=self._view(L.off_split_val, T * n_int, torch.float32).view(T, n_int),
            perm=self._view(L.off_perm, T * self.N, torch.int32).view(T, self.N),
            leaf_ofs=self._view(L.off_leaf_ofs, (1 << L.depth) + 1, torch.int32),
            leaf_pt=self._view(L.off_leaf_pt, T * (1 << L.depth), torch.int32).view(T, 1 << L.depth))


def atsne_forest_build(X, stream=None, opts=None, **kw):
    _dev(X, torch.float32, "X")
    N, D = X.shape
    o = opts or knn_opts(method="forest", **kw)
    L = ForestLayout()
    _raise(lib().atsne_forest_layout(N, D, ctypes.byref(o), ctypes.byref(L)))
    buf = torch.empty(L.bytes, dtype=torch.uint8, device=X.device)
    ws = _workspace(workspace_bytes(OP_FOREST_BUILD, N, D, 1, 0, o), X.device)
    _raise(lib().atsne_forest_build(_p(X), N, D, ctypes.byref(o), _p(buf), L.bytes, _p(ws),
                                    ws.numel(), _stream(stream)))
    return Forest(buf, L, N, D, o)


class ForestBuckets:
    """A forest's leaf buckets after points were added or removed (Sec. 5.3):
    perm [T][N] and per-tree leaf offsets, in one device buffer; the trees are
    those of `forest`."""

    def __init__(self, buf, forest, N, max_bucket):
        self.buf, self.forest, self.N, self.max_bucket = buf, forest, N, max_bucket

    def arrays(self):
        L, T = self.forest.layout, self.forest.layout.trees
        n_ofs = (1 << L.depth) + 1
        size = T * self.N * 4
        off = (size + 255) & ~255
        return dict(perm=self.buf[:size].view(torch.int32).view(T, self.N),
                    leaf_ofs=self.buf[off:off + T * n_ofs * 4].view(torch.int32).view(T, n_ofs))


def _buckets_buffer(forest, N, device):
    n = lib().atsne_forest_buckets_bytes(N, forest.layout.depth, forest.layout.trees)
    return torch.empty(max(int(n), 1), dtype=torch.uint8, device=device)


def atsne_forest_insert(X, forest, n_old, buckets=None, stream=None):
    """Rows n_old .. N-1 of X join every tree of `forest` (Sec. 5.3.1), after
    the buckets of the first n_old rows (`buckets`, or the forest's own when
    n_old is the number of points it was built on). Returns ForestBuckets."""
    _dev(X, torch.float32, "X")
    N, D = X.shape
    o = KnnOpts.from_buffer_copy(forest.opts)
    out = _buckets_buffer(forest, N, X.device)
    ws = _workspace(workspace_bytes(OP_FOREST_UPDATE, forest.N, D, 0, N, o), X.device)
    mb = _i32(0)
    _raise(lib().atsne_forest_insert(_p(X), forest.N, int(n_old), N, D, ctypes.byref(o), _p(forest.buf),
                                     _p(buckets.buf) if buckets is not None else None, _p(out), out.numel(),
                                     ctypes.byref(mb), _p(ws), ws.numel(), _stream(stream)))
    return ForestBuckets(out, forest, N, int(mb.value))


def atsne_forest_delete(forest, rows, buckets=None, stream=None):
    """The listed rows leave every tree (Sec. 5.3.2); the others are renumbered
    as the corpus rows are. Returns ForestBuckets."""
    _dev(rows, torch.int32, "rows")
    N = buckets.N if buckets is not None else forest.N
    o = KnnOpts.from_buffer_copy(forest.opts)
    R = rows.shape[0]
    out = _buckets_buffer(forest, N - R, forest.buf.device)
    ws = _workspace(workspace_bytes(OP_FOREST_UPDATE, forest.N, forest.D, 0, N, o), forest.buf.device)
    mb = _i32(0)
    _raise(lib().atsne_forest_delete(_p(rows), R, forest.N, N, forest.D, ctypes.byref(o), _p(forest.buf),
                                     _p(buckets.buf) if buckets is not None else None, _p(out), out.numel(),
                                     ctypes.byref(mb), _p(ws), ws.numel(), _stream(stream)))
    return ForestBuckets(out, forest, N - R, int(mb.value))


def atsne_forest_query(X, forest, k, checks=None, queries=None, queue_cap=None, stream=None, buckets=None):
    """Forest search (Sec. 4.2); with `buckets` (ForestBuckets), over the
    leaf buckets after points were added or removed."""
    _dev(X, torch.float32, "X")
    N, D = X.shape
    o = KnnOpts.from_buffer_copy(forest.opts)
    if checks is not None:
        o.checks = checks
    if queue_cap is not None:
        o.queue_cap = queue_cap
    S = 0
    if queries is not None:
        _dev(queries, torch.int32, "queries")
        S = queries.shape[0]
    rows = S if queries is not None else N
    idx = torch.empty((rows, k), dtype=torch.int32, device=X.device)
    d2 = torch.empty((rows, k), dtype=torch.float32, device=X.device)
    ev = torch.empty(rows, dtype=torch.int64, device=X.device)
    if buckets is not None:
        ob = KnnOpts.from_buffer_copy(o)
        ob.leaf_size = buckets.max_bucket
        ws = _workspace(workspace_bytes(OP_FOREST_QUERY, N, D, k, S, ob), X.device)
        _raise(lib().atsne_forest_query_buckets(_p(X), N, D, forest.N, _p(forest.buf), _p(buckets.buf),
                                                buckets.max_bucket, _p(queries), S, k, ctypes.byref(o), _p(idx),
                                                _p(d2), _p(ev), _p(ws), ws.numel(), _stream(stream)))
        return idx, d2, ev
    ws = _workspace(workspace_bytes(OP_FOREST_QUERY, N, D, k, S, o), X.device)
    _raise(lib().atsne_forest_query(_p(X), N, D, _p(forest.buf), _p(queries), S, k,
                                    ctypes.byref(o), _p(idx), _p(d2), _p(ev), _p(ws), ws.numel(),
                                    _stream(stream)))
    return idx, d2, ev


def atsne_check(stream=None):
    """Synchronise and raise if a kernel flagged bad input or an expired wait."""
    _raise(lib().atsne_check(_stream(stream)))


def set_wait_limit(ns=0):
    """Limit (ns) of the tensor kNN's pipeline waits; 0 restores the default."""
    _raise(lib().atsne_set_wait_limit(int(ns)))


def launch_count():
    """Kernel launches enqueued by the library since it was loaded."""
    return int(lib().atsne_launch_count())


def profile_enable(on=True):
    _raise(lib().atsne_profile_enable(1 if on else 0))


def profile_reset():
    _raise(lib().atsne_profile_reset())


def profile_read(kernel=None):
    n = _i64(0)
    ms = ctypes.c_double(0.0)
    _raise(lib().atsne_profile_read(kernel.encode() if kernel else None, ctypes.byref(n),
                                    ctypes.byref(ms)))
    return int(n.value), float(ms.value)
