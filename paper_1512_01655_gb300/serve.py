"""Serving: a growing corpus and its neighbourhood state kept on one GPU, with
insert requests (Sec. 5.3.1) and refinement requests (Sec. 4.3, Sec. 5.1.1)
processed by continuous batching.

A request is admitted, in arrival order, as soon as a stream slot is free and
its device memory fits in the free HBM. Its computation runs on its own stream
and overlaps the other admitted requests. Its write to the shared state (the
commit) is enqueued at admission on one state stream, so commits apply in
arrival order. A computation reads only rows of X, and rows of X are never
rewritten: an insert appends rows, and every request admitted after it waits
for that copy. Hence every request's result is the same alone and in the mix.

Insert of B points as rows [N, N + B):
  compute  the new rows' k nearest among X[:N + B] (exact) and their Gaussians
           (Eq. 3-4); for the existing rows, the new points inside their
           current radius d_i^Max, the farthest neighbour in N_i as it stands
           (atsne_row_dmax, then atsne_knn_cross with radii, kc = min(k, B)).
  commit   write the new rows (rho = 1); merge the candidates into the
           existing rows (Eq. 11); re-calibrate the existing rows.
Refine of S listed rows:
  compute  their k nearest among the current rows (the filter seeded with each
           row's current k-th distance) and their Gaussians.
  commit   write the rows (rho = 1).
Delete of R listed rows (Sec. 5.3.2): the points leave every neighbourhood
  (rho -= 1/k per point removed), the remaining rows move up in order with
  every index renumbered, and their Gaussians are calibrated again. Row
  numbers change, so a deletion is admitted only when no other request is in
  flight, and the requests after it are numbered against the state it leaves.
Update of R listed rows with R new vectors (Sec. 5.3.3: a changed point is
  removed and added again): the deletion of the rows, then the insertion of the
  new vectors as the last rows, admitted together like a deletion.

With a forest (forest_trees > 0) the state also keeps a randomized KD-forest
resident, built once on the initial rows, whose leaf buckets follow every
insertion and deletion (Sec. 5.3.1, Sec. 5.3.2), and an inserted point takes its
neighbourhood from a forest search (checks) instead of the exact kNN: the
paper's approximate insertion, whose rho_i is the forest's precision (Eq. 9,
estimated at start on sampled rows against their exact lists) until a
refinement makes the row exact. The reverse update of Eq. 11 stays exact.
The buckets change in arrival order on the state stream.

The symmetrised CSR P (Eq. 2, Eq. 10) of the current rows is kept resident too:
after commits it is rebuilt on the state stream, at most every csr_interval
seconds while requests keep arriving and always once the queue drains, so it
follows the state it was built from (csr_rows).
"""
import collections
import time

import numpy as np
import torch

from . import (OP_DELETE, OP_FOREST_QUERY, OP_FOREST_UPDATE, OP_KNN, OP_KNN_CROSS_RADIUS, OP_SYMMETRIZE,
               atsne_calibrate_P, atsne_commit_rows, atsne_delete_rows, atsne_forest_build,
               atsne_forest_delete, atsne_forest_insert, atsne_forest_query, atsne_knn, atsne_knn_cross,
               atsne_knn_precision, atsne_knn_rows, atsne_merge_neighbors, atsne_row_dmax,
               atsne_symmetrize, knn_opts, workspace_bytes)


class Request:
    """kind "insert" (points: float32 [B][D] host array), "refine" or "delete"
    (rows: int32 [S] host array of existing rows, numbered as the state is when
    the request is admitted), or "update" (both: the rows' new vectors);
    arrival in seconds."""

    def __init__(self, rid, kind, arrival, points=None, rows=None):
        self.rid, self.kind, self.arrival = rid, kind, float(arrival)
        self.points, self.rows = points, rows
        self.admitted = self.done = None
        self.first_row = None

    @property
    def size(self):
        return len(self.points) if self.kind in ("insert", "update") else len(self.rows)


class Server:
    def __init__(self, X0, capacity, k=90, perplexity=30.0, precision="fp32", slots=4,
                 reserve_bytes=1 << 30, device="cuda", forest_trees=0, checks=1024, seed=7,
                 csr_interval=0.1):
        self.dev = torch.device(device)
        N0, D = X0.shape
        if N0 < k + 1 or capacity < N0:
            raise ValueError("need k + 1 <= N0 <= capacity")
        self.k, self.perp, self.D, self.cap = k, float(perplexity), D, capacity
        self.opts = knn_opts(method="exact", precision=precision)
        f32, i32 = torch.float32, torch.int32
        self.X = torch.empty((capacity, D), dtype=f32, device=self.dev)
        self.X[:N0].copy_(torch.from_numpy(np.ascontiguousarray(X0, dtype=np.float32)))
        self.idx = torch.zeros((capacity, k), dtype=i32, device=self.dev)
        self.d2 = torch.zeros((capacity, k), dtype=f32, device=self.dev)
        self.P = torch.zeros((capacity, k), dtype=f32, device=self.dev)
        self.beta = torch.zeros(capacity, dtype=f32, device=self.dev)
        self.rho = torch.zeros(capacity, dtype=f32, device=self.dev)
        i, d = atsne_knn(self.X[:N0], k, opts=self.opts)
        self.idx[:N0].copy_(i)
        self.d2[:N0].copy_(d)
        atsne_calibrate_P(self.d2[:N0], self.perp, P_out=self.P[:N0], beta_out=self.beta[:N0])
        self.rho[:N0] = 1.0
        self.N = N0
        # the resident forest: trees of the initial rows, buckets updated in place of a rebuild
        self.forest = self.buckets = None
        self.rho_forest = 1.0
        if forest_trees > 0:
            self.fopts = knn_opts(method="forest", trees=forest_trees, checks=checks, leaf_size=1, seed=seed)
            self.checks = checks
            self.forest = atsne_forest_build(self.X[:N0], opts=self.fopts)
            sample = torch.arange(0, N0, max(1, N0 // 2048), dtype=torch.int32, device=self.dev)
            fi, _, _ = atsne_forest_query(self.X[:N0], self.forest, k, queries=sample)
            self.rho_forest = atsne_knn_precision(fi, self.idx[sample.long()])[1]
        # the resident CSR P, buffers for the full capacity
        self.row_ptr = torch.empty(capacity + 1, dtype=torch.int64, device=self.dev)
        self.col = torch.empty(2 * capacity * k, dtype=torch.int32, device=self.dev)
        self.val = torch.empty(2 * capacity * k, dtype=torch.float32, device=self.dev)
        self.nnz = torch.empty(1, dtype=torch.int64, device=self.dev)
        self.csr_ws = torch.empty(max(1, workspace_bytes(OP_SYMMETRIZE, capacity, 0, k)), dtype=torch.uint8,
                                  device=self.dev)
        self.csr_interval = csr_interval
        self.rebuild_csr(torch.cuda.current_stream(self.dev))
        self.csr_dirty, self.csr_at = False, 0.0
        torch.cuda.synchronize(self.dev)
        self.state = torch.cuda.Stream(self.dev)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(slots)]
        self.free = list(range(slots))
        self.reserve = reserve_bytes
        self.x_ready = None
        self.inflight = []

    def rebuild_csr(self, stream):
        """The symmetrised CSR P of rows [0, N) as the state stands, on `stream`."""
        N = self.N
        with torch.cuda.stream(stream):
            atsne_symmetrize(self.idx[:N], self.P[:N], stream=stream, trim=False,
                             out=(self.row_ptr, self.col, self.val, self.nnz), workspace=self.csr_ws)
        self.csr_rows = N

    def csr(self):
        """(row_ptr, col, val) of the resident CSR P (synchronises for nnz)."""
        torch.cuda.synchronize(self.dev)
        n = int(self.nnz.item())
        return self.row_ptr[:self.csr_rows + 1], self.col[:n], self.val[:n]

    # ---- admission ----
    def need_bytes(self, req):
        k, D, N = self.k, self.D, self.N
        n = req.size
        if req.kind == "insert":
            if self.forest is not None:
                fo = knn_opts(method="forest", trees=self.fopts.trees, checks=self.checks,
                              leaf_size=max(1, self.buckets.max_bucket if self.buckets else 1) + n)
                ws = workspace_bytes(OP_FOREST_QUERY, N + n, D, k, n, fo) + \
                    workspace_bytes(OP_FOREST_UPDATE, self.forest.N, D, 0, N + n, self.fopts) + \
                    2 * self.fopts.trees * (N + n) * 4
            else:
                ws = workspace_bytes(OP_KNN, N + n, D, k, n, self.opts)
            if N > 0:
                kc = min(k, n)
                ws += workspace_bytes(OP_KNN_CROSS_RADIUS, n, D, kc, N, self.opts) + N * (kc * 8 + 5)
        elif req.kind == "delete":
            ws = workspace_bytes(OP_DELETE, N, D, k)
        elif req.kind == "update":
            ins = Request(req.rid, "insert", req.arrival, points=req.points)
            return self.need_bytes(Request(req.rid, "delete", req.arrival, rows=req.rows)) + \
                self.need_bytes(ins)
        else:
            ws = workspace_bytes(OP_KNN, N, D, k, n, self.opts)
        return ws + n * (k * 12 + 8) + (1 << 20)

    def free_bytes(self):
        free, _ = torch.cuda.mem_get_info(self.dev)
        return free + torch.cuda.memory_reserved(self.dev) - torch.cuda.memory_allocated(self.dev)

    def fits(self, req):
        grow = req.size if req.kind == "insert" else req.size - len(req.rows) if req.kind == "update" else 0
        if self.N + grow > self.cap:
            raise ValueError("insert beyond the corpus capacity")
        return self.need_bytes(req) + self.reserve <= self.free_bytes()

    def admit_delete(self, req, now):
        """A deletion on the state stream, all earlier requests done."""
        st = self.state
        with torch.cuda.stream(st):
            rows = torch.from_numpy(np.ascontiguousarray(req.rows, dtype=np.int32)).to(self.dev)
            if self.forest is not None:  # the points leave every bucket (Sec. 5.3.2)
                self.buckets = atsne_forest_delete(self.forest, rows, buckets=self.buckets, stream=st)
            self.N = atsne_delete_rows(self.X, rows, self.perp, self.idx, self.d2, self.P, self.beta,
                                       self.rho, N=self.N, stream=st)
            done = torch.cuda.Event()
            done.record(st)
        self.csr_dirty = True
        self.x_ready = done  # later requests read the compacted rows
        req.admitted = now
        self.inflight.append((req, None, done, [rows]))

    def admit_update(self, req, now):
        """A deletion of the rows, then the insertion of their new vectors."""
        self.admit_delete(Request(req.rid, "delete", req.arrival, rows=req.rows), now)
        _, _, _, dkeep = self.inflight.pop()  # the insertion's commit follows it on the state stream
        ins = Request(req.rid, "insert", req.arrival, points=req.points)
        self.admit(ins, now)
        _, slot, done, keep = self.inflight.pop()
        req.first_row, req.admitted = ins.first_row, now
        self.inflight.append((req, slot, done, keep + dkeep))

    def admit(self, req, now):
        if req.kind == "delete":
            return self.admit_delete(req, now)
        if req.kind == "update":
            return self.admit_update(req, now)
        slot = self.free.pop(0)
        s = self.streams[slot]
        keep = []
        with torch.cuda.stream(s):
            if self.x_ready is not None:
                s.wait_event(self.x_ready)
            N0 = self.N
            if req.kind == "insert":
                B = req.size
                host = torch.from_numpy(np.ascontiguousarray(req.points, dtype=np.float32)).pin_memory()
                self.X[N0:N0 + B].copy_(host, non_blocking=True)
                self.x_ready = torch.cuda.Event()
                self.x_ready.record(s)
                rows = torch.arange(N0, N0 + B, dtype=torch.int32, device=self.dev)
                if self.forest is not None:
                    # the new points join the forest's buckets in arrival order (state
                    # stream), then their neighbourhoods come from a forest search
                    with torch.cuda.stream(self.state):
                        self.state.wait_event(self.x_ready)
                        self.buckets = atsne_forest_insert(self.X[:N0 + B], self.forest, N0,
                                                           buckets=self.buckets, stream=self.state)
                        fdone = torch.cuda.Event()
                        fdone.record(self.state)
                    s.wait_event(fdone)
                    ti, td, _ = atsne_forest_query(self.X[:N0 + B], self.forest, self.k, checks=self.checks,
                                                   queries=rows, buckets=self.buckets, stream=s)
                    keep.append(self.buckets.buf)
                else:
                    ti, td = atsne_knn(self.X[:N0 + B], self.k, queries=rows, opts=self.opts, stream=s)
                tp, tb = atsne_calibrate_P(td, self.perp, stream=s)
                cand = None
                if N0 > 0:
                    # the existing rows' radii d_i^Max (their farthest neighbour in
                    # N_i as it stands), taken on the state stream after the
                    # earlier commits (a radius only ever shrinks)
                    with torch.cuda.stream(self.state):
                        radius = atsne_row_dmax(self.d2[:N0], stream=self.state)
                        snap = torch.cuda.Event()
                        snap.record(self.state)
                    radius.record_stream(s)
                    s.wait_event(snap)
                    kc = min(self.k, B)
                    cand = atsne_knn_cross(self.X[:N0], self.X[N0:N0 + B], kc, opts=self.opts, stream=s,
                                           radius_d2=radius)
                    keep.append(radius)
                self.N = N0 + B
                req.first_row = N0
                keep += [host, rows, ti, td, tp, tb] + (list(cand) if cand else [])
            else:
                rows = torch.from_numpy(np.ascontiguousarray(req.rows, dtype=np.int32)).to(self.dev)
                # the rows' current k-th distances (taken after the earlier
                # commits) seed the exact search's filter
                with torch.cuda.stream(self.state):
                    hint = self.d2[:, self.k - 1].index_select(0, rows.long())
                    snap = torch.cuda.Event()
                    snap.record(self.state)
                hint.record_stream(s)
                s.wait_event(snap)
                ti, td = atsne_knn_rows(self.X[:N0], rows, self.k, hint_d2=hint, opts=self.opts, stream=s)
                keep.append(hint)
                tp, tb = atsne_calibrate_P(td, self.perp, stream=s)
                cand = None
                keep += [rows, ti, td, tp, tb]
            computed = torch.cuda.Event()
            computed.record(s)
        st = self.state
        with torch.cuda.stream(st):
            st.wait_event(computed)
            atsne_commit_rows(rows, ti, td, tp, tb, self.idx, self.d2, self.P, self.beta, self.rho,
                              stream=st)
            if req.kind == "insert" and self.forest is not None:
                self.rho[N0:N0 + req.size].fill_(self.rho_forest)  # approximate rows (Eq. 9)
            if cand is not None:
                atsne_merge_neighbors(self.idx[:N0], self.d2[:N0], cand[0], cand[1], N0, stream=st)
                atsne_calibrate_P(self.d2[:N0], self.perp, stream=st, P_out=self.P[:N0],
                                  beta_out=self.beta[:N0])
            done = torch.cuda.Event()
            done.record(st)
        for t in keep:
            if t.is_cuda:
                t.record_stream(st)
        req.admitted = now
        self.inflight.append((req, slot, done, keep))
        self.csr_dirty = True

    # ---- the loop ----
    def run(self, requests, clock=time.perf_counter, idle_sleep=2e-4):
        """Serve `requests` (arrival times in seconds from the start); returns
        them with admitted/done times and a summary."""
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        served = []
        t0 = clock()
        while pending or self.inflight:
            now = clock() - t0
            progress = False
            for item in list(self.inflight):
                req, slot, done, _ = item
                if done.query():
                    req.done = clock() - t0
                    self.inflight.remove(item)
                    if slot is not None:
                        self.free.append(slot)
                    served.append(req)
                    progress = True
            while pending and pending[0].arrival <= now and self.free:
                if pending[0].kind in ("delete", "update") and self.inflight:
                    break  # renumbering: wait until nothing else is in flight
                if not self.fits(pending[0]):
                    if not self.inflight:
                        raise MemoryError("request %d does not fit in free device memory"
                                          % pending[0].rid)
                    break
                self.admit(pending.popleft(), clock() - t0)
                progress = True
            # the resident CSR P follows the commits: rebuilt after the last one
            # enqueued, at most every csr_interval seconds while requests arrive
            now = clock() - t0
            if self.csr_dirty and (not self.inflight or now - self.csr_at >= self.csr_interval):
                self.rebuild_csr(self.state)
                self.csr_dirty, self.csr_at = False, now
                progress = True
            if not progress:
                time.sleep(idle_sleep)
        if self.csr_dirty:
            self.rebuild_csr(self.state)
            self.csr_dirty = False
        torch.cuda.synchronize(self.dev)
        return served, summarize(served)


def summarize(served):
    if not served:
        return {}
    lat = np.array([r.done - r.arrival for r in served])
    pts = sum(r.size for r in served)
    span = max(r.done for r in served) - min(r.arrival for r in served)
    out = {"requests": len(served), "points": int(pts), "seconds": round(span, 4),
           "points_per_s": round(pts / span, 1) if span > 0 else None,
           "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 3),
           "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 3)}
    for kind in ("insert", "refine", "delete", "update"):
        lk = np.array([r.done - r.arrival for r in served if r.kind == kind])
        if lk.size:
            out[kind] = {"requests": int(lk.size),
                         "p50_ms": round(float(np.percentile(lk, 50)) * 1e3, 3),
                         "p99_ms": round(float(np.percentile(lk, 99)) * 1e3, 3)}
    return out
