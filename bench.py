#!/usr/bin/env python
"""Benchmark of the A-tSNE similarity path (tSNE's P matrix) on one GB300.

Headline: one step = the exact P matrix of one batch of 1,000,000 x 128
non-negative Gamma(2, 1) features in 50 clusters (perplexity 30, k = 90):
    exact kNN (Eq. 8, Sec. 3.1) -> beta bisection (Eq. 3-4) -> symmetrised CSR P (Eq. 2)
with the distance contraction in BF16 on the tensor cores and the top-4k
candidates re-ranked in FP32 (recall >= 0.999 against FP32 checked), beside the
same step in FP32 (three BF16 passes, certified exact), the certified one-pass
BF16 mode and FP8 with per-row scales. value = N points / step time (whole job:
N points per rank, summed over ranks).

Beside it: the approximate path and the paper's refinement on the MNIST-shaped
workload (70000 x 784: forest build, forest kNN at checks 1024, rho of Eq. 9,
exact refinement of a brushed selection, CSR P^A), the forest's checks sweep,
serving with p50/p99 latency, the density views and batched refinement.

--impl reference times the FP64 CPU oracle (the plain restatement of the
method the library is checked against) on the host cores, on a bounded sample
of the same workload extrapolated to points/s.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

K_NN, PERPLEXITY = 90, 30.0
METRIC = "P-matrix points/s at k=90, FP32 vs BF16+rerank at recall≥0.999; p99 latency"

WORKLOADS = {
    "gamma1m": dict(N=1_000_000, D=128, seed=3, kind="gamma_clusters",
                    desc="1000000x128 fp32, non-negative Gamma(2,1) features times per-cluster "
                         "scales U(0.5,2), 50 clusters"),
    "gamma200k": dict(N=200_000, D=128, seed=3, kind="gamma_clusters",
                      desc="200000x128 fp32, Gamma-cluster features (profiling case)"),
    "mnist70k": dict(N=70000, D=784, seed=2, kind="sparse_prototypes",
                     desc="70000x784 fp32, integer values in [0,255], ~80% zeros, 10 sparse "
                          "prototypes + noise (MNIST-shaped)"),
    "mnist20k": dict(N=20000, D=784, seed=2, kind="sparse_prototypes",
                     desc="20000x784 fp32, MNIST-shaped sparse prototypes (profiling case)"),
    "gauss2k": dict(N=2000, D=64, seed=1, kind="gaussian_mixture",
                    desc="2000x64 fp32, 10 isotropic Gaussians (sigma 1, centres N(0,5^2))"),
}
PRECISIONS = ("fp32", "bf16", "bf16_approx", "fp8")
PREC_NAME = {"fp32": "FP32 (three BF16 passes, FP32 re-rank, certified exact)",
             "bf16": "BF16+rerank, certified (uncertified rows on the CUDA cores)",
             "bf16_approx": "BF16+rerank (one BF16 pass, top-4k re-ranked in FP32)",
             "fp8": "FP8 E4M3 with per-row scales + top-4k FP32 re-rank"}


def make_data(w):
    from paper_1512_01655_gb300 import synth
    if w["kind"] == "sparse_prototypes":
        X, labels = synth.sparse_prototypes(N=w["N"], D=w["D"], seed=w["seed"], return_labels=True)
    elif w["kind"] == "gamma_clusters":
        X, labels = synth.gamma_clusters(N=w["N"], D=w["D"], seed=w["seed"], return_labels=True)
    else:
        X, labels = synth.gaussian_mixture(w["N"], w["D"], seed=w["seed"], return_labels=True)
    return X, labels


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default="gamma1m",
                   help="the headline exact-P workload")
    p.add_argument("--precision", choices=PRECISIONS, default="bf16_approx",
                   help="precision of the headline step's distance contraction")
    p.add_argument("--fp32-steps", type=int, default=5, help="timed steps of the FP32 comparison")
    p.add_argument("--variant-reps", type=int, default=2,
                   help="timed runs of the certified BF16 and the FP8 variants (0: skip)")
    p.add_argument("--oracle-rows", type=int, default=48,
                   help="sampled rows whose kNN the oracle computes for the recall check")
    p.add_argument("--approx-workload", choices=sorted(WORKLOADS), default="mnist70k")
    p.add_argument("--approx-steps", type=int, default=5,
                   help="timed steps of the approximate path with refinement (0: skip)")
    p.add_argument("--trees", type=int, default=4)
    p.add_argument("--checks", type=int, default=1024)
    p.add_argument("--queue-cap", type=int, default=0, help="forest queue capacity (0 = auto)")
    p.add_argument("--refine", type=int, default=2000, help="points in the refined selection")
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--serve-max", type=int, default=2_000_000,
                   help="serving benchmark corpus size (0 to skip)")
    p.add_argument("--kde-reps", type=int, default=5,
                   help="timed density-view renders (0 to skip)")
    p.add_argument("--refine-batch-reps", type=int, default=3,
                   help="timed batched refinements of the 500000 x 256 workload (0 to skip)")
    p.add_argument("--checks-sweep", default="32,64,128,256,512,1024,2048,4096",
                   help="forest checks values for the rho sweep (empty to skip)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample", type=int, default=256)
    p.add_argument("--kernel-case", choices=["knn_tc", "bandwidth"], default=None,
                   help="run one small case of a kernel for a profiler and exit (no timing line): "
                        "knn_tc = the exact kNN of every --query-every-th row of the workload against "
                        "all rows; bandwidth = the exact path on the workload's first --case-rows rows")
    p.add_argument("--query-every", type=int, default=25)
    p.add_argument("--case-rows", type=int, default=100_000)
    return p.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (torchrun: one rank per GPU; replicas of the workload)
# ---------------------------------------------------------------------------
def dist_init(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    elif args.impl == "ours":
        torch.cuda.set_device(0)
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, v, device=None):
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu),
                                          "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
class Pipeline:
    """Buffers and the step of the whole path, all through the C ABI binding."""

    def __init__(self, at, X, labels, args, dev):
        import torch
        self.at, self.X, self.args = at, X, args
        N, D = X.shape
        self.N, self.D = N, D
        from paper_1512_01655_gb300 import synth
        sel = synth.refine_subsets(labels, 1, lo=args.refine, hi=args.refine, seed=4)[0]
        self.subset = torch.from_numpy(sel).to(dev)
        self.exact_opts = at.knn_opts(method="exact", precision="fp32")
        self.forest_opts = at.knn_opts(method="forest", trees=args.trees, checks=args.checks,
                                       leaf_size=1, seed=7, queue_cap=args.queue_cap)
        # the approximate path runs on its own stream beside the exact one: the
        # two are independent until rho, and their kernels are bound by different
        # units (integer issue and latency for the forest, tensor pipe and
        # gathers for the exact kNN). It is the longer of the two, so its stream
        # has the higher priority: its blocks are scheduled first when both wait.
        self.side = torch.cuda.Stream(device=dev, priority=-1)

    def step(self):
        import torch
        at, X = self.at, self.X
        main = torch.cuda.current_stream()
        side = self.side
        side.wait_stream(main)
        # approximate P^A (side stream)
        with torch.cuda.stream(side):
            forest = at.atsne_forest_build(X, opts=self.forest_opts, stream=side)
            idx_a, d2_a, _ = at.atsne_forest_query(X, forest, K_NN, stream=side)
            P_a, beta_a = at.atsne_calibrate_P(d2_a, PERPLEXITY, stream=side)
        # exact P (main stream)
        idx_e, d2_e = at.atsne_knn(X, K_NN, opts=self.exact_opts)
        P_e, _ = at.atsne_calibrate_P(d2_e, PERPLEXITY)
        csr_e = at.atsne_symmetrize(idx_e, P_e, trim=False)
        main.wait_stream(side)
        for t in (idx_a, d2_a, P_a, beta_a):
            t.record_stream(main)
        # precision of the approximate neighbourhoods (Eq. 9), before refinement
        rho_i, rho_sum = self._precision(idx_a, idx_e)
        self.rho_sum = rho_sum
        # refinement of a selection, then the CSR rebuild
        at.atsne_refine_subset(X, self.subset, PERPLEXITY, idx_a, d2_a, P_a, beta_a, rho_i)
        csr_a = at.atsne_symmetrize(idx_a, P_a, trim=False)
        return csr_e, csr_a, rho_i

    def _precision(self, a, e):
        import torch
        import ctypes
        at = self.at
        rows = a.shape[0]
        rho_i = torch.empty(rows, dtype=torch.float32, device=a.device)
        s = torch.empty(1, dtype=torch.float64, device=a.device)
        at._raise(at.lib().atsne_knn_precision(at._p(a), at._p(e), rows, K_NN, at._p(rho_i),
                                               at._p(s), at._stream()))
        return rho_i, s


def default_queue_cap(checks):
    # the library's default (queue_cap = 0): checks/2 as a power of two in [256, 4096]
    q = 256
    while q < checks // 2 and q < 4096:
        q <<= 1
    return q


# sources whose hash a recorded ncu traffic figure is tied to (profiles/dram_traffic.txt)
TRAFFIC_SOURCES = {
    "forest_traverse": ["forest_query.cu", "common.cuh", "internal.h"],
    "forest_traverse_u8": ["forest_query.cu", "common.cuh", "internal.h"],
    "forest_dist": ["forest_query.cu", "common.cuh", "internal.h"],
    "forest_dist_u8": ["forest_query.cu", "common.cuh", "internal.h"],
    "knn_tc": ["knn_tc.cu", "tc_ptx.cuh", "common.cuh", "internal.h", "warp_sort.cuh"],
}


def recorded_traffic(kernel, workload, variant=None):
    """DRAM bytes per launch of `kernel` on `workload` (and precision `variant`)
    from the committed ncu record, or None when there is none or the kernel's
    sources have changed."""
    import hashlib
    srcs = TRAFFIC_SOURCES.get(kernel)
    if not srcs:
        return None
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1512_01655_gb300", "csrc")
    try:
        for f in srcs:
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(fh.read())
        with open(os.path.join(ROOT, "profiles", "dram_traffic.txt")) as fh:
            for line in fh:
                parts = line.split()
                key = workload if variant is None else workload + ":" + variant
                if len(parts) == 4 and not line.startswith("#") and parts[0] == kernel \
                        and parts[1] == key and parts[2] == h.hexdigest():
                    return int(parts[3])
    except OSError:
        return None
    return None


def bench_serving(at, torch, dev, n_max, seed=5, precision="bf16", forest_trees=0, checks=1024):
    """Serving (Sec. 5.3.1 insertions, Sec. 4.3 refinements) with continuous
    batching: log-normal D = 50 points in 30 clusters, a corpus growing from
    100000 rows to n_max, the exact kNN in `precision`, 4 stream slots, admission by free
    HBM. One request sequence (half inserts of log-uniform 1000..50000 points,
    half refinements of log-uniform 500..50000 existing rows brushed from 1-3
    clusters, until the corpus is full) is served twice on a fresh server:
    closed loop (every request arriving at once) for the capacity, then open
    loop with Poisson arrivals offering 70% of that capacity in points/s
    (inter-arrival time exponential with mean size / rate). Latency = the
    completion of a request's state commit minus its arrival. Then one step of a
    sliding window on the full corpus (Sec. 5.3.2, Sec. 5.3.1): the oldest
    `window` rows deleted, `window` new points of the same distribution inserted.
    With forest_trees > 0 the server keeps a KD-forest resident and inserted
    points take their neighbourhoods from a forest search (the paper's
    approximate insertion); the CSR P is resident in both modes."""
    from paper_1512_01655_gb300 import synth
    from paper_1512_01655_gb300.serve import Request, Server
    window = 50_000
    X, labels = synth.lognormal_clusters(n_max + window, 50, seed=seed, return_labels=True)
    X_next = X[n_max:]
    X, labels = X[:n_max], labels[:n_max]
    N0 = 100_000
    rng = np.random.default_rng(seed + 1)
    seq, n = [], N0  # (kind, payload), in arrival order
    while n < n_max:
        if rng.random() < 0.5:
            b = min(int(np.exp(rng.uniform(np.log(1000), np.log(50000)))), n_max - n)
            seq.append(("insert", (n, n + b)))
            n += b
        else:
            sz = int(np.exp(rng.uniform(np.log(500), np.log(50000))))
            cl = rng.choice(30, size=int(rng.integers(1, 4)), replace=False)
            pool = np.flatnonzero(np.isin(labels[:n], cl))
            seq.append(("refine", np.sort(rng.choice(pool, size=min(sz, pool.size),
                                                     replace=False)).astype(np.int32)))

    def requests(arrivals):
        out = []
        for j, ((kind, pay), t) in enumerate(zip(seq, arrivals)):
            if kind == "insert":
                out.append(Request(j, "insert", t, points=X[pay[0]:pay[1]]))
            else:
                out.append(Request(j, "refine", t, rows=pay))
        return out

    sizes = np.array([(p[1] - p[0]) if k == "insert" else len(p) for k, p in seq], np.float64)
    kw = dict(capacity=n_max, k=K_NN, perplexity=PERPLEXITY, precision=precision, slots=4,
              forest_trees=forest_trees, checks=checks)
    srv = Server(X[:N0], **kw)
    _, closed = srv.run(requests(np.zeros(len(seq))))
    del srv
    torch.cuda.empty_cache()
    rate = 0.7 * closed["points_per_s"]
    arr = np.cumsum(rng.exponential(sizes / rate))
    srv = Server(X[:N0], **kw)
    _, opened = srv.run(requests(arr))
    at.atsne_check()
    # one sliding-window step: delete the oldest rows, insert as many new points
    win = [Request(0, "delete", 0.0, rows=np.arange(window, dtype=np.int32)),
           Request(1, "insert", 0.0, points=X_next)]
    done, _ = srv.run(win)
    at.atsne_check()
    lat = {r.kind: round((r.done - r.arrival) * 1e3, 3) for r in done}
    slide = {"rows": window, "corpus": srv.N, "delete_ms": lat["delete"],
             "delete_then_insert_ms": lat["insert"]}
    out = {"workload": "log-normal D=50, 30 clusters; corpus %d -> %d rows; %d requests; %s kNN; "
                       "4 slots" % (N0, srv.N, len(seq), precision),
           "precision": precision,
           "inserts": ("forest search (T=%d, checks=%d, buckets updated; rho of inserted rows %.4f)"
                       % (forest_trees, checks, srv.rho_forest)) if forest_trees else "exact kNN",
           "resident": "X, kNN lists, P_{j|i}, beta, rho, CSR P" + (", KD-forest and its buckets"
                                                                    if forest_trees else ""),
           "capacity_points_per_s": closed["points_per_s"], "offered_points_per_s": round(rate, 1)}
    out.update(opened)
    out["sliding_window"] = slide
    del srv
    torch.cuda.empty_cache()
    return out


def bench_kde(at, torch, dev, stream, labels, rho_i, reps, clk, peaks):
    """Density view, selected share, approximation map and lens (Sec. 5.2) of a
    stand-in 2-D layout of the workload's points (synth.embedding_2d: the
    optimiser is not part of this library), rho from the step's refined
    precision, one label selected; 1024 x 1024 pixels over [-13, 13]^2,
    h = 0.3, cutoff 4 h. Median of `reps` CUDA-event timed renders.
    Work model: every point contributes to the pixels within cutoff * h,
    about N * pi * (4h)^2 / pixel^2 Gaussian terms, one exp each; the bound is
    the SFU exponential rate, 16 per clock per SM (152 SMs)."""
    from paper_1512_01655_gb300 import synth
    Y = torch.from_numpy(synth.embedding_2d(labels, seed=6)).to(dev)
    sel = torch.from_numpy((labels == 3).astype(np.uint8)).to(dev)
    W = H = 1024
    x0 = y0 = -13.0
    px = 26.0 / W
    h, cut = 0.3, 4.0
    args = (Y, x0, y0, px, W, H, h)
    kw = dict(cutoff=cut, lens_k=2.0, rho=rho_i, selected=sel)
    for _ in range(2):
        at.atsne_kde_map(*args, **kw)
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        at.atsne_kde_map(*args, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    at.atsne_check()
    ms = sorted(ts)[len(ts) // 2]
    N = int(Y.shape[0])
    terms = N * np.pi * (cut * h) ** 2 / (px * px)
    mhz = (clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    peak = 152 * 16 * mhz * 1e6
    ach = terms / (ms / 1e3)
    return {"workload": "%d points (stand-in 2-D layout), %dx%d pixels, h=%.1f, cutoff %.0f h" % (N, W, H, h, cut),
            "ms": round(ms, 3), "pixels_per_s": round(W * H / (ms / 1e3), 1),
            "roofline": {"bound": "sfu", "achieved": round(ach / 1e12, 3), "peak": round(peak / 1e12, 3),
                         "unit": "T Gaussian terms/s (model N*pi*(cutoff*h)^2/pixel^2)",
                         "frac": round(ach / peak, 4)}}


def bench_refine_batch(at, torch, dev, stream, reps, peaks):
    """Batched refinement on its own workload: a 500000 x 256 corpus of 100
    Gaussian clusters (sigma 1, centres N(0, 4^2)) and 512 brushed selections
    of 200..20000 points (log-uniform, 1-3 clusters each), refined in one call
    (Sec. 4.3, 5.1.1). The state starts as the approximate one (forest kNN,
    T = 4, checks = 1024, and its Gaussians) and is restored before every call,
    outside the timed region, so each refinement starts from approximate rows
    (their k-th distances bound the filter). Median of `reps` CUDA-event timed
    calls after one warm-up, with the rule's column split and then with the
    split atsne_tune_knn picks for the union's shape; value = selected points
    (with repeats) per second and union rows per second."""
    from paper_1512_01655_gb300 import synth
    X, labels = synth.gaussian_mixture(500_000, 256, n_centres=100, centre_sigma=4.0, seed=4,
                                       return_labels=True)
    subs = synth.refine_subsets(labels, 512, lo=200, hi=20000, seed=4)
    N, D, k = X.shape[0], X.shape[1], K_NN
    Xd = torch.from_numpy(X).to(dev)
    lists = torch.from_numpy(np.concatenate(subs)).to(dev)
    total = int(lists.numel())
    idx0, d20 = at.atsne_knn(Xd, k, method="forest", trees=4, checks=1024, seed=7)
    P0, beta0 = at.atsne_calibrate_P(d20, PERPLEXITY)
    idx, d2, P, beta = idx0.clone(), d20.clone(), P0.clone(), beta0.clone()
    rho = torch.zeros(N, dtype=torch.float32, device=dev)

    def timed():
        ws = torch.empty(at.workspace_bytes(at.OP_REFINE_BATCH, N, D, k, total), dtype=torch.uint8,
                         device=dev)
        ts, cnt = [], None
        for it in range(reps + 1):
            for a, b in ((idx, idx0), (d2, d20), (P, P0), (beta, beta0)):
                a.copy_(b)
            rho.fill_(0.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cnt = at.atsne_refine_batch(Xd, lists, PERPLEXITY, idx, d2, P, beta, rho, workspace=ws)
            e1.record(stream)
            torch.cuda.synchronize()
            if it > 0:
                ts.append(e0.elapsed_time(e1))
        at.atsne_check()
        return sorted(ts)[len(ts) // 2], int(cnt.item())

    at.atsne_tune_clear()
    ms_rule, union = timed()
    rows_max = min(N, total)
    q = torch.arange(rows_max, dtype=torch.int32, device=dev)
    splits, _ = at.atsne_tune_knn(Xd, k, queries=q, precision="fp32")
    del q
    ms_tuned, union = timed()
    at.atsne_tune_clear()
    ms = min(ms_rule, ms_tuned)
    flops = 2.0 * union * N * D
    peak, peak_src = peak_of(peaks, "bf16_tflops")
    ach = flops / (ms / 1e3) / 1e12
    return {"workload": "500000x256 fp32, 100 Gaussian clusters; 512 selections of 200..20000 points; "
                        "state restored to the forest kNN (T=4, checks=1024) before every call",
            "selections": len(subs), "listed_points": total, "union_rows": union,
            "ms": round(ms, 2), "ms_rule_split": round(ms_rule, 2), "ms_tuned_split": round(ms_tuned, 2),
            "tuned_splits": splits,
            "listed_points_per_s": round(total / (ms / 1e3), 1),
            "union_rows_per_s": round(union / (ms / 1e3), 1),
            "tensor": {"achieved": round(ach, 1), "peak": peak, "unit": "TFLOP/s (algorithmic 2*U*N*D)",
                       "frac": round(ach / peak, 4), "tensor_passes": 3, "peak_source": peak_src}}


def algorithmic_flops_knn(Q, N, D):
    return 2.0 * Q * N * D


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def peak_of(peaks, key):
    """(value, source label) of a roofline denominator: the pool's measured
    figure when MEASURED_PEAKS.json holds it, else the recipe's fallback."""
    if key in peaks:
        kind = " (burst, of measured)" if key == "bf16_tflops" else " (of measured)"
        return float(peaks[key]), "MEASURED_PEAKS.json " + key + kind
    return FALLBACK_PEAKS[key], "fallback %g, no MEASURED_PEAKS.json (of fallback)" % FALLBACK_PEAKS[key]


class ExactStep:
    """The exact P matrix of one batch, all through the C ABI binding:
    exact kNN (prep, tensor-core contraction with fused filter, merge and
    re-rank) -> beta bisection -> symmetrised CSR P."""

    def __init__(self, at, X, precision):
        self.at, self.X = at, X
        self.opts = at.knn_opts(method="exact", precision=precision)

    def step(self):
        at = self.at
        idx, d2 = at.atsne_knn(self.X, K_NN, opts=self.opts)
        P, _ = at.atsne_calibrate_P(d2, PERPLEXITY)
        csr = at.atsne_symmetrize(idx, P, trim=False)
        return idx, csr


def timed_steps(torch, fn, steps, stream, l2_flush=None):
    """CUDA events on the launching stream around each step."""
    evs, out = [], None
    for _ in range(steps):
        if l2_flush is not None:
            l2_flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs], out


PROFILED = ["knn_order", "knn_prep", "knn_tc", "knn_tc_merge", "knn_fallback", "knn_bruteforce", "calibrate_beta",
            "sym_fwd", "sym_rev", "sym_len", "sym_write", "sym_sort_long", "sym_write_long",
            "scan_reduce", "scan_partials", "scan_down",
            "forest_traverse", "forest_traverse_u8", "forest_dist", "forest_dist_u8", "forest_u8_prep",
            "forest_choose", "forest_partial", "forest_sort_smem", "forest_sort_global", "forest_keys",
            "forest_scatter", "forest_leaf_pt", "refine_scatter", "knn_precision"]
SYM_PARTS = ("sym_fwd", "sym_rev", "sym_len", "sym_write", "sym_sort_long", "sym_write_long",
             "scan_reduce", "scan_partials", "scan_down")


def read_profile(at):
    out = {}
    for name in PROFILED:
        n, ms = at.profile_read(name)
        if n:
            out[name] = {"launches": n, "ms": ms}
    return out


def exact_rooflines(per_kernel, steps, N, D, k, nnz, passes, prec, peaks, workload):
    """Roofline lines of the exact path's kernels from their CUDA-event times
    per launch: the tensor-core kNN against the measured BF16 peak (FP8: twice
    it, the nominal ratio), the bandwidth-bound kernels against the measured HBM
    copy rate on their algorithmic bytes."""
    hbm, hbm_src = peak_of(peaks, "hbm_gbs")
    bf16, bf16_src = peak_of(peaks, "bf16_tflops")
    lines = {}
    if "knn_tc" in per_kernel:
        pk = per_kernel["knn_tc"]
        avg = pk["ms"] / pk["launches"]
        peak = bf16 * (2.0 if prec == "fp8" else 1.0)
        ach = algorithmic_flops_knn(N, N, D) / (avg / 1e3) / 1e12
        lines["knn_tc"] = {
            "kernel": "knn_tc", "bound": "tensor", "achieved": round(ach, 1), "peak": round(peak, 1),
            "unit": "TFLOP/s", "frac": round(ach / peak, 4), "launch_ms": round(avg, 3),
            "traffic": recorded_traffic("knn_tc", workload, prec),
            "algorithmic_flops_per_launch": algorithmic_flops_knn(N, N, D), "tensor_passes": passes,
            "peak_source": bf16_src + (" x 2 (FP8 nominal ratio)" if prec == "fp8" else "")}
    Dp = 64 * ((D + 63) // 64)
    bw = {
        # X read; BF16 copies (two in FP32 mode), norms and error statistics written
        "knn_prep": N * D * 4 + N * Dp * 2 * (2 if passes == 3 else 1) + N * 20,
        # d2 read; P and beta written
        "calibrate_beta": N * k * 8 + N * 4,
        # idx and P read; row_ptr, col and val written
        "symmetrize": N * k * 8 + (N + 1) * 8 + nnz * 8,
    }
    for name, bytes_ in bw.items():
        parts = SYM_PARTS if name == "symmetrize" else (name,)
        ms = sum(per_kernel[p]["ms"] for p in parts if p in per_kernel) / steps
        if ms <= 0:
            continue
        ach = bytes_ / (ms / 1e3) / 1e9
        lines[name] = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                       "frac": round(ach / hbm, 4), "ms": round(ms, 3), "algorithmic_bytes": int(bytes_),
                       "peak_source": hbm_src}
    if "calibrate_beta" in lines:
        lines["calibrate_beta"]["note"] = ("bound by the exponentials of the bisection (about 40-60 "
                                           "steps of k exp per row), not by its bytes")
    if "knn_tc_merge" in per_kernel:
        lines["knn_tc_merge"] = {"bound": "gather", "ms": round(per_kernel["knn_tc_merge"]["ms"] / steps, 3)}
    return lines


def oracle_recall(Xh, idx_by_prec, rows):
    """Eq. 9 precision of each mode's lists against the oracle's exact kNN on
    sampled rows, and the rows whose index set equals the oracle's where the
    k-th/(k+1)-th oracle distance gap exceeds 1e-4 (relative)."""
    import oracle
    from paper_1512_01655_gb300 import synth
    q = synth.sample_rows(Xh.shape[0], rows, seed=19)
    o_idx, o_d2 = oracle.knn_exact(Xh, K_NN + 1, queries=q)
    clear = (o_d2[:, K_NN] - o_d2[:, K_NN - 1]) / o_d2[:, K_NN] > 1e-4
    out = {"rows": int(len(q)), "rows_with_clear_gap": int(clear.sum())}
    for prec, idx in idx_by_prec.items():
        g = idx[q.astype(np.int64)]
        inter = [len(set(g[r]) & set(o_idx[r, :K_NN])) for r in range(len(q))]
        same = [set(g[r]) == set(o_idx[r, :K_NN]) for r in range(len(q)) if clear[r]]
        out[prec] = {"recall": round(float(np.mean(inter)) / K_NN, 6),
                     "clear_rows_identical": int(np.sum(same))}
    return out


def run_ours(args, world, rank, local, pg):
    import torch
    import paper_1512_01655_gb300 as at
    dev = torch.device("cuda", local)
    peaks = load_peaks()
    w = WORKLOADS[args.workload]
    Xh, labels = make_data(w)
    X = torch.from_numpy(Xh).to(dev)
    N, D = Xh.shape
    stream = torch.cuda.current_stream()
    l2_flush = None
    if Xh.nbytes < 256 * 2**20:
        l2_flush = torch.empty(256 * 2**20, dtype=torch.uint8, device=dev)

    # ---- headline: the exact P matrix in the headline precision ----
    head = ExactStep(at, X, args.precision)
    for _ in range(args.warmup):
        head.step()
    torch.cuda.synchronize()
    at.atsne_check()
    at.profile_enable(True)
    at.profile_reset()
    launches0 = at.launch_count()
    clocks = ClockSampler(local)
    barrier(pg)
    torch.cuda.synchronize()
    clocks.start()
    step_ms, out = timed_steps(torch, head.step, args.steps, stream, l2_flush)
    barrier(pg)
    clk = clocks.stop()
    launches = at.launch_count() - launches0
    per_kernel = read_profile(at)
    at.profile_enable(False)
    at.atsne_check()
    idx_head = out[0]
    nnz = int(out[1][3].item())
    total_ms = max_over_ranks(pg, sum(step_ms), dev)
    value = world * N * args.steps / (total_ms / 1e3)
    exact_bf16 = bool(torch.equal(X.to(torch.bfloat16).float(), X))  # low halves zero: one pass in FP32 mode

    def passes_of(prec):
        return 3 if prec == "fp32" and not exact_bf16 else 1

    passes = passes_of(args.precision)
    rooflines = exact_rooflines(per_kernel, args.steps, N, D, K_NN, nnz, passes, args.precision, peaks,
                                args.workload)
    roofline = rooflines.get("knn_tc")
    idx_by_prec = {args.precision: idx_head.cpu().numpy()}
    del out, idx_head
    torch.cuda.empty_cache()

    # ---- end to end through the API with host buffers: X from pinned memory,
    # the step, the CSR P (nnz, then row_ptr and the nnz columns and values)
    # back into pinned host buffers a caller keeps between steps ----
    e2e = None
    if args.e2e_steps > 0:
        Xpin = torch.from_numpy(Xh).pin_memory()
        cap = 2 * N * K_NN
        h_rp = torch.empty(N + 1, dtype=torch.int64).pin_memory()
        h_col = torch.empty(cap, dtype=torch.int32).pin_memory()
        h_val = torch.empty(cap, dtype=torch.float32).pin_memory()
        h_nz = torch.empty(1, dtype=torch.int64).pin_memory()
        e2e_ms, h2d, d2h = [], 0, 0
        for it in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            head.X = Xpin.to(dev, non_blocking=True)
            _, (rp, col, val, nz) = head.step()
            h_nz.copy_(nz, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            n_ = int(h_nz[0])
            h_rp.copy_(rp[:N + 1], non_blocking=True)
            h_col[:n_].copy_(col[:n_], non_blocking=True)
            h_val[:n_].copy_(val[:n_], non_blocking=True)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            if it > 0:
                e2e_ms.append((t1 - t0) * 1e3)
                h2d = Xpin.numel() * 4
                d2h = 8 + (N + 1) * 8 + n_ * 8
        head.X = X
        del Xpin, h_rp, h_col, h_val, h_nz
        e2e_total = max_over_ranks(pg, sum(e2e_ms), dev)
        e2e = {"value": round(world * N * len(e2e_ms) / (e2e_total / 1e3), 1),
               "unit": "points/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
        torch.cuda.empty_cache()

    # ---- the metric's comparison: the same step in FP32, then the certified
    # BF16 mode and FP8; recall (Eq. 9) against FP32 over all rows ----
    modes = {}
    head_recall = None
    order = [p for p in ("fp32", "bf16_approx", "bf16", "fp8") if p != args.precision]
    for prec in order:
        reps = args.fp32_steps if prec == "fp32" else args.variant_reps
        if reps <= 0:
            continue
        st = ExactStep(at, X, prec)
        st.step()
        torch.cuda.synchronize()
        at.profile_enable(True)
        at.profile_reset()
        ms, out = timed_steps(torch, st.step, reps, stream, l2_flush)
        pk = read_profile(at)
        at.profile_enable(False)
        at.atsne_check()
        med = sorted(ms)[len(ms) // 2]
        rl = exact_rooflines(pk, reps, N, D, K_NN, int(out[1][3].item()), passes_of(prec), prec, peaks,
                             args.workload)
        modes[prec] = {"what": PREC_NAME[prec], "steps": reps, "ms": round(med, 3),
                       "points_per_s": round(world * N / (med / 1e3), 1),
                       "stage_ms": {k_: round(v["ms"] / reps, 3) for k_, v in pk.items()},
                       "knn_tc": rl.get("knn_tc")}
        idx_by_prec[prec] = out[0].cpu().numpy()
        del out, st
        torch.cuda.empty_cache()
    if "fp32" in idx_by_prec:
        ref = torch.from_numpy(idx_by_prec["fp32"]).to(dev)
        for prec, idx in idx_by_prec.items():
            if prec != "fp32":
                r = round(at.atsne_knn_precision(torch.from_numpy(idx).to(dev), ref)[1], 7)
                if prec == args.precision:
                    head_recall = r
                else:
                    modes[prec]["recall_vs_fp32"] = r
        del ref
    recall_oracle = None
    if args.oracle_rows > 0 and rank == 0:
        recall_oracle = oracle_recall(Xh, idx_by_prec, args.oracle_rows)
    del idx_by_prec
    torch.cuda.empty_cache()

    # ---- the approximate path, its precision and the refinement ----
    approx = None
    if args.approx_steps > 0:
        approx = bench_approx(at, torch, dev, stream, args, peaks)
        torch.cuda.empty_cache()
    serving = None
    if args.serve_max > 0 and world == 1:
        serving = bench_serving(at, torch, dev, args.serve_max, precision="fp32", forest_trees=args.trees,
                                checks=args.checks)
        b = bench_serving(at, torch, dev, args.serve_max, precision="fp32")
        serving["exact_inserts"] = {kk: b[kk] for kk in ("inserts", "capacity_points_per_s", "points_per_s",
                                                         "p50_ms", "p99_ms", "insert", "refine", "sliding_window")}
    refine_batch = None
    if args.refine_batch_reps > 0:
        refine_batch = bench_refine_batch(at, torch, dev, stream, args.refine_batch_reps, peaks)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, Xh)

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": round(value, 1), "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else ("e4m3+f32" if args.precision == "fp8" else "bf16+f32"),
            "data": "synthetic (seeded Gamma-cluster features; no dataset)",
            "config": {"workload": w["desc"], "N": N, "D": D, "k": K_NN, "perplexity": PERPLEXITY,
                       "step": "exact kNN (Eq. 8) -> beta bisection (Eq. 3-4) -> symmetrised CSR P (Eq. 2)",
                       "precision": PREC_NAME[args.precision],
                       "l2": "input larger than L2" if l2_flush is None else "L2 flushed between steps",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "recall_vs_fp32": head_recall, "recall_vs_oracle": recall_oracle, "nnz_P": nnz,
            "stage_ms": {k_: round(v["ms"] / args.steps, 3) for k_, v in per_kernel.items()},
            "step_ms": [round(t, 3) for t in step_ms],
            "roofline": roofline, "bandwidth_kernels": {k_: v for k_, v in rooflines.items() if k_ != "knn_tc"},
            "modes": modes, "approx_path": approx, "refine_batch": refine_batch, "serving": serving,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": int(launches),
        }
        print(json.dumps(line))


def bench_approx(at, torch, dev, stream, args, peaks):
    """The approximate path on its own workload (MNIST-shaped by default): per
    step the exact FP32 P (reference for rho), the forest build (T trees, V = 5),
    the forest kNN at `checks`, its beta bisection, rho (Eq. 9), the exact
    refinement of a brushed selection and the CSR P^A (Sec. 4.2, 4.3), the two
    paths on two streams; then the forest's checks sweep and the density views."""
    w = WORKLOADS[args.approx_workload]
    Xh, labels = make_data(w)
    X = torch.from_numpy(Xh).to(dev)
    N, D = Xh.shape
    pipe = Pipeline(at, X, labels, args, dev)
    l2_flush = torch.empty(256 * 2**20, dtype=torch.uint8, device=dev) if Xh.nbytes < 256 * 2**20 else None
    for _ in range(3):
        pipe.step()
    torch.cuda.synchronize()
    at.atsne_check()
    at.profile_enable(True)
    at.profile_reset()
    step_ms, out = timed_steps(torch, pipe.step, args.approx_steps, stream, l2_flush)
    per_kernel = read_profile(at)
    at.profile_enable(False)
    at.atsne_check()
    csr_e, csr_a, rho_i = out
    rho_refined = float(rho_i.double().mean().item())
    rho = float(pipe.rho_sum.item()) / N
    med = sorted(step_ms)[len(step_ms) // 2]
    # the forest search: gather-bound, every evaluated point's row read once per
    # query (bytes when every value is an integer in [0, 255], else FP32), the
    # query row and the k outputs; traversal and distances taken together
    fparts = ("forest_u8_prep", "forest_traverse", "forest_traverse_u8", "forest_dist", "forest_dist_u8")
    need = max(args.checks, K_NN)
    u8 = D <= 2048 and bool(((X >= 0) & (X <= 255) & (X == torch.round(X))).all())
    vb = 1 if u8 else 4
    per_launch = N * ((need + 1) * D * vb + K_NN * 8)
    forest = None
    if "forest_traverse" in per_kernel:
        nl = per_kernel["forest_traverse"]["launches"]
        avg = sum(per_kernel[k_]["ms"] for k_ in fparts if k_ in per_kernel) / nl
        ach = per_launch / (avg / 1e3) / 1e9
        peak, peak_src = peak_of(peaks, "hbm_gbs")
        trn = "forest_traverse_u8" if u8 else "forest_traverse"
        dname = "forest_dist_u8" if u8 else "forest_dist"
        t_tr, t_di = recorded_traffic(trn, args.approx_workload), recorded_traffic(dname, args.approx_workload)
        forest = {"kernel": "forest_query (%s + %s)" % (trn, dname), "bound": "hbm", "achieved": round(ach, 1),
                  "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4), "launch_ms": round(avg, 3),
                  "traffic": t_tr + t_di if t_tr is not None and t_di is not None else None,
                  "algorithmic_bytes_per_launch": per_launch, "row_bytes_per_value": vb,
                  "traversal_ms": round(per_kernel.get(trn, per_kernel["forest_traverse"])["ms"] / nl, 3),
                  "traversal_bound": "instruction issue (queue and tree walk)",
                  "peak_source": peak_src}
    sweep = None
    if args.checks_sweep:
        sweep = []
        ref_idx, _ = at.atsne_knn(X, K_NN, opts=pipe.exact_opts)
        fr = at.atsne_forest_build(X, opts=pipe.forest_opts)
        for c in [int(v) for v in args.checks_sweep.split(",")]:
            at.atsne_forest_query(X, fr, K_NN, checks=c)
            ts = []
            for _ in range(3):
                if l2_flush is not None:
                    l2_flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                idx_c, _, ev_c = at.atsne_forest_query(X, fr, K_NN, checks=c)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            sweep.append({"checks": c, "rho": round(at.atsne_knn_precision(idx_c, ref_idx)[1], 5),
                          "evaluated_mean": round(float(ev_c.double().mean().item()), 1),
                          "ms": round(sorted(ts)[1], 3), "points_per_s": round(N / (sorted(ts)[1] / 1e3), 1)})
        at.atsne_check()
        del fr, ref_idx
    kde = None
    if args.kde_reps > 0:
        kde = bench_kde(at, torch, dev, stream, labels, rho_i, args.kde_reps, None, peaks)
    return {"workload": w["desc"], "N": N, "D": D,
            "step": "exact FP32 P and, on a second stream, forest build -> forest kNN -> beta -> rho -> "
                    "refinement of %d points -> CSR P^A" % int(pipe.subset.numel()),
            "forest": {"trees": args.trees, "top_var_dims": 5, "checks": args.checks, "leaf_size": 1,
                       "queue_cap": args.queue_cap or default_queue_cap(args.checks)},
            "ms_per_step": round(med, 3), "points_per_s": round(N / (med / 1e3), 1),
            "rho": round(rho, 5), "rho_after_refine": round(rho_refined, 5),
            "stage_ms": {k_: round(v["ms"] / args.approx_steps, 3) for k_, v in per_kernel.items()},
            "forest_query_roofline": forest, "checks_sweep": sweep, "kde": kde}


# ---------------------------------------------------------------------------
# oracle timing (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------
def oracle_sample_timing(Xh, sample_rows):
    """Time the oracle's exact P path on a sample of query rows and extrapolate
    to all N rows: the exact kNN and the bisection scale with the rows; the
    symmetrisation is timed on a 100000-row kNN graph of the same k and scaled
    by (N log N) / (n log n), the cost of its sort."""
    import oracle
    from paper_1512_01655_gb300 import synth
    N = Xh.shape[0]
    q = synth.sample_rows(N, sample_rows, seed=17)
    t = {}
    t0 = time.perf_counter()
    idx_e, d2_e = oracle.knn_exact(Xh, K_NN, queries=q)
    t["knn_exact"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.calibrate(d2_e, PERPLEXITY)
    t["calibrate"] = time.perf_counter() - t0
    n = min(N, 100_000)
    rng = np.random.default_rng(3)
    g_idx = ((np.arange(n)[:, None] + rng.integers(1, n, size=(n, K_NN))) % n).astype(np.int32)
    g_P = np.full((n, K_NN), 1.0 / K_NN)
    t0 = time.perf_counter()
    oracle.symmetrize(g_idx, g_P)
    t["symmetrize_%d_rows" % n] = time.perf_counter() - t0
    sym_full = t["symmetrize_%d_rows" % n] * (N * np.log(N * K_NN)) / (n * np.log(n * K_NN))
    per_row = (t["knn_exact"] + t["calibrate"]) / len(q)
    est = per_row * N + sym_full
    return N / est, t, len(q)


def cpu_baseline(args, Xh):
    import oracle
    value, t, n = oracle_sample_timing(Xh, args.cpu_sample)
    return {"value": round(value, 4), "unit": "points/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": ("FP64 exact kNN and beta bisection of %d sampled query rows against the full "
                       "corpus, extrapolated linearly to all rows; CSR symmetrisation timed on a "
                       "100000-row graph and scaled by N log N" % n),
            "seconds": {k_: round(v, 3) for k_, v in t.items()}}


def run_reference(args, world, rank, pg):
    if rank != 0:
        return
    import oracle
    w = WORKLOADS[args.workload]
    Xh, _ = make_data(w)
    sample = max(16, args.cpu_sample // 4)
    vals = []
    for it in range(args.warmup + args.steps):
        v, t, n = oracle_sample_timing(Xh, sample)
        if it >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    line = {
        "metric": METRIC,
        "value": round(value, 4), "unit": "points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded Gamma-cluster features; no dataset)",
        "config": {"workload": w["desc"], "N": w["N"], "D": w["D"], "k": K_NN, "perplexity": PERPLEXITY,
                   "step": "exact kNN (Eq. 8) -> beta bisection (Eq. 3-4) -> symmetrised CSR P (Eq. 2)"},
        "impl": "reference",
        "cpu_baseline": {"value": round(value, 4), "unit": "points/s", "kind": "oracle",
                         "cores": oracle.num_threads(),
                         "sample": "%d sampled query rows per step (FP64 exact kNN and bisection), "
                                   "extrapolated; symmetrisation timed on 100000 rows and scaled" % sample},
        "e2e": {"value": round(value, 4), "unit": "points/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def kernel_case(args):
    """A small case of one kernel for a profiler capture: a warm-up call and
    one more, in the headline precision."""
    import torch
    import paper_1512_01655_gb300 as at
    w = WORKLOADS[args.workload]
    Xh, _ = make_data(w)
    dev = torch.device("cuda", 0)
    if args.kernel_case == "knn_tc":
        X = torch.from_numpy(Xh).to(dev)
        q = torch.arange(0, X.shape[0], args.query_every, dtype=torch.int32, device=dev)
        o = at.knn_opts(method="exact", precision=args.precision)
        for _ in range(2):
            at.atsne_knn(X, K_NN, queries=q, opts=o)
        what = "%d query rows" % q.numel()
    else:
        X = torch.from_numpy(np.ascontiguousarray(Xh[:args.case_rows])).to(dev)
        o = at.knn_opts(method="exact", precision=args.precision)
        for _ in range(2):
            idx, d2 = at.atsne_knn(X, K_NN, opts=o)
            P, _ = at.atsne_calibrate_P(d2, PERPLEXITY)
            at.atsne_symmetrize(idx, P, trim=False)
        what = "%d rows" % X.shape[0]
    at.atsne_check()
    print("kernel case %s: %s, %s, %s" % (args.kernel_case, w["desc"], what, args.precision))


def main():
    args = parse()
    if args.kernel_case:
        kernel_case(args)
        return
    world, rank, local, pg = dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank, pg)
    else:
        run_ours(args, world, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
