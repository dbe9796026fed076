// C ABI entry points (declared in include/atsne.h): argument validation on the
// host, workspace layouts, the device status word, launch profiling, and the
// composition of kernels into the four operations.
#include <float.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace atsne {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";

atsne_status set_error(atsne_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

atsne_status cuda_error(cudaError_t e, const char *what) {
    return set_error(ATSNE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// device status word (one int per device, no allocation)
// ---------------------------------------------------------------------------
static __device__ int g_status_word;
static int *g_status_ptr[64];

int *device_status_word() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!g_status_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) return nullptr;
        g_status_ptr[dev] = static_cast<int *>(p);
    }
    return g_status_ptr[dev];
}

// ---------------------------------------------------------------------------
// launch profiling
// ---------------------------------------------------------------------------
namespace {
struct ProfRec {
    const char *name;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_pool;
size_t g_prof_used = 0;
constexpr size_t PROF_POOL = 8192;
}  // namespace

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

ProfScope::ProfScope(const char *kernel, cudaStream_t s) : slot(-1), stream(s) {
    if (!g_prof_on) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (g_prof_used >= g_prof_pool.size()) return;
    slot = (int)g_prof_used++;
    g_prof_pool[slot].name = kernel;
    cudaEventRecord(g_prof_pool[slot].a, stream);
}

ProfScope::~ProfScope() {
    if (slot >= 0) cudaEventRecord(g_prof_pool[slot].b, stream);
}

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
namespace {

__global__ void check_finite_kernel(const float4 *__restrict__ x4, int64_t n4,
                                    const float *__restrict__ tail, int64_t ntail, int *status) {
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = x4[i];
        bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w));
    }
    if (blockIdx.x == 0)
        for (int64_t i = threadIdx.x; i < ntail; i += blockDim.x) bad |= !isfinite(tail[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) raise_status(status, DEV_NONFINITE);
}

__global__ void check_indices_kernel(const int32_t *__restrict__ list, int64_t n, int64_t N,
                                     int *status) {
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        bad |= list[i] < 0 || list[i] >= N;
    if (__syncthreads_or(bad) && threadIdx.x == 0) raise_status(status, DEV_MALFORMED);
}

}  // namespace

atsne_status check_finite(const float *X, int64_t n, cudaStream_t stream) {
    const bool aligned = (reinterpret_cast<uintptr_t>(X) & 15) == 0;
    const int64_t n4 = aligned ? n / 4 : 0;
    const int64_t done = n4 * 4;
    const int grid = (int)hmin(4 * num_sms(), ceil_div(n4 > 0 ? n4 : 1, 256));
    return launch_kernel("check_finite", check_finite_kernel, grid, 256, 0, stream,
                         reinterpret_cast<const float4 *>(X), n4, X + done, n - done,
                         device_status_word());
}

atsne_status check_indices(const int32_t *list, int64_t n, int64_t N, cudaStream_t stream) {
    if (n <= 0) return ATSNE_OK;
    const int grid = (int)hmin(2 * num_sms(), ceil_div(n, 256));
    return launch_kernel("check_indices", check_indices_kernel, grid, 256, 0, stream, list, n, N,
                         device_status_word());
}

namespace {

atsne_knn_opts opts_or_default(const atsne_knn_opts *o) {
    atsne_knn_opts d;
    atsne_knn_opts_default(&d);
    return o ? *o : d;
}

atsne_status validate_knn_opts(const atsne_knn_opts &o) {
    if (o.method != ATSNE_KNN_EXACT && o.method != ATSNE_KNN_FOREST)
        return set_error(ATSNE_EINVAL, "knn: unknown method %d", o.method);
    if (o.precision != ATSNE_FP32 && o.precision != ATSNE_BF16_RERANK &&
        o.precision != ATSNE_FP32_CUDA_CORES && o.precision != ATSNE_FP8_RERANK &&
        o.precision != ATSNE_BF16_RERANK_APPROX)
        return set_error(ATSNE_EINVAL, "knn: unknown precision %d", o.precision);
    if (o.rerank_k < 0 || o.rerank_k > 4096)
        return set_error(ATSNE_EINVAL, "knn: rerank_k=%d not in [0, 4096]", o.rerank_k);
    if (o.method == ATSNE_KNN_FOREST) {
        if (o.trees < 1 || o.trees > 64) return set_error(ATSNE_EINVAL, "forest: trees=%d not in [1,64]", o.trees);
        if (o.top_var_dims < 1 || o.top_var_dims > 8)
            return set_error(ATSNE_EINVAL, "forest: top_var_dims=%d not in [1,8]", o.top_var_dims);
        if (o.checks < 1) return set_error(ATSNE_EINVAL, "forest: checks=%d < 1", o.checks);
        if (o.leaf_size < 1) return set_error(ATSNE_EINVAL, "forest: leaf_size=%d < 1", o.leaf_size);
        if (o.queue_cap != 0 && o.queue_cap < 2)
            return set_error(ATSNE_EINVAL, "forest: queue_cap=%d < 2", o.queue_cap);
    }
    return ATSNE_OK;
}

atsne_status validate_xk(const float *X, int64_t N, int32_t D, int32_t k) {
    if (!X) return set_error(ATSNE_EINVAL, "X is NULL");
    if (N < 2 || N > INT32_MAX) return set_error(ATSNE_EINVAL, "N=%lld not in [2, 2^31-1]", (long long)N);
    if (D < 1) return set_error(ATSNE_EINVAL, "D=%d < 1", D);
    if (k < 1 || (int64_t)k > N - 1) return set_error(ATSNE_EINVAL, "k=%d not in [1, N-1]", k);
    return ATSNE_OK;
}

// Queue capacity: the caller's, or checks/2 rounded up to a power of two in
// [256, 4096] (a bound the search reaches only when it would not have popped
// the evicted entries within its budget on the workloads measured).
int queue_capacity(const atsne_knn_opts &o) {
    if (o.queue_cap > 0) return o.queue_cap;
    int q = 256;
    while (q < o.checks / 2 && q < 4096) q <<= 1;
    return q;
}

ForestView forest_view(void *forest, int64_t N, int32_t D, const atsne_knn_opts &o) {
    atsne_forest_layout_t L;
    forest_layout(N, o.trees, o.leaf_size, &L);
    char *b = static_cast<char *>(forest);
    ForestView f;
    f.N = N;
    f.D = D;
    f.trees = o.trees;
    f.depth = L.depth;
    f.leaf_size = o.leaf_size;
    f.top_var_dims = o.top_var_dims;
    f.n_internal = L.n_internal;
    f.seed = o.seed;
    f.split_dim = reinterpret_cast<int32_t *>(b + L.off_split_dim);
    f.split_val = reinterpret_cast<float *>(b + L.off_split_val);
    f.perm = reinterpret_cast<int32_t *>(b + L.off_perm);
    f.leaf_ofs = reinterpret_cast<int32_t *>(b + L.off_leaf_ofs);
    f.leaf_pt = reinterpret_cast<int32_t *>(b + L.off_leaf_pt);
    return f;
}

bool exact_on_tensor_cores(const atsne_knn_opts &o, int32_t k) {
    return o.method == ATSNE_KNN_EXACT && o.precision != ATSNE_FP32_CUDA_CORES && k <= 200;
}

// Workspace layouts (sizing and carving share these).
size_t knn_ws(Carver &c, int64_t N, int32_t D, int32_t k, int64_t S, const atsne_knn_opts &o,
              void **forest, void **sub_ws, size_t *sub_bytes, TcPlan *plan = nullptr,
              TcWs *tws = nullptr) {
    if (exact_on_tensor_cores(o, k)) {
        const int64_t Q = S > 0 ? S : N;
        const TcPlan pl = tc_plan(N, D, Q, k, o.precision, o.rerank_k);
        if (plan) *plan = pl;
        tc_workspace(c, N, D, Q, S > 0, pl, tws);
    }
    if (o.method == ATSNE_KNN_FOREST) {
        const size_t fb = forest_layout(N, o.trees, o.leaf_size, nullptr);
        char *f = c.take<char>(fb);
        if (forest) *forest = f;
        Carver b(nullptr), q(nullptr);
        const size_t bb = forest_build_workspace(b, N, D, o.trees, o.leaf_size, nullptr);
        const size_t qb = forest_query_workspace(q, N, D, S > 0 ? S : N, k, o.checks, o.leaf_size, nullptr);
        const size_t need = bb > qb ? bb : qb;
        char *w = c.take<char>(need);
        if (sub_ws) *sub_ws = w;
        if (sub_bytes) *sub_bytes = need;
    }
    return c.bytes();
}

// Workspaces and forests are carved at 256-byte offsets from their base, and
// kernels read parts of them with 16-byte vector loads.
atsne_status check_base(const void *p, const char *what) {
    if (reinterpret_cast<uintptr_t>(p) & 255)
        return set_error(ATSNE_EINVAL, "%s: base address not 256-byte aligned", what);
    return ATSNE_OK;
}

// Selections of at least this many rows are refined on the tensor-core path.
constexpr int64_t REFINE_TC_MIN_ROWS = 128;

size_t refine_ws(Carver &c, int64_t N, int32_t D, int64_t S, int32_t k, int32_t **ti, float **td,
                 float **tp, float **tb, TcPlan *plan = nullptr, TcWs *tws = nullptr,
                 float **hint = nullptr) {
    int32_t *a = c.take<int32_t>((size_t)S * k);
    float *b = c.take<float>((size_t)S * k);
    float *p = c.take<float>((size_t)S * k);
    float *q = c.take<float>((size_t)(S > 0 ? S : 1));
    float *h = c.take<float>((size_t)(S > 0 ? S : 1));
    if (ti) *ti = a;
    if (td) *td = b;
    if (tp) *tp = p;
    if (tb) *tb = q;
    if (hint) *hint = h;
    if (S >= REFINE_TC_MIN_ROWS && k <= 200) {
        const TcPlan pl = tc_plan(N, D, S, k, ATSNE_FP32, 0);
        if (plan) *plan = pl;
        tc_workspace(c, N, D, S, true, pl, tws);
    }
    return c.bytes();
}

// kNN of Nq rows of another array among Nc corpus rows.
size_t cross_ws(Carver &c, int64_t Nq, int64_t Nc, int32_t D, int32_t k, const atsne_knn_opts &o,
                bool radius, TcPlan *plan, TcWs *tws) {
    if (exact_on_tensor_cores(o, k) && Nq > 0 && !(radius && o.precision == ATSNE_FP8_RERANK)) {
        TcPlan pl = tc_plan(Nc, D, Nq, k, o.precision, o.rerank_k);
        if (radius) pl.cap = RADIUS_CAP;  // only the points inside the radius are buffered
        if (plan) *plan = pl;
        tc_workspace(c, Nc, D, Nq, true, pl, tws);
    }
    return c.bytes();
}

// Autotuner: room for the largest candidate's tensor-core workspace.
constexpr int TUNE_MAX_CAND = 8;
size_t tune_ws(int64_t N, int32_t D, int32_t k, int64_t S, const atsne_knn_opts &o, int *cand, int *n_cand) {
    const int64_t Q = S > 0 ? S : N;
    int c_[TUNE_MAX_CAND];
    int *cs = cand ? cand : c_;
    const int n = tc_split_candidates(N, D, Q, k, o.precision, o.rerank_k, cs, TUNE_MAX_CAND);
    if (n_cand) *n_cand = n;
    size_t need = 0;
    for (int i = 0; i < n; ++i) {
        Carver c(nullptr);
        tc_workspace(c, N, D, Q, S > 0, tc_plan(N, D, Q, k, o.precision, o.rerank_k, cs[i]), nullptr);
        if (c.bytes() > need) need = c.bytes();
    }
    return need;
}

// Batched refinement: the union's rows (padded to min(N, total)), its bitmap,
// then the refinement of that many rows.
size_t refine_batch_ws(Carver &c, int64_t N, int32_t D, int64_t total, int32_t k, int32_t **rows,
                       uint32_t **bitmap, int32_t **ti, float **td, float **tp, float **tb,
                       TcPlan *plan, TcWs *tws, float **hint = nullptr) {
    const int64_t rows_max = total < N ? total : N;
    int32_t *r = c.take<int32_t>((size_t)(rows_max > 0 ? rows_max : 1));
    uint32_t *b = c.take<uint32_t>((size_t)((N + 31) / 32));
    if (rows) *rows = r;
    if (bitmap) *bitmap = b;
    return refine_ws(c, N, D, rows_max, k, ti, td, tp, tb, plan, tws, hint);
}

}  // namespace
}  // namespace atsne

namespace atsne {
namespace {
// The trees of a built forest and, for a buckets buffer, its views.
struct UpdateArgs {
    ForestView f;
    const int32_t *perm_in, *ofs_in;
    int64_t stride_in;
    BucketsView out;
    UpdateWs w;
};

atsne_status update_args(const float *X, int64_t N_built, int64_t n_in, int64_t n_out, int64_t ws_rows, int32_t D,
                         const atsne_knn_opts *opts, const void *forest, const void *buckets_in, void *buckets_out,
                         size_t out_bytes, void *workspace, size_t ws_bytes, const char *what, UpdateArgs *a) {
    atsne_knn_opts o = opts_or_default(opts);
    o.method = ATSNE_KNN_FOREST;
    atsne_status st = validate_knn_opts(o);
    if (st) return st;
    if (!forest || !buckets_out || (!buckets_in && n_in != N_built) || (X == nullptr && D < 1))
        return set_error(ATSNE_EINVAL, "%s: NULL pointer or buckets", what);
    if (N_built < 2 || N_built > INT32_MAX || n_in < 0 || n_out < 0 || n_in > INT32_MAX || n_out > INT32_MAX ||
        D < 1)
        return set_error(ATSNE_EINVAL, "%s: N_built=%lld rows %lld -> %lld D=%d", what, (long long)N_built,
                         (long long)n_in, (long long)n_out, D);
    a->f = forest_view(const_cast<void *>(forest), N_built, D, o);
    const int depth = a->f.depth;
    if (depth > 25) return set_error(ATSNE_EUNSUPPORTED, "%s: depth %d", what, depth);
    size_t off = 0;
    if (buckets_layout(n_out, depth, o.trees, &off) > out_bytes)
        return set_error(ATSNE_ENOMEM, "%s: buckets buffer of %zu bytes too small", what, out_bytes);
    if (buckets_in) {  // any overlap of the two byte ranges races the copy with its source
        const char *i0 = static_cast<const char *>(buckets_in);
        const char *i1 = i0 + buckets_layout(n_in, depth, o.trees, nullptr);
        const char *o0 = static_cast<const char *>(buckets_out);
        const char *o1 = o0 + out_bytes;
        if (i0 < o1 && o0 < i1)
            return set_error(ATSNE_EINVAL, "%s: buckets_in and buckets_out overlap", what);
    }
    if ((st = check_base(forest, what)) || (st = check_base(buckets_out, what)) ||
        (buckets_in && (st = check_base(buckets_in, what))) || (st = check_base(workspace, what)))
        return st;
    char *bo = static_cast<char *>(buckets_out);
    a->out.perm = reinterpret_cast<int32_t *>(bo);
    a->out.ofs = reinterpret_cast<int32_t *>(bo + off);
    if (buckets_in) {
        size_t off_in = 0;
        buckets_layout(n_in, depth, o.trees, &off_in);
        const char *bi = static_cast<const char *>(buckets_in);
        a->perm_in = reinterpret_cast<const int32_t *>(bi);
        a->ofs_in = reinterpret_cast<const int32_t *>(bi + off_in);
        a->stride_in = ((int64_t)1 << depth) + 1;
    } else {
        a->perm_in = a->f.perm;
        a->ofs_in = a->f.leaf_ofs;
        a->stride_in = 0;
    }
    Carver c(workspace);
    update_workspace(c, ws_rows, depth, o.trees, &a->w);
    if (!workspace || ws_bytes < c.bytes())
        return set_error(ATSNE_ENOMEM, "%s: workspace of %zu bytes, %zu needed", what, ws_bytes, c.bytes());
    return ATSNE_OK;
}

atsne_status read_max_bucket(const UpdateWs &w, int32_t *out, cudaStream_t stream) {
    int32_t v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, w.bmax, sizeof(int32_t), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_error(e, "forest update: read the largest bucket");
    if (out) *out = v;
    return ATSNE_OK;
}
}  // namespace
}  // namespace atsne

using namespace atsne;

extern "C" {

void atsne_knn_opts_default(atsne_knn_opts *o) {
    if (!o) return;
    o->method = ATSNE_KNN_EXACT;
    o->precision = ATSNE_FP32;
    o->trees = 4;
    o->top_var_dims = 5;
    o->checks = 1024;
    o->leaf_size = 1;
    o->queue_cap = 0;
    o->rerank_k = 0;
    o->seed = 0;
}

const char *atsne_last_error(void) { return g_err; }

int64_t atsne_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

size_t atsne_workspace_bytes(int32_t op, int64_t N, int32_t D, int32_t k, int64_t S,
                             const atsne_knn_opts *opts) {
    const atsne_knn_opts o = opts_or_default(opts);
    Carver c(nullptr);
    switch (op) {
    case ATSNE_OP_KNN:
        return knn_ws(c, N, D, k, S, o, nullptr, nullptr, nullptr);
    case ATSNE_OP_CALIBRATE:
        return 0;
    case ATSNE_OP_SYMMETRIZE:
        return symmetrize_workspace(c, N, k, nullptr);
    case ATSNE_OP_REFINE:
        return refine_ws(c, N, D, S, k, nullptr, nullptr, nullptr, nullptr);
    case ATSNE_OP_FOREST_BUILD:
        return forest_build_workspace(c, N, D, o.trees, o.leaf_size, nullptr);
    case ATSNE_OP_FOREST_QUERY:
        return forest_query_workspace(c, N, D, S > 0 ? S : N, k, o.checks, o.leaf_size, nullptr);
    case ATSNE_OP_KNN_CROSS:
        return cross_ws(c, S, N, D, k, o, false, nullptr, nullptr);
    case ATSNE_OP_DELETE:
        return delete_workspace(c, N, D, k, nullptr);
    case ATSNE_OP_FOREST_UPDATE:
        return update_workspace(c, S, forest_depth(N, o.leaf_size), o.trees, nullptr);
    case ATSNE_OP_TUNE_KNN:
        return exact_on_tensor_cores(o, k) ? tune_ws(N, D, k, S, o, nullptr, nullptr) : 0;
    case ATSNE_OP_KNN_CROSS_RADIUS:
        return cross_ws(c, S, N, D, k, o, true, nullptr, nullptr);
    case ATSNE_OP_REFINE_BATCH:
        return refine_batch_ws(c, N, D, S, k, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                               nullptr, nullptr);
    default:
        return 0;
    }
}

atsne_status atsne_knn(const float *X, int64_t N, int32_t D, const int32_t *queries, int64_t S,
                       int32_t k, const atsne_knn_opts *opts, int32_t *idx_out, float *d2_out,
                       void *workspace, size_t ws_bytes, void *stream_) {
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    atsne_status st = validate_xk(X, N, D, k);
    if (st) return st;
    const atsne_knn_opts o = opts_or_default(opts);
    if ((st = validate_knn_opts(o))) return st;
    if (!idx_out || !d2_out) return set_error(ATSNE_EINVAL, "knn: NULL output");
    if (queries && S < 0) return set_error(ATSNE_EINVAL, "knn: S=%lld < 0", (long long)S);
    const int64_t nq = queries ? S : N;
    if (nq == 0) return ATSNE_OK;
    Carver c(workspace);
    void *forest = nullptr, *sub = nullptr;
    size_t sub_bytes = 0;
    TcPlan plan;
    TcWs tws;
    knn_ws(c, N, D, k, queries ? S : 0, o, &forest, &sub, &sub_bytes, &plan, &tws);
    if (c.bytes() > 0 && (!workspace || ws_bytes < c.bytes()))
        return set_error(ATSNE_ENOMEM, "knn: workspace of %zu bytes, %zu needed", ws_bytes, c.bytes());
    if ((st = check_base(workspace, "knn workspace"))) return st;
    if (queries && (st = check_indices(queries, S, N, stream))) return st;
    if (exact_on_tensor_cores(o, k))  // the prep kernel checks X for non-finite values
        return knn_exact_tc(X, N, D, queries, nq, k, plan, tws, idx_out, d2_out, stream);
    if ((st = check_finite(X, N * (int64_t)D, stream))) return st;
    if (o.method == ATSNE_KNN_EXACT)
        return knn_bruteforce(X, N, D, queries, nq, k, idx_out, d2_out, stream);
    ForestView f = forest_view(forest, N, D, o);
    if ((st = forest_build_launch(X, f, sub, sub_bytes, stream))) return st;
    return forest_query_launch(X, f, queries, nq, k, o.checks, queue_capacity(o), idx_out, d2_out,
                               nullptr, sub, sub_bytes, stream);
}

atsne_status atsne_tune_knn(const float *X, int64_t N, int32_t D, const int32_t *queries, int64_t S,
                            int32_t k, const atsne_knn_opts *opts, int32_t *idx_out, float *d2_out,
                            void *workspace, size_t ws_bytes, void *stream_, int32_t *splits_out,
                            float *ms_out) {
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    atsne_status st = validate_xk(X, N, D, k);
    if (st) return st;
    const atsne_knn_opts o = opts_or_default(opts);
    if ((st = validate_knn_opts(o))) return st;
    if (!exact_on_tensor_cores(o, k))
        return set_error(ATSNE_EUNSUPPORTED, "tune: only the exact kNN on the tensor cores has a tunable");
    if (!idx_out || !d2_out) return set_error(ATSNE_EINVAL, "tune: NULL output");
    if (queries && S < 1) return set_error(ATSNE_EINVAL, "tune: S=%lld < 1", (long long)S);
    const int64_t Q = queries ? S : N;
    int cand[TUNE_MAX_CAND], n_cand = 0;
    const size_t need = tune_ws(N, D, k, queries ? S : 0, o, cand, &n_cand);
    if (!workspace || ws_bytes < need)
        return set_error(ATSNE_ENOMEM, "tune: workspace of %zu bytes, %zu needed", ws_bytes, need);
    if ((st = check_base(workspace, "tune workspace"))) return st;
    if (queries && (st = check_indices(queries, S, N, stream))) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int best = 0;
    float best_ms = FLT_MAX;
    for (int i = 0; i < n_cand && e == cudaSuccess && st == ATSNE_OK; ++i) {
        const TcPlan pl = tc_plan(N, D, Q, k, o.precision, o.rerank_k, cand[i]);
        Carver c(workspace);
        TcWs w;
        tc_workspace(c, N, D, Q, queries != nullptr, pl, &w);
        float ms = FLT_MAX;
        for (int rep = 0; rep < 3 && st == ATSNE_OK && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(e0, stream);
            if (e != cudaSuccess) break;
            st = knn_exact_tc(X, N, D, queries, Q, k, pl, w, idx_out, d2_out, stream);
            if (st) break;
            e = cudaEventRecord(e1, stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e == cudaSuccess && rep > 0 && t < ms) ms = t;  // the first run warms up
        }
        if (st == ATSNE_OK && e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = pl.splits;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) return st;
    if (e != cudaSuccess) return cuda_error(e, "tune");
    set_tuned_splits(N, D, Q, k, o.precision, o.rerank_k, best);
    if (splits_out) *splits_out = best;
    if (ms_out) *ms_out = best_ms;
    return ATSNE_OK;
}

atsne_status atsne_tune_clear(void) {
    clear_tuned_splits();
    return ATSNE_OK;
}

atsne_status atsne_calibrate_P(const float *d2, int64_t rows, int32_t k, float perplexity,
                               float tol, int32_t max_iter, float *P_cond_out, float *beta_out,
                               void *stream) {
    if (!d2 || !P_cond_out) return set_error(ATSNE_EINVAL, "calibrate: NULL pointer");
    if (rows < 0 || k < 1) return set_error(ATSNE_EINVAL, "calibrate: rows=%lld k=%d", (long long)rows, k);
    if (!(perplexity > 0.f) || !(perplexity < (float)k))
        return set_error(ATSNE_EINVAL, "calibrate: perplexity=%g not in (0, k=%d)", (double)perplexity, k);
    if (calibrate_smem_bytes(k) > 227 * 1024)
        return set_error(ATSNE_EUNSUPPORTED, "calibrate: k=%d too large", k);
    if (!(tol > 0.f)) tol = 1e-5f;
    if (max_iter <= 0) max_iter = 200;
    return calibrate_launch(d2, rows, k, perplexity, tol, max_iter, P_cond_out, beta_out,
                            static_cast<cudaStream_t>(stream));
}

atsne_status atsne_delete_rows(const int32_t *rows, int64_t R, float *X, int64_t N, int32_t D, int32_t k,
                               float perplexity, int32_t *idx, float *d2, float *P_cond, float *beta,
                               float *rho, void *workspace, size_t ws_bytes, void *stream) {
    if (!X || !idx || !d2 || !P_cond || (R > 0 && !rows))
        return set_error(ATSNE_EINVAL, "delete: NULL pointer");
    if (N < 1 || N > INT32_MAX || D < 1 || k < 1 || R < 0 || R > N)
        return set_error(ATSNE_EINVAL, "delete: N=%lld D=%d k=%d R=%lld", (long long)N, D, k, (long long)R);
    if (!(perplexity > 0.f) || !(perplexity < (float)k))
        return set_error(ATSNE_EINVAL, "delete: perplexity=%g not in (0, k=%d)", (double)perplexity, k);
    if (calibrate_smem_bytes(k) > 227 * 1024) return set_error(ATSNE_EUNSUPPORTED, "delete: k=%d too large", k);
    if (atsne_status st = check_base(workspace, "delete workspace")) return st;
    Carver c(workspace);
    DeleteWs w;
    delete_workspace(c, N, D, k, &w);
    if (ws_bytes < c.bytes()) return set_error(ATSNE_ENOMEM, "delete: workspace too small");
    return delete_launch(rows, R, X, N, D, k, perplexity, idx, d2, P_cond, beta, rho, w,
                         static_cast<cudaStream_t>(stream));
}

atsne_status atsne_symmetrize(const int32_t *idx, const float *P_cond, int64_t N, int32_t k,
                              int64_t *row_ptr, int32_t *col, float *val, int64_t *nnz_dev,
                              void *workspace, size_t ws_bytes, void *stream) {
    if (!idx || !P_cond || !row_ptr || !col || !val) return set_error(ATSNE_EINVAL, "symmetrize: NULL pointer");
    if (N < 2 || N > INT32_MAX || k < 1 || (int64_t)k > N - 1)
        return set_error(ATSNE_EINVAL, "symmetrize: N=%lld k=%d", (long long)N, k);
    if (k > 512) return set_error(ATSNE_EUNSUPPORTED, "symmetrize: k=%d above 512", k);
    Carver c(workspace);
    SymWs w;
    symmetrize_workspace(c, N, k, &w);
    if (!workspace || ws_bytes < c.bytes())
        return set_error(ATSNE_ENOMEM, "symmetrize: workspace of %zu bytes, %zu needed", ws_bytes, c.bytes());
    if (atsne_status st = check_base(workspace, "symmetrize workspace")) return st;
    return symmetrize_launch(idx, P_cond, N, k, row_ptr, col, val, nnz_dev, w,
                             static_cast<cudaStream_t>(stream));
}

atsne_status atsne_refine_subset(const float *X, int64_t N, int32_t D, const int32_t *subset,
                                 int64_t S, int32_t k, float perplexity, int32_t *idx, float *d2,
                                 float *P_cond, float *beta, float *rho, void *workspace,
                                 size_t ws_bytes, void *stream_) {
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    atsne_status st = validate_xk(X, N, D, k);
    if (st) return st;
    if (!subset || !idx || !d2 || !P_cond) return set_error(ATSNE_EINVAL, "refine: NULL pointer");
    if (S < 0) return set_error(ATSNE_EINVAL, "refine: S=%lld < 0", (long long)S);
    if (!(perplexity > 0.f) || !(perplexity < (float)k))
        return set_error(ATSNE_EINVAL, "refine: perplexity=%g not in (0, k=%d)", (double)perplexity, k);
    if (S == 0) return ATSNE_OK;
    Carver c(workspace);
    int32_t *ti;
    float *td, *tp, *tb, *hint;
    TcPlan plan;
    TcWs tws;
    refine_ws(c, N, D, S, k, &ti, &td, &tp, &tb, &plan, &tws, &hint);
    if (!workspace || ws_bytes < c.bytes())
        return set_error(ATSNE_ENOMEM, "refine: workspace of %zu bytes, %zu needed", ws_bytes, c.bytes());
    if ((st = check_base(workspace, "refine workspace"))) return st;
    if ((st = check_indices(subset, S, N, stream))) return st;
    if (S >= REFINE_TC_MIN_ROWS && k <= 200) {  // the prep kernel checks X for non-finite values
        // the rows' current k-th distances seed the threshold (a row that lists
        // k real points bounds its exact k-th distance; the certificate keeps
        // the result exact whatever the bound)
        if ((st = gather_hint_launch(subset, S, N, k, d2, hint, stream))) return st;
        if ((st = knn_exact_tc(X, N, D, subset, S, k, plan, tws, ti, td, stream, nullptr, nullptr, hint)))
            return st;
    } else {
        if ((st = check_finite(X, N * (int64_t)D, stream))) return st;
        if ((st = knn_bruteforce(X, N, D, subset, S, k, ti, td, stream))) return st;
    }
    if ((st = calibrate_launch(td, S, k, perplexity, 1e-5f, 200, tp, tb, stream))) return st;
    return refine_scatter_launch(subset, S, N, k, ti, td, tp, tb, idx, d2, P_cond, beta, rho, stream);
}

atsne_status atsne_refine_batch(const float *X, int64_t N, int32_t D, const int32_t *lists,
                                int64_t total, int32_t k, float perplexity, int32_t *idx, float *d2,
                                float *P_cond, float *beta, float *rho, int64_t *refined_count,
                                void *workspace, size_t ws_bytes, void *stream_) {
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    atsne_status st = validate_xk(X, N, D, k);
    if (st) return st;
    if ((!lists && total > 0) || !idx || !d2 || !P_cond)
        return set_error(ATSNE_EINVAL, "refine batch: NULL pointer");
    if (total < 0) return set_error(ATSNE_EINVAL, "refine batch: total=%lld < 0", (long long)total);
    if (!(perplexity > 0.f) || !(perplexity < (float)k))
        return set_error(ATSNE_EINVAL, "refine batch: perplexity=%g not in (0, k=%d)", (double)perplexity, k);
    if (total == 0) {
        if (refined_count) {
            cudaError_t e = cudaMemsetAsync(refined_count, 0, sizeof(int64_t), stream);
            if (e != cudaSuccess) return cuda_error(e, "refine batch: count");
        }
        return ATSNE_OK;
    }
    Carver c(workspace);
    int32_t *rows, *ti;
    uint32_t *bitmap;
    float *td, *tp, *tb, *hint;
    TcPlan plan;
    TcWs tws;
    refine_batch_ws(c, N, D, total, k, &rows, &bitmap, &ti, &td, &tp, &tb, &plan, &tws, &hint);
    if (!workspace || ws_bytes < c.bytes())
        return set_error(ATSNE_ENOMEM, "refine batch: workspace of %zu bytes, %zu needed", ws_bytes,
                         c.bytes());
    if ((st = check_base(workspace, "refine batch workspace"))) return st;
    if ((st = check_indices(lists, total, N, stream))) return st;
    const int64_t S = total < N ? total : N;
    if ((st = union_launch(lists, total, N, bitmap, rows, S, refined_count, stream))) return st;
    if (S >= REFINE_TC_MIN_ROWS && k <= 200) {  // the prep kernel checks X for non-finite values
        if ((st = gather_hint_launch(rows, S, N, k, d2, hint, stream))) return st;
        if ((st = knn_exact_tc(X, N, D, rows, S, k, plan, tws, ti, td, stream, nullptr, nullptr, hint)))
            return st;
    } else {
        if ((st = check_finite(X, N * (int64_t)D, stream))) return st;
        if ((st = knn_bruteforce(X, N, D, rows, S, k, ti, td, stream))) return st;
    }
    if ((st = calibrate_launch(td, S, k, perplexity, 1e-5f, 200, tp, tb, stream))) return st;
    return refine_scatter_launch(rows, S, N, k, ti, td, tp, tb, idx, d2, P_cond, beta, rho, stream);
}

atsne_status atsne_knn_rows(const float *X, int64_t N, int32_t D, const int32_t *queries, int64_t S,
                            int32_t k, const atsne_knn_opts *opts, const float *hint_d2,
                            int32_t *idx_out, float *d2_out, void *workspace, size_t ws_bytes,
                            void *stream_) {
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    atsne_status st = validate_xk(X, N, D, k);
    if (st) return st;
    const atsne_knn_opts o = opts_or_default(opts);
    if ((st = validate_knn_opts(o))) return st;
    if (o.method != ATSNE_KNN_EXACT) return set_error(ATSNE_EINVAL, "knn rows: exact method only");
    if (!queries || !idx_out || !d2_out) return set_error(ATSNE_EINVAL, "knn rows: NULL pointer");
    if (S < 0) return set_error(ATSNE_EINVAL, "knn rows: S=%lld < 0", (long long)S);
    if (S == 0) return ATSNE_OK;
    Carver c(workspace);
    void *forest = nullptr, *sub = nullptr;
    size_t sub_bytes = 0;
    TcPlan plan;
    TcWs tws;
    knn_ws(c, N, D, k, S, o, &forest, &sub, &sub_bytes, &plan, &tws);
    if (c.bytes() > 0 && (!workspace || ws_bytes < c.bytes()))
        return set_error(ATSNE_ENOMEM, "knn rows: workspace of %zu bytes, %zu needed", ws_bytes, c.bytes());
    if ((st = check_base(workspace, "knn rows workspace"))) return st;
    if ((st = check_indices(queries, S, N, stream))) return st;
    if (exact_on_tensor_cores(o, k))
        return knn_exact_tc(X, N, D, queries, S, k, plan, tws, idx_out, d2_out, stream, nullptr, nullptr,
                            hint_d2);
    if ((st = check_finite(X, N * (int64_t)D, stream))) return st;
    return knn_bruteforce(X, N, D, queries, S, k, idx_out, d2_out, stream);
}

atsne_status atsne_knn_cross(const float *Xq, int64_t Nq, const float *Xc, int64_t Nc, int32_t D,
                             int32_t k, const atsne_knn_opts *opts, const float *radius_d2,
                             int32_t *idx_out, float *d2_out, void *workspace, size_t ws_bytes,
                             void *stream_) {
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    const atsne_knn_opts o = opts_or_default(opts);
    atsne_status st = validate_knn_opts(o);
    if (st) return st;
    if (o.method != ATSNE_KNN_EXACT) return set_error(ATSNE_EINVAL, "knn cross: exact method only");
    if (!Xq || !Xc || !idx_out || !d2_out) return set_error(ATSNE_EINVAL, "knn cross: NULL pointer");
    if (Nq < 0 || Nq > INT32_MAX || Nc < 1 || Nc > INT32_MAX || D < 1 || k < 1 || (int64_t)k > Nc)
        return set_error(ATSNE_EINVAL, "knn cross: Nq=%lld Nc=%lld D=%d k=%d", (long long)Nq,
                         (long long)Nc, D, k);
    if (Nq == 0) return ATSNE_OK;
    Carver c(workspace);
    TcPlan plan;
    TcWs tws;
    cross_ws(c, Nq, Nc, D, k, o, radius_d2 != nullptr, &plan, &tws);
    if (c.bytes() > 0 && (!workspace || ws_bytes < c.bytes()))
        return set_error(ATSNE_ENOMEM, "knn cross: workspace of %zu bytes, %zu needed", ws_bytes, c.bytes());
    if ((st = check_base(workspace, "knn cross workspace"))) return st;
    // radius mode needs the certified keys: the FP8 variant takes the CUDA-core path
    const bool tc = exact_on_tensor_cores(o, k) && !(radius_d2 && o.precision == ATSNE_FP8_RERANK);
    if (tc)  // both prep kernels check their rows for non-finite values
        return knn_exact_tc(Xc, Nc, D, nullptr, Nq, k, plan, tws, idx_out, d2_out, stream, Xq, radius_d2);
    if ((st = check_finite(Xc, Nc * (int64_t)D, stream))) return st;
    if ((st = check_finite(Xq, Nq * (int64_t)D, stream))) return st;
    if ((st = knn_bruteforce_rows(Xc, Nc, D, nullptr, nullptr, nullptr, Nq, k, idx_out, d2_out, stream,
                                  Xq)))
        return st;
    return radius_d2 ? radius_filter_launch(idx_out, d2_out, Nq, k, radius_d2, stream) : ATSNE_OK;
}

atsne_status atsne_row_dmax(const float *d2, int64_t rows, int32_t k, float *dmax_out, void *stream) {
    if (rows < 0 || k < 1) return set_error(ATSNE_EINVAL, "row dmax: rows=%lld k=%d", (long long)rows, k);
    if (rows > 0 && (!d2 || !dmax_out)) return set_error(ATSNE_EINVAL, "row dmax: NULL pointer");
    return row_dmax_launch(d2, rows, k, dmax_out, static_cast<cudaStream_t>(stream));
}

atsne_status atsne_merge_neighbors(int32_t *idx, float *d2, int64_t rows, int32_t k,
                                   const int32_t *cand_idx, const float *cand_d2, int32_t kc,
                                   int32_t index_offset, uint8_t *changed, void *stream) {
    if (rows < 0 || k < 1 || kc < 0) return set_error(ATSNE_EINVAL, "merge neighbors: rows=%lld k=%d kc=%d",
                                                      (long long)rows, k, kc);
    if (rows == 0 || kc == 0) {
        if (rows > 0 && changed) {
            cudaError_t e = cudaMemsetAsync(changed, 0, (size_t)rows, static_cast<cudaStream_t>(stream));
            if (e != cudaSuccess) return cuda_error(e, "merge neighbors");
        }
        return ATSNE_OK;
    }
    if (!idx || !d2 || !cand_idx || !cand_d2) return set_error(ATSNE_EINVAL, "merge neighbors: NULL pointer");
    return merge_neighbors_launch(idx, d2, rows, k, cand_idx, cand_d2, kc, index_offset, changed,
                                  static_cast<cudaStream_t>(stream));
}

atsne_status atsne_commit_rows(const int32_t *rows, int64_t S, int64_t N, int32_t k, const int32_t *ti,
                               const float *td, const float *tp, const float *tb, int32_t *idx,
                               float *d2, float *P_cond, float *beta, float *rho, void *stream) {
    if (S < 0 || N < 1 || k < 1) return set_error(ATSNE_EINVAL, "commit rows: S=%lld N=%lld k=%d",
                                                  (long long)S, (long long)N, k);
    if (S == 0) return ATSNE_OK;
    if (!rows || !ti || !td || !tp || !idx || !d2 || !P_cond)
        return set_error(ATSNE_EINVAL, "commit rows: NULL pointer");
    if (!tb) beta = nullptr;
    return refine_scatter_launch(rows, S, N, k, ti, td, tp, tb, idx, d2, P_cond, beta, rho,
                                 static_cast<cudaStream_t>(stream));
}

atsne_status atsne_kde_map(const float *Y, int64_t N, const float *rho, const uint8_t *selected,
                           float x0, float y0, float pixel, int32_t width, int32_t height, float h,
                           float cutoff, float lens_k, float *f_out, float *s_out, float *a_out,
                           float *alpha_out, void *stream) {
    if (!Y) return set_error(ATSNE_EINVAL, "kde: Y is NULL");
    if (N < 1 || N > INT32_MAX) return set_error(ATSNE_EINVAL, "kde: N=%lld", (long long)N);
    if (width < 1 || height < 1 || !(pixel > 0.f) || !(h > 0.f) || !(cutoff >= 0.f) ||
        !isfinite(x0) || !isfinite(y0) || !isfinite(lens_k))
        return set_error(ATSNE_EINVAL, "kde: width=%d height=%d pixel=%g h=%g cutoff=%g", width, height,
                         (double)pixel, (double)h, (double)cutoff);
    return kde_launch(Y, N, rho, selected, x0, y0, pixel, width, height, h, cutoff, lens_k, f_out,
                      s_out, a_out, alpha_out, static_cast<cudaStream_t>(stream));
}

atsne_status atsne_knn_precision(const int32_t *idx_approx, const int32_t *idx_exact,
                                 int64_t rows, int32_t k, float *rho_i_out, double *rho_sum_dev,
                                 void *stream) {
    if (!idx_approx || !idx_exact) return set_error(ATSNE_EINVAL, "precision: NULL pointer");
    if (rows < 0 || k < 1 || k > 4096) return set_error(ATSNE_EINVAL, "precision: rows=%lld k=%d", (long long)rows, k);
    return precision_launch(idx_approx, idx_exact, rows, k, rho_i_out, rho_sum_dev,
                            static_cast<cudaStream_t>(stream));
}

atsne_status atsne_forest_layout(int64_t N, int32_t D, const atsne_knn_opts *opts,
                                 atsne_forest_layout_t *out) {
    atsne_knn_opts o = opts_or_default(opts);
    o.method = ATSNE_KNN_FOREST;
    atsne_status st = validate_knn_opts(o);
    if (st) return st;
    if (N < 2 || N > INT32_MAX || D < 1 || !out) return set_error(ATSNE_EINVAL, "forest layout: bad arguments");
    forest_layout(N, o.trees, o.leaf_size, out);
    return ATSNE_OK;
}

atsne_status atsne_forest_build(const float *X, int64_t N, int32_t D, const atsne_knn_opts *opts,
                                void *forest, size_t forest_bytes, void *workspace,
                                size_t ws_bytes, void *stream_) {
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    atsne_knn_opts o = opts_or_default(opts);
    o.method = ATSNE_KNN_FOREST;
    atsne_status st = validate_knn_opts(o);
    if (st) return st;
    if (!X || !forest || N < 2 || N > INT32_MAX || D < 1) return set_error(ATSNE_EINVAL, "forest build: bad arguments");
    if (forest_bytes < forest_layout(N, o.trees, o.leaf_size, nullptr))
        return set_error(ATSNE_ENOMEM, "forest build: forest buffer too small");
    if ((st = check_base(forest, "forest build: forest"))) return st;
    if ((st = check_base(workspace, "forest build: workspace"))) return st;
    if ((st = check_finite(X, N * (int64_t)D, stream))) return st;
    return forest_build_launch(X, forest_view(forest, N, D, o), workspace, ws_bytes, stream);
}

atsne_status atsne_forest_query(const float *X, int64_t N, int32_t D, const void *forest,
                                const int32_t *queries, int64_t S, int32_t k,
                                const atsne_knn_opts *opts, int32_t *idx_out, float *d2_out,
                                int64_t *evaluated_out, void *workspace, size_t ws_bytes,
                                void *stream_) {
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    atsne_status st = validate_xk(X, N, D, k);
    if (st) return st;
    atsne_knn_opts o = opts_or_default(opts);
    o.method = ATSNE_KNN_FOREST;
    if ((st = validate_knn_opts(o))) return st;
    if (!forest || !idx_out || !d2_out) return set_error(ATSNE_EINVAL, "forest query: NULL pointer");
    if (queries && S < 0) return set_error(ATSNE_EINVAL, "forest query: S < 0");
    if ((st = check_base(forest, "forest query: forest"))) return st;
    if ((st = check_base(workspace, "forest query: workspace"))) return st;
    const int64_t nq = queries ? S : N;
    if (nq == 0) return ATSNE_OK;
    if (queries && (st = check_indices(queries, S, N, stream))) return st;
    return forest_query_launch(X, forest_view(const_cast<void *>(forest), N, D, o), queries, nq, k,
                               o.checks, queue_capacity(o), idx_out, d2_out, evaluated_out, workspace,
                               ws_bytes, stream);
}

size_t atsne_forest_buckets_bytes(int64_t N, int32_t depth, int32_t trees) {
    if (N < 0 || depth < 0 || depth > 25 || trees < 1) return 0;
    return buckets_layout(N, depth, trees, nullptr);
}


atsne_status atsne_forest_insert(const float *X, int64_t N_built, int64_t N_old, int64_t N_new, int32_t D,
                                 const atsne_knn_opts *opts, const void *forest, const void *buckets_in,
                                 void *buckets_out, size_t out_bytes, int32_t *max_bucket_out, void *workspace,
                                 size_t ws_bytes, void *stream_) {
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (!X) return set_error(ATSNE_EINVAL, "forest insert: NULL X");
    if (N_new < N_old) return set_error(ATSNE_EINVAL, "forest insert: N_new=%lld < N_old=%lld",
                                        (long long)N_new, (long long)N_old);
    UpdateArgs a;
    atsne_status st = update_args(X, N_built, N_old, N_new, N_new, D, opts, forest, buckets_in, buckets_out,
                                  out_bytes, workspace, ws_bytes, "forest insert", &a);
    if (st) return st;
    if (N_new > N_old && (st = check_finite(X + N_old * (int64_t)D, (N_new - N_old) * (int64_t)D, stream)))
        return st;
    if ((st = forest_insert_launch(X, N_old, N_new, D, a.f, a.perm_in, a.ofs_in, a.stride_in, a.out, a.w, stream)))
        return st;
    return read_max_bucket(a.w, max_bucket_out, stream);
}

atsne_status atsne_forest_delete(const int32_t *rows, int64_t R, int64_t N_built, int64_t N, int32_t D,
                                 const atsne_knn_opts *opts, const void *forest, const void *buckets_in,
                                 void *buckets_out, size_t out_bytes, int32_t *max_bucket_out, void *workspace,
                                 size_t ws_bytes, void *stream_) {
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (R < 0 || R > N || (R > 0 && !rows))
        return set_error(ATSNE_EINVAL, "forest delete: R=%lld N=%lld", (long long)R, (long long)N);
    UpdateArgs a;
    atsne_status st = update_args(nullptr, N_built, N, N - R, N, D, opts, forest, buckets_in, buckets_out,
                                  out_bytes, workspace, ws_bytes, "forest delete", &a);
    if (st) return st;
    if ((st = forest_delete_launch(rows, R, N, a.f, a.perm_in, a.ofs_in, a.stride_in, a.out, a.w, stream)))
        return st;
    return read_max_bucket(a.w, max_bucket_out, stream);
}

atsne_status atsne_forest_query_buckets(const float *X, int64_t N, int32_t D, int64_t N_built, const void *forest,
                                        const void *buckets, int32_t max_bucket, const int32_t *queries, int64_t S,
                                        int32_t k, const atsne_knn_opts *opts, int32_t *idx_out, float *d2_out,
                                        int64_t *evaluated_out, void *workspace, size_t ws_bytes, void *stream_) {
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    atsne_status st = validate_xk(X, N, D, k);
    if (st) return st;
    atsne_knn_opts o = opts_or_default(opts);
    o.method = ATSNE_KNN_FOREST;
    if ((st = validate_knn_opts(o))) return st;
    if (!forest || !buckets || !idx_out || !d2_out)
        return set_error(ATSNE_EINVAL, "forest query buckets: NULL pointer");
    if (N_built < 2 || N_built > INT32_MAX || max_bucket < 1 || max_bucket > N)
        return set_error(ATSNE_EINVAL, "forest query buckets: N_built=%lld max_bucket=%d", (long long)N_built,
                         max_bucket);
    if (queries && S < 0) return set_error(ATSNE_EINVAL, "forest query buckets: S < 0");
    if ((st = check_base(forest, "forest query buckets")) || (st = check_base(buckets, "forest query buckets")) ||
        (st = check_base(workspace, "forest query buckets")))
        return st;
    ForestView f = forest_view(const_cast<void *>(forest), N_built, D, o);
    size_t off = 0;
    buckets_layout(N, f.depth, o.trees, &off);
    char *b = static_cast<char *>(const_cast<void *>(buckets));
    f.N = N;
    f.perm = reinterpret_cast<int32_t *>(b);
    f.leaf_ofs = reinterpret_cast<int32_t *>(b + off);
    f.ofs_stride = ((int64_t)1 << f.depth) + 1;
    f.leaf_size = max_bucket;
    const int64_t nq = queries ? S : N;
    if (nq == 0) return ATSNE_OK;
    if (queries && (st = check_indices(queries, S, N, stream))) return st;
    // the lists are sized for buckets of max_bucket points: a larger bucket is flagged
    if ((st = bucket_bound_check(f.leaf_ofs, o.trees, f.depth, max_bucket, stream))) return st;
    return forest_query_launch(X, f, queries, nq, k, o.checks, queue_capacity(o), idx_out, d2_out, evaluated_out,
                               workspace, ws_bytes, stream);
}

atsne_status atsne_check(void *stream) {
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_error(e, "check: stream synchronize");
    int *p = device_status_word();
    if (!p) return set_error(ATSNE_ECUDA, "check: no status word");
    int v = 0;
    e = cudaMemcpy(&v, p, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "check: read status");
    const int zero = 0;
    e = cudaMemcpy(p, &zero, sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "check: clear status");
    switch (v) {
    case DEV_OK:
        return ATSNE_OK;
    case DEV_NONFINITE:
        return set_error(ATSNE_EINVAL, "device: non-finite input");
    case DEV_MALFORMED:
        return set_error(ATSNE_EINVAL, "device: index out of range or malformed neighbour list");
    case DEV_TIMEOUT:
        return set_error(ATSNE_ETIMEOUT, "device: a bounded wait expired");
    default:
        return set_error(ATSNE_ECUDA, "device: unknown status %d", v);
    }
}

atsne_status atsne_set_wait_limit(uint64_t ns) {
    set_pipeline_wait_ns(ns);
    return ATSNE_OK;
}

atsne_status atsne_profile_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (on && g_prof_pool.empty()) {
        g_prof_pool.resize(PROF_POOL);
        for (auto &r : g_prof_pool) {
            r.name = "";
            if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
                g_prof_pool.clear();
                return set_error(ATSNE_ECUDA, "profile: event creation failed");
            }
        }
    }
    g_prof_on = on != 0;
    return ATSNE_OK;
}

atsne_status atsne_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_used = 0;
    return ATSNE_OK;
}

atsne_status atsne_profile_read(const char *kernel, int64_t *launches, double *total_ms) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int64_t n = 0;
    double ms = 0.0;
    for (size_t i = 0; i < g_prof_used; ++i) {
        const ProfRec &r = g_prof_pool[i];
        if (kernel && strcmp(kernel, r.name) != 0) continue;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return cuda_error(e, "profile: event synchronize");
        float t = 0.f;
        e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) return cuda_error(e, "profile: elapsed time");
        ms += t;
        ++n;
    }
    if (launches) *launches = n;
    if (total_ms) *total_ms = ms;
    return ATSNE_OK;
}

}  // extern "C"
