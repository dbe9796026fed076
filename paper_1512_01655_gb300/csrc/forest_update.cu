// Adding points to and removing points from a built forest (Sec. 5.3.1,
// Sec. 5.3.2). The split dimensions and values stay; only the leaf buckets
// change, so each tree gets its own leaf offsets:
//   insertion: a new point descends every tree by the search's rule (value
//              below the split: left child 2v + 1, else right child 2v + 2)
//              and joins the reached leaf's bucket after the points already
//              there, the new points in index order;
//   deletion:  the listed points leave every bucket, the others keep their
//              order and are renumbered as the corpus rows are (j becomes j
//              minus the number of deleted points below j).
// One thread per (tree, new point) descends; one thread per (tree, leaf)
// copies or compacts a bucket, so every bucket keeps its order without a sort
// of the whole tree; a per-tree block scan turns bucket sizes into offsets.
#include "common.cuh"
#include "internal.h"

namespace atsne {
namespace {

constexpr int FU_SCAN_THREADS = 1024;

__global__ void fu_descend_kernel(const float *__restrict__ X, int D, int64_t N_old, int64_t B, int T,
                                  int64_t n_int, const int32_t *__restrict__ split_dim,
                                  const float *__restrict__ split_val, int32_t *__restrict__ leaf) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= B * T) return;
    const int t = (int)(g / B);
    const int64_t b = g - (int64_t)t * B;
    const float *x = X + (N_old + b) * (int64_t)D;
    const int32_t *sd = split_dim + (int64_t)t * n_int;
    const float *sv = split_val + (int64_t)t * n_int;
    int64_t v = 0;
    while (v < n_int) v = x[sd[v]] < sv[v] ? 2 * v + 1 : 2 * v + 2;
    leaf[g] = (int32_t)(v - n_int);
}

// sizes[t][m + 1] = old size of bucket m (sizes[t][0] = 0); with `dead`, only
// the points that stay are counted.
__global__ void fu_sizes_kernel(const int32_t *__restrict__ perm_in, int64_t n_in, const int32_t *__restrict__ ofs_in,
                                int64_t stride_in, int T, int64_t L, const int32_t *__restrict__ dead,
                                int32_t *__restrict__ sizes) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= L * T) return;
    const int t = (int)(g / L);
    const int64_t m = g - (int64_t)t * L;
    const int32_t *oi = ofs_in + (int64_t)t * stride_in;
    int32_t n = oi[m + 1] - oi[m];
    if (dead) {
        const int32_t *pi = perm_in + (int64_t)t * n_in;
        n = 0;
        for (int32_t q = oi[m]; q < oi[m + 1]; ++q) n += dead[pi[q]] == 0;
    }
    sizes[(int64_t)t * (L + 1) + m + 1] = n;
    if (m == 0) sizes[(int64_t)t * (L + 1)] = 0;
}

__global__ void fu_count_new_kernel(const int32_t *__restrict__ leaf, int64_t B, int T, int64_t L,
                                    int32_t *__restrict__ sizes) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= B * T) return;
    const int t = (int)(g / B);
    atomicAdd(&sizes[(int64_t)t * (L + 1) + leaf[g] + 1], 1);
}

// In place, per tree (one block each): a[t][i] <- a[t][0] + ... + a[t][i].
__global__ void __launch_bounds__(FU_SCAN_THREADS) fu_scan_kernel(int32_t *__restrict__ ofs, int64_t L1) {
    __shared__ int32_t part[FU_SCAN_THREADS];
    int32_t *a = ofs + (int64_t)blockIdx.x * L1;
    const int64_t per = (L1 + FU_SCAN_THREADS - 1) / FU_SCAN_THREADS;
    const int64_t i0 = (int64_t)threadIdx.x * per;
    const int64_t i1 = i0 + per < L1 ? i0 + per : L1;
    int32_t s = 0;
    for (int64_t i = i0; i < i1; ++i) s += a[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < FU_SCAN_THREADS; o <<= 1) {
        const int32_t v = (int)threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int32_t run = threadIdx.x > 0 ? part[threadIdx.x - 1] : 0;
    for (int64_t i = i0; i < i1; ++i) {
        run += a[i];
        a[i] = run;
    }
}

// Insertion: the old bucket first, then a cursor for the new points.
__global__ void fu_copy_old_kernel(const int32_t *__restrict__ perm_in, int64_t N_old,
                                   const int32_t *__restrict__ ofs_in, int64_t stride_in, int T, int64_t L,
                                   const int32_t *__restrict__ ofs_out, int32_t *__restrict__ perm_out,
                                   int64_t N_new, int32_t *__restrict__ cursor) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= L * T) return;
    const int t = (int)(g / L);
    const int64_t m = g - (int64_t)t * L;
    const int32_t *oi = ofs_in + (int64_t)t * stride_in;
    const int32_t *pi = perm_in + (int64_t)t * N_old;
    int32_t *po = perm_out + (int64_t)t * N_new;
    int32_t w = ofs_out[(int64_t)t * (L + 1) + m];
    for (int32_t q = oi[m]; q < oi[m + 1]; ++q) po[w++] = pi[q];
    cursor[g] = w;
}

__global__ void fu_place_new_kernel(const int32_t *__restrict__ leaf, int64_t B, int T, int64_t L, int64_t N_old,
                                    int32_t *__restrict__ cursor, int32_t *__restrict__ perm_out, int64_t N_new) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= B * T) return;
    const int t = (int)(g / B);
    const int64_t b = g - (int64_t)t * B;
    const int32_t pos = atomicAdd(&cursor[(int64_t)t * L + leaf[g]], 1);
    perm_out[(int64_t)t * N_new + pos] = (int32_t)(N_old + b);
}

// Ascending order of a[0, n) by heapsort: O(n log n) in one thread, for the
// buckets that many new points reach at once (duplicate rows all land in one
// leaf), where an insertion sort would take O(n^2).
__device__ void heapsort_i32(int32_t *a, int32_t n) {
    auto sift = [&](int32_t r, int32_t end) {
        const int32_t x = a[r];
        for (;;) {
            int32_t c = 2 * r + 1;
            if (c >= end) break;
            if (c + 1 < end && a[c + 1] > a[c]) ++c;
            if (a[c] <= x) break;
            a[r] = a[c];
            r = c;
        }
        a[r] = x;
    };
    for (int32_t r = n / 2 - 1; r >= 0; --r) sift(r, n);
    for (int32_t end = n - 1; end > 0; --end) {
        const int32_t t = a[0];
        a[0] = a[end];
        a[end] = t;
        sift(0, end);
    }
}

// The new points of a bucket (placed by atomics) in index order: an insertion
// sort for the few a bucket usually gets, a heapsort beyond 32.
__global__ void fu_order_new_kernel(const int32_t *__restrict__ ofs_in, int64_t stride_in, int T, int64_t L,
                                    const int32_t *__restrict__ ofs_out, int32_t *__restrict__ perm_out,
                                    int64_t N_new, unsigned *__restrict__ bmax) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= L * T) return;
    const int t = (int)(g / L);
    const int64_t m = g - (int64_t)t * L;
    const int32_t *oi = ofs_in + (int64_t)t * stride_in;
    const int32_t *oo = ofs_out + (int64_t)t * (L + 1);
    int32_t *po = perm_out + (int64_t)t * N_new;
    const int32_t lo = oo[m] + (oi[m + 1] - oi[m]), hi = oo[m + 1];
    if (hi - lo > 32) {
        heapsort_i32(po + lo, hi - lo);
        atomicMax(bmax, (unsigned)(hi - oo[m]));
        return;
    }
    for (int32_t i = lo + 1; i < hi; ++i) {
        const int32_t x = po[i];
        int32_t j = i - 1;
        while (j >= lo && po[j] > x) {
            po[j + 1] = po[j];
            --j;
        }
        po[j + 1] = x;
    }
    atomicMax(bmax, (unsigned)(hi - oo[m]));
}

__global__ void fd_mark_kernel(const int32_t *__restrict__ rows, int64_t R, int64_t N, int32_t *__restrict__ dead,
                               int *status) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int32_t j = rows[r];
    if (j < 0 || j >= N) {
        raise_status(status, DEV_MALFORMED);
        return;
    }
    if (atomicExch(&dead[j], 1) != 0) raise_status(status, DEV_MALFORMED);
}

// Deletion: the bucket's remaining points, renumbered, in order.
__global__ void fd_compact_kernel(const int32_t *__restrict__ perm_in, int64_t N, const int32_t *__restrict__ ofs_in,
                                  int64_t stride_in, int T, int64_t L, const int32_t *__restrict__ dead,
                                  const int64_t *__restrict__ before, const int32_t *__restrict__ ofs_out,
                                  int32_t *__restrict__ perm_out, int64_t n_out, unsigned *__restrict__ bmax) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= L * T) return;
    const int t = (int)(g / L);
    const int64_t m = g - (int64_t)t * L;
    const int32_t *oi = ofs_in + (int64_t)t * stride_in;
    const int32_t *pi = perm_in + (int64_t)t * N;
    int32_t *po = perm_out + (int64_t)t * n_out;
    const int32_t w0 = ofs_out[(int64_t)t * (L + 1) + m];
    int32_t w = w0;
    for (int32_t q = oi[m]; q < oi[m + 1]; ++q) {
        const int32_t p = pi[q];
        if (dead[p]) continue;
        // a malformed list (raised in the status word) leaves more points than
        // n_out; the writes stay inside the tree's row regardless
        if (w < n_out) po[w] = (int32_t)(p - before[p]);
        ++w;
    }
    atomicMax(bmax, (unsigned)(w - w0));
}

}  // namespace

size_t buckets_layout(int64_t N, int depth, int trees, size_t *off_ofs) {
    Carver c(nullptr);
    c.take<int32_t>((size_t)trees * (size_t)(N > 0 ? N : 1));
    const size_t o = (c.off + 255) & ~size_t(255);
    c.take<int32_t>((size_t)trees * (((size_t)1 << depth) + 1));
    if (off_ofs) *off_ofs = o;
    return c.bytes();
}

size_t update_workspace(Carver &c, int64_t N, int depth, int trees, UpdateWs *ws) {
    UpdateWs w;
    const size_t n = (size_t)(N > 0 ? N : 1);
    w.leaf = c.take<int32_t>((size_t)trees * n);
    w.cursor = c.take<int32_t>((size_t)trees << depth);
    w.dead = c.take<int32_t>(n);
    w.before = c.take<int64_t>(n + 1);
    w.total = c.take<int64_t>(1);
    w.scan = c.take<int64_t>(scan_partials_count(N));
    w.bmax = c.take<int32_t>(1);
    if (ws) *ws = w;
    return c.bytes();
}

atsne_status forest_insert_launch(const float *X, int64_t N_old, int64_t N_new, int D, const ForestView &f,
                                  const int32_t *perm_in, const int32_t *ofs_in, int64_t stride_in,
                                  const BucketsView &out, const UpdateWs &w, cudaStream_t stream) {
    const int T = f.trees;
    const int64_t L = (int64_t)1 << f.depth, B = N_new - N_old;
    cudaError_t e = cudaMemsetAsync(w.bmax, 0, sizeof(int32_t), stream);
    if (e != cudaSuccess) return cuda_error(e, "forest insert memset");
    if (B > 0)
        ATSNE_TRY(launch_kernel("forest_update", fu_descend_kernel, ceil_div(B * T, 256), 256, 0, stream, X, D,
                                N_old, B, T, f.n_internal, (const int32_t *)f.split_dim, (const float *)f.split_val,
                                w.leaf));
    ATSNE_TRY(launch_kernel("forest_update", fu_sizes_kernel, ceil_div(L * T, 256), 256, 0, stream, perm_in, N_old,
                            ofs_in, stride_in, T, L, (const int32_t *)nullptr, out.ofs));
    if (B > 0)
        ATSNE_TRY(launch_kernel("forest_update", fu_count_new_kernel, ceil_div(B * T, 256), 256, 0, stream,
                                (const int32_t *)w.leaf, B, T, L, out.ofs));
    ATSNE_TRY(launch_kernel("forest_update", fu_scan_kernel, T, FU_SCAN_THREADS, 0, stream, out.ofs, L + 1));
    ATSNE_TRY(launch_kernel("forest_update", fu_copy_old_kernel, ceil_div(L * T, 256), 256, 0, stream, perm_in,
                            N_old, ofs_in, stride_in, T, L, (const int32_t *)out.ofs, out.perm, N_new, w.cursor));
    if (B > 0)
        ATSNE_TRY(launch_kernel("forest_update", fu_place_new_kernel, ceil_div(B * T, 256), 256, 0, stream,
                                (const int32_t *)w.leaf, B, T, L, N_old, w.cursor, out.perm, N_new));
    return launch_kernel("forest_update", fu_order_new_kernel, ceil_div(L * T, 256), 256, 0, stream, ofs_in,
                         stride_in, T, L, (const int32_t *)out.ofs, out.perm, N_new,
                         reinterpret_cast<unsigned *>(w.bmax));
}

atsne_status forest_delete_launch(const int32_t *rows, int64_t R, int64_t N, const ForestView &f,
                                  const int32_t *perm_in, const int32_t *ofs_in, int64_t stride_in,
                                  const BucketsView &out, const UpdateWs &w, cudaStream_t stream) {
    const int T = f.trees;
    const int64_t L = (int64_t)1 << f.depth;
    cudaError_t e = cudaMemsetAsync(w.dead, 0, sizeof(int32_t) * (size_t)N, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.bmax, 0, sizeof(int32_t), stream);
    if (e != cudaSuccess) return cuda_error(e, "forest delete memset");
    if (R > 0)
        ATSNE_TRY(launch_kernel("forest_update", fd_mark_kernel, ceil_div(R, 256), 256, 0, stream, rows, R, N,
                                w.dead, device_status_word()));
    ATSNE_TRY(scan_rowlen(w.dead, N, 0, w.before, w.total, w.scan, stream));
    ATSNE_TRY(launch_kernel("forest_update", fu_sizes_kernel, ceil_div(L * T, 256), 256, 0, stream, perm_in, N,
                            ofs_in, stride_in, T, L, (const int32_t *)w.dead, out.ofs));
    ATSNE_TRY(launch_kernel("forest_update", fu_scan_kernel, T, FU_SCAN_THREADS, 0, stream, out.ofs, L + 1));
    return launch_kernel("forest_update", fd_compact_kernel, ceil_div(L * T, 256), 256, 0, stream, perm_in, N,
                         ofs_in, stride_in, T, L, (const int32_t *)w.dead, (const int64_t *)w.before,
                         (const int32_t *)out.ofs, out.perm, N - R, reinterpret_cast<unsigned *>(w.bmax));
}

// Raises DEV_MALFORMED when a bucket of an updated forest holds more points
// than `bound`, the leaf size a search over the buckets sizes its lists by.
__global__ void fu_bucket_bound_kernel(const int32_t *__restrict__ ofs, int T, int64_t L, int bound, int *status) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= L * T) return;
    const int t = (int)(g / L);
    const int64_t m = g - (int64_t)t * L;
    const int32_t *o = ofs + (int64_t)t * (L + 1);
    if (o[m + 1] - o[m] > bound) raise_status(status, DEV_MALFORMED);
}

atsne_status bucket_bound_check(const int32_t *ofs, int trees, int depth, int bound, cudaStream_t stream) {
    const int64_t L = (int64_t)1 << depth;
    return launch_kernel("forest_update", fu_bucket_bound_kernel, ceil_div(L * trees, 256), 256, 0, stream, ofs,
                         trees, L, bound, device_status_word());
}

}  // namespace atsne
