// Small kernels: precision rho (Eq. 9), the row scatter of a refinement, and the
// byte copy of 8-bit integer data.
#include "common.cuh"
#include "internal.h"

namespace atsne {
namespace {

// rho_i = |N^A_i intersect N_i| / k, Eq. 9 (Sec. 4.1). One warp per row: the
// exact row is staged in shared memory and every approximate entry is looked
// up in it. Hit counts are summed as integers held in a double (exact), so
// the total does not depend on the order of the atomic additions.
__global__ void __launch_bounds__(128)
precision_kernel(const int32_t *__restrict__ a, const int32_t *__restrict__ e, int64_t rows, int k,
                 float *__restrict__ rho_i, double *__restrict__ hits_total) {
    extern __shared__ int ex[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t r = (int64_t)blockIdx.x * 4 + w;
    int *row = ex + w * k;
    int hits = 0;
    if (r < rows) {
        for (int t = lane; t < k; t += 32) row[t] = e[r * k + t];
        __syncwarp();
        for (int t = lane; t < k; t += 32) {
            const int j = a[r * k + t];
            bool found = false;
            for (int u = 0; u < k; ++u) found |= j >= 0 && row[u] == j;  // -1: absent
            hits += found;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) hits += __shfl_xor_sync(0xffffffffu, hits, o);
        if (lane == 0 && rho_i) rho_i[r] = (float)hits / (float)k;
    }
    __shared__ int cta_hits[4];
    if (lane == 0) cta_hits[w] = hits;
    __syncthreads();
    if (threadIdx.x == 0 && hits_total) {
        const int s = cta_hits[0] + cta_hits[1] + cta_hits[2] + cta_hits[3];
        if (s) atomicAdd(hits_total, (double)s);
    }
}

__global__ void scale_kernel(double *v, double f) { *v *= f; }

// Copy S refined rows (idx, d2, P) into their places in the [N][k] state and
// set beta and rho (Sec. 4.3: rho_i = 1 for a refined point).
__global__ void refine_scatter_kernel(const int32_t *__restrict__ subset, int64_t S, int64_t N, int k,
                                      const int32_t *__restrict__ ti, const float *__restrict__ td,
                                      const float *__restrict__ tp, const float *__restrict__ tb,
                                      int32_t *__restrict__ idx, float *__restrict__ d2,
                                      float *__restrict__ P, float *__restrict__ beta,
                                      float *__restrict__ rho) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= S * k) return;
    const int64_t s = e / k;
    const int t = (int)(e - s * k);
    const int64_t i = subset[s];
    if (i < 0 || i >= N) return;  // flagged by the caller's index check
    idx[i * k + t] = ti[e];
    d2[i * k + t] = td[e];
    P[i * k + t] = tp[e];
    if (t == 0) {
        if (beta) beta[i] = tb[s];
        if (rho) rho[i] = 1.f;
    }
}

// The union of listed rows: one bit per corpus row.
__global__ void mark_kernel(const int32_t *__restrict__ lists, int64_t total, int64_t N,
                            uint32_t *__restrict__ bitmap) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int64_t i = lists[e];
    if (i < 0 || i >= N) return;  // flagged by the caller's index check
    atomicOr(&bitmap[i >> 5], 1u << (i & 31));
}

// Ordered compaction of the bitmap by one block: thread t takes a contiguous
// run of words, a block-wide exclusive scan of the runs' popcounts gives each
// its output offset. The list is padded to out_rows with its first entry (a
// padded row repeats that point's refinement and writes the same values), or
// with -1 when no listed index was in range (such rows are never written).
constexpr int UNION_THREADS = 1024;
__global__ void __launch_bounds__(UNION_THREADS)
union_compact_kernel(const uint32_t *__restrict__ bitmap, int64_t words, int32_t *__restrict__ out,
                     int64_t out_rows, int64_t *__restrict__ count) {
    __shared__ int64_t warp_tot[UNION_THREADS / 32];
    __shared__ int64_t s_total;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t per = (words + UNION_THREADS - 1) / UNION_THREADS;
    const int64_t w0 = tid * per, w1 = w0 + per < words ? w0 + per : words;
    int64_t mine = 0;
    for (int64_t q = w0; q < w1; ++q) mine += __popc(bitmap[q]);
    int64_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        int64_t v = warp_tot[lane];
        int64_t vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) vi += t;
        }
        warp_tot[lane] = vi - v;  // exclusive prefix of the warps
        if (lane == 31) s_total = vi;
    }
    __syncthreads();
    int64_t pos = warp_tot[w] + incl - mine;
    for (int64_t q = w0; q < w1; ++q) {
        uint32_t b = bitmap[q];
        while (b) {
            const int bit = __ffs(b) - 1;
            b &= b - 1;
            if (pos < out_rows) out[pos] = (int32_t)(q * 32 + bit);
            ++pos;
        }
    }
    __syncthreads();
    const int64_t n = s_total < out_rows ? s_total : out_rows;
    const int32_t first = n > 0 ? out[0] : -1;  // -1: nothing valid listed (an error is flagged)
    for (int64_t r = n + tid; r < out_rows; r += UNION_THREADS) out[r] = first;
    if (tid == 0 && count) *count = s_total;
}

// Insertion of new points into existing neighbourhoods (Eq. 11, Sec. 5.3.1),
// for a batch: row i keeps the k smallest of its list and its kc candidates
// (indices + offset) under the (d^2, index) order. A candidate ties with the
// farthest listed point only at a larger index, so it enters exactly when it
// is strictly closer (Eq. 11's "<"). One warp per row; changed[i] = 1 if the
// list changed.
__global__ void __launch_bounds__(128)
merge_neighbors_kernel(int32_t *__restrict__ idx, float *__restrict__ d2, int64_t rows, int k,
                       const int32_t *__restrict__ cidx, const float *__restrict__ cd2, int kc,
                       int32_t offset, uint8_t *__restrict__ changed) {
    const int lane = threadIdx.x & 31;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= rows) return;
    int32_t *ri = idx + r * k;
    float *rd = d2 + r * k;
    const int32_t *ci = cidx + r * kc;
    const float *cd = cd2 + r * kc;
    // both lists are sorted; candidate t belongs to the k smallest of the
    // union when fewer than k entries precede it: its t predecessors among
    // the candidates and the listed entries below it (binary search). The
    // entering candidates are therefore a prefix of length m.
    int m = 0;
    for (int t = lane; t < kc; t += 32) {
        const float d = cd[t];
        const int32_t j = ci[t] + offset;
        int lo = 0, hi = k;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (rd[mid] < d || (rd[mid] == d && ri[mid] < j))
                lo = mid + 1;
            else
                hi = mid;
        }
        m += (t + lo < k) ? 1 : 0;
    }
    m = (int)__reduce_add_sync(0xffffffffu, (unsigned)m);
    if (lane == 0 && changed) changed[r] = m > 0;
    if (m == 0) return;
    // lane 0 merges from the back: the k - m first listed entries and the m
    // first candidates; position o is written after every entry it held was read
    if (lane == 0) {
        int a = k - m - 1, b = m - 1;
        for (int o = k - 1; o >= 0 && b >= 0; --o) {
            const bool take_b = a < 0 || cd[b] > rd[a] || (cd[b] == rd[a] && ci[b] + offset > ri[a]);
            if (take_b) {
                rd[o] = cd[b];
                ri[o] = ci[b] + offset;
                --b;
            } else {
                rd[o] = rd[a];
                ri[o] = ri[a];
                --a;
            }
        }
    }
}

// hint[s] = d2[rows[s]][k-1]: a listed row's current k-th squared distance,
// an upper bound of its exact one when the row lists k real points.
// d_i^Max of Eq. 11 over N_i as it stands: the largest distance among the
// row's present entries (+inf marks an absent one), +inf when none is left.
__global__ void row_dmax_kernel(const float *__restrict__ d2, int64_t rows, int k, float *__restrict__ dmax) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const float *r = d2 + i * k;
    float m = -1.f;
    for (int j = 0; j < k; ++j) {
        const float v = r[j];
        if (v < INFINITY) m = fmaxf(m, v);
    }
    dmax[i] = m < 0.f ? INFINITY : m;
}

__global__ void gather_hint_kernel(const int32_t *__restrict__ rows, int64_t S, int64_t N, int k,
                                   const float *__restrict__ d2, float *__restrict__ hint) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int64_t i = rows[s];
    hint[s] = (i >= 0 && i < N) ? d2[i * k + k - 1] : INFINITY;
}

// Byte copy of X (rows padded to Dp16 bytes with zeros) and, if nx8 is given,
// the rows' exact squared norms; *bad is raised if any value is not an integer
// in [0, 255] (then the copy is not used). One warp per row, four values per lane.
__global__ void __launch_bounds__(256) u8_copy_kernel(const float *__restrict__ X, int64_t N, int D,
                                                         int Dp16, uint8_t *__restrict__ xu8,
                                                         uint32_t *__restrict__ nx8, unsigned *bad) {
    const int lane = threadIdx.x & 31;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= N) return;
    const float *x = X + r * D;
    uint32_t *out = reinterpret_cast<uint32_t *>(xu8 + r * Dp16);
    uint32_t sq = 0;
    bool ok = true;
    for (int d4 = 4 * lane; d4 < Dp16; d4 += 128) {
        uint32_t word = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float v = d4 + i < D ? x[d4 + i] : 0.f;
            ok &= v >= 0.f && v <= 255.f && v == rintf(v);  // false for NaN
            const uint32_t b = ok ? (uint32_t)v : 0u;
            word |= b << (8 * i);
            sq += b * b;
        }
        out[d4 >> 2] = word;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicOr(bad, 1u);
    if (lane == 0 && nx8) nx8[r] = sq;
}

// ---- deletion (Sec. 5.3.2) ----
// dead[j] = 1 for every listed row; a row out of range or listed twice raises
// the status word.
__global__ void delete_mark_kernel(const int32_t *__restrict__ rows, int64_t R, int64_t N,
                                   int32_t *__restrict__ dead, int *status) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int32_t j = rows[r];
    if (j < 0 || j >= N) {
        raise_status(status, DEV_MALFORMED);
        return;
    }
    if (atomicExch(&dead[j], 1) != 0) raise_status(status, DEV_MALFORMED);
}

// One warp per row i that stays: its new row i - before[i] receives X's row,
// the entries that stay (renumbered j - before[j], in their order), absent
// entries (-1, +inf) for the rest, beta, and rho less 1/k per entry removed.
__global__ void __launch_bounds__(256)
delete_compact_kernel(const float *__restrict__ X, int64_t N, int D, int k, const int32_t *__restrict__ dead,
                      const int64_t *__restrict__ before, const int32_t *__restrict__ idx,
                      const float *__restrict__ d2, const float *__restrict__ beta,
                      const float *__restrict__ rho, float *__restrict__ Xo, int32_t *__restrict__ io,
                      float *__restrict__ d2o, float *__restrict__ bo, float *__restrict__ ro) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= N || dead[i]) return;
    const int64_t ni = i - before[i];
    for (int d = lane; d < D; d += 32) Xo[ni * D + d] = X[i * D + d];
    int c = 0, removed = 0;
    for (int t0 = 0; t0 < k; t0 += 32) {
        const int t = t0 + lane;
        const int32_t j = t < k ? idx[i * k + t] : -1;
        const bool gone = j >= 0 && dead[j];
        const bool stays = j >= 0 && !gone;
        removed += gone;
        const unsigned m = __ballot_sync(0xffffffffu, stays);
        if (stays) {
            const int pos = c + __popc(m & ((1u << lane) - 1u));
            io[ni * k + pos] = (int32_t)(j - before[j]);
            d2o[ni * k + pos] = d2[i * k + t];
        }
        c += __popc(m);
    }
    for (int t = c + lane; t < k; t += 32) {
        io[ni * k + t] = -1;
        d2o[ni * k + t] = INFINITY;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) removed += __shfl_xor_sync(0xffffffffu, removed, o);
    if (lane == 0) {
        if (beta) bo[ni] = beta[i];
        if (rho) ro[ni] = fmaxf(0.f, rho[i] - (float)removed / (float)k);
    }
}

}  // namespace

atsne_status row_dmax_launch(const float *d2, int64_t rows, int k, float *dmax, cudaStream_t stream) {
    if (rows <= 0) return ATSNE_OK;
    return launch_kernel("row_dmax", row_dmax_kernel, ceil_div(rows, 256), 256, 0, stream, d2, rows, k, dmax);
}

atsne_status gather_hint_launch(const int32_t *rows, int64_t S, int64_t N, int k, const float *d2,
                                float *hint, cudaStream_t stream) {
    if (S <= 0) return ATSNE_OK;
    return launch_kernel("gather_hint", gather_hint_kernel, ceil_div(S, 256), 256, 0, stream, rows, S, N,
                         k, d2, hint);
}

atsne_status merge_neighbors_launch(int32_t *idx, float *d2, int64_t rows, int k, const int32_t *cidx,
                                    const float *cd2, int kc, int32_t offset, uint8_t *changed,
                                    cudaStream_t stream) {
    if (rows <= 0) return ATSNE_OK;
    return launch_kernel("merge_neighbors", merge_neighbors_kernel, ceil_div(rows * 32, 128), 128, 0,
                         stream, idx, d2, rows, k, cidx, cd2, kc, offset, changed);
}

atsne_status union_launch(const int32_t *lists, int64_t total, int64_t N, uint32_t *bitmap,
                          int32_t *out, int64_t out_rows, int64_t *count, cudaStream_t stream) {
    const int64_t words = (N + 31) / 32;
    cudaError_t e = cudaMemsetAsync(bitmap, 0, sizeof(uint32_t) * (size_t)words, stream);
    if (e != cudaSuccess) return cuda_error(e, "union memset");
    if (total > 0)
        ATSNE_TRY(launch_kernel("refine_mark", mark_kernel, ceil_div(total, 256), 256, 0, stream, lists,
                                total, N, bitmap));
    return launch_kernel("refine_union", union_compact_kernel, 1, UNION_THREADS, 0, stream,
                         (const uint32_t *)bitmap, words, out, out_rows, count);
}

atsne_status precision_launch(const int32_t *a, const int32_t *e, int64_t rows, int k,
                              float *rho_i, double *rho_sum, cudaStream_t stream) {
    if (rho_sum) {
        cudaError_t err = cudaMemsetAsync(rho_sum, 0, sizeof(double), stream);
        if (err != cudaSuccess) return cuda_error(err, "precision memset");
    }
    if (rows > 0)
        ATSNE_TRY(launch_kernel("knn_precision", precision_kernel, ceil_div(rows, 4), 128,
                                sizeof(int) * 4 * k, stream, a, e, rows, k, rho_i, rho_sum));
    if (rho_sum)
        ATSNE_TRY(launch_kernel("knn_precision_scale", scale_kernel, 1, 1, 0, stream, rho_sum,
                                1.0 / (double)k));
    return ATSNE_OK;
}

atsne_status refine_scatter_launch(const int32_t *subset, int64_t S, int64_t N, int k, const int32_t *ti,
                                   const float *td, const float *tp, const float *tb, int32_t *idx,
                                   float *d2, float *P, float *beta, float *rho,
                                   cudaStream_t stream) {
    if (S <= 0) return ATSNE_OK;
    return launch_kernel("refine_scatter", refine_scatter_kernel, ceil_div(S * k, 256), 256, 0,
                         stream, subset, S, N, k, ti, td, tp, tb, idx, d2, P, beta, rho);
}

size_t delete_workspace(Carver &c, int64_t N, int D, int k, DeleteWs *ws) {
    DeleteWs w;
    w.dead = c.take<int32_t>((size_t)N);
    w.before = c.take<int64_t>((size_t)N + 1);
    w.total = c.take<int64_t>(1);
    w.scan = c.take<int64_t>(scan_partials_count(N));
    w.X = c.take<float>((size_t)N * D);
    w.idx = c.take<int32_t>((size_t)N * k);
    w.d2 = c.take<float>((size_t)N * k);
    w.beta = c.take<float>((size_t)N);
    w.rho = c.take<float>((size_t)N);
    if (ws) *ws = w;
    return c.bytes();
}

atsne_status delete_launch(const int32_t *rows, int64_t R, float *X, int64_t N, int D, int k, float perplexity,
                           int32_t *idx, float *d2, float *P, float *beta, float *rho, const DeleteWs &w,
                           cudaStream_t stream) {
    int *status = device_status_word();
    cudaError_t e = cudaMemsetAsync(w.dead, 0, sizeof(int32_t) * (size_t)N, stream);
    if (e != cudaSuccess) return cuda_error(e, "delete memset");
    if (R > 0)
        ATSNE_TRY(launch_kernel("delete_mark", delete_mark_kernel, ceil_div(R, 256), 256, 0, stream, rows, R, N,
                                w.dead, status));
    ATSNE_TRY(scan_rowlen(w.dead, N, 0, w.before, w.total, w.scan, stream));
    ATSNE_TRY(launch_kernel("delete_compact", delete_compact_kernel, ceil_div(N * 32, 256), 256, 0, stream,
                            (const float *)X, N, D, k, (const int32_t *)w.dead, (const int64_t *)w.before,
                            (const int32_t *)idx, (const float *)d2, (const float *)beta, (const float *)rho,
                            w.X, w.idx, w.d2, w.beta, w.rho));
    const int64_t n = N - R;
    if (n <= 0) return ATSNE_OK;
    e = cudaMemcpyAsync(X, w.X, sizeof(float) * (size_t)n * D, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(idx, w.idx, sizeof(int32_t) * (size_t)n * k, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d2, w.d2, sizeof(float) * (size_t)n * k, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess && rho)
        e = cudaMemcpyAsync(rho, w.rho, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, stream);
    if (e != cudaSuccess) return cuda_error(e, "delete copy");
    return calibrate_launch(d2, n, k, perplexity, 1e-5f, 200, P, beta, stream);
}

atsne_status u8_copy_launch(const char *name, const float *X, int64_t N, int D, int Dp16, uint8_t *xu8,
                            uint32_t *nx8, unsigned *bad, cudaStream_t stream) {
    return launch_kernel(name, u8_copy_kernel, ceil_div(N * 32, 256), 256, 0, stream, X, N, D, Dp16, xu8, nx8,
                         bad);
}

}  // namespace atsne
