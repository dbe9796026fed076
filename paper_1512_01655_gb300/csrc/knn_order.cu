// Order of rows and columns for the tensor-core exact kNN of a large point set
// against itself (Eq. 8). The streaming filter of the tensor kernel keeps every
// column below the current bound of a row; the bound falls only as near columns
// arrive, so the survivors it must buffer are about ksel (1 + ln(n / ksel)) when
// the columns come in random order. Grouping the points by their nearest of
// ORD_C centroids puts a row's neighbours mostly in its own group: each row tile
// first streams the column tiles of its own groups, which sets its bound near
// the final one, then all the others. The result does not depend on the order
// (the filter keeps a valid bound in any order and the merge returns the exact
// lists); only the work of the filter does.
//
// Centroids: ORD_ITERS Lloyd iterations (nearest centroid, then the mean of its
// points) over ORD_SAMPLE evenly spaced rows, started from evenly spaced rows.
// Order: a stable counting sort of all rows by nearest centroid.
#include "common.cuh"
#include "internal.h"

namespace atsne {
namespace {

constexpr int ORD_C = 64;          // centroids
constexpr int ORD_CC = 64;         // centroids per pass of the assignment
constexpr int ORD_SAMPLE = 32768;  // rows of the Lloyd iterations
constexpr int ORD_ITERS = 4;
constexpr int ORD_BLK = 1024;      // rows per block of the counting sort
constexpr int ORD_DC = 32;         // dimensions per shared-memory chunk of the centroids

// centroid c starts as row floor(c N / C)
__global__ void ord_init_kernel(const float *__restrict__ X, int64_t N, int D, float *__restrict__ cent) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)ORD_C * D) return;
    const int c = (int)(t / D), d = (int)(t - (int64_t)c * D);
    cent[t] = X[((int64_t)c * N / ORD_C) * D + d];
}

// ||centroid||^2, one warp per centroid
__global__ void ord_norm_kernel(const float *__restrict__ cent, int D, float *__restrict__ cn) {
    const int c = blockIdx.x, lane = threadIdx.x;
    float s = 0.f;
    for (int d = lane; d < D; d += 32) s = fmaf(cent[c * D + d], cent[c * D + d], s);
    s = warp_sum(s);
    if (lane == 0) cn[c] = s;
}

// label[i] = the centroid nearest to row i * stride (i < n): the smallest
// ||c||^2 - 2 x.c, ties to the lower centroid. One thread per row; the
// centroids, ORD_CC at a time, pass through shared memory ORD_DC dimensions
// at a time.
__global__ void __launch_bounds__(256) ord_assign_kernel(const float *__restrict__ X, int64_t n, int64_t stride,
                                                         int D, const float *__restrict__ cent,
                                                         const float *__restrict__ cn, int32_t *__restrict__ label) {
    __shared__ float cs[ORD_CC][ORD_DC];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < n;
    const float *x = X + (live ? i * stride : 0) * D;
    int best = 0;
    float bv = INFINITY;
    for (int cb = 0; cb < ORD_C; cb += ORD_CC) {
        float acc[ORD_CC];
#pragma unroll
        for (int c = 0; c < ORD_CC; ++c) acc[c] = 0.f;
        for (int d0 = 0; d0 < D; d0 += ORD_DC) {
            __syncthreads();
            for (int t = threadIdx.x; t < ORD_CC * ORD_DC; t += blockDim.x) {
                const int c = t / ORD_DC, d = d0 + (t - c * ORD_DC);
                cs[c][t - c * ORD_DC] = d < D ? cent[(cb + c) * D + d] : 0.f;
            }
            __syncthreads();
            float xv[ORD_DC];
#pragma unroll
            for (int j = 0; j < ORD_DC; ++j) xv[j] = d0 + j < D ? x[d0 + j] : 0.f;
#pragma unroll
            for (int c = 0; c < ORD_CC; ++c) {
                float a = acc[c];
#pragma unroll
                for (int j = 0; j < ORD_DC; ++j) a = fmaf(xv[j], cs[c][j], a);
                acc[c] = a;
            }
        }
#pragma unroll
        for (int c = 0; c < ORD_CC; ++c) {
            const float v = cn[cb + c] - 2.f * acc[c];
            if (v < bv) {
                bv = v;
                best = cb + c;
            }
        }
    }
    if (live) label[i] = best;
}

// sums and counts of the sample rows per centroid, one warp per row
__global__ void ord_accum_kernel(const float *__restrict__ X, int64_t n, int64_t stride, int D,
                                 const int32_t *__restrict__ label, float *__restrict__ sum,
                                 int *__restrict__ cnt) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int l = label[i];
    const float *x = X + i * stride * D;
    for (int d = lane; d < D; d += 32) atomicAdd(&sum[l * D + d], x[d]);
    if (lane == 0) atomicAdd(&cnt[l], 1);
}

// a centroid with points moves to their mean; one without keeps its place
__global__ void ord_update_kernel(float *__restrict__ cent, const float *__restrict__ sum,
                                  const int *__restrict__ cnt, int D) {
    const int c = blockIdx.x;
    const int m = cnt[c];
    if (m == 0) return;
    for (int d = threadIdx.x; d < D; d += blockDim.x) cent[c * D + d] = sum[c * D + d] / (float)m;
}

// per block of ORD_BLK rows, how many rows each centroid has
__global__ void ord_count_kernel(const int32_t *__restrict__ label, int64_t N, int32_t *__restrict__ bcnt) {
    __shared__ int h[ORD_C];
    for (int c = threadIdx.x; c < ORD_C; c += blockDim.x) h[c] = 0;
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * ORD_BLK;
    for (int t = threadIdx.x; t < ORD_BLK; t += blockDim.x)
        if (r0 + t < N) atomicAdd(&h[label[r0 + t]], 1);
    __syncthreads();
    for (int c = threadIdx.x; c < ORD_C; c += blockDim.x) bcnt[(int64_t)blockIdx.x * ORD_C + c] = h[c];
}

// the counts become each (block, centroid) pair's first position in the
// order (centroid-major, then block), and coff[c] the first position of c
__global__ void ord_scan_kernel(int32_t *__restrict__ bcnt, int nblk, int64_t N, int32_t *__restrict__ coff) {
    __shared__ int tot[ORD_C];
    const int c = threadIdx.x;
    if (c < ORD_C) {
        int s = 0;
        for (int b = 0; b < nblk; ++b) {
            const int v = bcnt[(int64_t)b * ORD_C + c];
            bcnt[(int64_t)b * ORD_C + c] = s;
            s += v;
        }
        tot[c] = s;
    }
    __syncthreads();
    if (c == 0) {
        int s = 0;
        for (int k = 0; k < ORD_C; ++k) {
            coff[k] = s;
            s += tot[k];
        }
        coff[ORD_C] = (int32_t)N;
    }
    __syncthreads();
    if (c < ORD_C)
        for (int b = 0; b < nblk; ++b) bcnt[(int64_t)b * ORD_C + c] += coff[c];
}

// rows placed in (centroid, row) order; one warp per block of ORD_BLK rows,
// walking them in order so that equal labels keep their row order
__global__ void ord_scatter_kernel(const int32_t *__restrict__ label, int64_t N, const int32_t *__restrict__ boff,
                                   int32_t *__restrict__ perm, int32_t *__restrict__ lab_sorted) {
    __shared__ int next[ORD_C];
    const int lane = threadIdx.x;
    for (int c = lane; c < ORD_C; c += 32) next[c] = boff[(int64_t)blockIdx.x * ORD_C + c];
    __syncwarp();
    const int64_t r0 = (int64_t)blockIdx.x * ORD_BLK;
    for (int s = 0; s < ORD_BLK; s += 32) {
        const int64_t r = r0 + s + lane;
        const bool live = r < N;
        const int l = live ? label[r] : ORD_C;  // ORD_C: no row
        const unsigned peers = __match_any_sync(0xffffffffu, l);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        const int base = live ? next[l] : 0;
        __syncwarp();
        if (live) {
            perm[base + rank] = (int32_t)r;
            lab_sorted[base + rank] = l;
            if (rank == 0) next[l] = base + __popc(peers);
        }
        __syncwarp();
    }
}

// row tile rt: the column tiles of the groups of its first and last rows
// (consecutive in the order), as (first tile, count)
__global__ void ord_prologue_kernel(const int32_t *__restrict__ lab_sorted, const int32_t *__restrict__ coff,
                                    int64_t N, int bm, int bn, int row_tiles, int col_tiles,
                                    int32_t *__restrict__ pro) {
    const int rt = blockIdx.x * blockDim.x + threadIdx.x;
    if (rt >= row_tiles) return;
    const int64_t p0 = (int64_t)rt * bm;
    const int64_t p1 = (p0 + bm < N ? p0 + bm : N) - 1;
    const int l0 = lab_sorted[p0], l1 = lab_sorted[p1];
    const int t0 = coff[l0] / bn;
    int t1 = (coff[l1 + 1] + bn - 1) / bn;
    if (t1 > col_tiles) t1 = col_tiles;
    pro[2 * rt] = t0;
    pro[2 * rt + 1] = t1 - t0;
}

}  // namespace

// Worth it where the filter, not the contraction, bounds the kernel: short rows
// (a tile's MMAs take D / 64 k-blocks against a fixed filter per tile).
bool knn_ordered(int64_t N, int D, bool list, const TcPlan &pl) {
    return !list && pl.splits == 1 && N >= ORD_MIN_ROWS && D <= ORD_MAX_DIM;
}

size_t order_workspace(Carver &c, int64_t N, int D, const TcPlan &pl, OrderWs *ws) {
    OrderWs w;
    const int64_t nblk = (N + ORD_BLK - 1) / ORD_BLK;
    w.cent = c.take<float>((size_t)ORD_C * D);
    w.cn = c.take<float>(ORD_C);
    w.sum = c.take<float>((size_t)ORD_C * D);
    w.cnt = c.take<int>(ORD_C);
    w.label = c.take<int32_t>((size_t)N);
    w.lab_sorted = c.take<int32_t>((size_t)N);
    w.perm = c.take<int32_t>((size_t)N);
    w.bcnt = c.take<int32_t>((size_t)nblk * ORD_C);
    w.coff = c.take<int32_t>(ORD_C + 1);
    w.pro = c.take<int32_t>((size_t)2 * pl.row_tiles);
    if (ws) *ws = w;
    return c.bytes();
}

atsne_status knn_order_launch(const float *X, int64_t N, int D, const TcPlan &pl, int bm, int bn,
                              const OrderWs &w, cudaStream_t stream) {
    const int64_t ns = N < ORD_SAMPLE ? N : ORD_SAMPLE;
    const int64_t stride = N / ns;
    ATSNE_TRY(launch_kernel("knn_order", ord_init_kernel, ceil_div((int64_t)ORD_C * D, 256), 256, 0, stream, X, N,
                            D, w.cent));
    for (int it = 0; it < ORD_ITERS; ++it) {
        ATSNE_TRY(launch_kernel("knn_order", ord_norm_kernel, ORD_C, 32, 0, stream, (const float *)w.cent, D, w.cn));
        ATSNE_TRY(launch_kernel("knn_order", ord_assign_kernel, ceil_div(ns, 256), 256, 0, stream, X, ns, stride, D,
                                (const float *)w.cent, (const float *)w.cn, w.label));
        cudaError_t e = cudaMemsetAsync(w.sum, 0, sizeof(float) * ORD_C * D, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.cnt, 0, sizeof(int) * ORD_C, stream);
        if (e != cudaSuccess) return cuda_error(e, "knn_order memset");
        ATSNE_TRY(launch_kernel("knn_order", ord_accum_kernel, ceil_div(ns * 32, 256), 256, 0, stream, X, ns, stride,
                                D, (const int32_t *)w.label, w.sum, w.cnt));
        ATSNE_TRY(launch_kernel("knn_order", ord_update_kernel, ORD_C, 128, 0, stream, w.cent, (const float *)w.sum,
                                (const int *)w.cnt, D));
    }
    ATSNE_TRY(launch_kernel("knn_order", ord_norm_kernel, ORD_C, 32, 0, stream, (const float *)w.cent, D, w.cn));
    ATSNE_TRY(launch_kernel("knn_order", ord_assign_kernel, ceil_div(N, 256), 256, 0, stream, X, N, (int64_t)1, D,
                            (const float *)w.cent, (const float *)w.cn, w.label));
    const int nblk = (int)((N + ORD_BLK - 1) / ORD_BLK);
    ATSNE_TRY(launch_kernel("knn_order", ord_count_kernel, nblk, 256, 0, stream, (const int32_t *)w.label, N,
                            w.bcnt));
    ATSNE_TRY(launch_kernel("knn_order", ord_scan_kernel, 1, ORD_C, 0, stream, w.bcnt, nblk, N, w.coff));
    ATSNE_TRY(launch_kernel("knn_order", ord_scatter_kernel, nblk, 32, 0, stream, (const int32_t *)w.label, N,
                            (const int32_t *)w.bcnt, w.perm, w.lab_sorted));
    const int col_tiles = (int)((N + bn - 1) / bn);
    return launch_kernel("knn_order", ord_prologue_kernel, ceil_div((int64_t)pl.row_tiles, 128), 128, 0, stream,
                         (const int32_t *)w.lab_sorted, (const int32_t *)w.coff, N, bm, bn, pl.row_tiles,
                         col_tiles, w.pro);
}

}  // namespace atsne
