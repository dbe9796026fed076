// Symmetrised joint P as CSR (Eq. 2 in the split form of Eq. 10, Sec. 4.3).
//
// Row i of P holds its forward entries j in N_i (k, fewer where a deletion
// left absent entries, index -1, Sec. 5.3.2) and one reverse entry for
// every j with i in N_j but j not in N_i; a mutual pair gets
// (p_{j|i} + p_{i|j}) / 2N on both sides. Steps:
//   1. sort_rows:   each conditional row sorted by column (warp bitonic) so
//                   membership tests are binary searches;
//   2. count:       for entry (i, j): is i in N_j? if not, row j gains one
//                   reverse-only entry (atomic count);
//   3. scan:        row_ptr[i] = sum_{i' < i} (own[i'] + rev[i']), own = the
//                   row's forward entries;
//   4. scatter:     forward entries land in place, in column order; mutual
//                   values are formed from the same two operands on both sides
//                   (bit-identical p_ij and p_ji); reverse-only entries are
//                   appended after the row's forward part;
//   5. sort_tails:  rows with reverse entries are sorted by column (warp in
//                   shared memory up to 1024 entries, one CTA per longer row).
// All passes are streaming or gather passes over N*k entries.
#include <limits.h>

#include "common.cuh"
#include "internal.h"

namespace atsne {
namespace {

constexpr int SORT_ROW_CAP = 1024;  // longest row a warp sorts in shared memory

template <int KP>
__global__ void __launch_bounds__(128)
sym_sort_rows_kernel(const int32_t *__restrict__ idx, const float *__restrict__ P, int64_t N, int k,
                     int32_t *__restrict__ scol, float *__restrict__ sval, int32_t *__restrict__ own,
                     int *status) {
    __shared__ int keys[4][KP];
    __shared__ float vals[4][KP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * 4 + w;
    if (i >= N) return;
    for (int t = lane; t < KP; t += 32) {
        int j = INT_MAX;
        float v = 0.f;
        if (t < k) {
            j = idx[i * k + t];
            v = P[i * k + t];
            if (j == -1) {  // an absent neighbour (Sec. 5.3.2): no entry
                j = INT_MAX;
                v = 0.f;
            } else if (j < 0 || j >= N || j == i) {
                raise_status(status, DEV_MALFORMED);
                j = INT_MAX;
            }
        }
        keys[w][t] = j;
        vals[w][t] = v;
    }
    __syncwarp();
    warp_bitonic_sort_smem(keys[w], vals[w], KP, lane);
    int c = 0;  // forward entries (absent ones sorted last)
    for (int t = lane; t < k; t += 32) {
        int j = keys[w][t];
        if (t > 0 && j != INT_MAX && j == keys[w][t - 1]) raise_status(status, DEV_MALFORMED);
        scol[i * k + t] = j;
        sval[i * k + t] = vals[w][t];
        c += j != INT_MAX;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) own[i] = c;
}

// rev[i] += own[i] - k, so that the scan of k + rev gives own + reverse entries.
__global__ void sym_rowlen_kernel(const int32_t *__restrict__ own, int64_t N, int k, int32_t *__restrict__ rev) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) rev[i] += own[i] - k;
}

__device__ __forceinline__ int find_in_row(const int32_t *__restrict__ row, int k, int key) {
    int lo = 0, hi = k;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int v = row[mid];
        if (v < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < k && row[lo] == key) ? lo : -1;
}

__global__ void sym_count_kernel(const int32_t *__restrict__ scol, int64_t N, int k,
                                 int32_t *__restrict__ rev) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * k) return;
    const int i = (int)(e / k);
    const int j = scol[e];
    if (j < 0 || j >= N) return;
    if (find_in_row(scol + (int64_t)j * k, k, i) < 0) atomicAdd(&rev[j], 1);
}

__global__ void sym_scatter_kernel(const int32_t *__restrict__ scol, const float *__restrict__ sval,
                                   int64_t N, int k, float inv2n,
                                   const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ own,
                                   int32_t *__restrict__ cursor,
                                   int32_t *__restrict__ col, float *__restrict__ val) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * k) return;
    const int i = (int)(e / k);
    const int t = (int)(e - (int64_t)i * k);
    const int j = scol[e];
    if (j < 0 || j >= N) return;
    const float v = sval[e];
    const int u = find_in_row(scol + (int64_t)j * k, k, i);
    float out;
    if (u >= 0) {
        out = (v + sval[(int64_t)j * k + u]) * inv2n;
    } else {
        out = v * inv2n;
        const int c = atomicAdd(&cursor[j], 1);
        const int64_t pos = row_ptr[j] + own[j] + c;
        col[pos] = i;
        val[pos] = out;
    }
    col[row_ptr[i] + t] = j;
    val[row_ptr[i] + t] = out;
}

// Rows with reverse entries: warp sort in shared memory, longer rows deferred.
__global__ void __launch_bounds__(128)
sym_sort_tails_kernel(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ own,
                      int64_t N, int32_t *__restrict__ col, float *__restrict__ val,
                      int32_t *__restrict__ long_rows, int32_t *__restrict__ n_long) {
    __shared__ int keys[4][SORT_ROW_CAP];
    __shared__ float vals[4][SORT_ROW_CAP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * 4 + w;
    if (i >= N) return;
    const int64_t b = row_ptr[i];
    const int len = (int)(row_ptr[i + 1] - b);
    if (len == own[i]) return;  // no reverse entries: already in column order
    if (len > SORT_ROW_CAP) {
        if (lane == 0) long_rows[atomicAdd(n_long, 1)] = (int)i;
        return;
    }
    int n = 32;
    while (n < len) n <<= 1;
    for (int t = lane; t < n; t += 32) {
        keys[w][t] = t < len ? col[b + t] : INT_MAX;
        vals[w][t] = t < len ? val[b + t] : 0.f;
    }
    __syncwarp();
    warp_bitonic_sort_smem(keys[w], vals[w], n, lane);
    for (int t = lane; t < len; t += 32) {
        col[b + t] = keys[w][t];
        val[b + t] = vals[w][t];
    }
}

// One CTA per long row, sorted in place in global memory by the bitonic
// network in its "flip" form: every merge starts by comparing mirrored
// positions and continues with half-cleaners, and every compare-exchange puts
// the smaller element at the lower position. Positions past the row's end act
// as +inf and never move, so exchanges with them are skipped.
__device__ __forceinline__ void ce_ascending(int32_t *col, float *val, int64_t a, int64_t c) {
    const int ka = col[a], kc = col[c];
    if (kc < ka) {
        col[a] = kc;
        col[c] = ka;
        const float va = val[a];
        val[a] = val[c];
        val[c] = va;
    }
}

__global__ void __launch_bounds__(1024)
sym_sort_long_kernel(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ long_rows,
                     const int32_t *__restrict__ n_long, int32_t *__restrict__ col,
                     float *__restrict__ val) {
    const int count = *n_long;
    for (int r = blockIdx.x; r < count; r += gridDim.x) {
        const int64_t i = long_rows[r];
        const int64_t b = row_ptr[i];
        const int64_t len = row_ptr[i + 1] - b;
        int64_t n = 1;
        while (n < len) n <<= 1;
        for (int64_t size = 2; size <= n; size <<= 1) {
            const int64_t half = size >> 1;
            for (int64_t t = threadIdx.x; t < (n >> 1); t += blockDim.x) {
                const int64_t blk = (t / half) * size, off = t % half;
                const int64_t a = blk + off, c = blk + size - 1 - off;
                if (c < len) ce_ascending(col + b, val + b, a, c);
            }
            __syncthreads();
            for (int64_t stride = half >> 1; stride > 0; stride >>= 1) {
                for (int64_t t = threadIdx.x; t < (n >> 1); t += blockDim.x) {
                    const int64_t a = 2 * t - (t & (stride - 1));
                    const int64_t c = a + stride;
                    if (c < len) ce_ascending(col + b, val + b, a, c);
                }
                __syncthreads();
            }
        }
    }
}

}  // namespace

size_t symmetrize_workspace(Carver &c, int64_t N, int k, SymWs *ws) {
    SymWs w;
    w.scol = c.take<int32_t>((size_t)N * k);
    w.sval = c.take<float>((size_t)N * k);
    w.rev = c.take<int32_t>((size_t)N);
    w.cursor = c.take<int32_t>((size_t)N);
    w.long_rows = c.take<int32_t>((size_t)N);
    w.n_long = c.take<int32_t>(1);
    w.own = c.take<int32_t>((size_t)N);
    w.scan = c.take<int64_t>(scan_partials_count(N));
    if (ws) *ws = w;
    return c.bytes();
}

atsne_status symmetrize_launch(const int32_t *idx, const float *P, int64_t N, int k,
                               int64_t *row_ptr, int32_t *col, float *val, int64_t *nnz_dev,
                               const SymWs &w, cudaStream_t stream) {
    int *status = device_status_word();
    cudaError_t e;
    e = cudaMemsetAsync(w.rev, 0, sizeof(int32_t) * N, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.cursor, 0, sizeof(int32_t) * N, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.n_long, 0, sizeof(int32_t), stream);
    if (e != cudaSuccess) return cuda_error(e, "symmetrize memset");
    const int grid4 = ceil_div(N, 4);
    if (k <= 128)
        ATSNE_TRY(launch_kernel("sym_sort_rows", sym_sort_rows_kernel<128>, grid4, 128, 0, stream,
                                idx, P, N, k, w.scol, w.sval, w.own, status));
    else if (k <= 256)
        ATSNE_TRY(launch_kernel("sym_sort_rows", sym_sort_rows_kernel<256>, grid4, 128, 0, stream,
                                idx, P, N, k, w.scol, w.sval, w.own, status));
    else if (k <= 512)
        ATSNE_TRY(launch_kernel("sym_sort_rows", sym_sort_rows_kernel<512>, grid4, 128, 0, stream,
                                idx, P, N, k, w.scol, w.sval, w.own, status));
    else
        return set_error(ATSNE_EUNSUPPORTED, "symmetrize: k=%d above 512", k);
    const int64_t M = N * k;
    ATSNE_TRY(launch_kernel("sym_count", sym_count_kernel, ceil_div(M, 256), 256, 0, stream, w.scol,
                            N, k, w.rev));
    ATSNE_TRY(launch_kernel("sym_count", sym_rowlen_kernel, ceil_div(N, 256), 256, 0, stream, w.own, N, k,
                            w.rev));
    ATSNE_TRY(scan_rowlen(w.rev, N, k, row_ptr, nnz_dev, w.scan, stream));
    ATSNE_TRY(launch_kernel("sym_scatter", sym_scatter_kernel, ceil_div(M, 256), 256, 0, stream,
                            w.scol, w.sval, N, k, (float)(0.5 / (double)N), row_ptr, w.own, w.cursor,
                            col, val));
    ATSNE_TRY(launch_kernel("sym_sort_tails", sym_sort_tails_kernel, grid4, 128, 0, stream, row_ptr,
                            w.own, N, col, val, w.long_rows, w.n_long));
    ATSNE_TRY(launch_kernel("sym_sort_long", sym_sort_long_kernel, 2 * num_sms(), 1024, 0, stream,
                            row_ptr, w.long_rows, w.n_long, col, val));
    return ATSNE_OK;
}

}  // namespace atsne
