// Exclusive scan of CSR row lengths (k + rev[i]) into int64 row offsets:
// reduce tiles of 4096 lengths, scan the tile sums in one CTA, then rescan
// each tile with its offset. Three streaming passes over N int32.
#include "common.cuh"
#include "internal.h"

namespace atsne {
namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *total) {
    __shared__ int64_t warp_tot[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;  // inclusive
    }
    __syncthreads();
    const int64_t before = (w > 0 ? warp_tot[w - 1] : 0) + x - v;
    if (total) *total = warp_tot[nw - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(SCAN_THREADS)
scan_reduce_kernel(const int32_t *__restrict__ rev, int64_t n, int add, int64_t *__restrict__ part) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t s = 0;
    for (int t = 0; t < SCAN_ITEMS; ++t) {
        const int64_t i = base + (int64_t)t * SCAN_THREADS + threadIdx.x;
        if (i < n) s += (int64_t)rev[i] + add;
    }
    int64_t total;
    block_exclusive_scan(s, &total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) scan_partials_kernel(int64_t *__restrict__ part, int64_t np) {
    const int64_t per = (np + blockDim.x - 1) / blockDim.x;
    const int64_t b = threadIdx.x * per, e = (np < b + per ? np : b + per);
    int64_t s = 0;
    for (int64_t i = b; i < e; ++i) s += part[i];
    int64_t off = block_exclusive_scan(s, nullptr);
    for (int64_t i = b; i < e; ++i) {
        const int64_t v = part[i];
        part[i] = off;
        off += v;
    }
}

__global__ void __launch_bounds__(SCAN_THREADS)
scan_down_kernel(const int32_t *__restrict__ rev, int64_t n, int add, const int64_t *__restrict__ part,
                 int64_t *__restrict__ out, int64_t *__restrict__ total_out) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t s = 0;
#pragma unroll
    for (int t = 0; t < SCAN_ITEMS; ++t) {
        const int64_t i = base + t;
        v[t] = i < n ? (int64_t)rev[i] + add : 0;
        s += v[t];
    }
    int64_t run = part[blockIdx.x] + block_exclusive_scan(s, nullptr);
#pragma unroll
    for (int t = 0; t < SCAN_ITEMS; ++t) {
        const int64_t i = base + t;
        if (i < n) out[i] = run;
        run += v[t];
    }
    if (base < n && base + SCAN_ITEMS >= n) {  // the thread holding the last element
        out[n] = run;
        if (total_out) *total_out = run;
    }
}

}  // namespace

size_t scan_partials_count(int64_t n) { return (size_t)ceil_div(n > 0 ? n : 1, SCAN_TILE); }

atsne_status scan_rowlen(const int32_t *rev, int64_t n, int add, int64_t *out, int64_t *total,
                         int64_t *part, cudaStream_t stream) {
    const int64_t np = (int64_t)scan_partials_count(n);
    ATSNE_TRY(launch_kernel("scan_reduce", scan_reduce_kernel, (int)np, SCAN_THREADS, 0, stream,
                            rev, n, add, part));
    ATSNE_TRY(launch_kernel("scan_partials", scan_partials_kernel, 1, 1024, 0, stream, part, np));
    return launch_kernel("scan_down", scan_down_kernel, (int)np, SCAN_THREADS, 0, stream, rev, n,
                         add, part, out, total);
}

}  // namespace atsne
