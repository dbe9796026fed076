// Symmetrised joint P as CSR (Eq. 2 in the split form of Eq. 10, Sec. 4.3).
//
// Row r of P is the union of its forward entries F_r = N_r (k, fewer where a
// deletion left absent entries, index -1, Sec. 5.3.2) and its reverse entries
// R_r = {i : r in N_i}; a column in both (a mutual pair) gets
// (p_{c|r} + p_{r|c}) / 2N, formed from the same two operands on both sides,
// so p_rc and p_cr are bit-identical; a column in one of them gets its one
// conditional / 2N. The transpose is a counting sort by target row:
//   1. fwd:      each conditional row sorted by column (warp bitonic, in
//                registers) and its entries counted into their target rows;
//   2. scan:     offsets of the reverse lists;
//   3. rev:      every entry (i -> j, p_{j|i}) placed in j's reverse list;
//   4. len:      row length |F_r| + |R_r| - |F_r and R_r| (each reverse entry
//                searched in the sorted forward row);
//   5. scan:     row_ptr;
//   6. write:    the reverse list sorted (warp bitonic in shared memory, or
//                for rows of more than SORT_ROW_CAP reverse entries a CTA
//                sort in global memory first), then every entry written
//                straight to its place: an entry's position in the union is
//                its rank in its own sorted list plus its rank in the other
//                one, less the mutual columns before it.
// Apart from the reverse placement (step 3, one scattered 8-byte write per
// entry) every pass streams rows.
#include <limits.h>

#include "common.cuh"
#include "internal.h"
#include "warp_sort.cuh"

namespace atsne {
namespace {

constexpr int SORT_ROW_CAP = 1024;  // longest reverse list a warp sorts in shared memory
constexpr int SYM_WARPS = 4;

// lower bound of key in the sorted a[0, n)
template <typename P>
__device__ __forceinline__ int lower_bound_i(P a, int n, int key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <int KP>
__global__ void __launch_bounds__(128)
sym_fwd_kernel(const int32_t *__restrict__ idx, const float *__restrict__ P, int64_t N, int k,
               int32_t *__restrict__ scol, float *__restrict__ sval, int32_t *__restrict__ own,
               int32_t *__restrict__ rcnt, int *status) {
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
            } else {
                atomicAdd(&rcnt[j], 1);
            }
        }
        keys[w][t] = j;
        vals[w][t] = v;
    }
    __syncwarp();
    warp_sort_pow2(keys[w], vals[w], KP, lane);
    __syncwarp();
    int c = 0;  // forward entries (absent ones sorted last)
    for (int t = lane; t < k; t += 32) {
        const int j = keys[w][t];
        if (t > 0 && j != INT_MAX && j == keys[w][t - 1]) raise_status(status, DEV_MALFORMED);
        scol[i * k + t] = j;
        sval[i * k + t] = vals[w][t];
        c += j != INT_MAX;
    }
    c = (int)__reduce_add_sync(0xffffffffu, (unsigned)c);
    if (lane == 0) own[i] = c;
}

// Entry (i -> j, p_{j|i}) into j's reverse list (order within a list is set
// by the atomic cursor; the write pass sorts each list).
__global__ void sym_rev_kernel(const int32_t *__restrict__ scol, const float *__restrict__ sval, int64_t N, int k,
                               const int64_t *__restrict__ roff, int32_t *__restrict__ cursor,
                               int32_t *__restrict__ rev_i, float *__restrict__ rev_p) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * k) return;
    const int j = scol[e];
    if (j < 0 || j >= N) return;
    const int64_t pos = roff[j] + atomicAdd(&cursor[j], 1);
    rev_i[pos] = (int32_t)(e / k);
    rev_p[pos] = sval[e];
}

// Row length |F| + |R| - |F and R|, one warp per row; the forward row is
// searched in shared memory.
template <int KP>
__global__ void __launch_bounds__(SYM_WARPS * 32)
sym_len_kernel(const int32_t *__restrict__ scol, const int32_t *__restrict__ own, int64_t N, int k,
               const int64_t *__restrict__ roff, const int32_t *__restrict__ rev_i, int32_t *__restrict__ len) {
    __shared__ int fc[SYM_WARPS][KP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t r = (int64_t)blockIdx.x * SYM_WARPS + w;
    if (r >= N) return;
    const int a = own[r];
    for (int t = lane; t < a; t += 32) fc[w][t] = scol[r * k + t];
    __syncwarp();
    const int64_t b0 = roff[r], m = roff[r + 1] - b0;
    int matched = 0;
    for (int64_t t = lane; t < m; t += 32) {
        const int key = rev_i[b0 + t];
        const int lb = lower_bound_i(fc[w], a, key);
        matched += lb < a && fc[w][lb] == key;
    }
    matched = (int)__reduce_add_sync(0xffffffffu, (unsigned)matched);
    if (lane == 0) len[r] = a + (int)m - matched;
}

// Writes row r of the CSR from its sorted forward row (fc/fv, a entries, in
// shared memory) and its sorted reverse list (ri/rp, m entries): an entry's
// place is its rank in its own list plus its rank in the other one, less the
// mutual columns before it. Warp-cooperative.
template <typename IP, typename VP>
__device__ __forceinline__ void sym_write_row(const int *fc, const float *fv, int a, IP ri, VP rp, int64_t m,
                                              float inv2n, int32_t *__restrict__ col, float *__restrict__ val,
                                              int64_t base, int lane) {
    const unsigned lt = (1u << lane) - 1u;
    // forward entries without a reverse partner
    int mc = 0;  // mutual columns among the forward entries so far
    for (int s0 = 0; s0 < a; s0 += 32) {
        const int s = s0 + lane;
        int key = INT_MAX;
        int64_t lb = 0;
        bool hit = false;
        if (s < a) {
            key = fc[s];
            int64_t lo = 0, hi = m;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (ri[mid] < key) lo = mid + 1;
                else hi = mid;
            }
            lb = lo;
            hit = lb < m && ri[lb] == key;
        }
        const unsigned hm = __ballot_sync(0xffffffffu, hit);
        if (s < a && !hit) {
            const int64_t pos = base + s + lb - (mc + __popc(hm & lt));
            col[pos] = key;
            val[pos] = fv[s] * inv2n;
        }
        mc += __popc(hm);
    }
    // reverse entries, mutual ones with both conditionals
    mc = 0;
    for (int64_t t0 = 0; t0 < m; t0 += 32) {
        const int64_t t = t0 + lane;
        int key = 0, lb = 0;
        bool hit = false;
        float p = 0.f;
        if (t < m) {
            key = ri[t];
            p = rp[t];
            lb = lower_bound_i(fc, a, key);
            hit = lb < a && fc[lb] == key;
        }
        const unsigned hm = __ballot_sync(0xffffffffu, hit);
        if (t < m) {
            const int64_t pos = base + t + lb - (mc + __popc(hm & lt));
            col[pos] = key;
            val[pos] = (hit ? fv[lb] + p : p) * inv2n;
        }
        mc += __popc(hm);
    }
}

template <int KP>
__global__ void __launch_bounds__(SYM_WARPS * 32)
sym_write_kernel(const int32_t *__restrict__ scol, const float *__restrict__ sval, const int32_t *__restrict__ own,
                 int64_t N, int k, float inv2n, const int64_t *__restrict__ roff, const int32_t *__restrict__ rev_i,
                 const float *__restrict__ rev_p, const int64_t *__restrict__ row_ptr, int32_t *__restrict__ col,
                 float *__restrict__ val, int32_t *__restrict__ long_rows, int32_t *__restrict__ n_long) {
    extern __shared__ __align__(16) unsigned char sw_smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int *fc = reinterpret_cast<int *>(sw_smem) + w * KP;
    float *fv = reinterpret_cast<float *>(sw_smem + SYM_WARPS * KP * 4) + w * KP;
    int *rk = reinterpret_cast<int *>(sw_smem + SYM_WARPS * KP * 8) + w * SORT_ROW_CAP;
    float *rv = reinterpret_cast<float *>(sw_smem + SYM_WARPS * (KP * 8 + SORT_ROW_CAP * 4)) + w * SORT_ROW_CAP;
    const int64_t r = (int64_t)blockIdx.x * SYM_WARPS + w;
    if (r >= N) return;
    const int64_t b0 = roff[r], m = roff[r + 1] - b0;
    if (m > SORT_ROW_CAP) {  // sorted in global memory first, written by sym_write_long_kernel
        if (lane == 0) long_rows[atomicAdd(n_long, 1)] = (int)r;
        return;
    }
    const int a = own[r];
    for (int t = lane; t < a; t += 32) {
        fc[t] = scol[r * k + t];
        fv[t] = sval[r * k + t];
    }
    int n = 32;
    while (n < m) n <<= 1;
    for (int t = lane; t < n; t += 32) {
        rk[t] = t < m ? rev_i[b0 + t] : INT_MAX;
        rv[t] = t < m ? rev_p[b0 + t] : 0.f;
    }
    __syncwarp();
    if (m > 1) warp_bitonic_sort_smem(rk, rv, n, lane);
    sym_write_row(fc, fv, a, rk, rv, m, inv2n, col, val, row_ptr[r], lane);
}

// One CTA per long reverse list, sorted in place in global memory by the
// bitonic network in its "flip" form: every merge starts by comparing
// mirrored positions and continues with half-cleaners, and every
// compare-exchange puts the smaller element at the lower position. Positions
// past the list's end act as +inf and never move, so exchanges with them are
// skipped.
__device__ __forceinline__ void ce_ascending(int32_t *key, float *val, int64_t a, int64_t c) {
    const int ka = key[a], kc = key[c];
    if (kc < ka) {
        key[a] = kc;
        key[c] = ka;
        const float va = val[a];
        val[a] = val[c];
        val[c] = va;
    }
}

__global__ void __launch_bounds__(1024)
sym_sort_long_kernel(const int64_t *__restrict__ roff, const int32_t *__restrict__ long_rows,
                     const int32_t *__restrict__ n_long, int32_t *__restrict__ rev_i, float *__restrict__ rev_p) {
    const int count = *n_long;
    for (int q = blockIdx.x; q < count; q += gridDim.x) {
        const int64_t r = long_rows[q];
        const int64_t b = roff[r];
        const int64_t len = roff[r + 1] - b;
        int64_t n = 1;
        while (n < len) n <<= 1;
        for (int64_t size = 2; size <= n; size <<= 1) {
            const int64_t half = size >> 1;
            for (int64_t t = threadIdx.x; t < (n >> 1); t += blockDim.x) {
                const int64_t blk = (t / half) * size, off = t % half;
                const int64_t a = blk + off, c = blk + size - 1 - off;
                if (c < len) ce_ascending(rev_i + b, rev_p + b, a, c);
            }
            __syncthreads();
            for (int64_t stride = half >> 1; stride > 0; stride >>= 1) {
                for (int64_t t = threadIdx.x; t < (n >> 1); t += blockDim.x) {
                    const int64_t a = 2 * t - (t & (stride - 1));
                    const int64_t c = a + stride;
                    if (c < len) ce_ascending(rev_i + b, rev_p + b, a, c);
                }
                __syncthreads();
            }
        }
    }
}

// The long rows, their reverse lists sorted in global memory.
template <int KP>
__global__ void __launch_bounds__(SYM_WARPS * 32)
sym_write_long_kernel(const int32_t *__restrict__ scol, const float *__restrict__ sval,
                      const int32_t *__restrict__ own, int k, float inv2n, const int64_t *__restrict__ roff,
                      const int32_t *__restrict__ rev_i, const float *__restrict__ rev_p,
                      const int64_t *__restrict__ row_ptr, int32_t *__restrict__ col, float *__restrict__ val,
                      const int32_t *__restrict__ long_rows, const int32_t *__restrict__ n_long) {
    __shared__ int fc[SYM_WARPS][KP];
    __shared__ float fv[SYM_WARPS][KP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int count = *n_long;
    for (int q = blockIdx.x * SYM_WARPS + w; q < count; q += gridDim.x * SYM_WARPS) {
        const int64_t r = long_rows[q];
        const int a = own[r];
        for (int t = lane; t < a; t += 32) {
            fc[w][t] = scol[r * k + t];
            fv[w][t] = sval[r * k + t];
        }
        __syncwarp();
        const int64_t b0 = roff[r];
        sym_write_row(fc[w], fv[w], a, rev_i + b0, rev_p + b0, roff[r + 1] - b0, inv2n, col, val, row_ptr[r],
                      lane);
        __syncwarp();
    }
}

template <int KP>
size_t sym_write_smem() {
    return (size_t)SYM_WARPS * (KP * 8 + SORT_ROW_CAP * 8);
}

template <int KP>
atsne_status symmetrize_t(const int32_t *idx, const float *P, int64_t N, int k, int64_t *row_ptr, int32_t *col,
                          float *val, int64_t *nnz_dev, const SymWs &w, cudaStream_t stream) {
    int *status = device_status_word();
    cudaError_t e = cudaMemsetAsync(w.rcnt, 0, sizeof(int32_t) * N, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.cursor, 0, sizeof(int32_t) * N, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.n_long, 0, sizeof(int32_t), stream);
    if (e != cudaSuccess) return cuda_error(e, "symmetrize memset");
    const int64_t M = N * k;
    const float inv2n = (float)(0.5 / (double)N);
    ATSNE_TRY(launch_kernel("sym_fwd", sym_fwd_kernel<KP>, ceil_div(N, 4), 128, 0, stream, idx, P, N, k, w.scol,
                            w.sval, w.own, w.rcnt, status));
    ATSNE_TRY(scan_rowlen(w.rcnt, N, 0, w.roff, w.rtot, w.scan, stream));
    ATSNE_TRY(launch_kernel("sym_rev", sym_rev_kernel, ceil_div(M, 256), 256, 0, stream,
                            (const int32_t *)w.scol, (const float *)w.sval, N, k, (const int64_t *)w.roff, w.cursor,
                            w.rev_i, w.rev_p));
    ATSNE_TRY(launch_kernel("sym_len", sym_len_kernel<KP>, ceil_div(N, SYM_WARPS), SYM_WARPS * 32, 0, stream,
                            (const int32_t *)w.scol, (const int32_t *)w.own, N, k, (const int64_t *)w.roff,
                            (const int32_t *)w.rev_i, w.len));
    ATSNE_TRY(scan_rowlen(w.len, N, 0, row_ptr, nnz_dev, w.scan, stream));
    const size_t smem = sym_write_smem<KP>();
    e = cudaFuncSetAttribute(sym_write_kernel<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "sym_write attribute");
    ATSNE_TRY(launch_kernel("sym_write", sym_write_kernel<KP>, ceil_div(N, SYM_WARPS), SYM_WARPS * 32, smem, stream,
                            (const int32_t *)w.scol, (const float *)w.sval, (const int32_t *)w.own, N, k, inv2n,
                            (const int64_t *)w.roff, (const int32_t *)w.rev_i, (const float *)w.rev_p,
                            (const int64_t *)row_ptr, col, val, w.long_rows, w.n_long));
    ATSNE_TRY(launch_kernel("sym_sort_long", sym_sort_long_kernel, 2 * num_sms(), 1024, 0, stream,
                            (const int64_t *)w.roff, (const int32_t *)w.long_rows, (const int32_t *)w.n_long,
                            w.rev_i, w.rev_p));
    return launch_kernel("sym_write_long", sym_write_long_kernel<KP>, 2 * num_sms(), SYM_WARPS * 32, 0, stream,
                         (const int32_t *)w.scol, (const float *)w.sval, (const int32_t *)w.own, k, inv2n,
                         (const int64_t *)w.roff, (const int32_t *)w.rev_i, (const float *)w.rev_p,
                         (const int64_t *)row_ptr, col, val, (const int32_t *)w.long_rows,
                         (const int32_t *)w.n_long);
}

}  // namespace

size_t symmetrize_workspace(Carver &c, int64_t N, int k, SymWs *ws) {
    SymWs w;
    w.scol = c.take<int32_t>((size_t)N * k);
    w.sval = c.take<float>((size_t)N * k);
    w.rev_i = c.take<int32_t>((size_t)N * k);
    w.rev_p = c.take<float>((size_t)N * k);
    w.rcnt = c.take<int32_t>((size_t)N);
    w.cursor = c.take<int32_t>((size_t)N);
    w.len = c.take<int32_t>((size_t)N);
    w.roff = c.take<int64_t>((size_t)N + 1);
    w.rtot = c.take<int64_t>(1);
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
    if (k <= 128) return symmetrize_t<128>(idx, P, N, k, row_ptr, col, val, nnz_dev, w, stream);
    if (k <= 256) return symmetrize_t<256>(idx, P, N, k, row_ptr, col, val, nnz_dev, w, stream);
    if (k <= 512) return symmetrize_t<512>(idx, P, N, k, row_ptr, col, val, nnz_dev, w, stream);
    return set_error(ATSNE_EUNSUPPORTED, "symmetrize: k=%d above 512", k);
}

}  // namespace atsne
