// Exact kNN by direct differences on the CUDA cores (Eq. 8, Sec. 3.1).
//
// Each CTA takes 32 queries and streams the whole corpus in tiles of 64
// points; 256 threads accumulate (q - c)^2 over 32-dimension slices (8 pairs
// per thread), then each warp folds a tile's 64 candidates per query into a
// per-query list of the best k in shared memory. A candidate enters only if it
// beats the list's current worst entry under the (distance, index) order, so
// after the first tiles almost every candidate costs one compare. The list's
// distances are then recomputed in the library's one summation order
// (group8_d2_pair, as the tensor-core merge computes them) and sorted, so a
// row's d2 does not depend on which kernel produced it. This kernel is the GPU
// path for small problems and the fallback for rows whose tensor-core
// candidates cannot be certified.
#include <float.h>
#include <limits.h>

#include "common.cuh"
#include "internal.h"

namespace atsne {
namespace {

constexpr int BF_QB = 32;       // queries per CTA
constexpr int BF_CB = 64;       // corpus points per tile
constexpr int BF_DC = 32;       // dimensions per slice
constexpr int BF_THREADS = 256;
// after the tiles, each warp's FP64 near-tie scratch lives in the tile buffers
static_assert(BF_CB * (BF_DC + 1) * 4 >= (BF_THREADS / 32) * TIE_MAX * 8, "near-tie distances fit the tile buffer");
static_assert(BF_QB * (BF_CB + 1) * 4 >= (BF_THREADS / 32) * TIE_MAX * 4, "near-tie positions fit the tile buffer");

// Work item s (0 <= s < nq, or < *rows_count when rows_list is given) is output
// row r = rows_list ? rows_list[s] : s, whose query point is qlist ? qlist[r] : r
// of X, or, with Xq (queries against another corpus), row r of Xq, with no
// point excluded. CTAs stride over blocks of 32 work items.
template <int KCAP>
__global__ void __launch_bounds__(BF_THREADS)
knn_bruteforce_kernel(const float *__restrict__ X, int64_t N, int D,
                      const int32_t *__restrict__ qlist, int64_t nq,
                      const int32_t *__restrict__ rows_list, const int32_t *__restrict__ rows_count,
                      int k, int32_t *__restrict__ idx_out, float *__restrict__ d2_out,
                      const float *__restrict__ Xq) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const bool cross = Xq != nullptr;
    const float *QX = cross ? Xq : X;
    float *Qs = reinterpret_cast<float *>(smem_raw);      // [QB][DC+1]
    float *Cs = Qs + BF_QB * (BF_DC + 1);                 // [CB][DC+1]
    float *Dt = Cs + BF_CB * (BF_DC + 1);                 // [QB][CB+1]
    float *td = Dt + BF_QB * (BF_CB + 1);                 // [QB][KCAP]
    int *tj = reinterpret_cast<int *>(td + BF_QB * KCAP); // [QB][KCAP]
    __shared__ int qid[BF_QB];
    __shared__ int64_t orow[BF_QB];
    __shared__ float thr_d[BF_QB];
    __shared__ int thr_j[BF_QB];
    __shared__ int thr_p[BF_QB];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n_items = rows_count ? (int64_t)*rows_count : nq;
    // the list keeps the (k+1)-th nearest too where it fits, so that a near tie
    // across the k-th place is settled in FP64
    const int kl = k + 1 <= KCAP ? k + 1 : k;
    for (int64_t q0 = (int64_t)blockIdx.x * BF_QB; q0 < n_items; q0 += (int64_t)gridDim.x * BF_QB) {
    if (tid < BF_QB) {
        const int64_t s = q0 + tid;
        int64_t r = -1;
        int q = -1;
        if (s < n_items) {
            r = rows_list ? rows_list[s] : s;
            q = cross ? (int)r : (qlist ? qlist[r] : (int)r);
        }
        qid[tid] = (q >= 0 && (cross || q < N)) ? q : -1;  // out-of-range queries are flagged by the caller
        orow[tid] = r;
        thr_d[tid] = INFINITY;
        thr_j[tid] = INT_MAX;
        thr_p[tid] = 0;
    }
    for (int t = tid; t < BF_QB * KCAP; t += BF_THREADS) {
        td[t] = INFINITY;
        tj[t] = INT_MAX;
    }
    __syncthreads();

    const int qi = tid >> 3, cg = tid & 7;
    for (int64_t c0 = 0; c0 < N; c0 += BF_CB) {
        float acc[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[m] = 0.f;
        for (int d0 = 0; d0 < D; d0 += BF_DC) {
            for (int t = tid; t < BF_QB * BF_DC; t += BF_THREADS) {
                int r = t / BF_DC, c = t - r * BF_DC;
                int q = qid[r];
                Qs[r * (BF_DC + 1) + c] = (q >= 0 && d0 + c < D) ? QX[(int64_t)q * D + d0 + c] : 0.f;
            }
            for (int t = tid; t < BF_CB * BF_DC; t += BF_THREADS) {
                int r = t / BF_DC, c = t - r * BF_DC;
                int64_t j = c0 + r;
                Cs[r * (BF_DC + 1) + c] = (j < N && d0 + c < D) ? X[j * D + d0 + c] : 0.f;
            }
            __syncthreads();
#pragma unroll 4
            for (int c = 0; c < BF_DC; ++c) {
                float qv = Qs[qi * (BF_DC + 1) + c];
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    float diff = qv - Cs[(cg + 8 * m) * (BF_DC + 1) + c];
                    acc[m] = fmaf(diff, diff, acc[m]);
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int m = 0; m < 8; ++m) Dt[qi * (BF_CB + 1) + cg + 8 * m] = acc[m];
        __syncthreads();

        // Fold the tile into the per-query lists; warp w owns queries 4w..4w+3.
        for (int r = warp * 4; r < warp * 4 + 4; ++r) {
            const int q = qid[r];
            if (q < 0) continue;
            float md = thr_d[r];
            int mj = thr_j[r], mp = thr_p[r];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = lane + 32 * h;
                const int64_t j = c0 + c;
                const bool valid = j < N && (cross || j != q);
                const float cd = valid ? Dt[r * (BF_CB + 1) + c] : INFINITY;
                const int cj = valid ? (int)j : INT_MAX;
                unsigned ball = __ballot_sync(0xffffffffu, pair_less(cd, cj, md, mj));
                while (ball) {
                    const int src = __ffs(ball) - 1;
                    ball &= ball - 1;
                    const float d = __shfl_sync(0xffffffffu, cd, src);
                    const int jj = __shfl_sync(0xffffffffu, cj, src);
                    if (!pair_less(d, jj, md, mj)) continue;
                    if (lane == 0) {
                        td[r * KCAP + mp] = d;
                        tj[r * KCAP + mp] = jj;
                    }
                    __syncwarp();
                    float bd = -INFINITY;
                    int bj = INT_MIN, bp = 0;
                    for (int s = lane; s < kl; s += 32) {
                        float sd = td[r * KCAP + s];
                        int sj = tj[r * KCAP + s];
                        if (pair_less(bd, bj, sd, sj)) {
                            bd = sd;
                            bj = sj;
                            bp = s;
                        }
                    }
                    warp_argmax_pair(bd, bj, bp);
                    md = bd;
                    mj = bj;
                    mp = bp;
                }
            }
            if (lane == 0) {
                thr_d[r] = md;
                thr_j[r] = mj;
                thr_p[r] = mp;
            }
        }
        __syncthreads();
    }

    // the tile buffers are free now: each warp's FP64 scratch for the near ties
    double *dm = reinterpret_cast<double *>(Cs) + warp * TIE_MAX;
    int *mp = reinterpret_cast<int *>(Dt) + warp * TIE_MAX;
    for (int r = warp * 4; r < warp * 4 + 4; ++r) {
        const int64_t o = orow[r];
        if (o < 0) continue;
        if (qid[r] >= 0) {
            // the list's distances in the library's one summation order
            const float *qrow = QX + (int64_t)qid[r] * D;
            const bool vec4 = (D & 3) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
                              (reinterpret_cast<uintptr_t>(qrow) & 15) == 0;
            const int g = lane >> 3, gl = lane & 7;
            for (int t0 = 0; t0 < kl; t0 += 8) {
                const int ta = t0 + g, tb = t0 + 4 + g;
                const int ja = ta < kl ? tj[r * KCAP + ta] : INT_MAX;
                const int jb = tb < kl ? tj[r * KCAP + tb] : INT_MAX;
                const float2 s2 = group8_d2_pair(qrow, ja != INT_MAX ? X + (int64_t)ja * D : qrow,
                                                 jb != INT_MAX ? X + (int64_t)jb * D : qrow, D, vec4, gl);
                if (gl == 0) {
                    if (ja != INT_MAX) td[r * KCAP + ta] = s2.x;
                    if (jb != INT_MAX) td[r * KCAP + tb] = s2.y;
                }
            }
            __syncwarp();
        }
        warp_bitonic_sort_smem(td + r * KCAP, tj + r * KCAP, KCAP, lane);
        if (qid[r] >= 0)
            fp64_near_ties(td + r * KCAP, tj + r * KCAP, kl, k, QX + (int64_t)qid[r] * D, X, D, dm, mp, lane);
        for (int t = lane; t < k; t += 32) {
            idx_out[o * k + t] = tj[r * KCAP + t];
            d2_out[o * k + t] = td[r * KCAP + t];
        }
    }
    __syncthreads();
    }
}

template <int KCAP>
atsne_status launch_bf(const float *X, int64_t N, int D, const int32_t *qlist, int64_t nq,
                       const int32_t *rows_list, const int32_t *rows_count, int k,
                       int32_t *idx_out, float *d2_out, cudaStream_t stream, const float *Xq) {
    const size_t smem = sizeof(float) * (BF_QB * (BF_DC + 1) + BF_CB * (BF_DC + 1) +
                                         BF_QB * (BF_CB + 1) + BF_QB * KCAP) +
                        sizeof(int) * BF_QB * KCAP;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(knn_bruteforce_kernel<KCAP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "knn_bruteforce attribute");
        attr_set = true;
    }
    const int grid = rows_count ? (int)hmin(2 * num_sms(), ceil_div(nq, BF_QB)) : ceil_div(nq, BF_QB);
    return launch_kernel(rows_count ? "knn_fallback" : "knn_bruteforce", knn_bruteforce_kernel<KCAP>,
                         grid, BF_THREADS, smem, stream, X, N, D, qlist, nq, rows_list, rows_count,
                         k, idx_out, d2_out, Xq);
}

}  // namespace

atsne_status knn_bruteforce(const float *X, int64_t N, int D, const int32_t *qlist, int64_t nq,
                            int k, int32_t *idx_out, float *d2_out, cudaStream_t stream) {
    return knn_bruteforce_rows(X, N, D, qlist, nullptr, nullptr, nq, k, idx_out, d2_out, stream);
}

atsne_status knn_bruteforce_rows(const float *X, int64_t N, int D, const int32_t *qlist,
                                 const int32_t *rows_list, const int32_t *rows_count, int64_t nq,
                                 int k, int32_t *idx_out, float *d2_out, cudaStream_t stream,
                                 const float *Xq) {
    if (nq <= 0) return ATSNE_OK;
    if (k <= 128) return launch_bf<128>(X, N, D, qlist, nq, rows_list, rows_count, k, idx_out, d2_out, stream, Xq);
    if (k <= 256) return launch_bf<256>(X, N, D, qlist, nq, rows_list, rows_count, k, idx_out, d2_out, stream, Xq);
    if (k <= 512) return launch_bf<512>(X, N, D, qlist, nq, rows_list, rows_count, k, idx_out, d2_out, stream, Xq);
    return set_error(ATSNE_EUNSUPPORTED, "knn: k=%d above the supported maximum of 512", k);
}

}  // namespace atsne
