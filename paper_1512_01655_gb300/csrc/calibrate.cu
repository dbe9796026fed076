// Per-point Gaussian bandwidth by bisection and the conditional rows P_{j|i}
// (Eq. 3 and Eq. 4, Sec. 3, over the kNN support of Eq. 8).
//
// One thread owns one row. A CTA of 128 threads stages its 128 contiguous rows
// (128*k floats, one coalesced sweep) into shared memory with an odd row
// stride, so the per-thread row walks are bank-conflict free; the P rows leave
// the same way. Each bisection step evaluates, for the shifted distances
// s_j = d_j - min d, w_j = exp(-beta s_j), Z = sum w_j and
// H = ln Z + beta sum_j w_j s_j / Z (nats), compares H with ln(perplexity) and
// halves the bracket exactly as the definition prescribes: start beta = 1,
// double while no upper bound is known, then bisect.
//
// A distance of +inf marks an absent neighbour (a neighbourhood shortened by a
// deletion, Sec. 5.3.2): it is outside N_i, takes no part in the sums and gets
// P = 0; a row without any neighbour gets P = 0 and beta = 0.
//
// Arithmetic: FP32 throughout. GB300 runs FP64 at 1/64 of the FP32 rate, and
// the parity bound for P (1e-5 absolute) needs H only to about 1e-6, which the
// 90-term FP32 sums give with a wide margin; the stopping tolerance defaults to
// 1e-5 nats for that reason.
#include <float.h>

#include "common.cuh"
#include "internal.h"

namespace atsne {
namespace {

constexpr int CAL_THREADS = 128;

// Bisection on beta over the shifted distances s_j of one row (returns the
// final beta and the normaliser Z); GAPS: the row holds absent entries (+inf).
template <bool GAPS>
__device__ __forceinline__ void bisect(const float *row, int k, float target, float tol, int max_iter,
                                       float &bf, float &Z) {
    float beta = 1.f, lo = 0.f, hi = INFINITY;
    for (int it = 1;; ++it) {
        bf = fminf(beta, FLT_MAX);
        float z = 0.f, ws = 0.f;
        for (int j = 0; j < k; ++j) {
            const float s = row[j];
            if (GAPS && s == INFINITY) continue;  // absent
            const float w = expf(-bf * s);
            z += w;
            ws = fmaf(w, s, ws);
        }
        const float H = logf(z) + bf * ws / z;
        Z = z;
        if (fabsf(H - target) < tol || it >= max_iter) break;
        if (H > target) {
            lo = beta;
            beta = isinf(hi) ? 2.f * beta : 0.5f * (beta + hi);
        } else {
            hi = beta;
            beta = 0.5f * (lo + beta);
        }
    }
}

__global__ void __launch_bounds__(CAL_THREADS)
calibrate_kernel(const float *__restrict__ d2, int64_t rows, int k, float perplexity, float target,
                 float tol, int max_iter, float *__restrict__ P, float *__restrict__ beta_out, int *status) {
    extern __shared__ float sm[];
    const int stride = k | 1;
    const int64_t r0 = (int64_t)blockIdx.x * CAL_THREADS;
    const int nr = (int)(rows - r0 < CAL_THREADS ? rows - r0 : CAL_THREADS);
    const float *src = d2 + r0 * k;
    for (int t = threadIdx.x; t < nr * k; t += CAL_THREADS) {
        int r = t / k, c = t - r * k;
        sm[r * stride + c] = src[t];
    }
    __syncthreads();

    if ((int)threadIdx.x < nr) {
        float *row = sm + threadIdx.x * stride;
        float dmin = INFINITY;
        bool valid = true;
        int present = 0;
        for (int j = 0; j < k; ++j) {
            float v = row[j];
            valid &= v >= 0.f;  // NaN and negative distances are errors; +inf is absent
            dmin = fminf(dmin, v);
            present += v < INFINITY;
        }
        if (!valid) raise_status(status, DEV_NONFINITE);
        if (dmin < INFINITY)
            for (int j = 0; j < k; ++j) row[j] -= dmin;  // s_j (+inf stays +inf)

        // the entropy over n present neighbours is at most log n, reached only
        // at beta = 0: when n <= perplexity the bisection's limit is beta = 0,
        // a uniform row, which is taken directly
        const bool flat = present > 0 && (float)present <= perplexity;
        float bf = 1.f, Z = 1.f;
        if (flat) bf = 0.f, Z = (float)present;
        // a full row (the usual case) skips the absent-entry test in the sums
        if (dmin < INFINITY && !flat) {
            if (present == k)
                bisect<false>(row, k, target, tol, max_iter, bf, Z);
            else
                bisect<true>(row, k, target, tol, max_iter, bf, Z);
        }
        if (dmin == INFINITY) bf = 0.f;  // no neighbour
        const float inv = dmin < INFINITY ? 1.f / Z : 0.f;
        for (int j = 0; j < k; ++j) row[j] = row[j] == INFINITY ? 0.f : expf(-bf * row[j]) * inv;
        if (beta_out) beta_out[r0 + threadIdx.x] = bf;
    }
    __syncthreads();
    float *dst = P + r0 * k;
    for (int t = threadIdx.x; t < nr * k; t += CAL_THREADS) {
        int r = t / k, c = t - r * k;
        dst[t] = sm[r * stride + c];
    }
}

}  // namespace

size_t calibrate_smem_bytes(int k) { return sizeof(float) * CAL_THREADS * (size_t)(k | 1); }

atsne_status calibrate_launch(const float *d2, int64_t rows, int k, float perplexity, float tol,
                              int max_iter, float *P, float *beta, cudaStream_t stream) {
    if (rows <= 0) return ATSNE_OK;
    const size_t smem = calibrate_smem_bytes(k);
    static size_t attr = 0;
    if (smem > 48 * 1024 && smem > attr) {
        cudaError_t e = cudaFuncSetAttribute(calibrate_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "calibrate attribute");
        attr = smem;
    }
    return launch_kernel("calibrate_beta", calibrate_kernel, ceil_div(rows, CAL_THREADS),
                         CAL_THREADS, smem, stream, d2, rows, k, perplexity, logf(perplexity), tol, max_iter, P,
                         beta, device_status_word());
}

}  // namespace atsne
