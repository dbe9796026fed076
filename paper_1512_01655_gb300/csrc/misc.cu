// Small kernels: precision rho (Eq. 9) and the row scatter of a refinement.
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
            for (int u = 0; u < k; ++u) found |= (row[u] == j);
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

}  // namespace

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

}  // namespace atsne
