// Density-based view of the embedding and its approximation map (Sec. 5.2):
// per pixel p of a W x H image over the 2-D embedding, with a Gaussian kernel
// G(d, h) = exp(-d^2 / (2 h^2)) / (2 pi h^2),
//   F = sum_i G(|p - y_i|, h),  S = sum_{i selected} G,  R = sum_i rho_i G,
//   f = F / N (Eq. 12),  s = S / F (Eq. 13, selected share),
//   a = R / F (Sec. 5.2.2, rho-weighted mean),  alpha = 1 - a^k (the lens).
// Points farther than cutoff * h from a pixel are left out of its sums
// (cutoff 0: every point counts).
//
// One CTA renders a 16 x 16 tile, one pixel per thread: it streams the points
// in index order, keeps those within reach of the tile (the tile's box widened
// by the cutoff radius) in shared memory in that order, and every thread
// accumulates its pixel's three sums over them. No atomics: each pixel's sums
// are taken in point order, so the image does not depend on scheduling.
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace atsne {
namespace {

constexpr int KT = 16;           // tile side in pixels
constexpr int KDE_THREADS = KT * KT;
constexpr int KDE_CHUNK = 1024;  // points examined per pass

__global__ void __launch_bounds__(KDE_THREADS)
kde_kernel(const float2 *__restrict__ Y, int64_t N, const float *__restrict__ rho,
           const uint8_t *__restrict__ sel, float x0, float y0, float px, int W, int H, float h,
           float cutoff, float lens_k, float *__restrict__ f_out, float *__restrict__ s_out,
           float *__restrict__ a_out, float *__restrict__ alpha_out) {
    __shared__ float2 ps[KDE_CHUNK];
    __shared__ float pw[KDE_CHUNK][2];  // selection weight, rho
    __shared__ int wcount[KDE_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ix = blockIdx.x * KT + (tid % KT), iy = blockIdx.y * KT + (tid / KT);
    // pixel centre and reach in FP32 with explicitly rounded operations: the
    // decision "within cutoff * h" is the kernel's and is restated exactly so
    const float cx = __fmaf_rn((float)ix + 0.5f, px, x0), cy = __fmaf_rn((float)iy + 0.5f, px, y0);
    const float r = cutoff > 0.f ? __fmul_rn(cutoff, h) : INFINITY;
    const float bx0 = x0 + (float)(blockIdx.x * KT) * px - r, bx1 = x0 + (float)((blockIdx.x + 1) * KT) * px + r;
    const float by0 = y0 + (float)(blockIdx.y * KT) * px - r, by1 = y0 + (float)((blockIdx.y + 1) * KT) * px + r;
    const float r2 = __fmul_rn(r, r);
    const float inv2h2 = 1.f / (2.f * h * h);
    const float norm = 1.f / (2.f * 3.14159265358979f * h * h);
    float F = 0.f, S = 0.f, R = 0.f;
    for (int64_t c0 = 0; c0 < N; c0 += KDE_CHUNK) {
        // keep the chunk's points within reach, in index order
        int n_keep = 0;
        for (int b = 0; b < KDE_CHUNK; b += KDE_THREADS) {
            const int64_t i = c0 + b + tid;
            float2 y = make_float2(0.f, 0.f);
            bool in = false;
            if (i < N) {
                y = Y[i];
                in = y.x >= bx0 && y.x <= bx1 && y.y >= by0 && y.y <= by1;
            }
            const unsigned m = __ballot_sync(0xffffffffu, in);
            if (lane == 0) wcount[warp] = __popc(m);
            __syncthreads();
            int before = n_keep, total = 0;
            for (int w = 0; w < KDE_THREADS / 32; ++w) {
                if (w < warp) before += wcount[w];
                total += wcount[w];
            }
            if (in) {
                const int pos = before + __popc(m & ((1u << lane) - 1u));
                ps[pos] = y;
                pw[pos][0] = sel ? (sel[i] ? 1.f : 0.f) : 0.f;
                pw[pos][1] = rho ? rho[i] : 1.f;
            }
            n_keep += total;
            __syncthreads();
        }
        for (int q = 0; q < n_keep; ++q) {
            const float dx = __fsub_rn(cx, ps[q].x), dy = __fsub_rn(cy, ps[q].y);
            const float d2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
            if (d2 <= r2) {
                const float g = norm * __expf(-d2 * inv2h2);
                F += g;
                S = fmaf(pw[q][0], g, S);
                R = fmaf(pw[q][1], g, R);
            }
        }
        __syncthreads();
    }
    if (ix < W && iy < H) {
        const int64_t o = (int64_t)iy * W + ix;
        const float a = F > 0.f ? R / F : 1.f;
        if (f_out) f_out[o] = F / (float)N;
        if (s_out) s_out[o] = F > 0.f ? S / F : 0.f;
        if (a_out) a_out[o] = a;
        if (alpha_out) alpha_out[o] = 1.f - powf(fmaxf(a, 0.f), lens_k);
    }
}

}  // namespace

atsne_status kde_launch(const float *Y, int64_t N, const float *rho, const uint8_t *selected, float x0,
                        float y0, float pixel, int W, int H, float h, float cutoff, float lens_k,
                        float *f_out, float *s_out, float *a_out, float *alpha_out,
                        cudaStream_t stream) {
    const dim3 grid((unsigned)ceil_div(W, KT), (unsigned)ceil_div(H, KT));
    return launch_kernel("kde_map", kde_kernel, grid, KDE_THREADS, 0, stream,
                         reinterpret_cast<const float2 *>(Y), N, rho, selected, x0, y0, pixel, W, H,
                         h, cutoff, lens_k, f_out, s_out, a_out, alpha_out);
}

}  // namespace atsne
