// Shared host/device helpers of the sm_103a library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "atsne.h"

namespace atsne {

// ---------------------------------------------------------------------------
// Host side: errors, workspace carving, launch profiling
// ---------------------------------------------------------------------------
atsne_status set_error(atsne_status st, const char *fmt, ...);
atsne_status cuda_error(cudaError_t e, const char *what);
int *device_status_word();  // device address of the status word (current device)

// Device status codes written by kernels (first writer wins).
enum : int { DEV_OK = 0, DEV_NONFINITE = 1, DEV_MALFORMED = 2, DEV_TIMEOUT = 3 };

// Carves 256-byte aligned slices out of a caller workspace. With base == nullptr
// it only measures, so one layout function serves sizing and carving.
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base(static_cast<char *>(b)) {}
    template <typename T>
    T *take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
    size_t bytes() const { return (off + 255) & ~size_t(255); }
};

// Brackets one kernel launch with CUDA events on its stream while profiling is on.
struct ProfScope {
    int slot;
    cudaStream_t stream;
    ProfScope(const char *kernel, cudaStream_t s);
    ~ProfScope();
};

void count_launch();  // one kernel launch enqueued by this library

// Launch `kern` on `stream`, bracketed by profiling events and counted.
template <typename... KArgs, typename... Args>
atsne_status launch_kernel(const char *name, void (*kern)(KArgs...), dim3 grid, dim3 block,
                           size_t smem, cudaStream_t stream, Args &&...args) {
    if (grid.x == 0 || grid.y == 0 || grid.z == 0) return ATSNE_OK;
    ProfScope prof(name, stream);
    kern<<<grid, block, smem, stream>>>(static_cast<KArgs>(args)...);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, name);
    return ATSNE_OK;
}

#define ATSNE_TRY(expr)                                                       \
    do {                                                                      \
        atsne_status st_ = (expr);                                            \
        if (st_ != ATSNE_OK) return st_;                                      \
    } while (0)

#define ATSNE_LAUNCH_CHECK(what)                                              \
    do {                                                                      \
        cudaError_t e_ = cudaGetLastError();                                  \
        if (e_ != cudaSuccess) return ::atsne::cuda_error(e_, what);          \
    } while (0)

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
inline int64_t hmin(int64_t a, int64_t b) { return a < b ? a : b; }
inline int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// ---------------------------------------------------------------------------
// Device side
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

__device__ __forceinline__ void raise_status(int *status, int code) {
    if (status) atomicCAS(status, DEV_OK, code);
}

// Total order on (distance, index) used for every neighbour list.
__device__ __forceinline__ bool pair_less(float da, int ja, float db, int jb) {
    return da < db || (da == db && ja < jb);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Lexicographic max of (d, j) over the warp; returns it in every lane.
__device__ __forceinline__ void warp_argmax_pair(float &d, int &j, int &pos) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float od = __shfl_xor_sync(0xffffffffu, d, o);
        int oj = __shfl_xor_sync(0xffffffffu, j, o);
        int op = __shfl_xor_sync(0xffffffffu, pos, o);
        if (pair_less(d, j, od, oj)) {
            d = od;
            j = oj;
            pos = op;
        }
    }
}

// FP32 squared distances ||q - xa||^2 and ||q - xb||^2 in the one summation
// order in which every exact kNN kernel returns its distances, so that a row's
// d2 does not depend on the kernel that computed it. The dimensions are cut
// into chunks of four; lane g of an 8-lane group sums the chunks g, g + 8,
// g + 16, ... as one FMA chain in dimension order, and the group's eight
// partial sums are added by a butterfly (xor 1, 2, 4), which leaves the same
// value in all eight lanes (floating-point addition commutes). Each group
// takes its own two points (pass q for an unused one); all 32 lanes of the
// warp call it together. vec4: D % 4 == 0 and all rows 16-byte aligned (the
// order is the same either way).
__device__ __forceinline__ float2 group8_d2_pair(const float *__restrict__ q, const float *__restrict__ xa,
                                                 const float *__restrict__ xb, int D, bool vec4, int gl) {
    float sa = 0.f, sb = 0.f;
    if (vec4) {
        const int n4 = D >> 2;
        const float4 *q4 = reinterpret_cast<const float4 *>(q);
        const float4 *a4 = reinterpret_cast<const float4 *>(xa);
        const float4 *b4 = reinterpret_cast<const float4 *>(xb);
#pragma unroll 4
        for (int j = gl; j < n4; j += 8) {
            const float4 qv = q4[j], av = a4[j], bv = b4[j];
            float df = qv.x - av.x;
            sa = fmaf(df, df, sa);
            df = qv.y - av.y;
            sa = fmaf(df, df, sa);
            df = qv.z - av.z;
            sa = fmaf(df, df, sa);
            df = qv.w - av.w;
            sa = fmaf(df, df, sa);
            df = qv.x - bv.x;
            sb = fmaf(df, df, sb);
            df = qv.y - bv.y;
            sb = fmaf(df, df, sb);
            df = qv.z - bv.z;
            sb = fmaf(df, df, sb);
            df = qv.w - bv.w;
            sb = fmaf(df, df, sb);
        }
    } else {
        for (int j = gl; 4 * j < D; j += 8) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int e = 4 * j + c;
                if (e < D) {
                    float df = q[e] - xa[e];
                    sa = fmaf(df, df, sa);
                    df = q[e] - xb[e];
                    sb = fmaf(df, df, sb);
                }
            }
        }
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    return make_float2(sa, sb);
}

// Near ties of a sorted neighbour list settled in FP64 (Eq. 8's order on
// exact distances): d[0, n) ascending with their points j[0, n) (FP32
// distances in the order of group8_d2_pair; entries of infinite distance are
// padding and their j is not read). Each such distance is within
// (m + 8) 2^-24 of its value, m = 4 ceil(D / 32) the terms of one lane's FMA
// chain: a rounded difference squares to within 2u + u^2 (u = 2^-24), the
// chain of m FMAs (exact products) and the three butterfly additions of
// positive terms add at most gamma_(m+3). Runs of neighbours
// whose FP32 gaps are within twice that bound, among the first k + 1, are
// recomputed as FP64 sums of squared differences of the query row xq and X's
// rows and put in (FP64 distance, index) order, their distances replaced by
// the FP64 values rounded to FP32. Outside such runs the FP32 order is the
// exact one. At most TIE_MAX members are recomputed (the rest keep the FP32
// order). Warp-cooperative; dm/mp are TIE_MAX doubles and ints of the warp's
// shared memory.
constexpr int TIE_MAX = 64;
__device__ __forceinline__ void fp64_near_ties(float *d, int *j, int n, int k, const float *__restrict__ xq,
                                               const float *__restrict__ X, int D, double *dm, int *mp,
                                               int lane) {
    const int m = n < k + 1 ? n : k + 1;
    const float band = 2.f * (float)(4 * ((D + 31) / 32) + 8) * 0x1p-24f;
    int nm = 0;
    for (int t0 = 0; t0 < m; t0 += 32) {
        const int t = t0 + lane;
        bool tie_prev = false, tie_next = false;
        // entries of infinite distance (a list's padding) are never members
        if (t < m && d[t] < INFINITY) {
            const float dt = d[t];
            if (t > 0) tie_prev = dt - d[t - 1] <= band * dt;
            if (t + 1 < m && d[t + 1] < INFINITY) tie_next = d[t + 1] - dt <= band * d[t + 1];
        }
        const bool mem = t < m && (tie_prev || tie_next);
        const unsigned mm = __ballot_sync(0xffffffffu, mem);
        const int pos = nm + __popc(mm & ((1u << lane) - 1u));
        if (mem && pos < TIE_MAX) mp[pos] = t;
        nm += __popc(mm);
    }
    if (nm == 0) return;
    if (nm > TIE_MAX) nm = TIE_MAX;
    __syncwarp();
    for (int i = 0; i < nm; ++i) {
        const float *xc = X + (int64_t)j[mp[i]] * D;
        double s = 0.0;
        for (int c = lane; c < D; c += 32) {
            const double df = (double)xq[c] - (double)xc[c];
            s = fma(df, df, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) dm[i] = s;
    }
    __syncwarp();
    if (lane == 0) {
        // each run of consecutive members: insertion sort by (FP64 distance, index)
        int a = 0;
        while (a < nm) {
            int b = a + 1;
            while (b < nm && mp[b] == mp[b - 1] + 1 && d[mp[b]] - d[mp[b - 1]] <= band * d[mp[b]]) ++b;
            for (int x = a + 1; x < b; ++x) {
                const double kd = dm[x];
                const int kj = j[mp[x]];
                int y = x - 1;
                while (y >= a && (dm[y] > kd || (dm[y] == kd && j[mp[y]] > kj))) {
                    dm[y + 1] = dm[y];
                    j[mp[y + 1]] = j[mp[y]];
                    --y;
                }
                dm[y + 1] = kd;
                j[mp[y + 1]] = kj;
            }
            for (int x = a; x < b; ++x) d[mp[x]] = (float)dm[x];
            a = b;
        }
    }
    __syncwarp();
}

// Order-preserving map of a float to uint32 (-0 folded onto +0, so that the
// ordering of values equals IEEE comparison order; inputs are finite).
__device__ __forceinline__ uint32_t float_key(float f) {
    f = f + 0.0f;  // -0 -> +0
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// In-warp bitonic sort of n (key, value) pairs held in shared memory,
// ascending by (key, value). n is a power of two; the caller pads the unused
// tail with entries that sort last.
template <typename K, typename V>
__device__ __forceinline__ void warp_bitonic_sort_smem(K *key, V *val, int n, int lane) {
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = lane; t < (n >> 1); t += 32) {
                int i = 2 * t - (t & (stride - 1));
                int j = i + stride;
                bool up = ((i & size) == 0);
                K ki = key[i], kj = key[j];
                V vi = val[i], vj = val[j];
                bool gt = (kj < ki) || (kj == ki && vj < vi);
                if (gt == up) {
                    key[i] = kj;
                    key[j] = ki;
                    val[i] = vj;
                    val[j] = vi;
                }
            }
            __syncwarp();
        }
    }
}

// Asynchronous global -> shared copies (cp.async): 4 or 16 bytes per call,
// completed in commit-group order; a thread's wait covers its own copies.
__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(float *dst, const float *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async_wait1() { cp_async_wait<1>(); }
__device__ __forceinline__ void cp_async_wait0() { cp_async_wait<0>(); }

#endif  // __CUDACC__

}  // namespace atsne
