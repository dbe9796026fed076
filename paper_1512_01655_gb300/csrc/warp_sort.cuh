// Warp-cooperative sorts and selections of (key, value) pairs held in shared
// memory.
#pragma once

#include "common.cuh"

namespace atsne {

// Warp-cooperative bitonic sort of n = 32 * R (key, value) pairs in shared
// memory, ascending by (key, value), carried out in registers: lane l holds
// elements l*R .. l*R + R - 1, so exchanges between elements fewer than R
// apart stay within a lane and the others are shuffles between lanes. It is
// the network of warp_bitonic_sort_smem (the same compare-exchanges in the
// same order), without a shared-memory round trip per exchange.
template <int R, typename K, typename V>
__device__ __forceinline__ void warp_sort_regs(K *key, V *val, int lane) {
    K k[R];
    V v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        k[r] = key[lane * R + r];
        v[r] = val[lane * R + r];
    }
    for (int size = 2; size <= 32 * R; size <<= 1) {
        const bool lane_up = ((lane * R) & size) == 0;  // direction of this lane's elements, size >= R
        for (int stride = size >> 1; stride >= R; stride >>= 1) {
            const int lm = stride / R;
            const bool keep_min = ((lane & lm) == 0) == lane_up;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const K pk = __shfl_xor_sync(0xffffffffu, k[r], lm);
                const V pv = __shfl_xor_sync(0xffffffffu, v[r], lm);
                const bool pless = pk < k[r] || (pk == k[r] && pv < v[r]);
                if (pless == keep_min) {
                    k[r] = pk;
                    v[r] = pv;
                }
            }
        }
#pragma unroll
        for (int stride = R >> 1; stride > 0; stride >>= 1) {
            if (stride < size) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r & stride) continue;
                    const bool up = ((lane * R + r) & size) == 0;
                    const int q = r + stride;
                    const bool gt = k[q] < k[r] || (k[q] == k[r] && v[q] < v[r]);
                    if (gt == up) {
                        const K tk = k[r];
                        k[r] = k[q];
                        k[q] = tk;
                        const V tv = v[r];
                        v[r] = v[q];
                        v[q] = tv;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        key[lane * R + r] = k[r];
        val[lane * R + r] = v[r];
    }
}

// Sort of n (a power of two, at least 32) pairs: in registers up to 512,
// else in shared memory.
template <typename K, typename V>
__device__ __forceinline__ void warp_sort_pow2(K *key, V *val, int n, int lane) {
    switch (n) {
        case 32: warp_sort_regs<1>(key, val, lane); break;
        case 64: warp_sort_regs<2>(key, val, lane); break;
        case 128: warp_sort_regs<4>(key, val, lane); break;
        case 256: warp_sort_regs<8>(key, val, lane); break;
        case 512: warp_sort_regs<16>(key, val, lane); break;
        default: warp_bitonic_sort_smem(key, val, n, lane);
    }
}

// Moves the entries of key[0, n) (32 < n <= 512) whose keys are at most the
// m-th smallest key (1 <= m <= n; every entry equal to it included) to
// positions [0, c) of key/val, in no particular order, and returns c when
// c <= cap; otherwise leaves both arrays unchanged and returns -1. The first m
// entries of the whole set in (key, value) order are then the first m of
// those c in that order. Keys are non-negative floats, compared through their
// bit patterns (which order them); the m-th is found by bisection on the bit
// pattern, counting with the warp's reduction. Entry t sits in lane t % 32.
// Warp-cooperative; n, m and cap uniform.
template <typename V>
__device__ __forceinline__ int warp_smallest_to_front(float *key, V *val, int n, int m, int cap, int lane) {
    constexpr int R = 16;
    uint32_t u[R];
    V v[R];
    uint32_t lo = 0xffffffffu, hi = 0u;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int t = r * 32 + lane;
        u[r] = 0xffffffffu;  // past n: above every key
        if (t < n) {
            u[r] = __float_as_uint(key[t]);
            v[r] = val[t];
            lo = min(lo, u[r]);
            hi = max(hi, u[r]);
        }
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    // the smallest T in [lo, hi] with at least m keys at or below it
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        int c0 = 0, c1 = 0;
#pragma unroll
        for (int r = 0; r < R; r += 2) {
            c0 += u[r] <= mid;
            c1 += u[r + 1] <= mid;
        }
        if ((int)__reduce_add_sync(0xffffffffu, (unsigned)(c0 + c1)) >= m) hi = mid;
        else lo = mid + 1;
    }
    int c0 = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) c0 += u[r] <= lo;
    const int c = (int)__reduce_add_sync(0xffffffffu, (unsigned)c0);
    if (c > cap) return -1;
    __syncwarp();  // every entry is in registers before the front is overwritten
    const unsigned below = (1u << lane) - 1u;
    int base = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const bool in = u[r] <= lo;
        const unsigned b = __ballot_sync(0xffffffffu, in);
        if (in) {
            const int pos = base + __popc(b & below);
            key[pos] = __uint_as_float(u[r]);
            val[pos] = v[r];
        }
        base += __popc(b);
    }
    __syncwarp();
    return c;
}

}  // namespace atsne
