// Warp-cooperative sorts of (key, value) pairs held in shared memory.
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

}  // namespace atsne
