// Forest of randomized KD-trees (Sec. 4.2): level-by-level build and a
// best-bin-first search with one priority queue across the forest.
//
// Storage is level-ordered and implicit: node v has children 2v+1, 2v+2, a
// node with n points gives the first ceil(n/2) in (value, index) order to its
// left child, so every node's segment of the permutation depends on N alone
// and the leaf boundaries leaf_ofs[] are shared by all trees.
//
// Build, per level l (all trees in the same launches):
//   choose : per node, spread of every dimension over the node's points
//            (n*sum x^2 - (sum x)^2, sums accumulated as float pairs with
//            error-free transformations), the V dimensions of largest spread,
//            and the split dimension picked by a counter-based SplitMix64 of
//            (seed, tree, node). Nodes larger than CHUNK points are summed in
//            CHUNK-point partials first (partial kernel) and combined in order.
//   keys   : 64-bit key (order-preserving float bits << 32 | point) per point,
//            padded per node to the next power of two.
//   sort   : bitonic network (all compare-exchanges ascending); segments up to
//            4096 keys sort in shared memory, longer ones take global passes
//            for the spans above 4096.
//   scatter: sorted points back into the permutation; split value = float
//            midpoint of the last left and first right value (+inf when the
//            node has fewer than two points).
// The search is in forest_query.cu.
#include <float.h>
#include <limits.h>

#include "common.cuh"
#include "internal.h"

namespace atsne {

int forest_depth(int64_t N, int leaf_size) {
    int h = 0;
    while (h < 40 && ((N + ((int64_t)1 << h) - 1) >> h) > leaf_size) ++h;
    return h;
}

size_t forest_layout(int64_t N, int trees, int leaf_size, atsne_forest_layout_t *out) {
    const int h = forest_depth(N, leaf_size);
    const int64_t n_int = ((int64_t)1 << h) - 1;
    Carver c(nullptr);
    atsne_forest_layout_t L;
    L.depth = h;
    L.trees = trees;
    L.n_internal = n_int;
    c.take<char>(0);
    L.off_split_dim = c.off;
    c.take<int32_t>((size_t)trees * (n_int > 0 ? n_int : 1));
    c.off = (c.off + 255) & ~size_t(255);
    L.off_split_val = c.off;
    c.take<float>((size_t)trees * (n_int > 0 ? n_int : 1));
    c.off = (c.off + 255) & ~size_t(255);
    L.off_perm = c.off;
    c.take<int32_t>((size_t)trees * N);
    c.off = (c.off + 255) & ~size_t(255);
    L.off_leaf_ofs = c.off;
    c.take<int32_t>(((size_t)1 << h) + 1);
    c.off = (c.off + 255) & ~size_t(255);
    L.off_leaf_pt = c.off;
    c.take<int32_t>((size_t)trees << h);
    L.bytes = c.bytes();
    if (out) *out = L;
    return L.bytes;
}

namespace {

constexpr int CHUNK = 1024;        // points per partial-sum chunk
constexpr int SMEM_SORT = 4096;    // keys per shared-memory bitonic block
constexpr int CHOOSE_THREADS = 256;

// ---- counter-based SplitMix64 (Steele, Lea, Flood 2014): output number c ----
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t c) {
    uint64_t z = seed + c * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// ---- float-pair (hi + lo) accumulation by error-free transformations ----
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
}
__device__ __forceinline__ void acc_point(float4 &a, float x) {
    // a = (s1 hi, s1 lo, s2 hi, s2 lo)
    two_sum_acc(a.x, a.y, x);
    const float p = x * x;
    const float pe = fmaf(x, x, -p);
    two_sum_acc(a.z, a.w, p);
    a.w += pe;
}
__device__ __forceinline__ void acc_pair(float4 &a, const float4 &b) {
    two_sum_acc(a.x, a.y, b.x);
    a.y += b.y;
    two_sum_acc(a.z, a.w, b.z);
    a.w += b.w;
}
// n * s2 - s1^2 as a normalised float pair (hi, lo).
__device__ __forceinline__ float2 spread_of(const float4 &a, float n) {
    const float s1h = a.x + a.y, s1l = a.y - (s1h - a.x);
    const float s2h = a.z + a.w, s2l = a.w - (s2h - a.z);
    const float p = n * s2h, pe = fmaf(n, s2h, -p) + n * s2l;
    const float q = s1h * s1h, qe = fmaf(s1h, s1h, -q) + 2.f * s1h * s1l;
    const float vh = p - q;
    const float bp = vh - p;
    const float ve = (p - (vh - bp)) + (-q - bp) + (pe - qe);
    const float h = vh + ve;
    return make_float2(h, ve - (h - vh));
}
__device__ __forceinline__ bool spread_greater(float2 a, int da, float2 b, int db) {
    if (a.x != b.x) return a.x > b.x;
    if (a.y != b.y) return a.y > b.y;
    return da < db;
}

__device__ __forceinline__ void node_segment(const int32_t *leaf_ofs, int h, int l, int64_t m,
                                             int64_t &lo, int64_t &hi) {
    lo = leaf_ofs[m << (h - l)];
    hi = leaf_ofs[(m + 1) << (h - l)];
}

__global__ void leaf_ofs_kernel(int64_t N, int h, int32_t *leaf_ofs) {
    const int64_t L = (int64_t)1 << h;
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m > L) return;
    if (m == L) {
        leaf_ofs[m] = (int32_t)N;
        return;
    }
    int64_t lo = 0, n = N;
    for (int l = 0; l < h; ++l) {
        const int64_t nl = (n + 1) >> 1;
        if ((m >> (h - 1 - l)) & 1) {
            lo += nl;
            n -= nl;
        } else {
            n = nl;
        }
    }
    leaf_ofs[m] = (int32_t)lo;
}

// leaf_pt[t][m]: the first point of leaf m of tree t, -1 for an empty leaf.
__global__ void leaf_pt_kernel(const int32_t *__restrict__ perm, const int32_t *__restrict__ leaf_ofs,
                               int64_t N, int h, int T, int32_t *__restrict__ leaf_pt) {
    const int64_t L = (int64_t)1 << h;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= L * T) return;
    const int t = (int)(g / L);
    const int64_t m = g - (int64_t)t * L;
    const int32_t a = leaf_ofs[m], b = leaf_ofs[m + 1];
    leaf_pt[g] = b > a ? perm[(int64_t)t * N + a] : -1;
}

__global__ void iota_kernel(int32_t *perm, int64_t N, int T) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < N * T) perm[g] = (int32_t)(g % N);
}

// Partial sums over CHUNK-point pieces of big nodes: grid (chunks, nodes, trees).
__global__ void __launch_bounds__(CHOOSE_THREADS)
partial_kernel(const float *__restrict__ X, int D, const int32_t *__restrict__ perm, int64_t N,
               const int32_t *__restrict__ leaf_ofs, int h, int l, int chunks,
               float4 *__restrict__ part) {
    const int ch = blockIdx.x, m = blockIdx.y, t = blockIdx.z;
    int64_t lo, hi;
    node_segment(leaf_ofs, h, l, m, lo, hi);
    const int64_t b = lo + (int64_t)ch * CHUNK, e = (hi < b + CHUNK ? hi : b + CHUNK);
    const int32_t *pt = perm + (int64_t)t * N;
    float4 *out = part + (((int64_t)t * gridDim.y + m) * chunks + ch) * D;
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int64_t q = b; q < e; ++q) acc_point(a, X[(int64_t)pt[q] * D + d]);
        out[d] = a;
    }
}

// Per node: spreads, top-V candidates, counter-based choice of the split dim.
__global__ void __launch_bounds__(CHOOSE_THREADS)
choose_kernel(const float *__restrict__ X, int D, const int32_t *__restrict__ perm, int64_t N,
              const int32_t *__restrict__ leaf_ofs, int h, int l, int chunks,
              const float4 *__restrict__ part, int V, uint64_t seed, int32_t *__restrict__ split_dim,
              float *__restrict__ split_val, int64_t n_int) {
    extern __shared__ float2 spread[];  // [D]
    const int m = blockIdx.x, t = blockIdx.y;
    const int64_t v = ((int64_t)1 << l) - 1 + m;
    int64_t lo, hi;
    node_segment(leaf_ofs, h, l, m, lo, hi);
    const float n = (float)(hi - lo);
    const int32_t *pt = perm + (int64_t)t * N;
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        if (chunks > 1) {
            const float4 *src = part + ((int64_t)t * gridDim.x + m) * chunks * D + d;
            for (int c = 0; c < chunks; ++c) acc_pair(a, src[(int64_t)c * D]);
        } else {
            for (int64_t q = lo; q < hi; ++q) acc_point(a, X[(int64_t)pt[q] * D + d]);
        }
        spread[d] = spread_of(a, n);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const int nV = V < D ? V : D;
        int chosen[8];
        for (int r = 0; r < nV; ++r) {
            float2 best = make_float2(-INFINITY, -INFINITY);
            int bd = INT_MAX;
            for (int d = lane; d < D; d += 32) {
                bool taken = false;
                for (int u = 0; u < r; ++u) taken |= (chosen[u] == d);
                if (!taken && spread_greater(spread[d], d, best, bd)) {
                    best = spread[d];
                    bd = d;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ox = __shfl_xor_sync(0xffffffffu, best.x, o);
                const float oy = __shfl_xor_sync(0xffffffffu, best.y, o);
                const int od = __shfl_xor_sync(0xffffffffu, bd, o);
                if (od != INT_MAX && (bd == INT_MAX || spread_greater(make_float2(ox, oy), od, best, bd))) {
                    best = make_float2(ox, oy);
                    bd = od;
                }
            }
            chosen[r] = bd;
        }
        if (lane == 0) {
            const uint64_t rr = splitmix64_at(seed, ((uint64_t)t << 32) + (uint64_t)v + 1u);
            split_dim[(int64_t)t * n_int + v] = chosen[rr % (uint64_t)nV];
            split_val[(int64_t)t * n_int + v] = INFINITY;
        }
    }
}

// keys[t][m * P + s]: (float key << 32 | point) for s < n, all-ones padding.
__global__ void keys_kernel(const float *__restrict__ X, int D, const int32_t *__restrict__ perm,
                            int64_t N, const int32_t *__restrict__ leaf_ofs, int h, int l, int64_t P,
                            const int32_t *__restrict__ split_dim, int64_t n_int, int T,
                            uint64_t *__restrict__ keys) {
    const int64_t per_tree = ((int64_t)1 << l) * P;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= per_tree * T) return;
    const int t = (int)(g / per_tree);
    const int64_t rem = g - (int64_t)t * per_tree;
    const int64_t m = rem / P, s = rem - m * P;
    int64_t lo, hi;
    node_segment(leaf_ofs, h, l, m, lo, hi);
    uint64_t key = ~0ull;
    if (s < hi - lo) {
        const int32_t p = perm[(int64_t)t * N + lo + s];
        const int dim = split_dim[(int64_t)t * n_int + ((int64_t)1 << l) - 1 + m];
        key = ((uint64_t)float_key(X[(int64_t)p * D + dim]) << 32) | (uint32_t)p;
    }
    keys[g] = key;
}

__device__ __forceinline__ void ce_asc(uint64_t *k, int a, int c) {
    const uint64_t x = k[a], y = k[c];
    if (y < x) {
        k[a] = y;
        k[c] = x;
    }
}

// Bitonic network (flip form) on 4096-key blocks in shared memory.
// mode 0: full sort of every aligned segment of `seg` (<= 4096) keys.
// mode 1: the half-cleaners with strides 2048..1 that finish a merge whose
//         larger spans were done by global passes.
__global__ void __launch_bounds__(1024)
sort_smem_kernel(uint64_t *__restrict__ keys, int64_t total, int seg, int mode) {
    __shared__ uint64_t sk[SMEM_SORT];
    const int64_t base = (int64_t)blockIdx.x * SMEM_SORT;
    for (int i = threadIdx.x; i < SMEM_SORT; i += blockDim.x)
        sk[i] = base + i < total ? keys[base + i] : ~0ull;
    __syncthreads();
    if (mode == 0) {
        for (int size = 2; size <= seg; size <<= 1) {
            const int half = size >> 1;
            for (int t = threadIdx.x; t < SMEM_SORT / 2; t += blockDim.x) {
                const int blk = (t / half) * size, off = t % half;
                ce_asc(sk, blk + off, blk + size - 1 - off);
            }
            __syncthreads();
            for (int stride = size >> 2; stride > 0; stride >>= 1) {
                for (int t = threadIdx.x; t < SMEM_SORT / 2; t += blockDim.x) {
                    const int a = 2 * t - (t & (stride - 1));
                    ce_asc(sk, a, a + stride);
                }
                __syncthreads();
            }
        }
    } else {
        for (int stride = SMEM_SORT >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < SMEM_SORT / 2; t += blockDim.x) {
                const int a = 2 * t - (t & (stride - 1));
                ce_asc(sk, a, a + stride);
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < SMEM_SORT; i += blockDim.x)
        if (base + i < total) keys[base + i] = sk[i];
}

// One global compare-exchange pass: flip=1 the mirrored first step of a merge
// of `size`, else a half-cleaner with `stride`.
__global__ void sort_global_kernel(uint64_t *__restrict__ keys, int64_t total, int64_t size,
                                   int64_t stride, int flip) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total / 2) return;
    int64_t a, c;
    if (flip) {
        const int64_t half = size >> 1;
        const int64_t blk = (t / half) * size, off = t % half;
        a = blk + off;
        c = blk + size - 1 - off;
    } else {
        a = 2 * t - (t & (stride - 1));
        c = a + stride;
    }
    const uint64_t x = keys[a], y = keys[c];
    if (y < x) {
        keys[a] = y;
        keys[c] = x;
    }
}

__global__ void scatter_kernel(const float *__restrict__ X, int D, int32_t *__restrict__ perm,
                               int64_t N, const int32_t *__restrict__ leaf_ofs, int h, int l,
                               int64_t P, const int32_t *__restrict__ split_dim,
                               float *__restrict__ split_val, int64_t n_int, int T,
                               const uint64_t *__restrict__ keys) {
    const int64_t per_tree = ((int64_t)1 << l) * P;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= per_tree * T) return;
    const int t = (int)(g / per_tree);
    const int64_t rem = g - (int64_t)t * per_tree;
    const int64_t m = rem / P, s = rem - m * P;
    int64_t lo, hi;
    node_segment(leaf_ofs, h, l, m, lo, hi);
    const int64_t n = hi - lo;
    if (s >= n) return;
    const uint32_t p = (uint32_t)(keys[g] & 0xffffffffu);
    perm[(int64_t)t * N + lo + s] = (int32_t)p;
    const int64_t nl = (n + 1) >> 1;
    if (n >= 2 && s == nl - 1) {
        const int64_t v = ((int64_t)1 << l) - 1 + m;
        const int dim = split_dim[(int64_t)t * n_int + v];
        const uint32_t pr = (uint32_t)(keys[g + 1] & 0xffffffffu);
        const float a = X[(int64_t)p * D + dim], b = X[(int64_t)pr * D + dim];
        split_val[(int64_t)t * n_int + v] = __fmul_rn(0.5f, __fadd_rn(a, b));
    }
}

struct BuildWs {
    uint64_t *keys;
    float4 *part;
    int64_t key_count;  // per launch (all trees)
};

int64_t pow2_at_least(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

}  // namespace

size_t forest_build_workspace(Carver &c, int64_t N, int D, int trees, int leaf_size, void *ws_out) {
    const int h = forest_depth(N, leaf_size);
    int64_t max_keys = 1;
    for (int l = 0; l < h; ++l) {
        const int64_t nmax = (N + ((int64_t)1 << l) - 1) >> l;
        max_keys = max_keys > (((int64_t)1 << l) * pow2_at_least(nmax))
                       ? max_keys
                       : (((int64_t)1 << l) * pow2_at_least(nmax));
    }
    BuildWs w;
    w.key_count = max_keys * trees;
    w.keys = c.take<uint64_t>((size_t)(w.key_count + SMEM_SORT));
    // partial sums exist only on levels whose nodes exceed CHUNK points
    int64_t max_parts = 1;
    for (int l = 0; l < h; ++l) {
        const int64_t nmax = (N + ((int64_t)1 << l) - 1) >> l;
        const int64_t ch = (nmax + CHUNK - 1) / CHUNK;
        if (ch > 1 && (((int64_t)1 << l) * ch) > max_parts) max_parts = ((int64_t)1 << l) * ch;
    }
    w.part = c.take<float4>((size_t)trees * (size_t)max_parts * D);
    if (ws_out) *static_cast<BuildWs *>(ws_out) = w;
    return c.bytes();
}

atsne_status forest_build_launch(const float *X, const ForestView &f, void *ws_base,
                                 size_t ws_bytes, cudaStream_t stream) {
    Carver c(ws_base);
    BuildWs w;
    forest_build_workspace(c, f.N, f.D, f.trees, f.leaf_size, &w);
    if (c.bytes() > ws_bytes) return set_error(ATSNE_ENOMEM, "forest build: workspace too small");
    const int h = f.depth, T = f.trees;
    ATSNE_TRY(launch_kernel("forest_leaf_ofs", leaf_ofs_kernel, ceil_div(((int64_t)1 << h) + 1, 256),
                            256, 0, stream, f.N, h, f.leaf_ofs));
    ATSNE_TRY(launch_kernel("forest_iota", iota_kernel, ceil_div(f.N * T, 256), 256, 0, stream, f.perm,
                            f.N, T));
    const size_t choose_smem = sizeof(float2) * (size_t)f.D;
    if (choose_smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(choose_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)choose_smem);
        if (e != cudaSuccess) return cuda_error(e, "forest choose attribute");
    }
    for (int l = 0; l < h; ++l) {
        const int64_t nodes = (int64_t)1 << l;
        const int64_t nmax = (f.N + nodes - 1) >> l;
        const int chunks = ceil_div(nmax, CHUNK);
        int threads = f.D >= CHOOSE_THREADS ? CHOOSE_THREADS : ((f.D + 31) / 32) * 32;
        if (threads < 32) threads = 32;
        if (chunks > 1)
            ATSNE_TRY(launch_kernel("forest_partial", partial_kernel, dim3(chunks, (unsigned)nodes, T),
                                    threads, 0, stream, X, f.D, f.perm, f.N, f.leaf_ofs, h, l, chunks,
                                    w.part));
        ATSNE_TRY(launch_kernel("forest_choose", choose_kernel, dim3((unsigned)nodes, T), threads,
                                choose_smem, stream, X, f.D, f.perm, f.N, f.leaf_ofs, h, l, chunks,
                                w.part, f.top_var_dims, f.seed, f.split_dim, f.split_val,
                                f.n_internal));
        const int64_t P = pow2_at_least(nmax);
        const int64_t total = nodes * P * T;
        ATSNE_TRY(launch_kernel("forest_keys", keys_kernel, ceil_div(total, 256), 256, 0, stream, X,
                                f.D, f.perm, f.N, f.leaf_ofs, h, l, P, f.split_dim, f.n_internal, T,
                                w.keys));
        const int blocks = ceil_div(total, SMEM_SORT);
        ATSNE_TRY(launch_kernel("forest_sort_smem", sort_smem_kernel, blocks, 1024, 0, stream, w.keys,
                                total, (int)(P < SMEM_SORT ? P : SMEM_SORT), 0));
        for (int64_t size = 2 * SMEM_SORT; size <= P; size <<= 1) {
            ATSNE_TRY(launch_kernel("forest_sort_global", sort_global_kernel, ceil_div(total / 2, 256),
                                    256, 0, stream, w.keys, total, size, (int64_t)0, 1));
            for (int64_t stride = size >> 2; stride >= SMEM_SORT; stride >>= 1)
                ATSNE_TRY(launch_kernel("forest_sort_global", sort_global_kernel,
                                        ceil_div(total / 2, 256), 256, 0, stream, w.keys, total, size,
                                        stride, 0));
            ATSNE_TRY(launch_kernel("forest_sort_smem", sort_smem_kernel, blocks, 1024, 0, stream,
                                    w.keys, total, (int)SMEM_SORT, 1));
        }
        ATSNE_TRY(launch_kernel("forest_scatter", scatter_kernel, ceil_div(total, 256), 256, 0, stream,
                                X, f.D, f.perm, f.N, f.leaf_ofs, h, l, P, f.split_dim, f.split_val,
                                f.n_internal, T, w.keys));
    }
    return launch_kernel("forest_leaf_pt", leaf_pt_kernel, ceil_div(((int64_t)T) << h, 256), 256, 0,
                         stream, f.perm, f.leaf_ofs, f.N, h, T, f.leaf_pt);
}

}  // namespace atsne
