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

// ---- the sums of x and x^2 per dimension over a range of points ----
//
// A block streams the rows of points pt[b..e) through shared memory in tiles
// of TP rows (two buffers, cp.async), W <= ACC_SLICE columns at a time;
// thread t accumulates columns 4t .. 4t+3 of the slice (one 16-byte shared
// load per row), in point order, into float pairs (acc_point).
constexpr int ACC_SLICE = 1024;         // columns per slice (256 threads x 4)
constexpr int ACC_TILE_FLOATS = 12288;  // floats per tile buffer (48 KB)


struct SliceGeom {
    int W, Wp, TP;  // columns, padded row length (multiple of 4), rows per tile
};
__host__ __device__ inline SliceGeom slice_geom(int D) {
    SliceGeom g;
    g.W = D < ACC_SLICE ? D : ACC_SLICE;
    g.Wp = (g.W + 3) & ~3;
    g.TP = ACC_TILE_FLOATS / g.Wp;
    if (g.TP > 32) g.TP = 32;
    return g;
}
// Threads of the blocks that call acc_slice: four columns each.
inline int acc_threads(int D) {
    const SliceGeom g = slice_geom(D);
    return ((g.Wp / 4 + 31) / 32) * 32;
}

// Accumulates columns [d0, d0 + W) of the points pt[b..e) into a[] (column
// d0 + 4 * threadIdx.x + i in a[i]). `tile` holds 2 * TP * Wp floats. Called
// by the whole block; returns with the tile buffers free.
__device__ void acc_slice(const float *__restrict__ X, int D, const int32_t *__restrict__ pt, int64_t b,
                          int64_t e, int d0, const SliceGeom &g, int W, float *tile, float4 (&a)[4]) {
    const int tid = threadIdx.x, nth = blockDim.x;
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    const bool v16 = (D & 3) == 0 && (d0 & 3) == 0 && (W & 3) == 0 &&
                     (reinterpret_cast<uintptr_t>(X) & 15) == 0;
    const int64_t n = e - b;
    const int64_t nt = (n + g.TP - 1) / g.TP;
    auto issue = [&](int64_t k) {
        float *buf = tile + (k & 1) * g.TP * g.Wp;
        const int64_t q0 = b + k * g.TP;
        const int rows = (int)(e - q0 < g.TP ? e - q0 : g.TP);
        // row r is `per` copies; thread tid takes copy tid % per of rows
        // tid / per, tid / per + step, ...
        const int per = v16 ? W >> 2 : W;
        const int step = nth / per > 0 ? nth / per : 1;
        for (int c0 = 0; c0 < per; c0 += nth) {
            const int c = c0 + (per >= nth ? tid : tid % per);
            const int r0 = per >= nth ? 0 : tid / per;
            if (c >= per || r0 >= step) continue;
            for (int r = r0; r < rows; r += step) {
                const float *src = X + (int64_t)pt[q0 + r] * D + d0;
                if (v16)
                    cp_async16(buf + r * g.Wp + 4 * c, src + 4 * c);
                else
                    cp_async4(buf + r * g.Wp + c, src + c);
            }
        }
        cp_async_commit();
    };
    const int c4 = 4 * tid;
    const bool full = c4 + 4 <= W;
    if (nt > 0) issue(0);
    for (int64_t k = 0; k < nt; ++k) {
        if (k + 1 < nt) {
            issue(k + 1);
            cp_async_wait1();
        } else {
            cp_async_wait0();
        }
        __syncthreads();
        const float *buf = tile + (k & 1) * g.TP * g.Wp + c4;
        const int rows = (int)(e - (b + k * g.TP) < g.TP ? e - (b + k * g.TP) : g.TP);
        if (full) {
            for (int r = 0; r < rows; ++r) {
                const float4 x = *reinterpret_cast<const float4 *>(buf + r * g.Wp);
                acc_point(a[0], x.x);
                acc_point(a[1], x.y);
                acc_point(a[2], x.z);
                acc_point(a[3], x.w);
            }
        } else if (c4 < W) {
            for (int r = 0; r < rows; ++r) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (c4 + i < W) acc_point(a[i], buf[r * g.Wp + i]);
            }
        }
        __syncthreads();
    }
}

// ---- 8-bit integer data: exact integer sums from the byte copy of X ----
// n * s2 - s1^2 exactly; the byte path runs only for N <= 2^18, so every term
// stays below 2^53 (and the FP64 sums of the definition are exact as well).
__device__ __forceinline__ uint64_t spread_exact(uint64_t s1, uint64_t s2, uint64_t n) { return n * s2 - s1 * s1; }

// Integer sums s1 (of x) and s2 (of x^2) of columns [d0, d0 + W) of the byte
// rows of points pt[b..e) (at most 65536 points, so s2 < 2^32): thread t takes
// columns d0 + 4t .. d0 + 4t + 3 (one 32-bit word per row). The rows stream
// through the same tile memory as acc_slice, in 16-byte pieces (cp.async).
__device__ void acc_slice_u8(const uint8_t *__restrict__ xu8, int Dp16, const int32_t *__restrict__ pt,
                             int64_t b, int64_t e, int d0, const SliceGeom &g, int W, float *tile_f,
                             uint32_t (&s1)[4], uint32_t (&s2)[4]) {
    const int tid = threadIdx.x, nth = blockDim.x;
#pragma unroll
    for (int i = 0; i < 4; ++i) s1[i] = s2[i] = 0u;
    uint8_t *tile = reinterpret_cast<uint8_t *>(tile_f);
    const int Wb = (W + 15) & ~15;  // bytes per tile row (the padding is the next columns or zeros)
    int TPb = g.TP * g.Wp * 4 / Wb;
    if (TPb > 64) TPb = 64;
    const int64_t n = e - b;
    const int64_t nt = (n + TPb - 1) / TPb;
    const int per = Wb >> 4;  // 16-byte pieces per row
    auto issue = [&](int64_t k) {
        uint8_t *buf = tile + (k & 1) * TPb * Wb;
        const int64_t q0 = b + k * TPb;
        const int rows = (int)(e - q0 < TPb ? e - q0 : TPb);
        const int step = nth / per > 0 ? nth / per : 1;
        for (int c0 = 0; c0 < per; c0 += nth) {
            const int c = c0 + (per >= nth ? tid : tid % per);
            const int r0 = per >= nth ? 0 : tid / per;
            if (c >= per || r0 >= step) continue;
            for (int r = r0; r < rows; r += step)
                cp_async16(reinterpret_cast<float *>(buf + r * Wb + 16 * c),
                           reinterpret_cast<const float *>(xu8 + (int64_t)pt[q0 + r] * Dp16 + d0 + 16 * c));
        }
        cp_async_commit();
    };
    const int c4 = 4 * tid;
    if (nt > 0) issue(0);
    for (int64_t k = 0; k < nt; ++k) {
        if (k + 1 < nt) {
            issue(k + 1);
            cp_async_wait1();
        } else {
            cp_async_wait0();
        }
        __syncthreads();
        const uint8_t *buf = tile + (k & 1) * TPb * Wb + c4;
        const int rows = (int)(e - (b + k * TPb) < TPb ? e - (b + k * TPb) : TPb);
        if (c4 < W) {
            for (int r = 0; r < rows; ++r) {
                const uint32_t w = *reinterpret_cast<const uint32_t *>(buf + r * Wb);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint32_t x = (w >> (8 * i)) & 0xffu;
                    s1[i] += x;
                    s2[i] += x * x;
                }
            }
        }
        __syncthreads();
    }
}

// Partial sums over CHUNK-point pieces of big nodes: grid (chunks, nodes, trees).
__global__ void __launch_bounds__(256)
partial_kernel(const float *__restrict__ X, int D, const int32_t *__restrict__ perm, int64_t N,
               const int32_t *__restrict__ leaf_ofs, int h, int l, int chunks,
               float4 *__restrict__ part, const uint8_t *__restrict__ xu8, int Dp16,
               const unsigned *__restrict__ u8_bad) {
    extern __shared__ __align__(16) float acc_tile[];
    const int ch = blockIdx.x, m = blockIdx.y, t = blockIdx.z;
    int64_t lo, hi;
    node_segment(leaf_ofs, h, l, m, lo, hi);
    const int64_t b = lo + (int64_t)ch * CHUNK, e = (hi < b + CHUNK ? hi : b + CHUNK);
    const int32_t *pt = perm + (int64_t)t * N;
    float4 *out = part + (((int64_t)t * gridDim.y + m) * chunks + ch) * D;
    const SliceGeom g = slice_geom(D);
    if (xu8 && *u8_bad == 0u) {  // byte rows: integer (s1, s2) in the first two words
        for (int d0 = 0; d0 < D; d0 += g.W) {
            const int W = D - d0 < g.W ? D - d0 : g.W;
            uint32_t s1[4], s2[4];
            acc_slice_u8(xu8, Dp16, pt, b, e, d0, g, W, acc_tile, s1, s2);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int c = 4 * threadIdx.x + i;
                if (c < W) out[d0 + c] = make_float4(__uint_as_float(s1[i]), __uint_as_float(s2[i]), 0.f, 0.f);
            }
        }
        return;
    }
    for (int d0 = 0; d0 < D; d0 += g.W) {
        const int W = D - d0 < g.W ? D - d0 : g.W;
        float4 a[4];
        acc_slice(X, D, pt, b, e, d0, g, W, acc_tile, a);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = 4 * threadIdx.x + i;
            if (c < W) out[d0 + c] = a[i];
        }
    }
}

// ---- top-V dimensions by spread ----
// Each lane keeps its best eight (spread, dim) pairs in registers, sorted by
// spread_greater; V rounds of a warp-wide argmax over the lanes' heads then
// give the V best in order. The spread is a float pair (hi, lo) or, for 8-bit
// integer data, the exact integer n * sum x^2 - (sum x)^2.
template <typename K>
struct TopN {
    K s[8];
    int d[8];
};
using Top8 = TopN<float2>;
using Top8u = TopN<uint64_t>;
__device__ __forceinline__ bool spread_greater(uint64_t a, int da, uint64_t b, int db) {
    if (a != b) return a > b;
    return da < db;
}
__device__ __forceinline__ void key_lowest(float2 &k) { k = make_float2(-INFINITY, -INFINITY); }
__device__ __forceinline__ void key_lowest(uint64_t &k) { k = 0ull; }  // empty slots carry dim INT_MAX
__device__ __forceinline__ float2 shfl_xor_key(float2 k, int o) {
    return make_float2(__shfl_xor_sync(0xffffffffu, k.x, o), __shfl_xor_sync(0xffffffffu, k.y, o));
}
__device__ __forceinline__ uint64_t shfl_xor_key(uint64_t k, int o) { return __shfl_xor_sync(0xffffffffu, k, o); }

template <typename K>
__device__ __forceinline__ void top8_init(TopN<K> &t) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        key_lowest(t.s[r]);
        t.d[r] = INT_MAX;
    }
}
template <typename K>
__device__ __forceinline__ void top8_insert(TopN<K> &t, K s, int d) {
    if (!spread_greater(s, d, t.s[7], t.d[7])) return;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        if (spread_greater(s, d, t.s[r], t.d[r])) {
            const K ts = t.s[r];
            const int td = t.d[r];
            t.s[r] = s;
            t.d[r] = d;
            s = ts;
            d = td;
        }
    }
}
// The split dimension of node v of tree t: one of the V best (counter-based
// draw). Whole warp; returns it on every lane.
template <typename K>
__device__ __forceinline__ int choose_from_top8(TopN<K> &t, int nV, uint64_t seed, int tree, int64_t v) {
    const uint64_t rr = splitmix64_at(seed, ((uint64_t)tree << 32) + (uint64_t)v + 1u);
    const int want = (int)(rr % (uint64_t)nV);
    int pick = 0;
    for (int r = 0; r < nV; ++r) {
        K best = t.s[0];
        int bd = t.d[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const K ok = shfl_xor_key(best, o);
            const int od = __shfl_xor_sync(0xffffffffu, bd, o);
            if (od != INT_MAX && (bd == INT_MAX || spread_greater(ok, od, best, bd))) {
                best = ok;
                bd = od;
            }
        }
        if (r == want) pick = bd;
        if (t.d[0] == bd) {  // the winning lane drops its head
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                t.s[q] = t.s[q + 1];
                t.d[q] = t.d[q + 1];
            }
            key_lowest(t.s[7]);
            t.d[7] = INT_MAX;
        }
    }
    return pick;
}

// Nodes of fewer than two points have every spread zero: the V best are the
// dimensions 0..V-1 (ties go to the smaller dimension).
__device__ __forceinline__ int choose_degenerate(int nV, uint64_t seed, int tree, int64_t v) {
    const uint64_t rr = splitmix64_at(seed, ((uint64_t)tree << 32) + (uint64_t)v + 1u);
    return (int)(rr % (uint64_t)nV);
}

// Per node (one block): spreads, top-V candidates, counter-based choice of
// the split dim. Nodes above CHUNK points combine their partial sums in order.
__global__ void __launch_bounds__(256)
choose_kernel(const float *__restrict__ X, int D, const int32_t *__restrict__ perm, int64_t N,
              const int32_t *__restrict__ leaf_ofs, int h, int l, int chunks,
              const float4 *__restrict__ part, int V, uint64_t seed, int32_t *__restrict__ split_dim,
              float *__restrict__ split_val, int64_t n_int, const uint8_t *__restrict__ xu8, int Dp16,
              const unsigned *__restrict__ u8_bad) {
    extern __shared__ __align__(16) float acc_tile[];
    const SliceGeom g = slice_geom(D);
    float2 *spread = reinterpret_cast<float2 *>(acc_tile + 2 * g.TP * g.Wp);  // [D]
    const int m = blockIdx.x, t = blockIdx.y;
    const int64_t v = ((int64_t)1 << l) - 1 + m;
    int64_t lo, hi;
    node_segment(leaf_ofs, h, l, m, lo, hi);
    const int nV = V < D ? V : D;
    if (hi - lo < 2) {
        if (threadIdx.x == 0) {
            split_dim[(int64_t)t * n_int + v] = choose_degenerate(nV, seed, t, v);
            split_val[(int64_t)t * n_int + v] = INFINITY;
        }
        return;
    }
    const float n = (float)(hi - lo);
    const int32_t *pt = perm + (int64_t)t * N;
    if (xu8 && *u8_bad == 0u) {  // byte rows: exact integer spreads
        uint64_t *sp = reinterpret_cast<uint64_t *>(spread);
        const uint64_t nn = (uint64_t)(hi - lo);
        if (chunks > 1) {
            for (int d = threadIdx.x; d < D; d += blockDim.x) {
                uint64_t s1 = 0, s2 = 0;
                const float4 *src = part + ((int64_t)t * gridDim.x + m) * chunks * D + d;
                for (int c = 0; c < chunks; ++c) {
                    const float4 q = src[(int64_t)c * D];
                    s1 += __float_as_uint(q.x);
                    s2 += __float_as_uint(q.y);
                }
                sp[d] = spread_exact(s1, s2, nn);
            }
        } else {
            for (int d0 = 0; d0 < D; d0 += g.W) {
                const int W = D - d0 < g.W ? D - d0 : g.W;
                uint32_t s1[4], s2[4];
                acc_slice_u8(xu8, Dp16, pt, lo, hi, d0, g, W, acc_tile, s1, s2);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int c = 4 * threadIdx.x + i;
                    if (c < W) sp[d0 + c] = spread_exact(s1[i], s2[i], nn);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            Top8u tp;
            top8_init(tp);
            for (int d = threadIdx.x; d < D; d += 32) top8_insert(tp, sp[d], d);
            const int dim = choose_from_top8(tp, nV, seed, t, v);
            if (threadIdx.x == 0) {
                split_dim[(int64_t)t * n_int + v] = dim;
                split_val[(int64_t)t * n_int + v] = INFINITY;
            }
        }
        return;
    }
    if (chunks > 1) {
        for (int d = threadIdx.x; d < D; d += blockDim.x) {
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 *src = part + ((int64_t)t * gridDim.x + m) * chunks * D + d;
            for (int c = 0; c < chunks; ++c) acc_pair(a, src[(int64_t)c * D]);
            spread[d] = spread_of(a, n);
        }
    } else {
        for (int d0 = 0; d0 < D; d0 += g.W) {
            const int W = D - d0 < g.W ? D - d0 : g.W;
            float4 a[4];
            acc_slice(X, D, pt, lo, hi, d0, g, W, acc_tile, a);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int c = 4 * threadIdx.x + i;
                if (c < W) spread[d0 + c] = spread_of(a[i], n);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        Top8 tp;
        top8_init(tp);
        for (int d = threadIdx.x; d < D; d += 32) top8_insert(tp, spread[d], d);
        const int dim = choose_from_top8(tp, nV, seed, t, v);
        if (threadIdx.x == 0) {
            split_dim[(int64_t)t * n_int + v] = dim;
            split_val[(int64_t)t * n_int + v] = INFINITY;
        }
    }
}

// Nodes of at most SMALL_NODE points: one warp per node; lane l accumulates
// the dimensions l, l + 32, ... (four at a time, four points' loads in flight
// together, accumulated in point order) and keeps its top eight.
constexpr int SMALL_NODE = 128;
constexpr int SMALL_WARPS = 8;

// Columns d0 + lane + 32 j (j < 4) over the node's points; FULL: all 128 in range.
template <bool FULL>
__device__ __forceinline__ void small_group(const float *__restrict__ X, int D, int d0, int lane, int cnt,
                                            const int (&pp)[4], float n, Top8 &tp) {
    // columns d0 + lane + 32 j (j < 4); four points per step, accumulated in point order
    float4 a[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) a[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int q = 0; q < cnt; q += 4) {
        float x[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int qq = q + i;
            const int sel = qq >> 5;
            const int pv = sel == 0 ? pp[0] : sel == 1 ? pp[1] : sel == 2 ? pp[2] : pp[3];
            const int p = __shfl_sync(0xffffffffu, pv, qq & 31);
            const float *r = X + (int64_t)p * D + d0 + lane;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                x[i][j] = qq < cnt && (FULL || d0 + lane + 32 * j < D) ? __ldg(r + 32 * j) : 0.f;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (q + i < cnt) {
#pragma unroll
                for (int j = 0; j < 4; ++j) acc_point(a[j], x[i][j]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int d = d0 + lane + 32 * j;
        if (FULL || d < D) top8_insert(tp, spread_of(a[j], n), d);
    }
}

// Byte rows: lane l takes columns g0 + 8 l .. g0 + 8 l + 7 of each 256-column
// group (one 8-byte load per point), exact integer sums, four points per step.
__device__ __forceinline__ void small_group_u8(const uint8_t *__restrict__ xu8, int Dp16, int D, int g0, int lane,
                                               int cnt, const int (&pp)[4], uint64_t n, Top8u &tp) {
    uint32_t s1[8], s2[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) s1[j] = s2[j] = 0u;
    const int c0 = g0 + 8 * lane;
    const bool in = c0 < Dp16;
    for (int q = 0; q < cnt; q += 4) {
        uint2 x[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int qq = q + i;
            const int sel = qq >> 5;
            const int pv = sel == 0 ? pp[0] : sel == 1 ? pp[1] : sel == 2 ? pp[2] : pp[3];
            const int p = __shfl_sync(0xffffffffu, pv, qq & 31);
            x[i] = qq < cnt && in ? __ldg(reinterpret_cast<const uint2 *>(xu8 + (int64_t)p * Dp16 + c0))
                                  : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t b = ((j < 4 ? x[i].x : x[i].y) >> (8 * (j & 3))) & 0xffu;
                s1[j] += b;
                s2[j] += b * b;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
        if (c0 + j < D) top8_insert(tp, spread_exact(s1[j], s2[j], n), c0 + j);
}

__global__ void __launch_bounds__(SMALL_WARPS * 32, 3)
choose_small_kernel(const float *__restrict__ X, int D, const int32_t *__restrict__ perm, int64_t N,
                    const int32_t *__restrict__ leaf_ofs, int h, int l, int V, uint64_t seed,
                    int32_t *__restrict__ split_dim, float *__restrict__ split_val, int64_t n_int,
                    const uint8_t *__restrict__ xu8, int Dp16, const unsigned *__restrict__ u8_bad) {
    const int lane = threadIdx.x & 31;
    const int64_t m = (int64_t)blockIdx.x * SMALL_WARPS + (threadIdx.x >> 5);
    const int t = blockIdx.y;
    if (m >= ((int64_t)1 << l)) return;
    const int64_t v = ((int64_t)1 << l) - 1 + m;
    int64_t lo, hi;
    node_segment(leaf_ofs, h, l, m, lo, hi);
    const int nV = V < D ? V : D;
    if (hi - lo < 2) {
        if (lane == 0) {
            split_dim[(int64_t)t * n_int + v] = choose_degenerate(nV, seed, t, v);
            split_val[(int64_t)t * n_int + v] = INFINITY;
        }
        return;
    }
    const float n = (float)(hi - lo);
    const int cnt = (int)(hi - lo);
    const int32_t *pt = perm + (int64_t)t * N;
    // the node's points, lane r holding points r, r + 32, r + 64 and r + 96
    int pp[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) pp[i] = lane + 32 * i < cnt ? pt[lo + lane + 32 * i] : 0;
    if (xu8 && *u8_bad == 0u) {  // byte rows: exact integer spreads
        Top8u tu;
        top8_init(tu);
        for (int g0 = 0; g0 < D; g0 += 256) small_group_u8(xu8, Dp16, D, g0, lane, cnt, pp, (uint64_t)cnt, tu);
        const int dim = choose_from_top8(tu, nV, seed, t, v);
        if (lane == 0) {
            split_dim[(int64_t)t * n_int + v] = dim;
            split_val[(int64_t)t * n_int + v] = INFINITY;
        }
        return;
    }
    Top8 tp;
    top8_init(tp);
    int d0 = 0;
    for (; d0 + 128 <= D; d0 += 128) small_group<true>(X, D, d0, lane, cnt, pp, n, tp);
    if (d0 < D) small_group<false>(X, D, d0, lane, cnt, pp, n, tp);
    const int dim = choose_from_top8(tp, nV, seed, t, v);
    if (lane == 0) {
        split_dim[(int64_t)t * n_int + v] = dim;
        split_val[(int64_t)t * n_int + v] = INFINITY;
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
    uint8_t *xu8;       // byte copy of X (N <= 2^18), else nullptr
    unsigned *u8_bad;
    int Dp16;
};

// The byte path (8-bit integer data) needs the partial sums exact: N <= 2^18.
constexpr int64_t BUILD_U8_MAX_N = int64_t(1) << 18;

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
    w.xu8 = nullptr;
    w.u8_bad = nullptr;
    w.Dp16 = (D + 15) & ~15;
    if (N <= BUILD_U8_MAX_N) {
        w.xu8 = c.take<uint8_t>((size_t)N * w.Dp16);
        w.u8_bad = c.take<unsigned>(1);
    }
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
    if (w.xu8) {  // 8-bit integer data: the spreads from a byte copy, exactly
        cudaError_t eb = cudaMemsetAsync(w.u8_bad, 0, sizeof(unsigned), stream);
        if (eb != cudaSuccess) return cuda_error(eb, "forest build memset");
        ATSNE_TRY(u8_copy_launch("forest_u8_prep", X, f.N, f.D, w.Dp16, w.xu8, nullptr, w.u8_bad, stream));
    }
    const SliceGeom sg = slice_geom(f.D);
    const size_t tile_smem = sizeof(float) * 2 * (size_t)sg.TP * sg.Wp;
    const size_t choose_smem = tile_smem + sizeof(float2) * (size_t)f.D;
    if (choose_smem > 227 * 1024)
        return set_error(ATSNE_EUNSUPPORTED, "forest build: D=%d needs %zu B of shared memory", f.D,
                         choose_smem);
    cudaError_t ea = cudaFuncSetAttribute(choose_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)choose_smem);
    if (ea == cudaSuccess)
        ea = cudaFuncSetAttribute(partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tile_smem);
    if (ea != cudaSuccess) return cuda_error(ea, "forest choose attribute");
    for (int l = 0; l < h; ++l) {
        const int64_t nodes = (int64_t)1 << l;
        const int64_t nmax = (f.N + nodes - 1) >> l;
        const int chunks = ceil_div(nmax, CHUNK);
        if (chunks > 1)
            ATSNE_TRY(launch_kernel("forest_partial", partial_kernel, dim3(chunks, (unsigned)nodes, T),
                                    acc_threads(f.D), tile_smem, stream, X, f.D, f.perm, f.N, f.leaf_ofs, h,
                                    l, chunks, w.part, (const uint8_t *)w.xu8, w.Dp16,
                                    (const unsigned *)w.u8_bad));
        if (nmax <= SMALL_NODE)
            ATSNE_TRY(launch_kernel("forest_choose", choose_small_kernel,
                                    dim3((unsigned)ceil_div(nodes, SMALL_WARPS), T), SMALL_WARPS * 32, 0,
                                    stream, X, f.D, f.perm, f.N, f.leaf_ofs, h, l, f.top_var_dims,
                                    f.seed, f.split_dim, f.split_val, f.n_internal, (const uint8_t *)w.xu8,
                                    w.Dp16, (const unsigned *)w.u8_bad));
        else
            ATSNE_TRY(launch_kernel("forest_choose", choose_kernel, dim3((unsigned)nodes, T),
                                    acc_threads(f.D), choose_smem, stream, X, f.D, f.perm, f.N, f.leaf_ofs, h, l, chunks,
                                    w.part, f.top_var_dims, f.seed, f.split_dim, f.split_val,
                                    f.n_internal, (const uint8_t *)w.xu8, w.Dp16, (const unsigned *)w.u8_bad));
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
