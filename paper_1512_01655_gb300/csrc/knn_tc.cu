// Exact kNN (Eq. 8, Sec. 3.1) on the tcgen05 tensor cores.
//
// Distances are ranked by key_j = ||x_j||^2 - 2 x_i.x_j (||x_i||^2 is common to
// a query row). The contraction x_i.x_j runs on the tensor cores in BF16 with
// FP32 accumulation in TMEM: one pass (x ~ hi) for the BF16 mode, three passes
// (x ~ hi + lo; hi.hi' + hi.lo' + lo.hi') for the FP32 mode. The N x N key
// matrix never leaves the SM:
//
//   knn_prep   x -> hi (+ lo) BF16 copies padded to Dp = 64*ceil(D/64), the
//              FP32 norm ||x||^2, and the norms of what the BF16 copies miss
//              (used to bound the key error).
//   knn_tc     persistent, warp-specialised: warp 0 issues TMA loads of
//              128-query x 64 and 256-point x 64 BF16 tiles (128-byte swizzle)
//              into a shared-memory ring; warp 1 issues tcgen05.mma
//              (M=128, N=256, K=16) into one of two TMEM accumulators; warps
//              2-5 read the other accumulator back (tcgen05.ld, one query row
//              per thread), form the keys, and append every key below the
//              row's running threshold tau to a per-(row, column split)
//              candidate buffer. Each thread also counts its buffered
//              distances in 64 buckets (8 per octave below an upper bound of
//              any distance of the row); tau is lowered to the upper edge of
//              the bucket in which the count reaches ksel, a valid bound on
//              the ksel-th distance within 9%. Buffers are sized for about
//              2.5x the survivors of a streaming top-ksel, so the exact
//              compaction of a full buffer (warp radix select) is rare.
//              When few query rows leave the SMs idle, the columns are cut
//              into splits (units ordered split-major); the splits of a row
//              then also count into one histogram per row in global memory,
//              so each split filters with the bound of the whole row.
//   knn_merge  one warp per query: one pass stages the keys below the
//              splits' lowest tau (+2E) in shared memory; there the k-th
//              smallest key is selected, every candidate within 2E of it (E
//              bounds the key error, see row_error_bound) is re-ranked by
//              FP32 direct differences, and a certificate is checked: if the
//              k-th exact distance is below ||x_i||^2 + min(tau) - E, no
//              point outside the buffers can belong to the k nearest, and
//              the row is exact. Rows that fail are listed for the
//              brute-force kernel.
//
// Every wait on an mbarrier is bounded (1 s); on expiry the CTA raises the
// device status word, stops issuing work, drains its own copies and MMAs and
// releases TMEM before it exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <float.h>
#include <limits.h>
#include <math.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"
#include "warp_sort.cuh"

namespace atsne {
namespace {

using namespace tc;

constexpr int TC_BM = 128;       // query rows per tile (TMEM lanes)
constexpr int TC_BN = 256;       // corpus points per tile (TMEM columns per accumulator)
constexpr int TC_BK = 64;        // BF16 per k-block (one 128-byte swizzle row)
constexpr uint64_t WAIT_NS = 1000000000ull;
constexpr int MERGE_WARPS = 4;
constexpr int RCAP = 256;        // candidates re-ranked per row at most (certified modes)
constexpr int MSTAGE = 1024;     // keys below tau staged per row for the merge's select
constexpr int RCAP_FP8 = 1024;   // modes without a certificate: the largest re-rank set (ksel <= 512)
constexpr int NBUCKET = 64;      // a thread's distance buckets: 2 octaves of d^2, 32 per octave
constexpr int HSHIFT = 18;       // float bits >> HSHIFT: exponent and 5 mantissa bits (32 per octave)
constexpr int GH_BUCKETS = 48;   // a row's global histogram (column splits): 6 octaves, 8 per octave
constexpr int GH_SHIFT = 20;

struct Cand {
    float key;
    int32_t idx;
};

// PASSES: 1 = one BF16 pass, 3 = BF16 hi/lo in three passes, 8 = one FP8
// (E4M3, per-row scale) pass. A k-block is one 128-byte swizzle row: 64 BF16
// or 128 FP8 values, four MMAs (K = 16 or 32).
// With PASSES = 3 and every low half zero (data exact in BF16, e.g. 8-bit
// integers) the two correction passes add exact zeros: the kernel then skips
// them and runs the same shared memory as MAX_STAGES single-pass stages.
//
// One-pass modes run eight epilogue warps (two per TMEM lane quadrant, each
// filtering half of a tile's columns) so that the filter keeps up with the
// shorter contraction; the shared memory then holds three stages. The
// three-pass mode keeps four epilogue warps and two double-width stages.
template <int PASSES>
struct TcCfg {
    static constexpr int NEPI = PASSES == 3 ? 4 : 8;      // epilogue warps
    static constexpr int HALVES = NEPI / 4;               // column parts of a tile per lane quadrant
    static constexpr int THREADS = 64 + 32 * NEPI;        // warp 0 TMA, warp 1 MMA, then the epilogue
    static constexpr int STAGES = PASSES == 3 ? 2 : 3;
    static constexpr int MAX_STAGES = PASSES == 3 ? 4 : 3;
    static constexpr int KE = PASSES == 8 ? 128 : TC_BK;  // elements per k-block
    static constexpr int A_BYTES = TC_BM * 128;
    static constexpr int B_BYTES = TC_BN * 128;
    // One-pass BF16 folds the column norms into the contraction: one more
    // K = 16 step multiplies a constant query slice (-1/2 three times) with
    // each corpus row's norm in three BF16 pieces, so the accumulator holds
    // x.y - ||y||^2 / 2 and the key is -2 times it (exact scaling).
    static constexpr bool FOLD = PASSES == 1;
    static constexpr int EXT_A_BYTES = TC_BM * 32;             // the constant slice, resident
    static constexpr int EXT_B_BYTES = FOLD ? TC_BN * 32 : 0;  // a tile's norm pieces, per stage
    static constexpr int STAGE_BYTES = (A_BYTES + B_BYTES) * (PASSES == 3 ? 2 : 1) + EXT_B_BYTES;
};

template <int PASSES>
struct __align__(1024) TcSmem {
    static constexpr int NEPI = TcCfg<PASSES>::NEPI;
    unsigned char stage[TcCfg<PASSES>::STAGES][TcCfg<PASSES>::STAGE_BYTES];
    unsigned char a_ext[TcCfg<PASSES>::FOLD ? TcCfg<PASSES>::EXT_A_BYTES : 16];  // 1024-aligned
    float ny[NEPI][2][32];      // per epilogue warp: two chunks' corpus norms (double-buffered)
    float ms[PASSES == 8 ? NEPI : 1][2][32];  // FP8: two chunks' -2 * corpus row scales
    // per epilogue warp: the 256 counters of the radix select of an exact compaction
    uint32_t sel_hist[NEPI][256];
    // per epilogue thread: buffered distances by bucket, two 16-bit counts per word
    uint32_t dhist[NEPI][NBUCKET / 2][32];
    // each half's current tau per query row, tagged with its work unit:
    // (unit << 32) | tau bits
    unsigned long long tau_sh[TcCfg<PASSES>::HALVES > 1 ? TcCfg<PASSES>::HALVES : 1][TcCfg<PASSES>::HALVES > 1 ? TC_BM : 1];
    uint64_t full[TcCfg<PASSES>::MAX_STAGES];
    uint64_t empty[TcCfg<PASSES>::MAX_STAGES];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t drain;
    uint64_t ext_bar;  // the constant query slice has landed
    // each unit's first column tile of the main stream, from the producer to
    // the epilogue (a ring of four units, one barrier each)
    uint64_t unit_bar[4];
    uint32_t unit_start[4];
    uint32_t tmem_base;
    int abort_flag;
    int zero;
};

struct TcParams {
    CUtensorMap tm_a_hi, tm_a_lo, tm_b_hi, tm_b_lo;
    CUtensorMap tm_a_ext, tm_b_ext;  // one-pass BF16: the norm slices
    const int32_t *pro;    // ordered rows and columns: per row tile, the first column tile of its
                           // groups and their count (streamed first); nullptr: natural order
    unsigned long long *clock;  // tiles issued by all CTAs (one split): where a unit's stream starts
    const float *nrm;      // [N] corpus ||x||^2
    const float *scale;    // FP8: [N] corpus row scales (x ~ scale * q)
    const float *qscale;   // FP8 with a query list: [Q] query row scales
    const float *qnrm;     // queries from another array: [Q] their ||x||^2 (no self exclusion)
    const float *radius;   // radius mode: [Q] squared radius per query row (else nullptr)
    const float *hint;     // [Q] upper bounds of each query row's k-th squared distance (or nullptr)
    const float4 *qst;     // queries from another array: their error statistics
    const float4 *st;      // corpus rows' error statistics (for listed queries)
    float acc_coef;        // FP32 accumulation term of the key error bound
    float sq_coef;         // the same for the folded norms, per max ||y||^2
    const unsigned *gmax;  // max ||x|| over the corpus (float bits)
    const unsigned *lo_max;  // max norm of the corpus' BF16 low halves (float bits), or nullptr
                             // when the queries' low halves are not covered by it
    const int32_t *qlist;  // query row -> corpus index (nullptr: identity)
    int64_t Q, N;
    int KB;                // Dp / 64
    int splits, cols_per_split, row_tiles;
    int ksel, cap;
    Cand *cand;            // [Q][splits * halves][cap]
    int4 *meta;            // [Q][splits * halves]: count, tau bits, overflow
    unsigned *row_hist;    // [Q][GH_BUCKETS]: buffered distances of all splits by bucket (splits > 1)
    int *status;
    uint64_t wait_ns;      // limit of each pipeline wait (the drains of issued copies and MMAs keep WAIT_NS)
};

// Absolute bucket of a squared distance on the thread grid (32 per octave),
// and the upper edge of bucket b.
__device__ __forceinline__ int dbucket(float d) { return (int)(__float_as_uint(fmaxf(d, 1e-30f)) >> HSHIFT); }
__device__ __forceinline__ float bucket_top(int b) { return __uint_as_float((uint32_t)(b + 1) << HSHIFT); }

// (mask << 1) | sign bit of v: one funnel shift per key.
__device__ __forceinline__ uint32_t sign_into_mask(float v, uint32_t mask) {
    uint32_t r;
    asm("shf.l.wrap.b32 %0, %1, %2, 1;" : "=r"(r) : "r"(__float_as_uint(v)), "r"(mask));
    return r;
}

__device__ __forceinline__ float key_of_bits(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Shared-memory add whose result is not needed (no wait on it).
__device__ __forceinline__ void red_add_shared(uint32_t *p, uint32_t v) { atomicAdd(p, v); }

// Adds one to hist[bin] for every active lane; must be called by the whole
// warp. Lanes that share a bin are combined into one shared-memory atomic: the
// keys of one query row mostly share their leading digits, so plain per-lane
// atomics would serialise 32 ways on a single bin.
__device__ __forceinline__ void warp_hist_add(uint32_t *hist, uint32_t bin, bool active) {
    const unsigned act = __ballot_sync(0xffffffffu, active);
    if (active) {
        const unsigned peers = __match_any_sync(act, bin);
        if ((peers & lanemask_lt()) == 0) atomicAdd(&hist[bin], (uint32_t)__popc(peers));
    }
}

// Radix select over (key) of `count` candidates fetched by get(i): returns the
// order-preserving bits of the kth smallest key (1-based) and, in n_less, how
// many keys are strictly smaller. Warp-cooperative (count and kth uniform over
// the warp); hist is 256 words of shared memory private to the warp.
// visit(fn) calls fn(valid, key) for every candidate, in iterations uniform
// over the warp.
template <typename Visit>
__device__ uint32_t warp_select_visit(Visit visit, int kth, uint32_t *hist, int lane, int &n_less) {
    uint32_t prefix = 0, mask = 0;
    int rem = kth;
    n_less = 0;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int i = lane; i < 256; i += 32) hist[i] = 0u;
        __syncwarp();
        visit([&](bool valid, float key) {
            const uint32_t u = float_key(key);
            warp_hist_add(hist, (u >> shift) & 255u, valid && (u & mask) == prefix);
        });
        __syncwarp();
        uint32_t c[8], sum = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            c[q] = hist[8 * lane + q];
            sum += c[q];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t excl = incl - sum;
        const bool mine = excl < (uint32_t)rem && (uint32_t)rem <= incl;
        const unsigned who = __ballot_sync(0xffffffffu, mine);
        const int src = who ? __ffs(who) - 1 : 31;
        int bin = 255;
        uint32_t before = 0;
        if (lane == src) {
            uint32_t acc = excl;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (acc + c[q] >= (uint32_t)rem) {
                    bin = 8 * lane + q;
                    before = acc;
                    break;
                }
                acc += c[q];
            }
        }
        bin = __shfl_sync(0xffffffffu, bin, src);
        before = __shfl_sync(0xffffffffu, before, src);
        rem -= (int)before;
        n_less += (int)before;
        prefix |= (uint32_t)bin << shift;
        mask |= 255u << shift;
        __syncwarp();
    }
    return prefix;
}

template <typename Get>
__device__ uint32_t warp_select(Get get, int count, int kth, uint32_t *hist, int lane, int &n_less) {
    return warp_select_visit(
        [&](auto fn) {
            for (int base = 0; base < count; base += 32) {
                const int i = base + lane;
                fn(i < count, i < count ? get(i) : 0.f);
            }
        },
        kth, hist, lane, n_less);
}

// ---------------------------------------------------------------------------
// prep: BF16 hi/lo copies, norms, error norms
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
knn_prep_kernel(const float *__restrict__ X, const int32_t *__restrict__ rows, int64_t nrows, int64_t N,
                int D, int Dp, int passes, __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo,
                float *__restrict__ nrm, float4 *__restrict__ stats, unsigned *__restrict__ gmax,
                __nv_bfloat16 *__restrict__ bext, __nv_bfloat16 *__restrict__ aext, int *status) {
    const int lane = threadIdx.x & 31;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    // the constant query slice of the folded norms: -1/2 in its first three columns
    if (aext && blockIdx.x == 0)
        for (int t = threadIdx.x; t < TC_BM * 16; t += blockDim.x)
            aext[t] = __float2bfloat16_rn((t & 15) < 3 ? -0.5f : 0.f);
    if (r >= nrows) return;
    int64_t src = rows ? rows[r] : r;
    if (src < 0 || src >= N) src = 0;  // flagged by the caller's index check
    const float *x = X + src * D;
    float n = 0.f, res = 0.f, l2 = 0.f;
    bool finite = true;
    for (int d = lane; d < Dp; d += 32) {
        const float v = d < D ? x[d] : 0.f;
        finite &= isfinite(v);
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const float r1 = v - __bfloat162float(h);
        hi[r * Dp + d] = h;
        n = fmaf(v, v, n);
        if (passes == 3) {
            const __nv_bfloat16 l = __float2bfloat16_rn(r1);
            const float lf = __bfloat162float(l);
            const float r2 = r1 - lf;
            lo[r * Dp + d] = l;
            res = fmaf(r2, r2, res);
            l2 = fmaf(lf, lf, l2);
        } else {
            res = fmaf(r1, r1, res);
        }
    }
    n = warp_sum(n);
    res = warp_sum(res);
    l2 = warp_sum(l2);
    if (bext && lane < 16) {
        // the row's FP32 squared norm as three BF16 pieces h1 + h2 + h3 (each
        // the rounded remainder of the previous: together within 2^-24 of it)
        const __nv_bfloat16 h1 = __float2bfloat16_rn(n);
        const float r1 = n - __bfloat162float(h1);
        const __nv_bfloat16 h2 = __float2bfloat16_rn(r1);
        const __nv_bfloat16 h3 = __float2bfloat16_rn(r1 - __bfloat162float(h2));
        bext[r * 16 + lane] = lane == 0 ? h1 : lane == 1 ? h2 : lane == 2 ? h3 : __float2bfloat16_rn(0.f);
    }
    if (!__all_sync(0xffffffffu, finite) && lane == 0) raise_status(status, DEV_NONFINITE);
    if (lane == 0 && nrm) {
        nrm[r] = n;
        const float a = sqrtf(n), e = sqrtf(res), l = sqrtf(l2);
        stats[r] = make_float4(a, e, l, 0.f);
        if (gmax) {  // corpus rows only
            atomicMax(&gmax[0], __float_as_uint(a));
            atomicMax(&gmax[1], __float_as_uint(e));
            atomicMax(&gmax[2], __float_as_uint(l));
        }
    }
}

// FP8 copies: per row the scale s = max|x| / 448 (448 = largest E4M3 value;
// s = 1 for a zero row) and the E4M3 bytes of x / s (round to nearest even),
// zero-padded to Dp bytes; ||x||^2 and max ||x|| as in knn_prep_kernel.
__global__ void __launch_bounds__(256)
knn_prep_fp8_kernel(const float *__restrict__ X, const int32_t *__restrict__ rows, int64_t nrows,
                    int64_t N, int D, int Dp, uint16_t *__restrict__ q8, float *__restrict__ scale,
                    float *__restrict__ nrm, unsigned *__restrict__ gmax, int *status) {
    const int lane = threadIdx.x & 31;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= nrows) return;
    int64_t src = rows ? rows[r] : r;
    if (src < 0 || src >= N) src = 0;  // flagged by the caller's index check
    const float *x = X + src * D;
    float m = 0.f, n = 0.f;
    bool finite = true;
    for (int d = lane; d < D; d += 32) {
        const float v = x[d];
        finite &= isfinite(v);
        m = fmaxf(m, fabsf(v));
        n = fmaf(v, v, n);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    n = warp_sum(n);
    if (!__all_sync(0xffffffffu, finite) && lane == 0) raise_status(status, DEV_NONFINITE);
    const float sc = m > 0.f ? __fdiv_rn(m, 448.f) : 1.f;
    uint16_t *out = q8 + r * (Dp >> 1);
    for (int d = 2 * lane; d < Dp; d += 64) {
        const float v0 = d < D ? x[d] : 0.f, v1 = d + 1 < D ? x[d + 1] : 0.f;
        out[d >> 1] = cvt_e4m3x2(__fdiv_rn(v1, sc), __fdiv_rn(v0, sc));
    }
    if (lane == 0) {
        scale[r] = sc;
        if (nrm) nrm[r] = n;
        if (gmax) atomicMax(&gmax[0], __float_as_uint(sqrtf(n)));
    }
}

// ---------------------------------------------------------------------------
// the fused contraction + filter kernel
// ---------------------------------------------------------------------------
// Bound on |estimated - true| key (= squared distance - ||x_i||^2) for query
// row statistics st = (||x||, residual norm of its BF16 copy, norm of its low
// part) against any corpus point (gmax: the corpus maxima of the same): the
// terms the BF16 copies drop (Cauchy-Schwarz on the residual norms), the FP32
// accumulation of the products, and the FP32 norms.
__device__ __forceinline__ float key_error_bound(float4 st, const unsigned *gmax, float acc_coef,
                                                 float sq_coef) {
    const float amax = __uint_as_float(gmax[0]);
    const float rmax = __uint_as_float(gmax[1]);
    const float lmax = __uint_as_float(gmax[2]);
    const float a = st.x, r = st.y, l = st.z;
    const float drop = l * lmax + r * amax + a * rmax;
    return 2.f * drop + acc_coef * a * amax + (4e-6f + sq_coef) * amax * amax + 4e-6f * a * a;
}

// The same bound over the corpus points of norm at most amax_cap only (a
// point farther in norm than sqrt(d) from the query is farther than sqrt(d)
// in distance). Their residuals are capped by the BF16 rounding bound:
// ||x - hi|| <= 2^-9 ||x|| and ||lo|| <= 2^-8 ||x|| (round to nearest, 8
// significand bits), plus a tiny absolute term for subnormal values.
__device__ __forceinline__ float key_error_bound_capped(float4 st, const unsigned *gmax, float acc_coef,
                                                        float sq_coef, float amax_cap) {
    const float amax = fminf(__uint_as_float(gmax[0]), amax_cap);
    const float rmax = fminf(__uint_as_float(gmax[1]), 0x1p-9f * amax + 1e-30f);
    const float lmax = fminf(__uint_as_float(gmax[2]), 0x1p-8f * amax + 1e-30f);
    const float a = st.x, r = st.y, l = st.z;
    const float drop = l * lmax + r * amax + a * rmax;
    return 2.f * drop + acc_coef * a * amax + (4e-6f + sq_coef) * amax * amax + 4e-6f * a * a;
}

// Fire-and-forget request of the 128-byte line holding p into L2.
__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<uint64_t>(p)));
}

// First column of the ti-th column tile of a work unit.
__device__ __forceinline__ int64_t unit_tile_col(int64_t c0, int64_t ti) { return c0 + ti * TC_BN; }

// With one split the CTAs walk the corpus together: a unit's stream starts at
// s0, the tile the CTAs have reached on average (the global count of issued
// tiles over the grid, modulo the unit's ntl tiles) and wraps around, so that
// units that start at different times still read the same tiles at the same
// time, which L2 then holds for all of them. With the columns in the order of
// knn_order.cu, row tile rt first streams its groups' pn column tiles from ps,
// then the others from s0 (moved past them if it falls among them). Any order
// gives the same result; only the filter's work and the DRAM traffic change.
// ps, pn: the unit's first group tile and group tile count (0, 0 without the order).
__device__ __forceinline__ int64_t tile_col(int64_t ps, int64_t pn, int64_t s0, int64_t c0, int64_t ntl,
                                            int64_t ti) {
    if (pn == 0 && s0 == 0) return unit_tile_col(c0, ti);
    if (ti < pn) return c0 + (ps + ti) * TC_BN;
    const int64_t j = ti - pn;
    int64_t st = s0;
    if (st >= ps && st < ps + pn) st = ps + pn == ntl ? 0 : ps + pn;
    const int64_t e0 = ps - st >= 0 ? ps - st : ps - st + ntl;  // the groups' tiles, counted from st
    int64_t t = st + (j < e0 ? j : j + pn);
    if (t >= ntl) t -= ntl;
    return c0 + t * TC_BN;
}

template <int PASSES>
__global__ void __launch_bounds__(TcCfg<PASSES>::THREADS, 1) knn_tc_kernel(const __grid_constant__ TcParams p) {
    using C = TcCfg<PASSES>;
    extern __shared__ __align__(16) unsigned char tc_raw[];
    const uint32_t pad = (1024u - (smem_u32(tc_raw) & 1023u)) & 1023u;
    TcSmem<PASSES> &s = *reinterpret_cast<TcSmem<PASSES> *>(tc_raw + pad);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // three passes unless every low half is zero; then single-pass stages
    const bool lo_on = PASSES == 3 && !(p.lo_max && *p.lo_max == 0u);
    const int nst = PASSES == 3 && !lo_on ? C::MAX_STAGES : C::STAGES;
    const int sbytes = PASSES == 3 && !lo_on ? C::STAGE_BYTES / 2 : C::STAGE_BYTES;

    if (threadIdx.x == 0) {
        for (int i = 0; i < C::MAX_STAGES; ++i) {
            mbar_init(&s.full[i], 1);
            mbar_init(&s.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&s.acc_full[i], 1);
            mbar_init(&s.acc_empty[i], 32 * C::NEPI);
        }
        mbar_init(&s.drain, 1);
        mbar_init(&s.ext_bar, 1);
        for (int i = 0; i < 4; ++i) mbar_init(&s.unit_bar[i], 1);
        s.abort_flag = 0;
        s.zero = 0;
        fence_mbar_init();
    }
    if (C::HALVES > 1)
        for (int i = threadIdx.x; i < C::HALVES * TC_BM; i += blockDim.x)
            (&s.tau_sh[0][0])[i] = ~0ull;  // tagged with no unit
    if (threadIdx.x == 32) {
        tma_prefetch_desc(&p.tm_a_hi);
        tma_prefetch_desc(&p.tm_b_hi);
        if (PASSES == 3) {
            tma_prefetch_desc(&p.tm_a_lo);
            tma_prefetch_desc(&p.tm_b_lo);
        }
        if (C::FOLD) {
            tma_prefetch_desc(&p.tm_a_ext);
            tma_prefetch_desc(&p.tm_b_ext);
        }
    }
    __syncthreads();
    if (warp == 1) {
        tmem_alloc(&s.tmem_base, 512);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = s.tmem_base;
    const int n_units = p.row_tiles * p.splits;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            uint32_t armed_phase[C::MAX_STAGES];
            bool armed[C::MAX_STAGES];
            for (int i = 0; i < C::MAX_STAGES; ++i) armed[i] = false;
            if (C::FOLD) {  // the constant query slice, once
                mbar_arrive_expect_tx(&s.ext_bar, C::EXT_A_BYTES);
                tma_load_2d(s.a_ext, &p.tm_a_ext, 0, 0, &s.ext_bar);
            }
            int un = 0;  // units begun by this CTA
            for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++un) {
                const int rt = u % p.row_tiles, sp = u / p.row_tiles;
                const int64_t c0 = (int64_t)sp * p.cols_per_split;
                const int64_t c1 = min(p.N, c0 + p.cols_per_split);
                const int64_t ntl = (c1 - c0 + TC_BN - 1) / TC_BN;
                int64_t s0 = 0;
                const int64_t ps = p.pro ? p.pro[2 * rt] : 0, pn = p.pro ? p.pro[2 * rt + 1] : 0;
                if (p.clock) {
                    s0 = (int64_t)((*(volatile unsigned long long *)p.clock / gridDim.x) % (unsigned long long)ntl);
                    s.unit_start[un & 3] = (uint32_t)s0;
                    mbar_arrive(&s.unit_bar[un & 3]);
                }
                for (int64_t ti = 0; ti < ntl && ok; ++ti) {
                    const int64_t ct = tile_col(ps, pn, s0, c0, ntl, ti);
                    for (int kb = 0; kb < p.KB; ++kb) {
                        if (!mbar_wait(&s.empty[stage], phase ^ 1u, &s.abort_flag, p.wait_ns)) {
                            ok = false;
                            break;
                        }
                        unsigned char *st = &s.stage[0][0] + stage * sbytes;
                        // the tile's norm pieces travel with its last k-block
                        const bool ext = C::FOLD && kb + 1 == p.KB;
                        mbar_arrive_expect_tx(&s.full[stage], sbytes - (ext ? 0 : C::EXT_B_BYTES));
                        armed[stage] = true;
                        armed_phase[stage] = phase;
                        tma_load_2d(st, &p.tm_a_hi, kb * C::KE, rt * TC_BM, &s.full[stage]);
                        tma_load_2d(st + C::A_BYTES, &p.tm_b_hi, kb * C::KE, (int)ct, &s.full[stage]);
                        if (ext) tma_load_2d(st + C::A_BYTES + C::B_BYTES, &p.tm_b_ext, 0, (int)ct, &s.full[stage]);
                        if (p.clock && kb == 0) atomicAdd(p.clock, 1ull);
                        if (PASSES == 3 && lo_on) {
                            tma_load_2d(st + C::A_BYTES + C::B_BYTES, &p.tm_a_lo, kb * TC_BK,
                                        rt * TC_BM, &s.full[stage]);
                            tma_load_2d(st + 2 * C::A_BYTES + C::B_BYTES, &p.tm_b_lo, kb * TC_BK,
                                        (int)ct, &s.full[stage]);
                        }
                        if (++stage == nst) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                }
            }
            if (!ok) {
                s.abort_flag = 1;
                raise_status(p.status, DEV_TIMEOUT);
                // let the copies already issued land before the CTA exits
                for (int i = 0; i < nst; ++i)
                    if (armed[i]) mbar_wait(&s.full[i], armed_phase[i], &s.zero, WAIT_NS);
            }
            if (C::FOLD) mbar_wait(&s.ext_bar, 0, &s.zero, WAIT_NS);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            const uint32_t idesc = PASSES == 8 ? idesc_e4m3_f32(TC_BM, TC_BN) : idesc_bf16_f32(TC_BM, TC_BN);
            int stage = 0, acc = 0;
            uint32_t phase = 0, acc_phase = 0;
            bool ok = true;
            if (C::FOLD && !mbar_wait(&s.ext_bar, 0, &s.abort_flag, p.wait_ns)) ok = false;
            for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
                const int sp = u / p.row_tiles;
                const int64_t c0 = (int64_t)sp * p.cols_per_split;
                const int64_t c1 = min(p.N, c0 + p.cols_per_split);
                const int64_t ntl = (c1 - c0 + TC_BN - 1) / TC_BN;
                for (int64_t ti = 0; ti < ntl && ok; ++ti) {
                    if (!mbar_wait(&s.acc_empty[acc], acc_phase ^ 1u, &s.abort_flag, p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    fence_after_sync();
                    const uint32_t d = tbase + (uint32_t)(acc * TC_BN);
                    for (int kb = 0; kb < p.KB; ++kb) {
                        if (!mbar_wait(&s.full[stage], phase, &s.abort_flag, p.wait_ns)) {
                            ok = false;
                            break;
                        }
                        fence_after_sync();
                        const uint32_t a_hi = smem_u32(&s.stage[0][0] + stage * sbytes);
                        const uint32_t b_hi = a_hi + C::A_BYTES;
                        const uint32_t a_lo = b_hi + C::B_BYTES;
                        const uint32_t b_lo = a_lo + C::A_BYTES;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {  // 32 bytes of each row per MMA
                            if (PASSES == 8)
                                mma_e4m3(d, sw128_kmajor_desc(a_hi + 32 * k), sw128_kmajor_desc(b_hi + 32 * k),
                                         idesc, (kb | k) != 0);
                            else
                                mma_bf16(d, sw128_kmajor_desc(a_hi + 32 * k), sw128_kmajor_desc(b_hi + 32 * k),
                                         idesc, (kb | k) != 0);
                            if (PASSES == 3 && lo_on) {
                                mma_bf16(d, sw128_kmajor_desc(a_hi + 32 * k),
                                         sw128_kmajor_desc(b_lo + 32 * k), idesc, 1u);
                                mma_bf16(d, sw128_kmajor_desc(a_lo + 32 * k),
                                         sw128_kmajor_desc(b_hi + 32 * k), idesc, 1u);
                            }
                        }
                        if (C::FOLD && kb + 1 == p.KB)  // the norms: -1/2 (h1 + h2 + h3) per column
                            mma_bf16(d, sw32_kmajor_desc(smem_u32(s.a_ext)), sw32_kmajor_desc(b_hi + C::B_BYTES),
                                     idesc, 1u);
                        mma_commit(&s.empty[stage]);
                        if (++stage == nst) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    if (!ok) break;
                    mma_commit(&s.acc_full[acc]);
                    if (++acc == 2) {
                        acc = 0;
                        acc_phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                s.abort_flag = 1;
                raise_status(p.status, DEV_TIMEOUT);
            }
            // all MMAs of this CTA complete before TMEM is released
            mma_commit(&s.drain);
            mbar_wait(&s.drain, 0, &s.zero, WAIT_NS);
        }
    } else {
        // ---------------- epilogue: keys, filter, per-row candidate buffers ----------------
        // Epilogue warp e reads TMEM lane quadrant (warp % 4); with two warps
        // per quadrant, warp e filters the columns [half * CW, half * CW + CW)
        // of every tile. Each thread owns one (query row, column split, half)
        // stream with its own buffer. The two halves of a row share their
        // bounds: each half bounds the kh-th smallest key it has seen (kh =
        // ksel / 2, rounded up), so the larger of the two halves' bounds has
        // at least ksel keys of the row below it.
        const int e = warp - 2;
        const int quarter = warp & 3;
        const int half = e >> 2;
        constexpr int CW = TC_BN / C::HALVES;  // columns of each tile filtered by this thread
        constexpr int NCH = CW / 32;           // 32-column TMEM loads per tile
        const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
        uint32_t *hist = s.sel_hist[e];
        const int subs = p.splits * C::HALVES;  // candidate buffers per query row
        int acc = 0;
        uint32_t acc_phase = 0;
        bool ok = true;
        int un = 0;  // units begun by this CTA
        for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++un) {
            const int rt = u % p.row_tiles, sp = u / p.row_tiles;
            const int64_t c0 = (int64_t)sp * p.cols_per_split;
            const int64_t c1 = min(p.N, c0 + p.cols_per_split);
            const int64_t ntl_u = (c1 - c0 + TC_BN - 1) / TC_BN;
            int64_t s0 = 0;  // where the producer started this unit's stream
            const int64_t ps = p.pro ? p.pro[2 * rt] : 0, pn = p.pro ? p.pro[2 * rt + 1] : 0;
            if (p.clock) {
                ok = mbar_wait(&s.unit_bar[un & 3], (uint32_t)((un >> 2) & 1), &s.abort_flag, p.wait_ns);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) {
                    if (lane == 0) {
                        s.abort_flag = 1;
                        raise_status(p.status, DEV_TIMEOUT);
                    }
                    break;
                }
                s0 = s.unit_start[un & 3];
            }
            const int64_t row = (int64_t)rt * TC_BM + quarter * 32 + lane;
            const bool cross = p.qnrm != nullptr;  // queries from another array than the corpus
            const int qraw = row < p.Q ? (cross ? (int)row : (p.qlist ? p.qlist[row] : (int)row)) : -1;
            const bool qv = qraw >= 0 && (cross || qraw < p.N);  // listed rows out of range are flagged by the caller
            const int qid = qv ? qraw : -1;
            Cand *buf = qv ? p.cand + ((size_t)row * subs + (size_t)sp * C::HALVES + half) * p.cap : nullptr;
            float tau = qv ? INFINITY : -INFINITY;
            float th = INFINITY;  // bound of this half's kh-th smallest key
            const int kh = C::HALVES > 1 ? (p.ksel + 1) / 2 : p.ksel;
            int cnt = 0, since = 0, rovf = 0;
            // radius mode: a fixed threshold, the row's squared radius as a key
            // widened by twice the key error bound, so that no point inside the
            // radius is filtered out; no top-k bookkeeping
            const bool rmode = p.radius != nullptr;
            // the thread's distance grid: NBUCKET buckets, 32 per octave of d^2,
            // below an anchor; first anchored at t0 = (||x|| + max||y||)^2 >= d
            const float nx = qv ? (cross ? p.qnrm[row] : p.nrm[qid]) : 0.f;
            const float ai = sqrtf(nx), amax = __uint_as_float(p.gmax[0]);
            const float t0 = (ai + amax) * (ai + amax) * 1.0001f + 1e-30f;
            int top = dbucket(t0);
            // With column splits, every split of a row also counts its buffered
            // distances in one histogram per row in global memory, on a fixed
            // grid below t0 (8 buckets per octave): the splits cover disjoint
            // columns and the counts only grow, so the bucket where the summed
            // count reaches ksel bounds the row's ksel-th distance for all of them.
            unsigned *gh = (p.splits > 1 && qv) ? p.row_hist + (size_t)row * GH_BUCKETS : nullptr;
            const int gbase = (int)(__float_as_uint(t0) >> GH_SHIFT) - (GH_BUCKETS - 1);
            auto global_tau = [&]() {
                int cum = 0, b = 0;
                for (; b < GH_BUCKETS; b += 4) {
                    const uint4 h4 = __ldcg(reinterpret_cast<const uint4 *>(gh + b));
                    if (cum + (int)(h4.x + h4.y + h4.z + h4.w) >= p.ksel) {
                        if ((cum += h4.x) >= p.ksel) break;
                        ++b;
                        if ((cum += h4.y) >= p.ksel) break;
                        ++b;
                        if ((cum += h4.z) >= p.ksel) break;
                        ++b;
                        break;
                    }
                    cum += h4.x + h4.y + h4.z + h4.w;
                }
                if (b < GH_BUCKETS)
                    tau = fminf(tau, __uint_as_float((uint32_t)(gbase + b + 1) << GH_SHIFT) - nx);
            };
            if (gh) global_tau();
            if ((rmode || (p.hint && PASSES != 8)) && qv) {  // FP8 keys carry no error bound
                // the radius (or the hint, an upper bound of the k-th squared
                // distance) as a key threshold, widened by twice the key error
                // bound so that no point inside is filtered out
                const float rad = rmode ? p.radius[row] : p.hint[row];
                if (isfinite(rad)) {
                    // the points that must pass lie within sqrt(rad) of the
                    // query, so their norms are at most ||x|| + sqrt(rad)
                    const float4 qs = cross ? p.qst[row] : p.st[qid];
                    const float widen =
                        2.f * key_error_bound_capped(qs, p.gmax, p.acc_coef, p.sq_coef,
                                                     qs.x + sqrtf(fmaxf(rad, 0.f)) * (1.f + 1e-6f) + 1e-30f) +
                        1e-6f * (fabsf(rad) + nx);
                    tau = fminf(tau, rad - nx + widen);
                    // the distance grid then only needs to reach the bound
                    const int ht = dbucket((rad + widen) * 1.0001f) + 1;
                    if (ht < top) top = ht;
                }
            }
            bool rebased = rmode || (p.hint && PASSES != 8);
            // largest and smallest buffered keys, for the first re-anchoring of the grid
            float kmx = -INFINITY, kmn = INFINITY;
            uint32_t *dh = &s.dhist[e][0][lane];
            for (int bw = 0; bw < NBUCKET / 2; ++bw) dh[bw * 32] = 0;
            // recount the buffered distances on the grid below `top`
            auto recount = [&]() {
                for (int bw = 0; bw < NBUCKET / 2; ++bw) dh[bw * 32] = 0;
                for (int i = 0; i < cnt; ++i) {
                    int bk = dbucket(nx + buf[i].key) - (top - (NBUCKET - 1));
                    if (bk < NBUCKET) {
                        bk = max(bk, 0);
                        dh[(bk >> 1) * 32] += 1u << ((bk & 1) * 16);
                    }
                }
            };
            // corpus norms of the first tile of the unit, then one tile ahead
            // (lane l holds columns l, l + 32, ... of this thread's part)
            float nyn[NCH], msn[NCH];
#pragma unroll
            for (int q = 0; q < NCH; ++q) {
                const int64_t cc = tile_col(ps, pn, s0, c0, ntl_u, 0) + half * CW + q * 32 + lane;
                nyn[q] = !C::FOLD && cc < c1 ? p.nrm[cc] : INFINITY;
                if (PASSES == 8) msn[q] = cc < c1 ? -2.f * p.scale[cc] : 0.f;
            }
            // FP8: x_i . x_j ~ s_i s_j (q_i . q_j); the row's scale, the
            // columns' -2 s_j beside their norms
            const float si = PASSES == 8 && qv ? (p.qscale ? p.qscale[row] : p.scale[qid]) : 1.f;
            // the partner half may still be on an earlier unit: its bound is
            // taken only when its tag is this unit
            volatile unsigned long long *tau_mine =
                &s.tau_sh[C::HALVES > 1 ? half : 0][C::HALVES > 1 ? quarter * 32 + lane : 0];
            volatile unsigned long long *tau_peer =
                &s.tau_sh[C::HALVES > 1 ? half ^ 1 : 0][C::HALVES > 1 ? quarter * 32 + lane : 0];
            auto share_tau = [&]() {
                if (C::HALVES > 1) *tau_mine = ((unsigned long long)u << 32) | __float_as_uint(th);
            };
            share_tau();
            const int64_t ntl = (c1 - c0 + TC_BN - 1) / TC_BN;
            for (int64_t ti = 0; ti < ntl; ++ti) {
                const int64_t ct = tile_col(ps, pn, s0, c0, ntl_u, ti);
                float nyc[NCH], msc[NCH];
#pragma unroll
                for (int q = 0; q < NCH; ++q) {
                    nyc[q] = nyn[q];
                    msc[q] = msn[q];
                }
                if (!C::FOLD && ti + 1 < ntl) {
                    const int64_t cn = tile_col(ps, pn, s0, c0, ntl_u, ti + 1);
#pragma unroll
                    for (int q = 0; q < NCH; ++q) {
                        const int64_t cc = cn + half * CW + q * 32 + lane;
                        nyn[q] = cc < c1 ? p.nrm[cc] : INFINITY;
                        if (PASSES == 8) msn[q] = cc < c1 ? -2.f * p.scale[cc] : 0.f;
                    }
                }
                ok = mbar_wait(&s.acc_full[acc], acc_phase, &s.abort_flag, p.wait_ns);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) {
                    if (lane == 0) {
                        s.abort_flag = 1;
                        raise_status(p.status, DEV_TIMEOUT);
                    }
                    break;
                }
                fence_after_sync();
                const uint32_t taddr = tbase + lane_base + (uint32_t)(acc * TC_BN + half * CW);
                const int colb0 = (int)ct + half * CW;  // first column of this thread's part
                // the query's own column, if in this part (none for another array's queries)
                const int self_off = cross ? INT_MIN / 2 : qid - colb0;
                // filter threshold: finite, so that a padded column (key +inf)
                // never passes even while tau is +inf
                const float tf = fminf(tau, FLT_MAX);
                const float2 ntau = make_float2(-tf, -tf);
                const float2 m2 = make_float2(-2.f, -2.f);
                const float2 si2 = make_float2(si, si);
                // two register sets: the next chunk's load is in flight while
                // this one's keys are filtered
                uint32_t ra[32], rb[32];
                tmem_ld32(taddr, ra);
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    uint32_t(&r)[32] = (c & 1) ? rb : ra;
                    uint32_t(&rn)[32] = (c & 1) ? ra : rb;
                    // norms (and FP8 scales) of the chunk's columns, double-buffered:
                    // the buffer written here was last read two chunks ago, before
                    // the previous chunk's __syncwarp
                    float *nyw = s.ny[e][c & 1];
                    float *msw = s.ms[PASSES == 8 ? e : 0][c & 1];
                    if (!C::FOLD) nyw[lane] = nyc[c];
                    if (PASSES == 8) msw[lane] = msc[c];
                    tmem_ld_wait(r);
                    if (c + 1 < NCH) tmem_ld32(taddr + (uint32_t)((c + 1) * 32), rn);
                    __syncwarp();
                    // keys two at a time (packed FP32), each key's survivor bit
                    // the sign of key - tau (exact: a difference of two floats
                    // is negative exactly when the first is smaller). With the
                    // norms folded in, key - tau is one packed FMA of the
                    // accumulator (-2 acc - tau, -2 acc exact) and a survivor's
                    // key is -2 times its accumulator value.
                    float kk[32];
                    uint32_t mask = 0;
                    const float4 *ny4 = reinterpret_cast<const float4 *>(nyw);
                    const float4 *ms4 = reinterpret_cast<const float4 *>(msw);
                    float dd[32];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        float2 a01 = make_float2(__uint_as_float(r[4 * q + 0]), __uint_as_float(r[4 * q + 1]));
                        float2 a23 = make_float2(__uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
                        if (C::FOLD) {
                            const float2 d01 = __ffma2_rn(m2, a01, ntau), d23 = __ffma2_rn(m2, a23, ntau);
                            kk[4 * q + 0] = a01.x;
                            kk[4 * q + 1] = a01.y;
                            kk[4 * q + 2] = a23.x;
                            kk[4 * q + 3] = a23.y;
                            dd[4 * q + 0] = d01.x;
                            dd[4 * q + 1] = d01.y;
                            dd[4 * q + 2] = d23.x;
                            dd[4 * q + 3] = d23.y;
                            continue;
                        }
                        const float4 n4 = ny4[q];
                        float2 k01, k23;
                        if (PASSES == 8) {
                            const float4 g4 = ms4[q];
                            k01 = __ffma2_rn(__fmul2_rn(a01, si2), make_float2(g4.x, g4.y), make_float2(n4.x, n4.y));
                            k23 = __ffma2_rn(__fmul2_rn(a23, si2), make_float2(g4.z, g4.w), make_float2(n4.z, n4.w));
                        } else {
                            k01 = __ffma2_rn(m2, a01, make_float2(n4.x, n4.y));
                            k23 = __ffma2_rn(m2, a23, make_float2(n4.z, n4.w));
                        }
                        const float2 d01 = __fadd2_rn(k01, ntau), d23 = __fadd2_rn(k23, ntau);
                        kk[4 * q + 0] = k01.x;
                        kk[4 * q + 1] = k01.y;
                        kk[4 * q + 2] = k23.x;
                        kk[4 * q + 3] = k23.y;
                        dd[4 * q + 0] = d01.x;
                        dd[4 * q + 1] = d01.y;
                        dd[4 * q + 2] = d23.x;
                        dd[4 * q + 3] = d23.y;
                    }
                    // four independent shift chains of eight keys (a single chain
                    // of 32 dependent shifts would be the filter's critical path)
                    uint32_t mq[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                    for (int j = 7; j >= 0; --j)
#pragma unroll
                        for (int g = 0; g < 4; ++g) mq[g] = sign_into_mask(dd[8 * g + j], mq[g]);  // key 8g+j -> bit j
                    mask = mq[0] | (mq[1] << 8) | (mq[2] << 16) | (mq[3] << 24);
                    const int so = self_off - c * 32;
                    if (so >= 0 && so < 32) mask &= ~(1u << so);
                    if (C::FOLD) {  // columns past the corpus (their accumulators read 0)
                        const int64_t vc = c1 - (int64_t)(colb0 + c * 32);
                        if (vc < 32) mask &= vc <= 0 ? 0u : (1u << vc) - 1u;
                    }
                    if (__any_sync(0xffffffffu, mask != 0)) {
                        // walk this row's survivors one per step (a chunk rarely
                        // holds more than one or two of a row's): the warp takes
                        // as many steps as the largest count of any lane, not
                        // the union of survivor positions, and every step is the
                        // same straight-line code for all lanes (a lane with no
                        // survivor left adds nothing), so the walk carries no
                        // divergent branch. A survivor's key is picked from the
                        // 32 key registers by a tree of selects on the bits of
                        // its position (no round trip through shared memory,
                        // whose pipe the MMA operand reads and the copies keep
                        // busy), appended (key, column) to the thread's buffer
                        // and counted in its bucket by a fire-and-forget shared add.
                        const int colb = colb0 + c * 32;
                        since += __popc(mask);
                        const int steps = (int)__reduce_max_sync(0xffffffffu, (unsigned)__popc(mask));
                        for (int st = 0; st < steps; ++st) {
                            const bool has = mask != 0;
                            const int j0 = (__ffs(mask) - 1) & 31;
                            mask &= mask - 1;
                            float t16[16], t8[8], t4[4], t2[2];
#pragma unroll
                            for (int i = 0; i < 16; ++i) t16[i] = (j0 & 1) ? kk[2 * i + 1] : kk[2 * i];
#pragma unroll
                            for (int i = 0; i < 8; ++i) t8[i] = (j0 & 2) ? t16[2 * i + 1] : t16[2 * i];
#pragma unroll
                            for (int i = 0; i < 4; ++i) t4[i] = (j0 & 4) ? t8[2 * i + 1] : t8[2 * i];
#pragma unroll
                            for (int i = 0; i < 2; ++i) t2[i] = (j0 & 8) ? t4[2 * i + 1] : t4[2 * i];
                            const float key = C::FOLD ? -2.f * ((j0 & 16) ? t2[1] : t2[0]) : ((j0 & 16) ? t2[1] : t2[0]);
                            const int col = colb + j0;
                            if (rmode) {  // no compaction: a full buffer sends the row to the fallback
                                if (has) {
                                    if (cnt < p.cap)
                                        buf[cnt++] = Cand{key, col};
                                    else
                                        rovf = 1;
                                }
                                continue;
                            }
                            if (has) buf[cnt] = Cand{key, col};
                            cnt += has;
                            const float dd2 = nx + key;
                            kmx = has ? fmaxf(kmx, key) : kmx;
                            kmn = has ? fminf(kmn, key) : kmn;
                            const int bk = dbucket(dd2) - (top - (NBUCKET - 1));
                            // distances above the grid are not counted
                            const int bc = min(max(bk, 0), NBUCKET - 1);
                            red_add_shared(dh + (bc >> 1) * 32,
                                           has && bk < NBUCKET ? 1u << ((bc & 1) * 16) : 0u);
                            if (gh && has) {
                                const int gb = (int)(__float_as_uint(fmaxf(dd2, 1e-30f)) >> GH_SHIFT) - gbase;
                                atomicAdd(gh + min(max(gb, 0), GH_BUCKETS - 1), 1u);
                            }
                        }
                    }
                }
                fence_before_sync();
                __syncwarp();
                mbar_arrive(&s.acc_empty[acc]);
                if (++acc == 2) {
                    acc = 0;
                    acc_phase ^= 1u;
                }
                if (rmode) continue;  // the threshold is fixed
                // Once kh keys are buffered, the largest of them bounds the
                // kh-th (and, with ksel buffered, the ksel-th) smallest, and
                // the grid is re-anchored and recounted: the first anchor
                // bounds the largest distance any point could have, which can
                // lie octaves above the neighbourhood. With one buffer per row
                // (kh = ksel) the new grid ends at twice the smallest buffered
                // distance, kept within [dmx / 8, dmx] (dmx the largest): on
                // spread-out data the final ksel-th distance lies far below
                // the largest of the first distances, near their smallest.
                // A half's ksel-th lies above its first kh keys, and its grid
                // ends at the largest. Any anchor gives a valid bound
                // (distances above the grid are not counted); one too high
                // leaves the ksel-th in the lowest bucket, which also counts
                // every distance below the grid, until the buffer fills.
                if (!rebased && cnt >= kh) {
                    rebased = true;
                    th = fminf(th, kmx);
                    if (cnt >= p.ksel) tau = fminf(tau, kmx);
                    const float dmx = nx + kmx, dmn = nx + kmn;
                    const float anchor = C::HALVES > 1 ? dmx : fminf(dmx, fmaxf(2.f * dmn, 0.125f * dmx));
                    const int nt = dbucket(anchor * 1.0001f) + 1;
                    if (nt < top) {
                        top = nt;
                        recount();
                        since = 32;
                    }
                }
                // lower tau to the upper edge of the bucket holding the ksel-th
                // distance, th to that of the bucket holding the kh-th; the
                // warp updates together once any lane has 32 new survivors
                if (__any_sync(0xffffffffu, since >= 32 && cnt >= kh) && since > 0 && cnt >= kh) {
                    uint32_t hw[NBUCKET / 2];
#pragma unroll
                    for (int bw = 0; bw < NBUCKET / 2; ++bw) hw[bw] = dh[bw * 32];
                    int cum = 0, bk = NBUCKET, bh = NBUCKET;
#pragma unroll
                    for (int b2 = 0; b2 < NBUCKET; ++b2) {
                        cum += (int)((hw[b2 >> 1] >> ((b2 & 1) * 16)) & 0xffffu);
                        if (bh == NBUCKET && cum >= kh) bh = b2;
                        if (bk == NBUCKET && cum >= p.ksel) bk = b2;
                    }
                    if (bk < NBUCKET) tau = fminf(tau, bucket_top(top - (NBUCKET - 1) + bk) - nx);
                    if (bh < NBUCKET) th = fminf(th, bucket_top(top - (NBUCKET - 1) + bh) - nx);
                    since = 0;
                    // The lowest bucket also counts every distance below the
                    // grid; when it holds the ksel-th, that distance may lie
                    // far lower. The grid then slides down by its own span:
                    // the old lowest bucket becomes the new highest, with its
                    // whole count (those distances lie at or below its top, so
                    // the count never exceeds the true one at any edge and the
                    // bounds stay valid), and later survivors are counted on
                    // the finer, lower grid. No buffered entry is reread.
                    // The grid never slides below the bucket of the smallest
                    // distance the buckets tell apart (dbucket(0)).
                    if (bk == 0 && top - 2 * (NBUCKET - 1) >= dbucket(0.f)) {
                        const uint32_t c0 = hw[0] & 0xffffu;
                        for (int bw = 0; bw < NBUCKET / 2; ++bw) dh[bw * 32] = 0;
                        dh[(NBUCKET / 2 - 1) * 32] = c0 << 16;
                        top -= NBUCKET - 1;
                    }
                }
                if (gh) global_tau();
                if (C::HALVES > 1) {  // with the other half of the row: ksel keys below the larger bound
                    share_tau();
                    const unsigned long long pv = *tau_peer;
                    if ((int)(pv >> 32) == u) tau = fminf(tau, fmaxf(th, __uint_as_float((uint32_t)pv)));
                }
                // a buffer that the next tile could overflow is compacted exactly
                unsigned m = __ballot_sync(0xffffffffu, cnt > p.cap - CW);
                if (m) __syncwarp();
                const unsigned compacted = m;
                while (m) {
                    const int l = __ffs(m) - 1;
                    m &= m - 1;
                    Cand *b = reinterpret_cast<Cand *>(
                        __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(buf), l));
                    const int n = __shfl_sync(0xffffffffu, cnt, l);
                    int n_less = 0;
                    const uint32_t tk = warp_select([&](int i) { return b[i].key; }, n, p.ksel, hist,
                                                    lane, n_less);
                    const int eq_quota = p.ksel - n_less;
                    int wpos = 0, eq_seen = 0;
                    for (int base = 0; base < n; base += 32) {
                        const int i = base + lane;
                        Cand e2{INFINITY, -1};
                        if (i < n) e2 = b[i];
                        const uint32_t uk = float_key(e2.key);
                        const bool lt = i < n && uk < tk;
                        const bool eq = i < n && uk == tk;
                        const unsigned eqm = __ballot_sync(0xffffffffu, eq);
                        const int eq_rank = eq_seen + __popc(eqm & lanemask_lt());
                        const bool keep = lt || (eq && eq_rank < eq_quota);
                        const unsigned km = __ballot_sync(0xffffffffu, keep);
                        if (keep) b[wpos + __popc(km & lanemask_lt())] = e2;
                        wpos += __popc(km);
                        eq_seen += __popc(eqm);
                    }
                    __syncwarp();
                    if (lane == l) {
                        cnt = wpos;
                        tau = fminf(tau, key_of_bits(tk));  // never raised: dropped keys stay above it
                    }
                }
                if ((compacted >> lane) & 1u) {
                    // re-base the buckets below the new tau and recount the kept entries
                    top = dbucket((nx + tau) * 1.0001f) + 1;
                    recount();
                    rebased = true;
                    since = 0;
                }
            }
            if (!ok) break;
            if (qv)
                p.meta[(size_t)row * subs + (size_t)sp * C::HALVES + half] =
                    make_int4(cnt, __float_as_int(tau), rovf, 0);
        }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 1) tmem_dealloc(tbase, 512);
}

// ---------------------------------------------------------------------------
// merge, FP32 rerank and certificate
// ---------------------------------------------------------------------------
struct MergeParams {
    const Cand *cand;
    const int4 *meta;
    int splits, cap;
    int64_t Q, N;
    const int32_t *qlist;
    // ordered rows and columns (knn_order.cu): position -> row; the kernel's
    // rows, norms and candidate columns are positions, the outputs rows
    const int32_t *perm;
    const float *X;
    int D, k, ksel;
    int rc, mst;            // re-rank set and staged keys per row (shared memory)
    const float *nrm;
    const float4 *stats;
    const float *Xq;        // queries from another array (row r = Xq[r]), else nullptr
    const float *qnrm;
    const float4 *qstats;
    const unsigned *gmax;
    float acc_coef;        // (K steps of 16 + 8) * 2^-21
    float sq_coef;         // folded norms: acc_coef / 2, else 0
    int32_t *idx_out;
    float *d2_out;
    int32_t *flag_rows;
    int32_t *flag_count;
};

// Bound on |estimated - true| squared distance for query i and any point j:
// the terms the BF16 copies drop (Cauchy-Schwarz on the residual norms), the
// FP32 accumulation of the products, and the FP32 norms.
__device__ __forceinline__ float row_error_bound(const MergeParams &p, float4 st) {
    return key_error_bound(st, p.gmax, p.acc_coef, p.sq_coef);
}

// CERT (FP32 and BF16 modes): the k nearest, certified exact or sent to the
// brute-force kernel. Otherwise (approximate modes): the SEL = ksel best keys
// re-ranked in FP32 and the k best of them kept, without a certificate.
// p.mst keys are staged per row, p.rc candidates re-ranked at most. Without a
// certificate the staged keys are read once, by the collection of the re-rank
// set, so the re-rank set takes their place (p.rc <= p.mst) and five blocks
// fit on an SM instead of four.
size_t merge_smem_bytes(bool cert, int rc, int mst) {
    return (size_t)MERGE_WARPS * (256 * 4 + (size_t)mst * 8 + (cert ? (size_t)rc * 8 : 0) + TIE_MAX * 12);
}

template <bool CERT>
__global__ void __launch_bounds__(MERGE_WARPS * 32, CERT ? 4 : 5) knn_merge_kernel(MergeParams p) {
    extern __shared__ __align__(16) unsigned char mg_smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t *hist = reinterpret_cast<uint32_t *>(mg_smem) + w * 256;
    const int MST = p.mst, RC = p.rc;
    const int RCS = CERT ? RC : 0;  // the re-rank set's own region (else it is the staging region)
    float *sk = reinterpret_cast<float *>(mg_smem + MERGE_WARPS * 1024) + w * MST;
    int *sj = reinterpret_cast<int *>(mg_smem + MERGE_WARPS * (1024 + MST * 4)) + w * MST;
    float *rdw = CERT ? reinterpret_cast<float *>(mg_smem + MERGE_WARPS * (1024 + MST * 8)) + w * RC : sk;
    int *rjw = CERT ? reinterpret_cast<int *>(mg_smem + MERGE_WARPS * (1024 + MST * 8 + RC * 4)) + w * RC : sj;
    double *dmw = reinterpret_cast<double *>(mg_smem + MERGE_WARPS * (1024 + MST * 8 + RCS * 8)) + w * TIE_MAX;
    int *mpw = reinterpret_cast<int *>(mg_smem + MERGE_WARPS * (1024 + MST * 8 + RCS * 8 + TIE_MAX * 8)) +
               w * TIE_MAX;
    const int sel = CERT ? p.k : p.ksel;  // rank of the key that bounds the re-rank set
    const int64_t row = (int64_t)blockIdx.x * MERGE_WARPS + w;
    if (row >= p.Q) return;
    const bool cross = p.Xq != nullptr;
    const int qid = cross ? (int)row : (p.qlist ? p.qlist[row] : (int)row);
    const int64_t orow = p.perm ? p.perm[row] : row;  // the output row (and the query's row of X)
    const int S = p.splits;
    const Cand *cb = p.cand + (size_t)row * S * p.cap;
    const int4 *mt = p.meta + (size_t)row * S;

    // totals over the splits
    int total = 0, ovf = 0;
    float tau_min = INFINITY;
    for (int u = lane; u < S; u += 32) {
        const int4 m = mt[u];
        total += min(max(m.x, 0), p.cap);
        ovf |= m.z;
        tau_min = fminf(tau_min, __int_as_float(m.y));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        total += __shfl_xor_sync(0xffffffffu, total, o);
        ovf |= __shfl_xor_sync(0xffffffffu, ovf, o);
        tau_min = fminf(tau_min, __shfl_xor_sync(0xffffffffu, tau_min, o));
    }
    bool good = !ovf && total >= sel && qid >= 0 && (cross || qid < p.N);
    int nr = 0;
    if (good) {
        // One pass over the buffers stages every (key, index) at or below
        // tau_min. When at least sel keys lie below tau_min, the sel-th
        // smallest key theta lies among them and is selected there; otherwise
        // the buffers are walked again. Re-rank bands reaching above tau_min
        // are collected from the buffers.
        // the row's buffers requested into L2 at once (the staging pass below
        // walks them one 512-byte step at a time)
        for (int u = 0; u < S; ++u) {
            const int c = min(max(mt[u].x, 0), p.cap);
            const char *bb = reinterpret_cast<const char *>(cb + (size_t)u * p.cap);
            for (int o = lane * 128; o < c * (int)sizeof(Cand); o += 32 * 128) prefetch_l2(bb + o);
        }
        const float E = CERT ? row_error_bound(p, cross ? p.qstats[row] : p.stats[qid]) : 0.f;
        const float slim = tau_min;  // the select needs no key above tau_min
        int ns = 0, nlt = 0;
        for (int u0 = 0; u0 < S; u0 += 32) {
          const int cu = u0 + lane < S ? min(max(mt[u0 + lane].x, 0), p.cap) : 0;  // the counts of 32 splits at once
          for (int j = 0; j < 32 && u0 + j < S; ++j) {
            const int c = __shfl_sync(0xffffffffu, cu, j);
            const Cand *b = cb + (size_t)(u0 + j) * p.cap;
            // two candidates per lane in one 16-byte load; two such loads
            // in flight per step (positions past c are not staged)
            auto load2 = [&](int i, Cand &e0, Cand &e1) {
                e0 = Cand{INFINITY, -1};
                e1 = Cand{INFINITY, -1};
                if (i + 1 < c) {
                    const float4 v = __ldcs(reinterpret_cast<const float4 *>(b + i));
                    e0 = Cand{v.x, __float_as_int(v.y)};
                    e1 = Cand{v.z, __float_as_int(v.w)};
                } else if (i < c) {
                    e0 = b[i];
                }
            };
            auto stage2 = [&](int i, Cand e0, Cand e1) {
                nlt += (e0.key < tau_min) + (e1.key < tau_min);
                const bool t0 = i < c && e0.key <= slim, t1 = i + 1 < c && e1.key <= slim;
                const unsigned m0 = __ballot_sync(0xffffffffu, t0);
                const unsigned m1 = __ballot_sync(0xffffffffu, t1);
                const unsigned lt = lanemask_lt();
                const int pos = ns + __popc(m0 & lt) + __popc(m1 & lt);
                if (t0 && pos < MST) {
                    sk[pos] = e0.key;
                    sj[pos] = e0.idx;
                }
                if (t1 && pos + t0 < MST) {
                    sk[pos + t0] = e1.key;
                    sj[pos + t0] = e1.idx;
                }
                ns += __popc(m0) + __popc(m1);
            };
            for (int base = 0; base < c; base += 128) {
                const int i = base + 2 * lane;
                Cand e0, e1, e2, e3;
                load2(i, e0, e1);
                load2(i + 64, e2, e3);
                stage2(i, e0, e1);
                stage2(i + 64, e2, e3);
            }
          }
        }
        nlt = (int)__reduce_add_sync(0xffffffffu, (unsigned)nlt);
        __syncwarp();
        int n_less = 0;
        const bool staged = nlt >= sel && ns <= MST;
        uint32_t prefix;
        if (staged) {
            prefix = warp_select([&](int i) { return sk[i]; }, ns, sel, hist, lane, n_less);
        } else {
            prefix = warp_select_visit(
                [&](auto fn) {
                    for (int u = 0; u < S; ++u) {
                        const int c = min(max(mt[u].x, 0), p.cap);
                        const Cand *b = cb + (size_t)u * p.cap;
                        for (int base = 0; base < c; base += 32) {
                            const int i = base + lane;
                            fn(i < c, i < c ? b[i].key : 0.f);
                        }
                    }
                },
                sel, hist, lane, n_less);
        }
        const float theta = key_of_bits(prefix);
        // the re-rank set, collected in two bands of keys: (-inf, theta] then
        // (theta, lim]
        auto take_batch = [&](bool take, int idx) {
            const unsigned tm = __ballot_sync(0xffffffffu, take);
            const int pos = nr + __popc(tm & lanemask_lt());
            if (take && pos < RC) rjw[pos] = idx;
            nr += __popc(tm);
        };
        auto collect = [&](float lo, float hi) {  // keys in (lo, hi]
            if (staged && hi <= slim) {  // all staged: every key up to slim was
                for (int base = 0; base < ns; base += 32) {
                    const int i = base + lane;
                    const bool in = i < ns && sk[i] > lo && sk[i] <= hi;
                    const int idx = i < ns ? sj[i] : -1;
                    // without a certificate the set is compacted in place
                    // (position <= i): the batch is read before it is written
                    if (!CERT) __syncwarp();
                    take_batch(in, idx);
                }
            } else {
                for (int u = 0; u < S; ++u) {
                    const int c = min(max(mt[u].x, 0), p.cap);
                    const Cand *b = cb + (size_t)u * p.cap;
                    for (int base = 0; base < c; base += 32) {
                        const int i = base + lane;
                        Cand e{INFINITY, -1};
                        if (i < c) e = b[i];
                        take_batch(i < c && e.key > lo && e.key <= hi, e.idx);
                    }
                }
            }
        };
        // ordered columns: the collected positions mapped to rows of X, four
        // loads in flight per lane (one at a time per batch of the collection
        // would wait on each)
        auto map_rows = [&](int from, int to) {
            if (!p.perm) return;
            for (int t0 = from; t0 < to; t0 += 128) {
                int v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int t = t0 + 32 * q + lane;
                    v[q] = t < to ? p.perm[rjw[t]] : 0;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int t = t0 + 32 * q + lane;
                    if (t < to) rjw[t] = v[q];
                }
            }
            __syncwarp();
        };
        const float *xq = cross ? p.Xq + (int64_t)row * p.D : p.X + (p.perm ? orow : (int64_t)qid) * p.D;
        const bool vec4 = (p.D & 3) == 0 && (reinterpret_cast<uintptr_t>(p.X) & 15) == 0 &&
                          (reinterpret_cast<uintptr_t>(xq) & 15) == 0;
        // exact FP32 distances of rjw[from, to) in the library's one summation
        // order (group8_d2_pair), eight candidates per warp step
        auto rerank = [&](int from, int to) {
            // every candidate row requested into L2 first (rows of at most
            // 1 KB: longer ones gain less than the requests cost)
            for (int t = from + lane; p.D <= 256 && t < to; t += 32) {
                const char *xr = reinterpret_cast<const char *>(p.X + (int64_t)rjw[t] * p.D);
                for (int o = 0; o < p.D * 4; o += 128) prefetch_l2(xr + o);
            }
            const int g = lane >> 3, gl = lane & 7;
            for (int t0 = from; t0 < to; t0 += 8) {
                const int ta = t0 + g, tb = t0 + 4 + g;
                const float *xa = ta < to ? p.X + (int64_t)rjw[ta] * p.D : xq;
                const float *xb = tb < to ? p.X + (int64_t)rjw[tb] * p.D : xq;
                const float2 s2 = group8_d2_pair(xq, xa, xb, p.D, vec4, gl);
                if (gl == 0) {
                    if (ta < to) rdw[ta] = s2.x;
                    if (tb < to) rdw[tb] = s2.y;
                }
            }
        };
        collect(-INFINITY, theta);
        const int nr1 = nr;
        float Ec = E;  // the key error bound the band and the certificate use
        if (nr1 > RC) good = false;
        __syncwarp();
        if (good && CERT) {
            // the candidates at or below theta are sel >= k real points: the
            // largest of their exact distances bounds the k-th nearest one, so
            // only points of norm at most ||x|| + sqrt(that) can be nearer, and
            // the bound is taken over those points only
            map_rows(0, nr1);
            rerank(0, nr1);
            __syncwarp();
            float dk0 = 0.f;
            for (int t = lane; t < nr1; t += 32) dk0 = fmaxf(dk0, rdw[t]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dk0 = fmaxf(dk0, __shfl_xor_sync(0xffffffffu, dk0, o));
            const float4 st = cross ? p.qstats[row] : p.stats[qid];
            Ec = fminf(E, key_error_bound_capped(st, p.gmax, p.acc_coef, p.sq_coef,
                                                  st.x + sqrtf(dk0) * (1.f + 1e-6f) + 1e-30f));
            collect(theta, theta + 2.f * Ec);
            if (nr > RC) good = false;
            __syncwarp();
            if (good) {
                map_rows(nr1, nr);
                rerank(nr1, nr);
            }
        } else if (good) {
            map_rows(0, nr1);
            rerank(0, nr1);
        }
        __syncwarp();
        if (good && nr >= p.k) {
            // only the first k + 1 in (distance, index) order are needed: a
            // set of 129 to 512 is cut to the entries at or below its
            // (k + 1)-th distance first when at most 128 remain
            const int m1 = nr < p.k + 1 ? nr : p.k + 1;
            int nsrt = nr;
            if (nr > 128 && nr <= 512) {
                const int c = warp_smallest_to_front(rdw, rjw, nr, m1, 128, lane);
                if (c >= 0) nsrt = c;
            }
            int ns2 = 32;
            while (ns2 < nsrt) ns2 <<= 1;
            for (int t = nsrt + lane; t < ns2; t += 32) {
                rdw[t] = INFINITY;
                rjw[t] = INT_MAX;
            }
            __syncwarp();
            warp_sort_pow2(rdw, rjw, ns2, lane);
            __syncwarp();
            // near ties among the first k + 1 ordered as the exact distances are
            fp64_near_ties(rdw, rjw, nr, p.k, xq, p.X, p.D, dmw, mpw, lane);
            if (CERT) {
                const float dk = rdw[p.k - 1];
                const float nx = cross ? p.qnrm[row] : p.nrm[qid];
                const float lb = nx + tau_min - Ec;
                // certified: no point outside the buffers can be closer than dk
                good = isinf(tau_min) || dk < lb * (1.f - 1e-6f);
            }
        } else {
            good = false;
        }
    }
    if (good) {
        for (int t = lane; t < p.k; t += 32) {
            p.idx_out[orow * p.k + t] = rjw[t];
            p.d2_out[orow * p.k + t] = rdw[t];
        }
    } else if (lane == 0) {
        p.flag_rows[atomicAdd(p.flag_count, 1)] = (int)orow;
    }
}

// Radius mode (queries from another array): every buffered candidate is
// re-ranked by FP32 direct differences, the ones strictly inside the row's
// squared radius are kept in (d^2, index) order, the first k written and the
// rest of the row padded with (-1, +inf). Rows whose buffers overflowed, or
// that hold more than RCAP candidates, go to the brute-force kernel (then
// radius_filter_kernel applies the same rule).
__global__ void __launch_bounds__(MERGE_WARPS * 32) radius_merge_kernel(MergeParams p, const float *radius) {
    __shared__ float rd_s[MERGE_WARPS][RCAP];
    __shared__ int rj_s[MERGE_WARPS][RCAP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t row = (int64_t)blockIdx.x * MERGE_WARPS + w;
    if (row >= p.Q) return;
    float *rdw = rd_s[w];
    int *rjw = rj_s[w];
    const int S = p.splits;
    const Cand *cb = p.cand + (size_t)row * S * p.cap;
    const int4 *mt = p.meta + (size_t)row * S;
    int total = 0, ovf = 0;
    for (int u = lane; u < S; u += 32) {
        const int4 m = mt[u];
        total += min(max(m.x, 0), p.cap);
        ovf |= m.z;
    }
    total = (int)__reduce_add_sync(0xffffffffu, (unsigned)total);
    ovf = (int)__reduce_or_sync(0xffffffffu, (unsigned)ovf);
    if (ovf || total > RCAP) {
        if (lane == 0) p.flag_rows[atomicAdd(p.flag_count, 1)] = (int)row;
        return;
    }
    int nr = 0;
    for (int u = 0; u < S; ++u) {
        const int c = min(max(mt[u].x, 0), p.cap);
        const Cand *b = cb + (size_t)u * p.cap;
        for (int i = lane; i < c; i += 32) rjw[nr + i] = b[i].idx;
        nr += c;
    }
    __syncwarp();
    const float *xq = p.Xq + (int64_t)row * p.D;
    const bool vec4 = (p.D & 3) == 0 && (reinterpret_cast<uintptr_t>(p.X) & 15) == 0 &&
                      (reinterpret_cast<uintptr_t>(xq) & 15) == 0;
    // the library's one summation order (group8_d2_pair), eight candidates per step
    {
        const int g = lane >> 3, gl = lane & 7;
        for (int t0 = 0; t0 < nr; t0 += 8) {
            const int ta = t0 + g, tb = t0 + 4 + g;
            const float *xa = ta < nr ? p.X + (int64_t)rjw[ta] * p.D : xq;
            const float *xb = tb < nr ? p.X + (int64_t)rjw[tb] * p.D : xq;
            const float2 s2 = group8_d2_pair(xq, xa, xb, p.D, vec4, gl);
            if (gl == 0) {
                if (ta < nr) rdw[ta] = s2.x;
                if (tb < nr) rdw[tb] = s2.y;
            }
        }
    }
    __syncwarp();
    const float rad = radius[row];
    int ns2 = 32;
    while (ns2 < nr) ns2 <<= 1;
    for (int t = lane; t < ns2; t += 32) {
        if (t >= nr || !(rdw[t] < rad)) {
            rdw[t] = INFINITY;
            rjw[t] = INT_MAX;
        }
    }
    __syncwarp();
    warp_bitonic_sort_smem(rdw, rjw, ns2, lane);
    for (int t = lane; t < p.k; t += 32) {
        const bool in = t < ns2 && rjw[t] != INT_MAX;
        p.idx_out[row * p.k + t] = in ? rjw[t] : -1;
        p.d2_out[row * p.k + t] = in ? rdw[t] : INFINITY;
    }
}

// Entries at or beyond the row's squared radius become (-1, +inf); rows are
// sorted, so they form a suffix.
__global__ void radius_filter_kernel(int32_t *idx, float *d2, int64_t rows, int k, const float *radius) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * k) return;
    if (!(d2[e] < radius[e / k])) {
        d2[e] = INFINITY;
        idx[e] = -1;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    return fn;
}

atsne_status make_bf16_map(CUtensorMap *m, const void *base, int64_t rows, int Dp, int box_rows) {
    auto enc = tensor_map_encoder();
    if (!enc) return set_error(ATSNE_ECUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)Dp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)Dp * 2};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
                     es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(ATSNE_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return ATSNE_OK;
}

// Rows of 16 BF16 (32 bytes: the norm slices of the folded one-pass mode),
// box_rows rows per copy in the 32-byte swizzle layout.
atsne_status make_ext_map(CUtensorMap *m, const void *base, int64_t rows, int box_rows) {
    auto enc = tensor_map_encoder();
    if (!enc) return set_error(ATSNE_ECUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {16u, (cuuint64_t)rows};
    cuuint64_t strides[1] = {32u};
    cuuint32_t box[2] = {16u, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
                     es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(ATSNE_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return ATSNE_OK;
}

// The FP32 accumulation term of the key error bound: (K steps of 16 + 8) * 2^-21,
// the folded norms adding one step in the one-pass BF16 mode.
float acc_coef_of(const TcPlan &pl) {
    return (float)((pl.passes * pl.Dp / 16 + (pl.passes == 1 ? 1 : 0) + 8) * (1.0 / (1 << 21)));
}

atsne_status make_u8_map(CUtensorMap *m, const void *base, int64_t rows, int Dp, int box_rows) {
    auto enc = tensor_map_encoder();
    if (!enc) return set_error(ATSNE_ECUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)Dp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)Dp};
    cuuint32_t box[2] = {128u, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), dims, strides, box,
                     es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(ATSNE_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return ATSNE_OK;
}

template <int PASSES>
size_t tc_smem_bytes() {
    return sizeof(TcSmem<PASSES>) + 1024;
}
static_assert(sizeof(TcSmem<1>) + 1024 <= 232448, "tensor kNN shared memory above 227 KB");
static_assert(GH_BUCKETS % 4 == 0, "row histograms are read as uint4");
static_assert(sizeof(TcSmem<3>) + 1024 <= 232448, "tensor kNN shared memory above 227 KB");
static_assert(sizeof(TcSmem<8>) + 1024 <= 232448, "tensor kNN shared memory above 227 KB");

}  // namespace

namespace {
std::atomic<uint64_t> g_wait_ns{WAIT_NS};
}  // namespace

uint64_t pipeline_wait_ns() { return g_wait_ns.load(); }
void set_pipeline_wait_ns(uint64_t ns) { g_wait_ns.store(ns ? ns : WAIT_NS); }

atsne_status radius_filter_launch(int32_t *idx, float *d2, int64_t rows, int k, const float *radius,
                                  cudaStream_t stream) {
    if (rows <= 0) return ATSNE_OK;
    return launch_kernel("radius_filter", radius_filter_kernel, ceil_div(rows * k, 256), 256, 0, stream,
                         idx, d2, rows, k, radius);
}

// Column splits chosen by atsne_tune_knn, per problem shape (process-wide).
namespace {
struct TunedSplit {
    int64_t N, Q;
    int D, k, precision, rerank_k, splits;
};
std::mutex g_tuned_mu;
std::vector<TunedSplit> g_tuned;
}  // namespace

int tuned_splits(int64_t N, int D, int64_t Q, int k, int precision, int rerank_k) {
    std::lock_guard<std::mutex> g(g_tuned_mu);
    for (const TunedSplit &t : g_tuned)
        if (t.N == N && t.Q == Q && t.D == D && t.k == k && t.precision == precision && t.rerank_k == rerank_k)
            return t.splits;
    return 0;
}

void set_tuned_splits(int64_t N, int D, int64_t Q, int k, int precision, int rerank_k, int splits) {
    std::lock_guard<std::mutex> g(g_tuned_mu);
    for (TunedSplit &t : g_tuned)
        if (t.N == N && t.Q == Q && t.D == D && t.k == k && t.precision == precision && t.rerank_k == rerank_k) {
            t.splits = splits;
            return;
        }
    g_tuned.push_back({N, Q, D, k, precision, rerank_k, splits});
}

void clear_tuned_splits() {
    std::lock_guard<std::mutex> g(g_tuned_mu);
    g_tuned.clear();
}

int tc_split_candidates(int64_t N, int D, int64_t Q, int k, int precision, int rerank_k, int *out, int max_out) {
    const int64_t row_tiles = (Q + TC_BM - 1) / TC_BM;
    const int64_t units[] = {0, 152, 304, 608, 1216, 2048, 4096, 8192};
    int n = 0;
    for (int64_t u : units) {
        if (n == max_out) break;
        const int want = u == 0 ? 1 : (int)((u + row_tiles - 1) / row_tiles);
        const int s = tc_plan(N, D, Q, k, precision, rerank_k, want).splits;
        bool dup = false;
        for (int i = 0; i < n; ++i) dup |= out[i] == s;
        if (!dup) out[n++] = s;
    }
    return n;
}

TcPlan tc_plan(int64_t N, int D, int64_t Q, int k, int precision, int rerank_k, int splits) {
    TcPlan pl;
    pl.passes = precision == ATSNE_FP32 ? 3 : precision == ATSNE_FP8_RERANK ? 8 : 1;
    pl.certify = precision != ATSNE_FP8_RERANK && precision != ATSNE_BF16_RERANK_APPROX;
    const int ke = pl.passes == 8 ? 128 : TC_BK;  // elements per 128-byte row
    pl.Dp = ((D + ke - 1) / ke) * ke;
    pl.row_tiles = (int)((Q + TC_BM - 1) / TC_BM);
    const int64_t col_tiles = (N + TC_BN - 1) / TC_BN;
    // (row tile, column split) units: one split per row tile when the row tiles
    // alone give every SM at least two units (a split restarts the streaming
    // top-k, whose k' ln(n / k') survivors dominate the epilogue), else about
    // 2048 units, each at least 4 column tiles long
    if (splits <= 0) splits = tuned_splits(N, D, Q, k, precision, rerank_k);
    int64_t S = splits > 0 ? splits : pl.row_tiles >= 304 ? 1 : (2048 + pl.row_tiles - 1) / pl.row_tiles;
    const int64_t max_s = (col_tiles + 3) / 4;
    if (S > max_s) S = max_s;
    if (S < 1) S = 1;
    const int64_t tiles_per = (col_tiles + S - 1) / S;
    pl.cols_per_split = (int)(tiles_per * TC_BN);
    pl.splits = (int)((N + pl.cols_per_split - 1) / pl.cols_per_split);
    int ks = rerank_k > 0 ? rerank_k : (pl.passes == 3 ? k + 38 : !pl.certify ? 4 * k : 2 * k);
    if (!pl.certify && ks > RCAP_FP8 / 2) ks = RCAP_FP8 / 2;
    if (ks < k) ks = k;
    pl.ksel = ks;
    // A streaming top-ksel over n columns in random order admits about
    // ksel (1 + ln(n / ksel)) keys; the bucketed threshold somewhat more.
    // The buffer holds 2.5x the model so that the exact compaction of a full
    // buffer (a radix select per row) stays rare. With two halves per row
    // (one-pass modes) each half buffers about half of the row's survivors
    // after its first ksel, and holds 1.25x the model.
    pl.halves = pl.passes == 3 ? 1 : 2;
    const int cw = TC_BN / pl.halves;  // columns of a tile one buffer takes
    const double ncol = (double)hmin(N, (int64_t)pl.cols_per_split);
    const double model = ks * (1.0 + log(fmax(1.0, ncol / ks)));
    int64_t cap = (int64_t)ceil((pl.halves == 1 ? 2.5 : 1.25) * model) + cw;
    if (cap < (8 / pl.halves) * ks + cw) cap = (8 / pl.halves) * ks + cw;
    // the epilogue's bucket counts are 16 bits and never exceed the buffer's size
    if (cap > 65504) cap = 65504;
    pl.cap = (int)((cap + 31) / 32 * 32);
    return pl;
}

size_t tc_workspace(Carver &c, int64_t N, int D, int64_t Q, bool list, const TcPlan &pl, TcWs *ws) {
    TcWs w;
    const size_t per = pl.passes == 8 ? (size_t)pl.Dp / 2 : (size_t)pl.Dp;  // 16-bit words per row
    w.hi = c.take<uint16_t>((size_t)N * per);
    w.lo = pl.passes == 3 ? c.take<uint16_t>((size_t)N * per) : nullptr;
    w.qhi = list ? c.take<uint16_t>((size_t)Q * per) : nullptr;
    w.qlo = (list && pl.passes == 3) ? c.take<uint16_t>((size_t)Q * per) : nullptr;
    w.scale = pl.passes == 8 ? c.take<float>((size_t)N) : nullptr;
    w.qscale = (list && pl.passes == 8) ? c.take<float>((size_t)Q) : nullptr;
    w.qnrm = list ? c.take<float>((size_t)Q) : nullptr;  // queries from another array
    w.qstats = list ? c.take<float>((size_t)Q * 4) : nullptr;
    w.nrm = c.take<float>((size_t)N);
    w.stats = c.take<float>((size_t)N * 4);
    w.gmax = c.take<unsigned>(4);
    w.cand = c.take<char>((size_t)Q * pl.splits * pl.halves * pl.cap * sizeof(Cand));
    w.meta = c.take<char>((size_t)Q * pl.splits * pl.halves * sizeof(int4));
    w.row_hist = pl.splits > 1 ? c.take<unsigned>((size_t)Q * GH_BUCKETS) : nullptr;
    w.flag_rows = c.take<int32_t>((size_t)Q);
    w.flag_count = c.take<int32_t>(1);
    w.bext = pl.passes == 1 ? c.take<uint16_t>((size_t)N * 16) : nullptr;
    w.aext = pl.passes == 1 ? c.take<uint16_t>((size_t)TC_BM * 16) : nullptr;
    w.ordered = knn_ordered(N, D, list, pl);
    // the global column clock where many units stream a corpus larger than L2
    // on short rows (longer rows keep the natural start; the contraction, not
    // the copies, sets their pace)
    w.clock = pl.splits == 1 && N >= ORD_MIN_ROWS && D <= ORD_MAX_DIM ? c.take<unsigned long long>(1) : nullptr;
    if (w.ordered) order_workspace(c, N, D, pl, &w.ord);
    if (ws) *ws = w;
    return c.bytes();
}

atsne_status knn_exact_tc(const float *X, int64_t N, int D, const int32_t *qlist, int64_t Q, int k,
                          const TcPlan &pl, const TcWs &w, int32_t *idx_out, float *d2_out,
                          cudaStream_t stream, const float *Xq, const float *radius, const float *hint) {
    int *status = device_status_word();
    cudaError_t e = cudaMemsetAsync(w.gmax, 0, 4 * sizeof(unsigned), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.flag_count, 0, sizeof(int32_t), stream);
    if (e == cudaSuccess && w.clock) e = cudaMemsetAsync(w.clock, 0, sizeof(unsigned long long), stream);
    if (e == cudaSuccess && w.row_hist)
        e = cudaMemsetAsync(w.row_hist, 0, (size_t)Q * GH_BUCKETS * sizeof(unsigned), stream);
    // a unit that a timed-out kernel never finished reads as an empty buffer
    if (e == cudaSuccess)
        e = cudaMemsetAsync(w.meta, 0, (size_t)Q * pl.splits * pl.halves * sizeof(int4), stream);
    if (e != cudaSuccess) return cuda_error(e, "knn_tc memset");
    const bool fp8 = pl.passes == 8;
    const void *a_hi = w.hi, *a_lo = w.lo;
    const bool ordered = w.ordered && !qlist && !Xq;
    if (fp8) {
        if (ordered) ATSNE_TRY(knn_order_launch(X, N, D, pl, TC_BM, TC_BN, w.ord, stream));
        ATSNE_TRY(launch_kernel("knn_prep", knn_prep_fp8_kernel, ceil_div(N * 32, 256), 256, 0, stream, X,
                                ordered ? (const int32_t *)w.ord.perm : (const int32_t *)nullptr, N, N, D,
                                pl.Dp, w.hi, w.scale, w.nrm, w.gmax, status));
        if (Xq) {
            ATSNE_TRY(launch_kernel("knn_prep", knn_prep_fp8_kernel, ceil_div(Q * 32, 256), 256, 0, stream,
                                    Xq, (const int32_t *)nullptr, Q, Q, D, pl.Dp, w.qhi, w.qscale, w.qnrm,
                                    (unsigned *)nullptr, status));
            a_hi = w.qhi;
        } else if (qlist) {
            ATSNE_TRY(launch_kernel("knn_prep", knn_prep_fp8_kernel, ceil_div(Q * 32, 256), 256, 0, stream,
                                    X, qlist, Q, N, D, pl.Dp, w.qhi, w.qscale, (float *)nullptr,
                                    (unsigned *)nullptr, status));
            a_hi = w.qhi;
        }
    } else {
        auto *hi = reinterpret_cast<__nv_bfloat16 *>(w.hi);
        auto *lo = reinterpret_cast<__nv_bfloat16 *>(w.lo);
        // ordered rows and columns: the copies, norms and statistics in the order
        if (ordered) ATSNE_TRY(knn_order_launch(X, N, D, pl, TC_BM, TC_BN, w.ord, stream));
        ATSNE_TRY(launch_kernel("knn_prep", knn_prep_kernel, ceil_div(N * 32, 256), 256, 0, stream, X,
                                ordered ? (const int32_t *)w.ord.perm : (const int32_t *)nullptr, N, N, D,
                                pl.Dp, pl.passes, hi, lo, w.nrm,
                                reinterpret_cast<float4 *>(w.stats), w.gmax,
                                reinterpret_cast<__nv_bfloat16 *>(w.bext),
                                reinterpret_cast<__nv_bfloat16 *>(w.aext), status));
        if (Xq) {
            ATSNE_TRY(launch_kernel("knn_prep", knn_prep_kernel, ceil_div(Q * 32, 256), 256, 0, stream, Xq,
                                    (const int32_t *)nullptr, Q, Q, D, pl.Dp, pl.passes,
                                    reinterpret_cast<__nv_bfloat16 *>(w.qhi),
                                    reinterpret_cast<__nv_bfloat16 *>(w.qlo), w.qnrm,
                                    reinterpret_cast<float4 *>(w.qstats), (unsigned *)nullptr,
                                    (__nv_bfloat16 *)nullptr, (__nv_bfloat16 *)nullptr, status));
            a_hi = w.qhi;
            a_lo = w.qlo;
        } else if (qlist) {
            ATSNE_TRY(launch_kernel("knn_prep", knn_prep_kernel, ceil_div(Q * 32, 256), 256, 0, stream, X,
                                    qlist, Q, N, D, pl.Dp, pl.passes,
                                    reinterpret_cast<__nv_bfloat16 *>(w.qhi),
                                    reinterpret_cast<__nv_bfloat16 *>(w.qlo), (float *)nullptr,
                                    (float4 *)nullptr, (unsigned *)nullptr, (__nv_bfloat16 *)nullptr,
                                    (__nv_bfloat16 *)nullptr, status));
            a_hi = w.qhi;
            a_lo = w.qlo;
        }
    }
    TcParams p;
    memset(&p, 0, sizeof(p));
    if (fp8) {
        ATSNE_TRY(make_u8_map(&p.tm_a_hi, a_hi, (qlist || Xq) ? Q : N, pl.Dp, TC_BM));
        ATSNE_TRY(make_u8_map(&p.tm_b_hi, w.hi, N, pl.Dp, TC_BN));
    } else {
        ATSNE_TRY(make_bf16_map(&p.tm_a_hi, a_hi, (qlist || Xq) ? Q : N, pl.Dp, TC_BM));
        ATSNE_TRY(make_bf16_map(&p.tm_b_hi, w.hi, N, pl.Dp, TC_BN));
    }
    if (pl.passes == 1) {
        ATSNE_TRY(make_ext_map(&p.tm_a_ext, w.aext, TC_BM, TC_BM));
        ATSNE_TRY(make_ext_map(&p.tm_b_ext, w.bext, N, TC_BN));
    } else {
        p.tm_a_ext = p.tm_a_hi;
        p.tm_b_ext = p.tm_b_hi;
    }
    if (pl.passes == 3) {
        ATSNE_TRY(make_bf16_map(&p.tm_a_lo, a_lo, (qlist || Xq) ? Q : N, pl.Dp, TC_BM));
        ATSNE_TRY(make_bf16_map(&p.tm_b_lo, w.lo, N, pl.Dp, TC_BN));
    } else {
        p.tm_a_lo = p.tm_a_hi;
        p.tm_b_lo = p.tm_b_hi;
    }
    p.scale = w.scale;
    p.qscale = (qlist || Xq) ? w.qscale : nullptr;
    p.qnrm = Xq ? w.qnrm : nullptr;
    p.radius = radius;
    p.hint = hint;
    p.pro = ordered ? w.ord.pro : nullptr;
    p.clock = w.clock;
    p.qst = reinterpret_cast<const float4 *>(w.qstats);
    p.st = reinterpret_cast<const float4 *>(w.stats);
    p.acc_coef = acc_coef_of(pl);
    p.sq_coef = pl.passes == 1 ? 0.5f * p.acc_coef : 0.f;
    p.nrm = w.nrm;
    p.gmax = w.gmax;
    // queries that are corpus rows have the corpus' low halves
    p.lo_max = pl.passes == 3 && !Xq ? w.gmax + 2 : nullptr;
    p.qlist = qlist;
    p.Q = Q;
    p.N = N;
    p.KB = pl.Dp / (fp8 ? 128 : TC_BK);
    p.splits = pl.splits;
    p.cols_per_split = pl.cols_per_split;
    p.row_tiles = pl.row_tiles;
    p.ksel = pl.ksel;
    p.cap = pl.cap;
    p.cand = reinterpret_cast<Cand *>(w.cand);
    p.meta = reinterpret_cast<int4 *>(w.meta);
    p.row_hist = w.row_hist;
    p.status = status;
    p.wait_ns = pipeline_wait_ns();
    const int units = pl.row_tiles * pl.splits;
    const int grid = (int)hmin(units, num_sms());
    if (pl.passes == 3) {
        const size_t smem = tc_smem_bytes<3>();
        e = cudaFuncSetAttribute(knn_tc_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "knn_tc attribute");
        ATSNE_TRY(launch_kernel("knn_tc", knn_tc_kernel<3>, grid, TcCfg<3>::THREADS, smem, stream, p));
    } else if (fp8) {
        const size_t smem = tc_smem_bytes<8>();
        e = cudaFuncSetAttribute(knn_tc_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "knn_tc attribute");
        ATSNE_TRY(launch_kernel("knn_tc", knn_tc_kernel<8>, grid, TcCfg<8>::THREADS, smem, stream, p));
    } else {
        const size_t smem = tc_smem_bytes<1>();
        e = cudaFuncSetAttribute(knn_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "knn_tc attribute");
        ATSNE_TRY(launch_kernel("knn_tc", knn_tc_kernel<1>, grid, TcCfg<1>::THREADS, smem, stream, p));
    }
    MergeParams m;
    m.cand = p.cand;
    m.meta = p.meta;
    m.splits = pl.splits * pl.halves;  // candidate buffers per row
    m.cap = pl.cap;
    m.Q = Q;
    m.N = N;
    m.qlist = qlist;
    m.perm = ordered ? w.ord.perm : nullptr;
    m.X = X;
    m.D = D;
    m.k = k;
    m.nrm = w.nrm;
    m.stats = reinterpret_cast<const float4 *>(w.stats);
    m.Xq = Xq;
    m.qnrm = w.qnrm;
    m.qstats = reinterpret_cast<const float4 *>(w.qstats);
    m.gmax = w.gmax;
    m.acc_coef = acc_coef_of(pl);
    m.sq_coef = pl.passes == 1 ? 0.5f * m.acc_coef : 0.f;
    m.idx_out = idx_out;
    m.d2_out = d2_out;
    m.flag_rows = w.flag_rows;
    m.flag_count = w.flag_count;
    m.ksel = pl.ksel;
    if (radius) {
        ATSNE_TRY(launch_kernel("knn_tc_merge", radius_merge_kernel, ceil_div(Q, MERGE_WARPS),
                                MERGE_WARPS * 32, 0, stream, m, radius));
        ATSNE_TRY(knn_bruteforce_rows(X, N, D, qlist, w.flag_rows, w.flag_count, Q, k, idx_out, d2_out,
                                      stream, Xq));
        return launch_kernel("radius_filter", radius_filter_kernel, ceil_div(Q * k, 256), 256, 0, stream,
                             idx_out, d2_out, Q, k, radius);
    }
    if (!pl.certify) {
        // the re-rank set is the ksel best keys (ties included); the staged
        // keys are those below the lowest tau, about twice as many
        int rc = 64;
        while (rc < pl.ksel + pl.ksel / 4) rc <<= 1;
        m.rc = rc < RCAP_FP8 ? rc : RCAP_FP8;
        m.mst = 2 * m.rc;
        const size_t ms = merge_smem_bytes(false, m.rc, m.mst);
        e = cudaFuncSetAttribute(knn_merge_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ms);
        if (e != cudaSuccess) return cuda_error(e, "knn_tc_merge attribute");
        ATSNE_TRY(launch_kernel("knn_tc_merge", knn_merge_kernel<false>, ceil_div(Q, MERGE_WARPS),
                                MERGE_WARPS * 32, ms, stream, m));
    } else {
        m.rc = RCAP;
        m.mst = MSTAGE;
        const size_t ms = merge_smem_bytes(true, m.rc, m.mst);
        e = cudaFuncSetAttribute(knn_merge_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ms);
        if (e != cudaSuccess) return cuda_error(e, "knn_tc_merge attribute");
        ATSNE_TRY(launch_kernel("knn_tc_merge", knn_merge_kernel<true>, ceil_div(Q, MERGE_WARPS),
                                MERGE_WARPS * 32, ms, stream, m));
    }
    return knn_bruteforce_rows(X, N, D, qlist, w.flag_rows, w.flag_count, Q, k, idx_out, d2_out, stream,
                               Xq);
}

}  // namespace atsne
