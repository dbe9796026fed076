// Forest search (Sec. 4.2): best-bin-first over all T trees with one priority
// queue ordered by the distance to the decision boundary, stopped once a budget
// of `checks` distinct points has been evaluated.
//
// The visiting order never depends on distances (no pruning by the current
// k-th distance), so each query runs in two phases inside one warp:
//   1. traversal: queue pops, descents and de-duplication only. A descent
//      round covers five levels below the current node: each lane loads one
//      of the 31 subtree nodes and compares the query with its split, one
//      ballot gives the path, and the far children along it are pushed, so a
//      17-level descent costs four memory round trips and no serial
//      level-by-level walk. Queue entries are 64-bit words (key bits << 32 |
//      tree << 26 | node), so one integer compare orders them by (key, tree,
//      node). The queue is spread over the 32 lanes (ColQueue): pops and
//      evictions take a warp-wide min or max reduction and one
//      warp-cooperative column rescan, insertions one store. The points
//      collected are appended to a per-warp list in the workspace.
//   2. evaluation: the warp streams the collected points' rows eight at a time
//      (FP32 direct differences, float4 loads when D % 4 == 0) and keeps the k
//      best in shared memory under the (distance, index) order.
// Warps fetch queries from a global counter; the grid is sized by occupancy.
//
// Cut-off (all-rows mode). Popped keys never decrease (a descent adds squares to
// the popped key), so the search pops its entries in key order and stops at some
// last key K. Leaving out every push with key > C does not change which entries
// at or below C are popped, nor their order: an entry's fate in the bounded queue
// (kept or evicted) depends only on the entries below it, and the queue's minimum
// is the same while it holds any entry at or below C. So a search run with a
// cut-off C that reaches its budget is the search without one, and most pushes
// (and nearly all evictions) are skipped. A search that runs dry under its
// cut-off is run again without one. The queries are taken in the leaf order of
// tree 0; every FQ_SEED_GAP-th one (a seed, handed out first) runs without a
// cut-off and records its K, and the others take FQ_CUT_FACTOR times the larger
// K of the seeds on either side (neighbouring leaves: similar densities).
#include <float.h>
#include <limits.h>

#include "common.cuh"
#include "internal.h"

namespace atsne {
namespace {

constexpr int FQ_WARPS = 4;
constexpr int FQ_MAX_SLOTS = 4096;  // warps of the persistent grid (one seen bitmap each)
constexpr int FQ_KCAP = 128;
constexpr int SUB_DEPTH = 5;        // levels fetched per descent round (31 nodes, one per lane)
constexpr int FQ_SEED_GAP = 32;     // one seed query per this many, in tree-0 leaf order
constexpr float FQ_CUT_FACTOR = 3.f;

struct FqArgs {
    const float *X;
    int64_t N;
    int D, T, h, k, checks, qcap;
    int64_t n_int;
    const int32_t *split_dim;
    const float *split_val;
    const int32_t *perm;
    const int32_t *leaf_ofs;
    const int32_t *leaf_pt;
    int leaf_size;
    const int32_t *qlist;
    int64_t nq;
    int32_t *idx_out;
    float *d2_out;
    int64_t *evaluated_out;
    uint32_t *seen;    // [slots][words]
    int64_t words;
    int32_t *marked;   // [slots][mark_cap]
    int64_t mark_cap;
    int *next_query;
    float *kseed;      // [n_seeds] last popped key of each seed (NaN until written)
    int64_t n_seeds;
};

__device__ __forceinline__ uint64_t qpack(float key, int tree, int node) {
    return ((uint64_t)__float_as_uint(key) << 32) | ((uint64_t)tree << 26) | (uint64_t)node;
}

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
    const uint32_t hi = __reduce_min_sync(FULL, (uint32_t)(v >> 32));
    const uint32_t lo = __reduce_min_sync(FULL, (uint32_t)(v >> 32) == hi ? (uint32_t)v : 0xffffffffu);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
    const uint32_t hi = __reduce_max_sync(FULL, (uint32_t)(v >> 32));
    const uint32_t lo = __reduce_max_sync(FULL, (uint32_t)(v >> 32) == hi ? (uint32_t)v : 0u);
    return ((uint64_t)hi << 32) | lo;
}

// Bounded min-queue of distinct packed entries, spread over 32 columns in
// shared memory (lane l owns col[l * stride ...], filled in slots 0..cnt-1).
// Each lane keeps its column's count, minimum and maximum (and their slots) in
// registers; the warp keeps the total and an upper bound of the maximum.
//   pop:    the minimum over the lanes' minima; its column is closed up and
//           rescanned by the whole warp.
//   push:   into a column with room (round robin), or, when the queue is full,
//           in place of the maximum if smaller, that column then rescanned.
// All lanes call each operation with the same arguments. As entries are
// distinct, the queue holds the same set as any bounded min-queue that evicts
// its maximum, given the same pushes and pops.
struct ColQueue {
    uint64_t *col;
    int stride, cap;
    int lcap, cnt;    // this lane's column: capacity, entries
    uint64_t mn, mx;  // this lane's minimum (~0 if empty) and maximum (0 if empty)
    int mns, mxs;     // their slots
    int n;            // entries held (warp-uniform)
    uint64_t hmax;    // upper bound of the maximum held (warp-uniform)
    int rr;           // next column tried by an insertion (warp-uniform)
};

__device__ __forceinline__ void cq_init(ColQueue &q, uint64_t *col, int cap, int lane) {
    q.col = col;
    q.cap = cap;
    q.stride = (cap + 31) >> 5;
    q.lcap = (cap - lane + 31) >> 5;
    q.cnt = 0;
    q.mn = ~0ull;
    q.mx = 0;
    q.mns = q.mxs = -1;
    q.n = 0;
    q.hmax = 0;
    q.rr = 0;
}

// Lane w's column minimum (MIN) or maximum and its slot, found by the whole warp.
template <bool MIN>
__device__ __forceinline__ void cq_rescan(ColQueue &q, int w, int lane) {
    const int c = __shfl_sync(FULL, q.cnt, w);
    const uint64_t *cw = q.col + w * q.stride;
    uint64_t best = MIN ? ~0ull : 0ull;
    int bs = -1;
    for (int s = lane; s < c; s += 32) {
        const uint64_t e = cw[s];
        if (MIN ? e < best : e > best) {
            best = e;
            bs = s;
        }
    }
    const uint64_t g = MIN ? warp_min_u64(best) : warp_max_u64(best);
    const unsigned hit = __ballot_sync(FULL, bs >= 0 && best == g);
    const int slot = hit ? __shfl_sync(FULL, bs, __ffs(hit) - 1) : -1;
    if (lane == w) {
        if (MIN) {
            q.mn = hit ? g : ~0ull;
            q.mns = slot;
        } else {
            q.mx = hit ? g : 0ull;
            q.mxs = slot;
        }
    }
}

__device__ __forceinline__ uint64_t cq_pop(ColQueue &q, int lane) {
    const uint64_t top = warp_min_u64(q.mn);
    const int w = __ffs(__ballot_sync(FULL, q.cnt > 0 && q.mn == top)) - 1;
    if (lane == w) {
        uint64_t *cw = q.col + w * q.stride;
        const int last = q.cnt - 1, hole = q.mns;
        if (hole != last) cw[hole] = cw[last];
        if (q.mxs == last) q.mxs = hole;
        q.cnt = last;
        if (last == 0) {
            q.mx = 0;
            q.mxs = -1;
        }
    }
    __syncwarp();
    cq_rescan<true>(q, w, lane);
    --q.n;
    return top;
}

__device__ __forceinline__ void cq_push(ColQueue &q, uint64_t x, int lane) {
    if (q.n == q.cap) {
        if (x >= q.hmax) return;
        const uint64_t m = warp_max_u64(q.mx);
        q.hmax = m;
        if (x >= m) return;
        const int w = __ffs(__ballot_sync(FULL, q.cnt > 0 && q.mx == m)) - 1;
        if (lane == w) {
            q.col[w * q.stride + q.mxs] = x;
            if (x < q.mn) {
                q.mn = x;
                q.mns = q.mxs;
            }
        }
        __syncwarp();
        cq_rescan<false>(q, w, lane);
        q.hmax = warp_max_u64(q.mx);
        return;
    }
    const unsigned nf = __ballot_sync(FULL, q.cnt < q.lcap);
    const unsigned rot = __funnelshift_r(nf, nf, q.rr);
    const int t = (q.rr + __ffs(rot) - 1) & 31;
    if (lane == t) {
        q.col[t * q.stride + q.cnt] = x;
        if (x < q.mn) {
            q.mn = x;
            q.mns = q.cnt;
        }
        if (x > q.mx) {
            q.mx = x;
            q.mxs = q.cnt;
        }
        ++q.cnt;
    }
    q.rr = (t + 1) & 31;
    ++q.n;
    if (x > q.hmax) q.hmax = x;
}

// Pushes the entries of the lanes with `valid` set, in lane order. With no
// pop in between, the queue ends up holding the same set in any order; when
// it is full at the start, entries at or above the bound are rejected at once.
__device__ __forceinline__ void cq_push_lanes(ColQueue &q, uint64_t e, bool valid, int lane) {
    unsigned m = __ballot_sync(FULL, valid && (q.n < q.cap || e < q.hmax));
    while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1;
        cq_push(q, __shfl_sync(FULL, e, j), lane);
    }
}

// Descend tree `tr` from node v (queue key `key`) to a leaf, pushing the far
// child of every node passed whose key is at most `cut`; returns the leaf index. Each round covers up to
// five levels: lane j < 31 loads node j of the five-level subtree below the
// current node and compares the query with its split, a ballot of the
// outcomes gives the path, and lane j < (levels) pushes the far child of the
// path's node on level j. With PT (one point per leaf) the last round also
// fetches the points of the subtree's leaves and `pt` returns the reached
// leaf's point (-1 if empty). Node ids fit in 26 bits.
template <bool PT>
__device__ __forceinline__ int descend(const FqArgs &A, const float *qv, ColQueue &q, int tr, int v,
                                       float key, float cut, int lane, int &pt) {
    const int32_t *sd = A.split_dim + (int64_t)tr * A.n_int;
    const float *sv = A.split_val + (int64_t)tr * A.n_int;
    const int32_t *lpt = A.leaf_pt + ((int64_t)tr << A.h);
    const int n_int = (int)A.n_int;
    pt = -1;
    if (PT && v >= n_int) pt = lpt[v - n_int];
    while (v < n_int) {
        const int lv = 31 - __clz(v + 1);
        const int d = min(SUB_DEPTH, A.h - lv);
        const bool last = lv + d == A.h;
        int node = 0, lp = -1;
        bool left = false;
        float fk = INFINITY;
        if (lane < (1 << d) - 1) {
            const int j = 31 - __clz(lane + 1);
            node = ((v + 1) << j) - 1 + (lane + 1 - (1 << j));
            const float qd = qv[sd[node]];
            const float val = sv[node];
            left = qd < val;
            const float diff = __fsub_rn(qd, val);
            fk = __fadd_rn(key, __fmul_rn(diff, diff));
        }
        if (PT && last && lane < (1 << d)) lp = lpt[((v + 1) << d) - 1 + lane - n_int];
        const unsigned lm = __ballot_sync(FULL, left);
        int c = 0, my_c = 0;
#pragma unroll 1
        for (int j = 0; j < d; ++j) {
            if (lane == j) my_c = c;
            c = ((lm >> c) & 1u) ? 2 * c + 1 : 2 * c + 2;
        }
        const float pk = __shfl_sync(FULL, fk, my_c);
        const int pn = __shfl_sync(FULL, node, my_c);
        const uint64_t e = qpack(pk, tr, ((lm >> my_c) & 1u) ? 2 * pn + 2 : 2 * pn + 1);
        cq_push_lanes(q, e, lane < d && !isinf(pk) && pk <= cut, lane);
        const int o = c + 1 - (1 << d);  // offset of the reached node on its level
        if (PT && last) pt = __shfl_sync(FULL, lp, o);
        v = ((v + 1) << d) - 1 + o;
    }
    return v - n_int;
}

__global__ void __launch_bounds__(FQ_WARPS * 32) forest_query_kernel(FqArgs A) {
    extern __shared__ __align__(16) unsigned char fq_smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const size_t heap_b = (size_t)((A.qcap + 31) >> 5) * 32 * 8;
    const size_t q_b = ((size_t)A.D * 4 + 15) & ~size_t(15);
    unsigned char *base = fq_smem + w * (heap_b + q_b + FQ_KCAP * 8);
    uint64_t *qcol = reinterpret_cast<uint64_t *>(base);
    float *qv = reinterpret_cast<float *>(base + heap_b);
    float *td = reinterpret_cast<float *>(base + heap_b + q_b);
    int *tj = reinterpret_cast<int *>(td + FQ_KCAP);

    const int slot = blockIdx.x * FQ_WARPS + w;
    uint32_t *seen = A.seen + (int64_t)slot * A.words;
    int32_t *marked = A.marked + (int64_t)slot * A.mark_cap;
    const int64_t need = A.checks > A.k ? A.checks : A.k;
    const bool vec4 = (A.D & 3) == 0 && (reinterpret_cast<uintptr_t>(A.X) & 15) == 0;

    for (;;) {
        int64_t s = 0;
        if (lane == 0) s = atomicAdd(A.next_query, 1);
        s = __shfl_sync(0xffffffffu, s, 0);
        if (s >= A.nq) break;
        float cut = INFINITY;
        int64_t seed = -1;
        if (!A.qlist) {
            // all-rows mode walks the points in the leaf order of tree 0, so warps
            // running at the same time search neighbouring points (shared rows in
            // L2): the seeds first, then the positions between them
            int64_t pos;
            if (s < A.n_seeds) {
                seed = s;
                pos = s * FQ_SEED_GAP;
            } else {
                const int64_t j = s - A.n_seeds;
                pos = j / (FQ_SEED_GAP - 1) * FQ_SEED_GAP + j % (FQ_SEED_GAP - 1) + 1;
                const int64_t a = pos / FQ_SEED_GAP;
                const float ka = __ldcg(A.kseed + a);
                const float kb = a + 1 < A.n_seeds ? __ldcg(A.kseed + a + 1) : ka;
                // a seed still running reads NaN: no cut-off
                if (ka >= 0.f && kb >= 0.f) cut = FQ_CUT_FACTOR * fmaxf(ka, kb);
            }
            s = A.perm[pos];
        }
        const int64_t qi = A.qlist ? A.qlist[s] : s;
        if (qi < 0 || qi >= A.N) continue;  // flagged by the caller's index check
        const float *xq = A.X + qi * A.D;
        for (int d = lane; d < A.D; d += 32) qv[d] = xq[d];
        for (int t = lane; t < FQ_KCAP; t += 32) {
            td[t] = INFINITY;
            tj[t] = INT_MAX;
        }
        int64_t n_marked, evaluated;
        float kfin = 0.f;  // key of the last pop whose leaf was scanned
        ColQueue q;
        // ---- phase 1: traversal (a second time, without cut-off, if the first ran dry) ----
        for (;;) {
            if (lane == 0) {
                atomicOr(&seen[qi >> 5], 1u << (qi & 31));
                marked[0] = (int32_t)qi;
            }
            n_marked = 1;
            evaluated = 0;
            cq_init(q, qcol, A.qcap, lane);
            __syncwarp();

            auto scan_leaf = [&](int tr, int m) {
                const int s0 = A.leaf_ofs[m];
                const int cnt = A.leaf_ofs[m + 1] - s0;
                const int32_t *pt = A.perm + (int64_t)tr * A.N + s0;
                for (int b = 0; b < cnt; b += 32) {
                    const int q = b + lane;
                    int32_t p = -1;
                    bool fresh = false;
                    if (q < cnt) {
                        p = pt[q];
                        fresh = !((__ldcg(&seen[p >> 5]) >> (p & 31)) & 1u);
                    }
                    const unsigned fm = __ballot_sync(0xffffffffu, fresh);
                    if (fresh) {
                        atomicOr(&seen[p >> 5], 1u << (p & 31));
                        marked[n_marked + __popc(fm & ((1u << lane) - 1u))] = p;
                    }
                    n_marked += __popc(fm);
                    evaluated += __popc(fm);
                    __syncwarp();
                }
            };
            if (A.leaf_size == 1) {
                // one point per leaf: the seen test of step i is resolved after the
                // descent of step i + 1 (descents never read the bitmap; a step made
                // past the stopping point only adds queue entries that are not used)
                int pend_p = -1, pending = 0;
                uint32_t pend_w = 0;
                float pend_key = 0.f;
                auto resolve = [&]() {
                    if (pending) kfin = pend_key;
                    pending = 0;
                    if (pend_p >= 0 && !((pend_w >> (pend_p & 31)) & 1u)) {
                        if (lane == 0) {
                            atomicOr(&seen[pend_p >> 5], 1u << (pend_p & 31));
                            marked[n_marked] = pend_p;
                        }
                        ++n_marked;
                        ++evaluated;
                    }
                    pend_p = -1;
                };
                for (int t = 0;;) {
                    int hp_ = -1;
                    float key = 0.f;
                    if (t < A.T) {
                        descend<true>(A, qv, q, t, 0, 0.f, cut, lane, hp_);
                        ++t;
                    } else {
                        if (q.n == 0) break;
                        const uint64_t e = cq_pop(q, lane);
                        key = __uint_as_float((uint32_t)(e >> 32));
                        const int tr = (int)((e >> 26) & 63u);
                        const int v = (int)(e & ((1u << 26) - 1u));
                        descend<true>(A, qv, q, tr, v, key, cut, lane, hp_);
                    }
                    // the word is loaded now and only read at the next step
                    uint32_t hw = hp_ >= 0 ? __ldcg(&seen[hp_ >> 5]) : 0u;
                    const int prev = pend_p;
                    resolve();
                    __syncwarp();
                    if (evaluated >= need) break;
                    if (hp_ >= 0 && hp_ == prev) hw |= 1u << (prev & 31);
                    pend_p = hp_;
                    pend_w = hw;
                    pend_key = key;
                    pending = 1;
                }
                resolve();
                __syncwarp();
            } else {
                int unused;
                for (int t = 0; t < A.T && evaluated < need; ++t) {
                    scan_leaf(t, descend<false>(A, qv, q, t, 0, 0.f, cut, lane, unused));
                    kfin = 0.f;
                }
                while (evaluated < need && q.n > 0) {
                    const uint64_t e = cq_pop(q, lane);
                    const float key = __uint_as_float((uint32_t)(e >> 32));
                    const int tr = (int)((e >> 26) & 63u);
                    const int v = (int)(e & ((1u << 26) - 1u));
                    scan_leaf(tr, descend<false>(A, qv, q, tr, v, key, cut, lane, unused));
                    kfin = key;
                }
            }
            if (evaluated >= need || isinf(cut)) break;
            // the cut-off left too few entries: clear this attempt's marks, search again
            for (int64_t u = lane; u < n_marked; u += 32) {
                const int32_t p = marked[u];
                atomicAnd(&seen[p >> 5], ~(1u << (p & 31)));
            }
            __syncwarp();
            cut = INFINITY;
        }
        if (seed >= 0 && lane == 0) A.kseed[seed] = kfin;
        // the queue ran dry with fewer than k points: lowest-index unseen points
        for (int64_t b = 0; evaluated < A.k && b < A.N; b += 32) {
            const int64_t p = b + lane;
            const bool fresh = p < A.N && !((__ldcg(&seen[p >> 5]) >> (p & 31)) & 1u);
            unsigned fm = __ballot_sync(0xffffffffu, fresh);
            const int64_t room = A.k - evaluated;
            if (__popc(fm) > room) {  // keep the `room` lowest-index lanes
                unsigned keep = 0, rest = fm;
                for (int64_t r = 0; r < room; ++r) {
                    keep |= rest & (0u - rest);
                    rest &= rest - 1u;
                }
                fm = keep;
            }
            const bool take = (fm >> lane) & 1u;
            if (take) {
                atomicOr(&seen[p >> 5], 1u << (p & 31));
                marked[n_marked + __popc(fm & ((1u << lane) - 1u))] = (int32_t)p;
            }
            n_marked += __popc(fm);
            evaluated += __popc(fm);
            __syncwarp();
        }

        // ---- phase 2: distances of the collected points, k best kept ----
        float md = INFINITY;
        int mj = INT_MAX, mp = 0;
        auto insert = [&](float dist, int p) {
            if (!pair_less(dist, p, md, mj)) return;
            if (lane == 0) {
                td[mp] = dist;
                tj[mp] = p;
            }
            __syncwarp();
            float bd = -INFINITY;
            int bj = INT_MIN, bp = 0;
            for (int u = lane; u < A.k; u += 32) {
                if (pair_less(bd, bj, td[u], tj[u])) {
                    bd = td[u];
                    bj = tj[u];
                    bp = u;
                }
            }
            warp_argmax_pair(bd, bj, bp);
            md = bd;
            mj = bj;
            mp = bp;
            __syncwarp();
        };
        for (int64_t b0 = 1; b0 < n_marked; b0 += 32) {
            const int64_t nb = n_marked - b0 < 32 ? n_marked - b0 : 32;
            const int my = lane < nb ? marked[b0 + lane] : -1;
            for (int g = 0; g < nb; g += 8) {
                int pj[8];
                float acc[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    pj[u] = __shfl_sync(0xffffffffu, my, (g + u) & 31);
                    if (g + u >= nb) pj[u] = -1;
                    acc[u] = 0.f;
                }
                if (vec4) {
                    const float4 *q4 = reinterpret_cast<const float4 *>(qv);
                    for (int d = lane; d < (A.D >> 2); d += 32) {
                        const float4 qq = q4[d];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            if (pj[u] < 0) continue;
                            const float4 xv = reinterpret_cast<const float4 *>(A.X + (int64_t)pj[u] * A.D)[d];
                            float df = qq.x - xv.x;
                            acc[u] = fmaf(df, df, acc[u]);
                            df = qq.y - xv.y;
                            acc[u] = fmaf(df, df, acc[u]);
                            df = qq.z - xv.z;
                            acc[u] = fmaf(df, df, acc[u]);
                            df = qq.w - xv.w;
                            acc[u] = fmaf(df, df, acc[u]);
                        }
                    }
                } else {
                    for (int d = lane; d < A.D; d += 32) {
                        const float qq = qv[d];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            if (pj[u] < 0) continue;
                            const float df = qq - A.X[(int64_t)pj[u] * A.D + d];
                            acc[u] = fmaf(df, df, acc[u]);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float dist = warp_sum(acc[u]);
                    if (pj[u] >= 0) insert(dist, pj[u]);
                }
            }
        }

        warp_bitonic_sort_smem(td, tj, FQ_KCAP, lane);
        for (int t = lane; t < A.k; t += 32) {
            A.idx_out[s * A.k + t] = tj[t];
            A.d2_out[s * A.k + t] = td[t];
        }
        if (lane == 0 && A.evaluated_out) A.evaluated_out[s] = evaluated;
        for (int64_t u = lane; u < n_marked; u += 32) {
            const int32_t p = marked[u];
            atomicAnd(&seen[p >> 5], ~(1u << (p & 31)));
        }
        __syncwarp();
    }
}

size_t fq_smem_bytes(int D, int qcap) {
    return FQ_WARPS * ((size_t)((qcap + 31) >> 5) * 32 * 8 + (((size_t)D * 4 + 15) & ~size_t(15)) +
                       FQ_KCAP * 8);
}

}  // namespace

size_t forest_query_workspace(Carver &c, int64_t N, int64_t nq, int k, int checks, int leaf_size,
                              void *ws_out) {
    FqArgs a{};
    a.words = (N + 31) / 32;
    const int64_t need = checks > k ? checks : k;
    a.mark_cap = need + leaf_size + k + 1;
    a.seen = c.take<uint32_t>((size_t)FQ_MAX_SLOTS * a.words);
    a.marked = c.take<int32_t>((size_t)FQ_MAX_SLOTS * a.mark_cap);
    a.next_query = c.take<int>(1);
    a.n_seeds = (nq + FQ_SEED_GAP - 1) / FQ_SEED_GAP;
    a.kseed = c.take<float>((size_t)a.n_seeds + 1);
    if (ws_out) *static_cast<FqArgs *>(ws_out) = a;
    return c.bytes();
}

atsne_status forest_query_launch(const float *X, const ForestView &f, const int32_t *qlist,
                                 int64_t nq, int k, int checks, int qcap, int32_t *idx_out,
                                 float *d2_out, int64_t *evaluated_out, void *ws_base,
                                 size_t ws_bytes, cudaStream_t stream) {
    if (k > FQ_KCAP) return set_error(ATSNE_EUNSUPPORTED, "forest query: k=%d above %d", k, FQ_KCAP);
    if (f.depth > 25 || f.trees > 64)
        return set_error(ATSNE_EUNSUPPORTED, "forest query: depth %d / %d trees beyond the packed queue",
                         f.depth, f.trees);
    Carver c(ws_base);
    FqArgs a;
    forest_query_workspace(c, f.N, nq, k, checks, f.leaf_size, &a);
    if (c.bytes() > ws_bytes) return set_error(ATSNE_ENOMEM, "forest query: workspace too small");
    const size_t smem = fq_smem_bytes(f.D, qcap);
    if (smem > 227 * 1024)
        return set_error(ATSNE_EUNSUPPORTED,
                         "forest query: queue_cap %d with D=%d needs %zu B of shared memory", qcap, f.D,
                         smem);
    cudaError_t e = cudaFuncSetAttribute(forest_query_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "forest query attribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, forest_query_kernel, FQ_WARPS * 32, smem);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    const int grid = (int)hmin(hmin((int64_t)per_sm * num_sms(), FQ_MAX_SLOTS / FQ_WARPS),
                               ceil_div(nq, FQ_WARPS));
    e = cudaMemsetAsync(a.seen, 0, sizeof(uint32_t) * (size_t)grid * FQ_WARPS * a.words, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.next_query, 0, sizeof(int), stream);
    if (e == cudaSuccess)  // 0xff bytes: NaN, a seed not yet searched
        e = cudaMemsetAsync(a.kseed, 0xff, sizeof(float) * (size_t)(a.n_seeds + 1), stream);
    if (e != cudaSuccess) return cuda_error(e, "forest query memset");
    a.X = X;
    a.N = f.N;
    a.D = f.D;
    a.T = f.trees;
    a.h = f.depth;
    a.k = k;
    a.checks = checks;
    a.qcap = qcap;
    a.n_int = f.n_internal;
    a.split_dim = f.split_dim;
    a.split_val = f.split_val;
    a.perm = f.perm;
    a.leaf_ofs = f.leaf_ofs;
    a.leaf_pt = f.leaf_pt;
    a.leaf_size = f.leaf_size;
    a.qlist = qlist;
    a.nq = nq;
    a.idx_out = idx_out;
    a.d2_out = d2_out;
    a.evaluated_out = evaluated_out;
    return launch_kernel("forest_query", forest_query_kernel, grid, FQ_WARPS * 32, smem, stream, a);
}

}  // namespace atsne
