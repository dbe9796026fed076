// Forest search (Sec. 4.2): best-bin-first over all T trees with one priority
// queue ordered by the distance to the decision boundary, stopped once a budget
// of `checks` distinct points has been evaluated.
//
// The visiting order never depends on distances (no pruning by the current
// k-th distance), so each query runs in two phases inside one warp:
//   1. traversal: queue pops, descents and de-duplication only. A descent
//      fetches the next five levels below the current node in one round (one
//      node per lane, 31 independent loads), then walks them with shuffles, so
//      a 17-level descent costs four memory round trips instead of 17. Queue
//      entries are 64-bit words (key bits << 32 | tree << 26 | node), so one
//      integer compare orders them by (key, tree, node). A full queue keeps an
//      upper bound of its maximum, so most rejected pushes cost one compare.
//      The points collected are appended to a per-warp list in the workspace.
//   2. evaluation: the warp streams the collected points' rows four at a time
//      (FP32 direct differences, float4 loads when D % 4 == 0) and keeps the k
//      best in shared memory under the (distance, index) order.
// Warps fetch queries from a global counter; the grid is sized by occupancy.
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
};

__device__ __forceinline__ uint64_t qpack(float key, int tree, int node) {
    return ((uint64_t)__float_as_uint(key) << 32) | ((uint64_t)tree << 26) | (uint64_t)node;
}

// Bounded min-queue: when full, a new entry replaces the largest (a leaf of the
// heap) if it is smaller. `hmax` is an upper bound of the entries held (raised
// on every insertion, lowered to the exact maximum whenever one is searched),
// so a full queue rejects x >= hmax without searching. All lanes call it with
// the same arguments; lane 0 writes.
__device__ void q_push(uint64_t *hp, int &hn, uint64_t &hmax, int cap, uint64_t x, int lane) {
    int pos;
    if (hn == cap) {
        if (x >= hmax) return;
        uint64_t mx = 0;
        int mp = -1;
        for (int i = cap / 2 + lane; i < cap; i += 32) {
            const uint64_t e = hp[i];
            if (mp < 0 || e > mx) {
                mx = e;
                mp = i;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t om = __shfl_xor_sync(0xffffffffu, mx, o);
            const int op = __shfl_xor_sync(0xffffffffu, mp, o);
            if (op >= 0 && (mp < 0 || om > mx)) {
                mx = om;
                mp = op;
            }
        }
        hmax = mx;
        if (!(x < mx)) return;
        pos = mp;
    } else {
        pos = hn++;
        if (x > hmax) hmax = x;
    }
    if (lane == 0) {
        while (pos > 0) {
            const int par = (pos - 1) >> 1;
            const uint64_t pe = hp[par];
            if (!(x < pe)) break;
            hp[pos] = pe;
            pos = par;
        }
        hp[pos] = x;
    }
    __syncwarp();
}

__device__ uint64_t q_pop(uint64_t *hp, int &hn, int lane) {
    const uint64_t top = hp[0];
    __syncwarp();
    const int n = --hn;
    if (lane == 0 && n > 0) {
        const uint64_t x = hp[n];
        int pos = 0;
        for (;;) {
            int c = 2 * pos + 1;
            if (c >= n) break;
            uint64_t cv = hp[c];
            if (c + 1 < n) {
                const uint64_t cr = hp[c + 1];
                if (cr < cv) {
                    cv = cr;
                    ++c;
                }
            }
            if (!(cv < x)) break;
            hp[pos] = cv;
            pos = c;
        }
        hp[pos] = x;
    }
    __syncwarp();
    return top;
}

// Descend tree `tr` from node v (queue key `key`) to a leaf, pushing the far
// child of every node passed; returns the leaf index. Node ids fit in 26 bits.
__device__ int descend(const FqArgs &A, const float *qv, uint64_t *hp, int &hn, uint64_t &hmax,
                       int tr, int v, float key, int lane) {
    const int32_t *sd = A.split_dim + (int64_t)tr * A.n_int;
    const float *sv = A.split_val + (int64_t)tr * A.n_int;
    const int n_int = (int)A.n_int;
    while (v < n_int) {
        const int lv = 31 - __clz(v + 1);
        const int d = min(SUB_DEPTH, A.h - lv);
        int dim = 0;
        float val = 0.f;
        if (lane < (1 << d) - 1) {
            const int j = 31 - __clz(lane + 1);
            const int node = ((v + 1) << j) - 1 + (lane + 1 - (1 << j));
            dim = sd[node];
            val = sv[node];
        }
        int c = 0, vg = v;
#pragma unroll 1
        for (int j = 0; j < d; ++j) {
            const int cd = __shfl_sync(0xffffffffu, dim, c);
            const float cs = __shfl_sync(0xffffffffu, val, c);
            const float qd = qv[cd];
            const bool left = qd < cs;
            const float diff = __fsub_rn(qd, cs);
            const float fk = __fadd_rn(key, __fmul_rn(diff, diff));
            if (!isinf(fk)) q_push(hp, hn, hmax, A.qcap, qpack(fk, tr, left ? 2 * vg + 2 : 2 * vg + 1), lane);
            c = left ? 2 * c + 1 : 2 * c + 2;
            vg = left ? 2 * vg + 1 : 2 * vg + 2;
        }
        v = vg;
    }
    return v - n_int;
}

// One point per leaf: descend as above and return the reached leaf's point (-1
// if empty) and the seen-bitmap word holding it. The last round fetches the
// points of all leaves of its subtree together with the split data; the word is
// loaded after the walk and only read at the next step.
struct LeafHit {
    int p;
    uint32_t word;
};

__device__ LeafHit descend_pt(const FqArgs &A, const float *qv, uint64_t *hp, int &hn,
                              uint64_t &hmax, const uint32_t *seen, int tr, int v, float key,
                              int lane) {
    const int32_t *sd = A.split_dim + (int64_t)tr * A.n_int;
    const float *sv = A.split_val + (int64_t)tr * A.n_int;
    const int32_t *lpt = A.leaf_pt + ((int64_t)tr << A.h);
    const int n_int = (int)A.n_int;
    int p = -1;
    if (v >= n_int) {
        p = lpt[v - n_int];
    } else {
        while (v < n_int) {
            const int lv = 31 - __clz(v + 1);
            const int d = min(SUB_DEPTH, A.h - lv);
            const bool last = lv + d == A.h;
            int dim = 0, lp = -1;
            float val = 0.f;
            if (lane < (1 << d) - 1) {
                const int j = 31 - __clz(lane + 1);
                const int node = ((v + 1) << j) - 1 + (lane + 1 - (1 << j));
                dim = sd[node];
                val = sv[node];
            }
            if (last && lane < (1 << d)) lp = lpt[((v + 1) << d) - 1 + lane - n_int];
            int c = 0, vg = v;
#pragma unroll 1
            for (int j = 0; j < d; ++j) {
                const int cd = __shfl_sync(0xffffffffu, dim, c);
                const float cs = __shfl_sync(0xffffffffu, val, c);
                const float qd = qv[cd];
                const bool left = qd < cs;
                const float diff = __fsub_rn(qd, cs);
                const float fk = __fadd_rn(key, __fmul_rn(diff, diff));
                if (!isinf(fk)) q_push(hp, hn, hmax, A.qcap, qpack(fk, tr, left ? 2 * vg + 2 : 2 * vg + 1), lane);
                c = left ? 2 * c + 1 : 2 * c + 2;
                vg = left ? 2 * vg + 1 : 2 * vg + 2;
            }
            if (last) p = __shfl_sync(0xffffffffu, lp, c + 1 - (1 << d));
            v = vg;
        }
    }
    return LeafHit{p, p >= 0 ? __ldcg(&seen[p >> 5]) : 0u};
}

__global__ void __launch_bounds__(FQ_WARPS * 32) forest_query_kernel(FqArgs A) {
    extern __shared__ __align__(16) unsigned char fq_smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const size_t heap_b = ((size_t)A.qcap * 8 + 15) & ~size_t(15);
    const size_t q_b = ((size_t)A.D * 4 + 15) & ~size_t(15);
    unsigned char *base = fq_smem + w * (heap_b + q_b + FQ_KCAP * 8);
    uint64_t *hp = reinterpret_cast<uint64_t *>(base);
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
        // all-rows mode walks the points in the leaf order of tree 0, so warps
        // running at the same time search neighbouring points (shared rows in L2)
        if (!A.qlist) s = A.perm[s];
        const int64_t qi = A.qlist ? A.qlist[s] : s;
        if (qi < 0 || qi >= A.N) continue;  // flagged by the caller's index check
        const float *xq = A.X + qi * A.D;
        for (int d = lane; d < A.D; d += 32) qv[d] = xq[d];
        for (int t = lane; t < FQ_KCAP; t += 32) {
            td[t] = INFINITY;
            tj[t] = INT_MAX;
        }
        if (lane == 0) {
            atomicOr(&seen[qi >> 5], 1u << (qi & 31));
            marked[0] = (int32_t)qi;
        }
        int64_t n_marked = 1, evaluated = 0;
        int hn = 0;
        uint64_t hmax = 0;
        __syncwarp();

        // ---- phase 1: traversal ----
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
            int pend_p = -1;
            uint32_t pend_w = 0;
            auto resolve = [&]() {
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
                LeafHit hit;
                if (t < A.T) {
                    hit = descend_pt(A, qv, hp, hn, hmax, seen, t, 0, 0.f, lane);
                    ++t;
                } else {
                    if (hn == 0) break;
                    const uint64_t e = q_pop(hp, hn, lane);
                    const float key = __uint_as_float((uint32_t)(e >> 32));
                    const int tr = (int)((e >> 26) & 63u);
                    const int v = (int)(e & ((1u << 26) - 1u));
                    hit = descend_pt(A, qv, hp, hn, hmax, seen, tr, v, key, lane);
                }
                const int prev = pend_p;
                resolve();
                __syncwarp();
                if (evaluated >= need) break;
                if (hit.p >= 0 && hit.p == prev) hit.word |= 1u << (prev & 31);
                pend_p = hit.p;
                pend_w = hit.word;
            }
            resolve();
            __syncwarp();
        } else {
            for (int t = 0; t < A.T && evaluated < need; ++t)
                scan_leaf(t, descend(A, qv, hp, hn, hmax, t, 0, 0.f, lane));
            while (evaluated < need && hn > 0) {
                const uint64_t e = q_pop(hp, hn, lane);
                const float key = __uint_as_float((uint32_t)(e >> 32));
                const int tr = (int)((e >> 26) & 63u);
                const int v = (int)(e & ((1u << 26) - 1u));
                scan_leaf(tr, descend(A, qv, hp, hn, hmax, tr, v, key, lane));
            }
        }
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
    return FQ_WARPS * ((((size_t)qcap * 8 + 15) & ~size_t(15)) + (((size_t)D * 4 + 15) & ~size_t(15)) +
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
    (void)nq;
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
