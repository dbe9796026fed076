// Forest search (Sec. 4.2): best-bin-first over all T trees with one priority
// queue ordered by the distance to the decision boundary, stopped once a budget
// of `checks` distinct points has been evaluated.
//
// The visiting order never depends on distances (no pruning by the current
// k-th distance), so the search runs as two kernels, one warp per query in each:
//   1. traversal (forest_traverse_kernel): queue pops, descents and
//      de-duplication only. A descent
//      round covers five levels below the current node: each lane loads one
//      of the 31 subtree nodes and compares the query with its split, one
//      ballot gives the path, and the far children along it are pushed, so a
//      17-level descent costs four memory round trips and no serial
//      level-by-level walk. Queue entries are 64-bit words (key bits << 32 |
//      tree << 26 | node), so one integer compare orders them by (key, tree,
//      node). The queue is spread over the 32 lanes (ColQueue), each lane
//      keeping its column sorted: pops and evictions take one warp-wide min
//      or max reduction and one load by the owning lane, insertions a short
//      shift inside one column. The points collected are written to the
//      query's list in the workspace.
//   2. evaluation (forest_dist_kernel): the warp streams the listed points'
//      rows eight at a time (float4 loads into registers when D % 4 == 0, two
//      pieces of each row in flight; built for 32 warps per SM, so that enough
//      bytes are in flight to cover the L2 latency), takes FP32 direct
//      differences, reduces the eight rows at once (nine shuffles), and keeps
//      the k best under the (distance, index) order in a buffer of FD_BUF
//      pairs: new candidates below the current k-th pair are appended, and a
//      full buffer is sorted and cut back to k.
// The queries go in chunks (the lists of a chunk fit in FQ_MARK_BUDGET bytes);
// traversal warps fetch queries from a global counter. On 8-bit integer data
// (a byte copy of X with a device flag, written first) the traversal holds the
// query as bytes (more warps per SM) and the distances come from the byte rows;
// the FP32 variants are launched too and return at once.
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
#include <type_traits>
#include <limits.h>

#include "common.cuh"
#include "internal.h"

namespace atsne {
namespace {

constexpr int FQ_WARPS = 4;
constexpr int FQ_MAX_SLOTS = 5120;  // traversal warps of the persistent grid (one seen bitmap each)
constexpr int FQ_KCAP = 128;        // largest k
constexpr int64_t FQ_MARK_BUDGET = int64_t(1) << 30;  // bytes of point lists per chunk
constexpr int FD_MAX_WARPS = 4;     // distance kernel: warps per block (fewer for very long rows)
constexpr int FD_BUF = 256;         // (distance, index) pairs per distance warp
constexpr int FD_U8_PIECES = 4;     // byte rows: 16-byte pieces per lane at most (D <= 2048)
enum { FD_F32 = 0, FD_F32V = 1, FD_U8 = 2 };
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
    int64_t ofs_stride;  // 0: leaf offsets shared by the trees; else per tree
    const int32_t *qlist;
    int64_t w0, nw;    // work items of this chunk: leaf positions of tree 0, or list entries
    int64_t *evaluated_out;
    uint32_t *seen;    // [slots][words]
    int64_t words;
    int32_t *marked;   // [nw][mark_cap] points collected (entry 0: the query itself)
    int32_t *n_marked; // [nw] entries of each list (0: no list)
    int64_t mark_cap;
    int *next_query;
    float *kseed;      // last popped key of each seed (NaN until written)
    int64_t chunk;     // work items per chunk (a multiple of FQ_SEED_GAP)
    const uint8_t *xu8;      // byte copy of X, when every value is an integer in [0, 255]
    const unsigned *u8_bad;
    int Dp16;
    int *status;
};

struct FdArgs {
    const float *X;
    const uint8_t *xu8;      // X as bytes ([N][Dp16]) when every value is an integer in [0, 255]
    const uint32_t *nx8;     // their exact squared norms
    const unsigned *u8_bad;  // nonzero: some value is not such an integer (FP32 rows used)
    int Dp16;
    int D, k;
    bool list_mode;
    int64_t w0, nw;
    const int32_t *marked;
    const int32_t *n_marked;
    int64_t mark_cap;
    int32_t *idx_out;
    float *d2_out;
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
// shared memory. Lane l owns column l (col[l * stride ...]) and keeps it
// sorted, largest first, in a circular buffer of `stride` slots starting at
// its head slot h; its count, minimum (the tail) and maximum (the head) live
// in registers. Every lane reads and writes only its own column.
//   pop:    the minimum over the lanes' minima (one warp reduction); the owner
//           drops its tail and loads the next one.
//   push:   into a column with room (round robin): the owner moves its
//           entries below the new one a slot toward the tail and stores it.
//   evict:  when the queue is full, the maximum over the lanes' maxima (one
//           warp reduction) is dropped by its owner (head advanced), unless
//           the new entry is larger, which is dropped instead.
// As entries are distinct, the queue holds the same set as any bounded
// min-queue that evicts its maximum, given the same pushes and pops.
struct ColQueue {
    uint64_t *col;    // this lane's column
    int stride, cap;
    int lcap, cnt, h; // this lane's column: capacity, entries, head slot
    uint64_t mn, mx;  // this lane's minimum (~0 if empty) and maximum (0 if empty)
    int n;            // entries held (warp-uniform)
    uint64_t hmax;    // upper bound of the maximum held (warp-uniform)
    int rr;           // next column tried by an insertion (warp-uniform)
};

__device__ __forceinline__ void cq_init(ColQueue &q, uint64_t *col, int cap, int lane) {
    q.stride = (cap + 31) >> 5;
    q.col = col + lane * q.stride;
    q.cap = cap;
    q.lcap = (cap - lane + 31) >> 5;
    q.cnt = 0;
    q.h = 0;
    q.mn = ~0ull;
    q.mx = 0;
    q.n = 0;
    q.hmax = 0;
    q.rr = 0;
}

__device__ __forceinline__ int cq_wrap(const ColQueue &q, int i) { return i >= q.stride ? i - q.stride : i; }

// Stores x in this lane's column (which has room), keeping it sorted.
__device__ __forceinline__ void cq_insert(ColQueue &q, uint64_t x) {
    int i = q.cnt;
    while (i > 0) {
        const uint64_t y = q.col[cq_wrap(q, q.h + i - 1)];
        if (y > x) break;
        q.col[cq_wrap(q, q.h + i)] = y;
        --i;
    }
    q.col[cq_wrap(q, q.h + i)] = x;
    ++q.cnt;
    if (x < q.mn) q.mn = x;
    if (x > q.mx) q.mx = x;
}

__device__ __forceinline__ uint64_t cq_pop(ColQueue &q, int lane) {
    const uint64_t top = warp_min_u64(q.mn);
    if (q.cnt > 0 && q.mn == top) {  // one lane: entries are distinct
        --q.cnt;
        if (q.cnt > 0) {
            q.mn = q.col[cq_wrap(q, q.h + q.cnt - 1)];
        } else {
            q.mn = ~0ull;
            q.mx = 0;
        }
    }
    --q.n;
    return top;
}

// One entry (the same in all lanes).
__device__ __forceinline__ void cq_push(ColQueue &q, uint64_t x, int lane) {
    if (q.n == q.cap) {
        if (x >= q.hmax) return;
        const uint64_t m = warp_max_u64(q.mx);
        q.hmax = m;  // stays an upper bound after the eviction
        if (x >= m) return;
        if (q.cnt > 0 && q.mx == m) {  // the owner of the maximum drops it and takes x
            q.h = cq_wrap(q, q.h + 1);
            --q.cnt;
            q.mx = q.cnt > 0 ? q.col[q.h] : 0ull;
            if (q.cnt == 0) q.mn = ~0ull;
            cq_insert(q, x);
        }
        return;
    }
    const unsigned nf = __ballot_sync(FULL, q.cnt < q.lcap);
    const unsigned rot = __funnelshift_r(nf, nf, q.rr);
    const int t = (q.rr + __ffs(rot) - 1) & 31;
    if (lane == t) cq_insert(q, x);
    q.rr = (t + 1) & 31;
    ++q.n;
    if (x > q.hmax) q.hmax = x;
}

// Pushes the entries of the lanes with `valid` set. With no pop in between,
// the queue ends up holding the same set in any order; when it is full at the
// start, entries at or above the bound are rejected at once. When the queue has room
// for all of them in distinct columns they are inserted at once (each by the
// owner of its column), else one by one in lane order.
__device__ __forceinline__ void cq_push_lanes(ColQueue &q, uint64_t e, bool valid, int lane) {
    unsigned m;
    if (q.n < q.cap)
        m = __ballot_sync(FULL, valid);
    else
        m = __ballot_sync(FULL, valid && e < q.hmax);
    if (!m) return;
    const int np = __popc(m);
    const unsigned room = __ballot_sync(FULL, q.cnt < q.lcap);
    if (np == 1 && q.n < q.cap) {  // the common case: one entry, into the next column with room
        const uint64_t x = __shfl_sync(FULL, e, __ffs(m) - 1);
        const unsigned rot = __funnelshift_r(room, room, q.rr);
        const int t = (q.rr + __ffs(rot) - 1) & 31;
        if (lane == t) cq_insert(q, x);
        q.rr = (t + 1) & 31;
        ++q.n;
        if (x > q.hmax) q.hmax = x;
        return;
    }
    if (q.n + np <= q.cap && __popc(room) >= np) {
        // the r-th pushing lane's entry goes to the r-th column with room,
        // counting from column q.rr
        const unsigned rot = __funnelshift_r(room, room, q.rr);
        const int my = (lane - q.rr) & 31;
        const int rho = __popc(rot & ((1u << my) - 1u));
        const bool take = ((rot >> my) & 1u) && rho < np;
        unsigned mm = m;
        for (int i = 0; i < rho && i < np; ++i) mm &= mm - 1u;
        const uint64_t x = __shfl_sync(FULL, e, take ? __ffs(mm) - 1 : 0);
        if (take) cq_insert(q, x);
        q.rr = (q.rr + np) & 31;
        q.n += np;
        q.hmax = ~0ull;  // unknown until the next eviction
        return;
    }
    while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1;
        cq_push(q, __shfl_sync(FULL, e, j), lane);
    }
}

// A lane's fixed place in a five-level descent subtree (lane l < 31 holds
// subtree node l in level order): its level, its offset below the subtree
// root's first descendant on that level, the bit of its parent's outcome that
// leads to it, and the set of its ancestors (itself included).
struct SubLane {
    int lvl, off, par;
    bool left;         // a left child: reached when the parent's query value is below its split
    unsigned anc;      // lanes of the node and its ancestors
    unsigned lvl_mask; // lane j < 5: the lanes of subtree level j
};

__device__ __forceinline__ SubLane sub_lane(int lane) {
    SubLane L;
    L.lvl = 31 - __clz(lane + 1);
    L.off = lane - (1 << L.lvl);
    L.par = lane > 0 ? (lane - 1) >> 1 : 0;
    L.left = (lane & 1) != 0;
    L.anc = 0;
    for (int a = lane; ; a = (a - 1) >> 1) {
        L.anc |= 1u << a;
        if (a == 0) break;
    }
    L.lvl_mask = lane < 5 ? ((1u << ((2 << lane) - 1)) - 1u) & ~((1u << ((1 << lane) - 1)) - 1u) : 0u;
    return L;
}

// Descend tree `tr` from node v (queue key `key`) to a leaf, pushing the far
// child of every node passed whose key is at most `cut`; returns the leaf index. Each round covers up to
// five levels: lane j < 31 loads node j of the five-level subtree below the
// current node and compares the query with its split, a ballot of the
// outcomes gives the path, and lane j < (levels) pushes the far child of the
// path's node on level j. A node is on the path when every node from the
// subtree root down to it is the child its parent's outcome selects: one
// ballot of "my parent leads to me" tested against each lane's ancestor set.
// With PT (one point per leaf) the last round also fetches the points of the
// subtree's leaves and `pt` returns the reached leaf's point (-1 if empty).
// Node ids fit in 26 bits.
template <bool PT, typename QT>
__device__ __forceinline__ int descend(const FqArgs &A, const QT *qv, ColQueue &q, int tr, int v,
                                       float key, float cut, int lane, const SubLane &L, int &pt) {
    const int64_t tb = (int64_t)tr * A.n_int;
    const int32_t *sd = A.split_dim + tb;
    const float *sv = A.split_val + tb;
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
        const bool in_sub = lane < (1 << d) - 1;
        if (in_sub) {
            // lane = node (lane + 1 - 2^j) of level j below v, j = floor(log2(lane + 1))
            node = ((v + 1) << L.lvl) + L.off;
            const float qd = (float)qv[sd[node]];
            const float val = sv[node];
            left = qd < val;
            const float diff = __fsub_rn(qd, val);
            fk = __fadd_rn(key, __fmul_rn(diff, diff));
        }
        if (PT && last && lane < (1 << d)) lp = lpt[((v + 1) << d) - 1 + lane - n_int];
        const unsigned lm = __ballot_sync(FULL, left);
        const unsigned okm = __ballot_sync(FULL, in_sub && (lane == 0 || (((lm >> L.par) & 1u) != 0) == L.left));
        const unsigned pm = __ballot_sync(FULL, in_sub && (okm & L.anc) == L.anc);  // one node per level
        const int my_c = lane < d ? __ffs(pm & L.lvl_mask) - 1 : 0;
        const int cl = 31 - __clz(pm);  // the path's node on the last level of the round
        const int c = 2 * cl + 2 - (int)((lm >> cl) & 1u);
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

// QB: the query held as bytes (8-bit integer data: the same values, a quarter
// of the shared memory, so more warps fit); the host launches both variants and
// the byte copy's device flag lets one of them run.
template <bool QB>
__global__ void __launch_bounds__(FQ_WARPS * 32, QB ? 8 : 7) forest_traverse_kernel(FqArgs A) {
    using QT = typename std::conditional<QB, uint8_t, float>::type;
    if (QB != (A.xu8 != nullptr && *A.u8_bad == 0u)) return;
    extern __shared__ __align__(16) unsigned char fq_smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const SubLane SL = sub_lane(lane);
    const size_t heap_b = (size_t)((A.qcap + 31) >> 5) * 32 * 8;
    const size_t q_b = QB ? (size_t)A.Dp16 : ((size_t)A.D * 4 + 15) & ~size_t(15);
    unsigned char *base = fq_smem + w * (heap_b + q_b);
    uint64_t *qcol = reinterpret_cast<uint64_t *>(base);
    QT *qv = reinterpret_cast<QT *>(base + heap_b);

    const int slot = blockIdx.x * FQ_WARPS + w;
    uint32_t *seen = A.seen + (int64_t)slot * A.words;
    const int need = A.checks > A.k ? A.checks : A.k;

    for (;;) {
        int64_t c = 0;
        if (lane == 0) c = atomicAdd(A.next_query, 1);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= A.nw) break;
        float cut = INFINITY;
        int64_t seed = -1, t, qi, row;
        if (!A.qlist) {
            // all-rows mode walks the points in the leaf order of tree 0, so warps
            // running at the same time search neighbouring points (shared rows in
            // L2): the chunk's seeds first, then the positions between them
            const int64_t ns = (A.nw + FQ_SEED_GAP - 1) / FQ_SEED_GAP;
            if (c < ns) {
                t = c * FQ_SEED_GAP;
            } else {
                const int64_t j = c - ns;
                t = j / (FQ_SEED_GAP - 1) * FQ_SEED_GAP + j % (FQ_SEED_GAP - 1) + 1;
            }
            const int64_t wpos = A.w0 + t, a = wpos / FQ_SEED_GAP;
            if (t % FQ_SEED_GAP == 0) {
                seed = a;
            } else {
                const float ka = __ldcg(A.kseed + a);
                // the seed after the chunk's last block belongs to the next chunk
                const float kb = (a + 1) * FQ_SEED_GAP < A.w0 + A.nw ? __ldcg(A.kseed + a + 1) : ka;
                // a seed still running reads NaN: no cut-off
                if (ka >= 0.f && kb >= 0.f) cut = FQ_CUT_FACTOR * fmaxf(ka, kb);
            }
            qi = row = A.perm[wpos];
        } else {
            t = c;
            row = A.w0 + c;
            qi = A.qlist[row];
        }
        int32_t *marked = A.marked + t * A.mark_cap;
        if (qi < 0 || qi >= A.N) {  // flagged by the caller's index check
            if (lane == 0) A.n_marked[t] = 0;
            continue;
        }
        if constexpr (QB) {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(A.xu8 + qi * A.Dp16);
            for (int d = lane; d < (A.Dp16 >> 2); d += 32) reinterpret_cast<uint32_t *>(qv)[d] = src[d];
        } else {
            const float *xq = A.X + qi * A.D;
            for (int d = lane; d < A.D; d += 32) qv[d] = xq[d];
        }
        int n_marked, evaluated;  // at most mark_cap
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
                const int32_t *lo = A.leaf_ofs + (int64_t)tr * A.ofs_stride;
                const int s0 = lo[m];
                int cnt = lo[m + 1] - s0;
                // a bucket larger than the leaf size the list was sized for (a
                // caller's stale bucket bound) is cut to the list's room and flagged
                if (cnt > A.mark_cap - n_marked) {
                    if (lane == 0) raise_status(A.status, DEV_MALFORMED);
                    cnt = (int)(A.mark_cap - n_marked);
                }
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
            if (A.leaf_size == 1 && A.ofs_stride == 0) {
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
                        descend<true, QT>(A, qv, q, t, 0, 0.f, cut, lane, SL, hp_);
                        ++t;
                    } else {
                        if (q.n == 0) break;
                        const uint64_t e = cq_pop(q, lane);
                        key = __uint_as_float((uint32_t)(e >> 32));
                        const int tr = (int)((e >> 26) & 63u);
                        const int v = (int)(e & ((1u << 26) - 1u));
                        descend<true, QT>(A, qv, q, tr, v, key, cut, lane, SL, hp_);
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
                    scan_leaf(t, descend<false, QT>(A, qv, q, t, 0, 0.f, cut, lane, SL, unused));
                    kfin = 0.f;
                }
                while (evaluated < need && q.n > 0) {
                    const uint64_t e = cq_pop(q, lane);
                    const float key = __uint_as_float((uint32_t)(e >> 32));
                    const int tr = (int)((e >> 26) & 63u);
                    const int v = (int)(e & ((1u << 26) - 1u));
                    scan_leaf(tr, descend<false, QT>(A, qv, q, tr, v, key, cut, lane, SL, unused));
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

        if (lane == 0) {
            A.n_marked[t] = (int32_t)n_marked;
            if (A.evaluated_out) A.evaluated_out[row] = evaluated;
        }
        for (int64_t u = lane; u < n_marked; u += 32) {
            const int32_t p = marked[u];
            atomicAnd(&seen[p >> 5], ~(1u << (p & 31)));
        }
        __syncwarp();
    }
}

// Sums of eight rows' partial sums over the warp with nine shuffles: each lane
// ends with the total of row ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 +
// ((lane >> 2) & 1) (four lanes per row).
template <typename T>
__device__ __forceinline__ T warp_sum8(T (&v)[8], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const T send = b4 ? v[u] : v[u + 4];
        const T keep = b4 ? v[u + 4] : v[u];
        v[u] = keep + __shfl_xor_sync(FULL, send, 16);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const T send = b3 ? v[u] : v[u + 2];
        const T keep = b3 ? v[u + 2] : v[u];
        v[u] = keep + __shfl_xor_sync(FULL, send, 8);
    }
    const T send = b2 ? v[0] : v[1];
    T r = (b2 ? v[1] : v[0]) + __shfl_xor_sync(FULL, send, 4);
    r += __shfl_xor_sync(FULL, r, 2);
    r += __shfl_xor_sync(FULL, r, 1);
    return r;
}

// Distances of each query to its listed points (entry 0, the query, left out)
// and the k best under the (distance, index) order, written sorted.
// MODE: FD_F32 / FD_F32V (FP32 rows, scalar or float4 loads) or FD_U8 (byte
// rows, QP 16-byte pieces per lane). The host launches an FP32 and, where byte
// rows are possible, a byte instantiation; each returns at once unless the
// prep kernel's finding (every value an integer in [0, 255] or not) selects it.
template <int MODE, int QP>
__global__ void __launch_bounds__(FD_MAX_WARPS * 32, 8) forest_dist_kernel(FdArgs A) {
    constexpr bool U8 = MODE == FD_U8, VEC = MODE == FD_F32V;
    const bool u8_ok = A.xu8 != nullptr && *A.u8_bad == 0u;
    if (U8 != u8_ok) return;
    extern __shared__ __align__(16) unsigned char fd_smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int Dp = (A.D + 3) & ~3;
    float *qv = reinterpret_cast<float *>(fd_smem) + (size_t)w * Dp;
    float *bd = reinterpret_cast<float *>(fd_smem + (size_t)nwarp * Dp * 4) + w * FD_BUF;
    int *bj = reinterpret_cast<int *>(bd + (size_t)nwarp * FD_BUF);
    const int D = A.D, D4 = D >> 2, k = A.k;
    const int64_t stride = (int64_t)gridDim.x * nwarp;
    const int C16 = A.Dp16 >> 4;  // 16-byte pieces per byte row

    for (int64_t t = (int64_t)blockIdx.x * nwarp + w; t < A.nw; t += stride) {
        const int n = A.n_marked[t];
        if (n == 0) continue;
        const int32_t *list = A.marked + t * A.mark_cap;
        const int32_t qi = list[0];
        const int64_t row = A.list_mode ? A.w0 + t : qi;
        const float *xq = A.X + (int64_t)qi * D;
        uint4 qb[QP];
        int nq8 = 0;
        if constexpr (U8) {
#pragma unroll
            for (int j = 0; j < QP; ++j) {
                const int c = lane + 32 * j;
                qb[j] = c < C16 ? reinterpret_cast<const uint4 *>(A.xu8 + (int64_t)qi * A.Dp16)[c]
                                : make_uint4(0u, 0u, 0u, 0u);
            }
            nq8 = (int)A.nx8[qi];
        } else {
            for (int d = lane; d < D; d += 32) qv[d] = xq[d];
        }
        for (int u = lane; u < FD_BUF; u += 32) {
            bd[u] = INFINITY;
            bj[u] = INT_MAX;
        }
        __syncwarp();
        const int nr = n - 1;
        int fill = 0;
        bool sorted = false;
        float thr_d = INFINITY;
        int thr_j = INT_MAX;
        auto sort_cut = [&]() {
            for (int u = fill + lane; u < FD_BUF; u += 32) {
                bd[u] = INFINITY;
                bj[u] = INT_MAX;
            }
            __syncwarp();
            warp_bitonic_sort_smem(bd, bj, FD_BUF, lane);
            fill = k;
            sorted = true;
            thr_d = bd[k - 1];
            thr_j = bj[k - 1];
        };
        int my = 0;
        for (int b0 = 0; b0 < nr; b0 += 8) {
            if ((b0 & 31) == 0) my = b0 + lane < nr ? list[1 + b0 + lane] : 0;
            int pj[8];
            float acc[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                pj[u] = __shfl_sync(FULL, my, (b0 + u) & 31);
                if (b0 + u >= nr) pj[u] = pj[0];  // a valid row, its sum unused
                acc[u] = 0.f;
            }
            int dot8 = 0;
            if constexpr (U8) {
                // |q - x|^2 = |q|^2 + |x|^2 - 2 q.x, every term an exact integer
                // (below 2^31 for D <= 2048)
                unsigned dp[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) dp[u] = 0u;
#pragma unroll
                for (int j = 0; j < QP; ++j) {
                    const int c = lane + 32 * j;
                    if (c < C16) {
                        uint4 xv[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            xv[u] = __ldg(reinterpret_cast<const uint4 *>(A.xu8 + (int64_t)pj[u] * A.Dp16) + c);
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            dp[u] = __dp4a(xv[u].x, qb[j].x, dp[u]);
                            dp[u] = __dp4a(xv[u].y, qb[j].y, dp[u]);
                            dp[u] = __dp4a(xv[u].z, qb[j].z, dp[u]);
                            dp[u] = __dp4a(xv[u].w, qb[j].w, dp[u]);
                        }
                    }
                }
                dot8 = (int)warp_sum8(dp, lane);
            } else if constexpr (VEC) {
                const float4 *q4 = reinterpret_cast<const float4 *>(qv);
#pragma unroll 2
                for (int c = lane; c < D4; c += 32) {
                    const float4 qq = q4[c];
                    float4 xv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        xv[u] = __ldg(reinterpret_cast<const float4 *>(A.X + (int64_t)pj[u] * D) + c);
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        float df = qq.x - xv[u].x;
                        acc[u] = fmaf(df, df, acc[u]);
                        df = qq.y - xv[u].y;
                        acc[u] = fmaf(df, df, acc[u]);
                        df = qq.z - xv[u].z;
                        acc[u] = fmaf(df, df, acc[u]);
                        df = qq.w - xv[u].w;
                        acc[u] = fmaf(df, df, acc[u]);
                    }
                }
            } else {
                for (int c = lane; c < D; c += 32) {
                    const float qq = qv[c];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const float df = qq - __ldg(A.X + (int64_t)pj[u] * D + c);
                        acc[u] = fmaf(df, df, acc[u]);
                    }
                }
            }
            const int u = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
            const bool own = (lane & 3) == 0 && b0 + u < nr;
            const int p = __shfl_sync(FULL, my, (b0 + u) & 31);
            float dist;
            if constexpr (U8)
                dist = (float)(nq8 + (int)A.nx8[p] - 2 * dot8);
            else
                dist = warp_sum8(acc, lane);
            const bool cand = own && pair_less(dist, p, thr_d, thr_j);
            const unsigned m = __ballot_sync(FULL, cand);
            if (m) {
                if (cand) {
                    const int pos = fill + __popc(m & ((1u << lane) - 1u));
                    bd[pos] = dist;
                    bj[pos] = p;
                }
                fill += __popc(m);
                sorted = false;
                __syncwarp();
                if (fill + 8 > FD_BUF) sort_cut();
            }
        }
        if (!sorted) sort_cut();
        for (int u = lane; u < k; u += 32) {
            A.idx_out[row * k + u] = bj[u];
            A.d2_out[row * k + u] = bd[u];
        }
        __syncwarp();
    }
}

size_t fq_smem_bytes(int D, int qcap, bool qb) {
    return FQ_WARPS * ((size_t)((qcap + 31) >> 5) * 32 * 8 +
                       (qb ? (size_t)((D + 15) & ~15) : (((size_t)D * 4 + 15) & ~size_t(15))));
}

size_t fd_warp_bytes(int D) { return (size_t)((D + 3) & ~3) * 4 + FD_BUF * 8; }

template <int MODE, int QP>
atsne_status fd_launch_t(const FdArgs &a, int warps, cudaStream_t stream) {
    const size_t smem = warps * fd_warp_bytes(a.D);
    cudaError_t e = cudaFuncSetAttribute(forest_dist_kernel<MODE, QP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "forest distances attribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, forest_dist_kernel<MODE, QP>, warps * 32, smem);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    const int grid = (int)hmin((int64_t)per_sm * num_sms(), ceil_div(a.nw, warps));
    return launch_kernel(MODE == FD_U8 ? "forest_dist_u8" : "forest_dist", forest_dist_kernel<MODE, QP>, grid,
                         warps * 32, smem, stream, a);
}

int64_t fq_mark_cap(int k, int checks, int leaf_size) {
    const int64_t need = checks > k ? checks : k;
    return need + leaf_size + k + 1;
}
int64_t fq_chunk(int64_t nq, int64_t mark_cap) {
    int64_t c = FQ_MARK_BUDGET / (mark_cap * 4) / FQ_SEED_GAP * FQ_SEED_GAP;
    if (c < FQ_SEED_GAP) c = FQ_SEED_GAP;
    return nq < c ? (nq > 0 ? nq : 1) : c;
}

struct FqU8 {
    uint8_t *xu8 = nullptr;
    uint32_t *nx8 = nullptr;
    unsigned *bad = nullptr;
    int Dp16 = 0;
};
// Byte rows are used up to D = 2048 (16-byte pieces per lane in registers;
// exact int32 distances).
bool fq_u8_ok(int D) { return D <= 32 * 16 * FD_U8_PIECES; }

// Workspace layout of one search (sizing when c has no base).
size_t fq_workspace(Carver &c, int64_t N, int D, int64_t nq, int k, int checks, int leaf_size, FqArgs *ws_out,
                    FqU8 *u8_out) {
    FqArgs a{};
    a.words = (N + 31) / 32;
    a.mark_cap = fq_mark_cap(k, checks, leaf_size);
    a.chunk = fq_chunk(nq, a.mark_cap);
    a.seen = c.take<uint32_t>((size_t)FQ_MAX_SLOTS * a.words);
    a.marked = c.take<int32_t>((size_t)a.chunk * a.mark_cap);
    a.n_marked = c.take<int32_t>((size_t)a.chunk);
    a.next_query = c.take<int>(1);
    a.kseed = c.take<float>((size_t)(nq / FQ_SEED_GAP) + 2);
    FqU8 u{};
    if (fq_u8_ok(D)) {
        u.Dp16 = (D + 15) & ~15;
        u.xu8 = c.take<uint8_t>((size_t)N * u.Dp16);
        u.nx8 = c.take<uint32_t>((size_t)N);
        u.bad = c.take<unsigned>(1);
    }
    if (ws_out) *ws_out = a;
    if (u8_out) *u8_out = u;
    return c.bytes();
}

}  // namespace

size_t forest_query_workspace(Carver &c, int64_t N, int D, int64_t nq, int k, int checks, int leaf_size,
                              void *ws_out) {
    return fq_workspace(c, N, D, nq, k, checks, leaf_size, static_cast<FqArgs *>(ws_out), nullptr);
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
    FqU8 u8;
    fq_workspace(c, f.N, f.D, nq, k, checks, f.leaf_size, &a, &u8);
    if (c.bytes() > ws_bytes) return set_error(ATSNE_ENOMEM, "forest query: workspace too small");
    if (nq == 0) return ATSNE_OK;
    const size_t smem = fq_smem_bytes(f.D, qcap, false);
    if (smem > 227 * 1024)
        return set_error(ATSNE_EUNSUPPORTED,
                         "forest query: queue_cap %d with D=%d needs %zu B of shared memory", qcap, f.D,
                         smem);
    const int fd_warps = (int)hmin(FD_MAX_WARPS, (int64_t)(227 * 1024 / fd_warp_bytes(f.D)));
    if (fd_warps < 1)
        return set_error(ATSNE_EUNSUPPORTED, "forest query: rows of D=%d do not fit in shared memory", f.D);
    const size_t smem_b = fq_smem_bytes(f.D, qcap, true);
    auto grid_of = [&](auto kern, size_t sm, int &grid) -> cudaError_t {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (err != cudaSuccess) return err;
        int per_sm = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FQ_WARPS * 32, sm);
        if (err != cudaSuccess || per_sm < 1) per_sm = 1;
        grid = (int)hmin(hmin((int64_t)per_sm * num_sms(), FQ_MAX_SLOTS / FQ_WARPS),
                         ceil_div(hmin(nq, a.chunk), FQ_WARPS));
        return cudaSuccess;
    };
    int grid = 0, grid_b = 0;
    cudaError_t e = grid_of(forest_traverse_kernel<false>, smem, grid);
    if (e == cudaSuccess && u8.xu8) e = grid_of(forest_traverse_kernel<true>, smem_b, grid_b);
    if (e != cudaSuccess) return cuda_error(e, "forest query attribute");
    const int grid_max = grid > grid_b ? grid : grid_b;
    e = cudaMemsetAsync(a.seen, 0, sizeof(uint32_t) * (size_t)grid_max * FQ_WARPS * a.words, stream);
    if (e == cudaSuccess)  // 0xff bytes: NaN, a seed not yet searched
        e = cudaMemsetAsync(a.kseed, 0xff, sizeof(float) * (size_t)(nq / FQ_SEED_GAP + 2), stream);
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
    a.ofs_stride = f.ofs_stride;
    a.qlist = qlist;
    a.evaluated_out = evaluated_out;
    a.xu8 = u8.xu8;
    a.u8_bad = u8.bad;
    a.Dp16 = u8.Dp16;
    a.status = device_status_word();
    FdArgs b;
    b.X = X;
    b.D = f.D;
    b.k = k;
    b.list_mode = qlist != nullptr;
    b.marked = a.marked;
    b.n_marked = a.n_marked;
    b.mark_cap = a.mark_cap;
    b.idx_out = idx_out;
    b.d2_out = d2_out;
    b.xu8 = u8.xu8;
    b.nx8 = u8.nx8;
    b.u8_bad = u8.bad;
    b.Dp16 = u8.Dp16;
    if (u8.xu8) {
        e = cudaMemsetAsync(u8.bad, 0, sizeof(unsigned), stream);
        if (e != cudaSuccess) return cuda_error(e, "forest query memset");
        ATSNE_TRY(u8_copy_launch("forest_u8_prep", X, f.N, f.D, u8.Dp16, u8.xu8, u8.nx8, u8.bad, stream));
    }
    const bool vec = (f.D & 3) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
    for (int64_t w0 = 0; w0 < nq; w0 += a.chunk) {
        a.w0 = b.w0 = w0;
        a.nw = b.nw = hmin(a.chunk, nq - w0);
        e = cudaMemsetAsync(a.next_query, 0, sizeof(int), stream);
        if (e != cudaSuccess) return cuda_error(e, "forest query memset");
        atsne_status st = launch_kernel("forest_traverse", forest_traverse_kernel<false>, grid, FQ_WARPS * 32,
                                        smem, stream, a);
        if (st == ATSNE_OK && u8.xu8)
            st = launch_kernel("forest_traverse_u8", forest_traverse_kernel<true>, grid_b, FQ_WARPS * 32, smem_b,
                               stream, a);
        if (st != ATSNE_OK) return st;
        // the FP32 and byte instantiations; the prep kernel's finding picks one
        st = vec ? fd_launch_t<FD_F32V, 1>(b, fd_warps, stream) : fd_launch_t<FD_F32, 1>(b, fd_warps, stream);
        if (st != ATSNE_OK) return st;
        if (b.xu8) {
            st = b.Dp16 <= 32 * 16 * 2 ? fd_launch_t<FD_U8, 2>(b, fd_warps, stream)
                                       : fd_launch_t<FD_U8, FD_U8_PIECES>(b, fd_warps, stream);
            if (st != ATSNE_OK) return st;
        }
    }
    return ATSNE_OK;
}

}  // namespace atsne
