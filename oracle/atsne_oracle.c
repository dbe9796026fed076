/*
 * FP64 CPU oracle for the A-tSNE high-dimensional similarity path
 * (Pezzotti et al., "Approximated and User Steerable tSNE for Progressive
 * Visual Analytics").
 *
 * TEST INFRASTRUCTURE ONLY. This is the plain, slow restatement of the method
 * that the GPU library is checked against. Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg load it. It shares no code,
 * header, table or helper with the CUDA library, and the library never calls
 * it.
 *
 * Functions and the passage each one follows:
 *   oracle_knn_exact     Eq. 8 (Sec. 3.1): the K = floor(3 mu) nearest points
 *   oracle_calibrate     Eq. 3 and Eq. 4 (Sec. 3) over the kNN support of Eq. 8
 *   oracle_symmetrize    Eq. 2 and its split form Eq. 10 (Sec. 3, Sec. 4.3)
 *   oracle_forest_build  Sec. 4.2: T randomized KD-trees, each split on a
 *                        random dimension among the V of highest variance
 *   oracle_forest_query  Sec. 4.2: one priority queue across the forest,
 *                        ordered by distance to the decision boundary, stopped
 *                        after a budget of evaluated points ("checks")
 *   oracle_refine        Sec. 4.3 and Sec. 5.1.1: exact neighbourhood of the
 *                        selected points, new Gaussian, rho_i = 1
 *   oracle_precision     Eq. 9 (Sec. 4.1)
 *   oracle_kde           Eq. 12, Eq. 13 and the approximation map of Sec. 5.2.2
 *   oracle_knn_cross     Eq. 8 across two point sets (insertion, Sec. 5.3.1)
 *   oracle_delete        Sec. 5.3.2: points leave every neighbourhood, rho_i
 *                        falls by 1/k per point removed, rows renumbered
 *   oracle_forest_insert Sec. 5.3.1: a new point joins the forest by a descent
 *                        of every tree to a leaf
 *   oracle_forest_delete Sec. 5.3.2: a deleted point leaves every tree
 *   oracle_insert        Eq. 11 (Sec. 5.3.1): new points enter the existing
 *                        neighbourhoods they fall inside
 *
 * Readings taken where the paper is silent are stated at each function.
 * Compile with -ffp-contract=off: the forest's float decisions (split value,
 * queue key) are specified as separately rounded float operations.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Sorted bounded list of the k best (distance, index) pairs.               */
/* Order: distance ascending, then index ascending (the tie rule).          */
/* ------------------------------------------------------------------------ */
static int pair_less(double da, int32_t ja, double db, int32_t jb)
{
    return (da < db) || (da == db && ja < jb);
}

static void best_insert(double *bd, int32_t *bj, int k, int *cnt, double d, int32_t j)
{
    int pos;
    if (*cnt == k) {
        if (!pair_less(d, j, bd[k - 1], bj[k - 1])) return;
        pos = k - 1;
    } else {
        pos = (*cnt)++;
    }
    while (pos > 0 && pair_less(d, j, bd[pos - 1], bj[pos - 1])) {
        bd[pos] = bd[pos - 1];
        bj[pos] = bj[pos - 1];
        --pos;
    }
    bd[pos] = d;
    bj[pos] = j;
}

static double sq_dist(const float *a, const float *b, int32_t D)
{
    double s = 0.0;
    for (int32_t t = 0; t < D; ++t) {
        double diff = (double)a[t] - (double)b[t];
        s += diff * diff;
    }
    return s;
}

/*
 * Exact kNN, Eq. 8 (Sec. 3.1). For every query i (all rows when queries is
 * NULL, else the S listed rows) the k points j != i with the smallest
 * ||x_i - x_j||^2, computed by direct differences in FP64, listed in
 * ascending (distance, index) order. Exact duplicates (distance 0) are
 * ordinary neighbours; only j == i is excluded (the k != i of Eq. 3).
 * Returns 0 on success, 1 on bad arguments.
 */
int oracle_knn_exact(const float *X, int64_t N, int32_t D, const int32_t *queries,
                     int64_t S, int32_t k, int32_t *idx_out, double *d2_out)
{
    if (!X || !idx_out || !d2_out || N < 2 || D < 1 || k < 1 || (int64_t)k > N - 1) return 1;
    int64_t Q = queries ? S : N;
    if (queries)
        for (int64_t s = 0; s < S; ++s)
            if (queries[s] < 0 || queries[s] >= N) return 1;
#pragma omp parallel for schedule(dynamic, 2)
    for (int64_t s = 0; s < Q; ++s) {
        int64_t i = queries ? (int64_t)queries[s] : s;
        double *bd = d2_out + s * k;
        int32_t *bj = idx_out + s * k;
        int cnt = 0;
        const float *xi = X + i * D;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            best_insert(bd, bj, k, &cnt, sq_dist(xi, X + j * D, D), (int32_t)j);
        }
    }
    return 0;
}

/*
 * Gaussian bandwidth by bisection, Eq. 3 and Eq. 4 (Sec. 3), with the sum of
 * Eq. 3's denominator taken over the neighbourhood N_i only (reading of
 * Eq. 8: the rows of the sparse P_{j|i} must sum to one).
 *
 * Work with beta = 1/(2 sigma^2). For a row with distances d_1..d_k let
 * s_j = d_j - min_l d_l (the common factor exp(-beta min d) cancels between
 * numerator and denominator of Eq. 3, so P is unchanged in exact arithmetic).
 * With w_j = exp(-beta s_j), Z = sum w_j, p_j = w_j / Z the entropy in nats is
 *     H = ln Z + beta * sum_j p_j s_j,
 * and Eq. 4's 2^{H_2} = mu is H = ln mu. H decreases in beta, so bisection:
 * start beta = 1, lo = 0, hi = +inf; if H > ln mu raise beta (double it while
 * hi is infinite, else midpoint), otherwise lower it to the midpoint with lo.
 * Stop when |H - ln mu| < tol or after max_iter evaluations; the outputs are
 * the p_j, beta and exp(H) of the last evaluation.
 * A distance of +inf marks an absent neighbour (a neighbourhood left with
 * fewer than k points by a deletion, Sec. 5.3.2): it is outside N_i, so it
 * takes no part in the sums and gets p = 0. A row with no neighbour at all
 * gets p = 0, beta = 0, perplexity 0 and no iteration.
 */
int oracle_calibrate(const double *d2, int64_t rows, int32_t k, double perplexity, double tol,
                     int32_t max_iter, double *P_out, double *beta_out, double *perp_out,
                     int32_t *iters_out)
{
    if (!d2 || !P_out || rows < 0 || k < 1 || !(perplexity > 0.0) || max_iter < 1) return 1;
    const double target = log(perplexity);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < rows; ++r) {
        const double *d = d2 + r * k;
        double *p = P_out + r * k;
        double dmin = INFINITY;
        int32_t present = 0;
        for (int32_t j = 0; j < k; ++j) {
            if (d[j] < dmin) dmin = d[j];
            present += !isinf(d[j]);
        }
        if (present > 0 && (double)present <= perplexity) {
            /* H over n present neighbours is at most log n, attained only at
             * beta = 0: the target log(perplexity) >= log n is met in the
             * limit beta -> 0, the uniform distribution over N_i */
            for (int32_t j = 0; j < k; ++j) p[j] = isinf(d[j]) ? 0.0 : 1.0 / present;
            if (beta_out) beta_out[r] = 0.0;
            if (perp_out) perp_out[r] = (double)present;
            if (iters_out) iters_out[r] = 0;
            continue;
        }
        if (isinf(dmin)) {  /* no neighbour */
            for (int32_t j = 0; j < k; ++j) p[j] = 0.0;
            if (beta_out) beta_out[r] = 0.0;
            if (perp_out) perp_out[r] = 0.0;
            if (iters_out) iters_out[r] = 0;
            continue;
        }
        double beta = 1.0, lo = 0.0, hi = INFINITY, H = 0.0, Z = 0.0;
        int32_t it;
        for (it = 1;; ++it) {
            double ws = 0.0;
            Z = 0.0;
            for (int32_t j = 0; j < k; ++j) {
                if (isinf(d[j])) {  /* absent */
                    p[j] = 0.0;
                    continue;
                }
                double s = d[j] - dmin;
                double w = exp(-beta * s);
                p[j] = w;
                Z += w;
                ws += w * s;
            }
            H = log(Z) + beta * ws / Z;
            if (fabs(H - target) < tol || it >= max_iter) break;
            if (H > target) {
                lo = beta;
                beta = isinf(hi) ? 2.0 * beta : 0.5 * (beta + hi);
            } else {
                hi = beta;
                beta = 0.5 * (lo + beta);
            }
        }
        for (int32_t j = 0; j < k; ++j) p[j] /= Z;
        if (beta_out) beta_out[r] = beta;
        if (perp_out) perp_out[r] = exp(H);
        if (iters_out) iters_out[r] = it;
    }
    return 0;
}

/*
 * Symmetrisation, Eq. 2 written in the split form of Eq. 10 (Sec. 4.3):
 * every stored conditional p_{j|i} (j in N_i) contributes p_{j|i}/(2N) to both
 * p_ij and p_ji. Emit the 2Nk contributions, sort them by (row, column) and
 * add the ones that land on the same entry. Output is CSR with ascending
 * columns; there is no diagonal because j != i.
 */
typedef struct {
    int64_t r;
    int32_t c;
    double v;
} trip_t;

static int trip_cmp(const void *a, const void *b)
{
    const trip_t *x = (const trip_t *)a, *y = (const trip_t *)b;
    if (x->r != y->r) return x->r < y->r ? -1 : 1;
    if (x->c != y->c) return x->c < y->c ? -1 : 1;
    return 0;
}

int oracle_symmetrize(const int32_t *idx, const double *P, int64_t N, int32_t k,
                      int64_t *row_ptr, int32_t *col, double *val, int64_t *nnz_out)
{
    if (!idx || !P || !row_ptr || !col || !val || N < 1 || k < 1) return 1;
    int64_t M = 0;
    trip_t *t = (trip_t *)malloc(sizeof(trip_t) * (size_t)(2 * N * (int64_t)k));
    if (!t) return 2;
    const double scale = 1.0 / (2.0 * (double)N);
    for (int64_t i = 0; i < N; ++i)
        for (int32_t a = 0; a < k; ++a) {
            int32_t j = idx[i * k + a];
            if (j == -1) continue;  /* an absent neighbour (Sec. 5.3.2) */
            if (j < 0 || j >= N || j == i) {
                free(t);
                return 1;
            }
            double v = P[i * k + a] * scale;
            t[M++] = (trip_t){i, j, v};
            t[M++] = (trip_t){j, (int32_t)i, v};
        }
    qsort(t, (size_t)M, sizeof(trip_t), trip_cmp);
    int64_t nnz = 0;
    for (int64_t i = 0; i <= N; ++i) row_ptr[i] = 0;
    for (int64_t m = 0; m < M; ++m) {
        if (nnz > 0 && t[m].r == t[m - 1].r && t[m].c == t[m - 1].c) {
            val[nnz - 1] += t[m].v;
        } else {
            col[nnz] = t[m].c;
            val[nnz] = t[m].v;
            row_ptr[t[m].r + 1]++;
            nnz++;
        }
    }
    for (int64_t i = 0; i < N; ++i) row_ptr[i + 1] += row_ptr[i];
    free(t);
    if (nnz_out) *nnz_out = nnz;
    return 0;
}

/*
 * Precision, Eq. 9 (Sec. 4.1): rho_i = |N^A_i intersect N_i| / |N_i| with
 * |N_i| = k, and rho = mean_i rho_i.
 */
int oracle_precision(const int32_t *idx_a, const int32_t *idx_e, int64_t rows, int32_t k,
                     double *rho_i, double *rho_mean)
{
    if (!idx_a || !idx_e || rows < 0 || k < 1) return 1;
    double total = 0.0;
    for (int64_t r = 0; r < rows; ++r) {
        int64_t hits = 0;
        for (int32_t a = 0; a < k; ++a)
            for (int32_t e = 0; e < k; ++e)
                if (idx_a[r * k + a] >= 0 && idx_a[r * k + a] == idx_e[r * k + e]) {
                    hits++;
                    break;
                }
        double v = (double)hits / (double)k;
        if (rho_i) rho_i[r] = v;
        total += v;
    }
    if (rho_mean) *rho_mean = rows > 0 ? total / (double)rows : 0.0;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Randomized KD-forest (Sec. 4.2)                                          */
/* ------------------------------------------------------------------------ */

/*
 * SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the c-th output (c >= 1) of the stream seeded with
 * `seed` is mix(seed + c * 0x9E3779B97F4A7C15). Used as a counter-based
 * generator so that the random split choice of (tree, node) does not depend
 * on the order nodes are built in.
 */
uint64_t oracle_splitmix64_at(uint64_t seed, uint64_t c)
{
    uint64_t z = seed + c * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Depth of the implicit tree: the least h with ceil(N / 2^h) <= leaf_size. */
int32_t oracle_forest_depth(int64_t N, int32_t leaf_size)
{
    int32_t h = 0;
    while (h < 62 && ((N + ((int64_t)1 << h) - 1) >> h) > leaf_size) ++h;
    return h;
}

/*
 * Leaf boundaries of the implicit tree: a node holding n points gives the
 * first ceil(n/2) (in split order) to its left child and the rest to its
 * right child, so every node's segment of the permutation depends on N only.
 * ofs has 2^h + 1 entries; leaf m covers [ofs[m], ofs[m+1]).
 */
int oracle_forest_leaf_offsets(int64_t N, int32_t h, int64_t *ofs)
{
    if (!ofs || h < 0 || h > 40) return 1;
    int64_t L = (int64_t)1 << h;
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(L + 1));
    if (!tmp) return 2;
    ofs[0] = 0;
    ofs[1] = N;
    for (int32_t l = 0; l < h; ++l) {
        int64_t n_nodes = (int64_t)1 << l;
        for (int64_t m = 0; m < n_nodes; ++m) {
            int64_t lo = ofs[m], hi = ofs[m + 1];
            tmp[2 * m] = lo;
            tmp[2 * m + 1] = lo + (hi - lo + 1) / 2;
        }
        tmp[2 * n_nodes] = N;
        memcpy(ofs, tmp, sizeof(int64_t) * (size_t)(2 * n_nodes + 1));
    }
    free(tmp);
    return 0;
}

typedef struct {
    float v;
    int32_t p;
} vp_t;

static int vp_cmp(const void *a, const void *b)
{
    const vp_t *x = (const vp_t *)a, *y = (const vp_t *)b;
    if (x->v < y->v) return -1;
    if (x->v > y->v) return 1;
    return (x->p > y->p) - (x->p < y->p);
}

typedef struct {
    double s;
    int32_t d;
} vd_t;

/* Higher spread first, then lower dimension index. */
static int vd_cmp(const void *a, const void *b)
{
    const vd_t *x = (const vd_t *)a, *y = (const vd_t *)b;
    if (x->s > y->s) return -1;
    if (x->s < y->s) return 1;
    return (x->d > y->d) - (x->d < y->d);
}

/*
 * Build T randomized KD-trees (Sec. 4.2). Readings of what the paper leaves
 * open:
 *  - spread of dimension d over a node's n points is ranked by
 *    n * sum x^2 - (sum x)^2 (n^2 times the variance), sums in FP64 over the
 *    node's points in permutation order; the V dimensions of largest spread
 *    (ties to the lower index) are the candidates;
 *  - the split dimension is candidate r mod min(V, D), r = SplitMix64 output
 *    number (t * 2^32 + node + 1) of `seed`;
 *  - the node's points are sorted by (value along that dimension, point
 *    index); the first ceil(n/2) go left. The split value is the float
 *    midpoint 0.5f * (a + b) of the last left and first right value; a node
 *    with fewer than two points gets +inf (every query goes left);
 *  - trees are level-ordered: node v has children 2v+1, 2v+2; internal nodes
 *    are 0 .. 2^h - 2, leaf m is node 2^h - 1 + m.
 * Outputs: split_dim[T][2^h - 1], split_val[T][2^h - 1], perm[T][N] (the
 * points in leaf order), leaf_ofs[2^h + 1] (shared by all trees).
 */
int oracle_forest_build(const float *X, int64_t N, int32_t D, int32_t T, int32_t V,
                        int32_t leaf_size, uint64_t seed, int32_t *split_dim, float *split_val,
                        int32_t *perm, int64_t *leaf_ofs)
{
    if (!X || N < 1 || D < 1 || T < 1 || V < 1 || leaf_size < 1 || !split_dim || !split_val ||
        !perm || !leaf_ofs)
        return 1;
    const int32_t h = oracle_forest_depth(N, leaf_size);
    if (oracle_forest_leaf_offsets(N, h, leaf_ofs)) return 2;
    const int64_t n_internal = ((int64_t)1 << h) - 1;
    const int32_t nV = V < D ? V : D;
    int rc = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t t = 0; t < T; ++t) {
        int32_t *pt = perm + (int64_t)t * N;
        for (int64_t p = 0; p < N; ++p) pt[p] = (int32_t)p;
        double *s1 = (double *)malloc(sizeof(double) * (size_t)D);
        double *s2 = (double *)malloc(sizeof(double) * (size_t)D);
        vd_t *rank = (vd_t *)malloc(sizeof(vd_t) * (size_t)D);
        vp_t *buf = (vp_t *)malloc(sizeof(vp_t) * (size_t)N);
        if (!s1 || !s2 || !rank || !buf) {
#pragma omp atomic write
            rc = 2;
        } else {
            for (int32_t l = 0; l < h; ++l) {
                for (int64_t m = 0; m < ((int64_t)1 << l); ++m) {
                    const int64_t v = ((int64_t)1 << l) - 1 + m;
                    const int64_t lo = leaf_ofs[m << (h - l)];
                    const int64_t hi = leaf_ofs[(m + 1) << (h - l)];
                    const int64_t n = hi - lo;
                    for (int32_t d = 0; d < D; ++d) s1[d] = s2[d] = 0.0;
                    for (int64_t q = lo; q < hi; ++q) {
                        const float *x = X + (int64_t)pt[q] * D;
                        for (int32_t d = 0; d < D; ++d) {
                            double xv = (double)x[d];
                            s1[d] += xv;
                            s2[d] += xv * xv;
                        }
                    }
                    for (int32_t d = 0; d < D; ++d) {
                        rank[d].s = (double)n * s2[d] - s1[d] * s1[d];
                        rank[d].d = d;
                    }
                    qsort(rank, (size_t)D, sizeof(vd_t), vd_cmp);
                    uint64_t r = oracle_splitmix64_at(seed, ((uint64_t)t << 32) + (uint64_t)v + 1u);
                    const int32_t dim = rank[r % (uint64_t)nV].d;
                    for (int64_t q = lo; q < hi; ++q) {
                        buf[q - lo].v = X[(int64_t)pt[q] * D + dim];
                        buf[q - lo].p = pt[q];
                    }
                    qsort(buf, (size_t)n, sizeof(vp_t), vp_cmp);
                    for (int64_t q = lo; q < hi; ++q) pt[q] = buf[q - lo].p;
                    float sv = INFINITY;
                    if (n >= 2) {
                        const int64_t nl = (n + 1) / 2;
                        float a = buf[nl - 1].v, b = buf[nl].v;
                        sv = 0.5f * (a + b);
                    }
                    split_dim[(int64_t)t * n_internal + v] = dim;
                    split_val[(int64_t)t * n_internal + v] = sv;
                }
            }
        }
        free(s1);
        free(s2);
        free(rank);
        free(buf);
    }
    return rc;
}

/* Queue entry: (key, tree, node), ordered lexicographically. */
typedef struct {
    float key;
    int32_t tree;
    int64_t node;
} qent_t;

static int qent_less(const qent_t *a, const qent_t *b)
{
    if (a->key != b->key) return a->key < b->key;
    if (a->tree != b->tree) return a->tree < b->tree;
    return a->node < b->node;
}

/* Bounded queue kept as an ascending array (front = next to visit). When it
 * is full, a new entry replaces the current largest entry if it is smaller
 * than it and is dropped otherwise. */
typedef struct {
    qent_t *e;
    int64_t n, cap;
} pq_t;

static void pq_push(pq_t *q, qent_t x)
{
    if (q->n == q->cap) {
        if (!qent_less(&x, &q->e[q->n - 1])) return;
        q->n--;
    }
    int64_t pos = q->n++;
    while (pos > 0 && qent_less(&x, &q->e[pos - 1])) {
        q->e[pos] = q->e[pos - 1];
        --pos;
    }
    q->e[pos] = x;
}

static qent_t pq_pop(pq_t *q)
{
    qent_t x = q->e[0];
    memmove(q->e, q->e + 1, sizeof(qent_t) * (size_t)(q->n - 1));
    q->n--;
    return x;
}

/*
 * Forest search for the kNN of corpus points (Sec. 4.2). Readings:
 *  - one queue for all trees, key = float sum over the descent of the squared
 *    distance to each boundary passed, (q[dim] - split)^2, each addition and
 *    product rounded separately in float; ties by (tree, node);
 *  - first every tree is descended from its root in order 0..T-1, then
 *    entries are popped in key order, each popped node descended to a leaf;
 *    a descent pushes the far child of every node it passes (not when its
 *    key is +inf, which only happens for the empty right child of a node
 *    with fewer than two points);
 *  - every point of a reached leaf not yet seen by this query is evaluated
 *    (the query point itself counts as seen); "checks" is the budget of
 *    evaluated points, and the search stops at the end of the leaf in which
 *    the count of evaluated points reaches max(checks, k), or when the queue
 *    is empty;
 *  - the queue holds at most qcap entries (pq_push above);
 *  - the result is the k best evaluated points by (squared distance in FP64,
 *    index); should the queue run dry with fewer than k points evaluated the
 *    list is completed with the lowest-index points not yet seen.
 * No pruning by the current k-th distance is applied, so the visited order
 * does not depend on checks and a larger budget only extends it.
 */
/* State of one forest search. */
typedef struct {
    const float *X, *xq;
    int64_t N, n_internal;
    int32_t D, k;
    const int32_t *split_dim, *perm;
    const float *split_val;
    const int64_t *leaf_ofs;
    unsigned char *seen;
    pq_t *pq;
    double *bd;
    int32_t *bj;
    int cnt;
    int64_t evaluated;
    int64_t ofs_stride;  /* 0: one leaf-offset array for all trees; else per tree */
} search_t;

/* Descend from (tree, node, key) to a leaf, pushing the far child of every
 * node passed, then evaluate the leaf's unseen points. */
static void descend_and_scan(search_t *s, int32_t tr, int64_t v, float key)
{
    while (v < s->n_internal) {
        const int32_t dim = s->split_dim[(int64_t)tr * s->n_internal + v];
        const float sv = s->split_val[(int64_t)tr * s->n_internal + v];
        const float qd = s->xq[dim];
        const int64_t nearc = qd < sv ? 2 * v + 1 : 2 * v + 2;
        const int64_t farc = qd < sv ? 2 * v + 2 : 2 * v + 1;
        const float diff = qd - sv;
        const float sq = diff * diff;
        const float fk = key + sq;
        if (!isinf(fk)) {
            qent_t e = {fk, tr, farc};
            pq_push(s->pq, e);
        }
        v = nearc;
    }
    const int64_t m = v - s->n_internal;
    const int32_t *pt = s->perm + (int64_t)tr * s->N;
    const int64_t *lo = s->leaf_ofs + (int64_t)tr * s->ofs_stride;
    for (int64_t q = lo[m]; q < lo[m + 1]; ++q) {
        const int32_t p = pt[q];
        if (s->seen[p]) continue;
        s->seen[p] = 1;
        s->evaluated++;
        best_insert(s->bd, s->bj, s->k, &s->cnt, sq_dist(s->xq, s->X + (int64_t)p * s->D, s->D), p);
    }
}

/*
 * Forest search for the kNN of corpus points (Sec. 4.2). Readings:
 *  - one queue for all trees, key = float sum over the descent of the squared
 *    distance to each boundary passed, (q[dim] - split)^2, each product and
 *    addition rounded separately in float; ties by (tree, node);
 *  - first every tree is descended from its root in order 0..T-1, then
 *    entries are popped in key order, each popped node descended to a leaf;
 *    a descent pushes the far child of every node it passes (not when its
 *    key is +inf, which only happens for the empty right child of a node
 *    with fewer than two points);
 *  - every point of a reached leaf not yet seen by this query is evaluated
 *    (the query point itself counts as seen); "checks" is the budget of
 *    evaluated points, and the search stops at the end of the leaf in which
 *    the count of evaluated points reaches max(checks, k), or when the queue
 *    is empty;
 *  - the queue holds at most qcap entries (pq_push above);
 *  - the result is the k best evaluated points by (squared distance in FP64,
 *    index); should the queue run dry with fewer than k points evaluated the
 *    list is completed with the lowest-index points not yet seen.
 * No pruning by the current k-th distance is applied, so the visiting order
 * does not depend on checks and a larger budget only extends it.
 */
int oracle_forest_query_ex(const float *X, int64_t N, int32_t D, int32_t T, int32_t h,
                           const int32_t *split_dim, const float *split_val, const int32_t *perm,
                           const int64_t *leaf_ofs, int64_t ofs_stride, const int32_t *queries,
                           int64_t S, int32_t k, int32_t checks, int32_t qcap, int32_t *idx_out,
                           double *d2_out, int64_t *evaluated_out)
{
    if (!X || N < 2 || D < 1 || T < 1 || h < 0 || k < 1 || (int64_t)k > N - 1 || qcap < 1 ||
        !idx_out || !d2_out || !split_dim || !split_val || !perm || !leaf_ofs)
        return 1;
    const int64_t Q = queries ? S : N;
    if (queries)
        for (int64_t s = 0; s < S; ++s)
            if (queries[s] < 0 || queries[s] >= N) return 1;
    const int64_t need = checks > k ? checks : k;
    int rc = 0;
#pragma omp parallel
    {
        unsigned char *seen = (unsigned char *)calloc((size_t)N, 1);
        pq_t pq;
        pq.e = (qent_t *)malloc(sizeof(qent_t) * (size_t)qcap);
        pq.cap = qcap;
        if (!seen || !pq.e) {
#pragma omp atomic write
            rc = 2;
        } else {
#pragma omp for schedule(dynamic, 4)
            for (int64_t s = 0; s < Q; ++s) {
                const int64_t qi = queries ? (int64_t)queries[s] : s;
                search_t st = {X, X + qi * D, N, ((int64_t)1 << h) - 1, D, k,
                               split_dim, perm, split_val, leaf_ofs, seen, &pq,
                               d2_out + s * k, idx_out + s * k, 0, 0, ofs_stride};
                memset(seen, 0, (size_t)N);
                seen[qi] = 1;
                pq.n = 0;
                for (int32_t t = 0; t < T && st.evaluated < need; ++t)
                    descend_and_scan(&st, t, 0, 0.0f);
                while (st.evaluated < need && pq.n > 0) {
                    qent_t e = pq_pop(&pq);
                    descend_and_scan(&st, e.tree, e.node, e.key);
                }
                for (int64_t p = 0; st.cnt < k && p < N; ++p)
                    if (!seen[p]) {
                        seen[p] = 1;
                        st.evaluated++;
                        best_insert(st.bd, st.bj, k, &st.cnt, sq_dist(st.xq, X + p * D, D),
                                    (int32_t)p);
                    }
                if (evaluated_out) evaluated_out[s] = st.evaluated;
            }
        }
        free(seen);
        free(pq.e);
    }
    return rc;
}

int oracle_forest_query(const float *X, int64_t N, int32_t D, int32_t T, int32_t h,
                        const int32_t *split_dim, const float *split_val, const int32_t *perm,
                        const int64_t *leaf_ofs, const int32_t *queries, int64_t S, int32_t k,
                        int32_t checks, int32_t qcap, int32_t *idx_out, double *d2_out,
                        int64_t *evaluated_out)
{
    return oracle_forest_query_ex(X, N, D, T, h, split_dim, split_val, perm, leaf_ofs, 0, queries, S, k,
                                  checks, qcap, idx_out, d2_out, evaluated_out);
}

/*
 * Insertion into the forest, Sec. 5.3.1: the points N_old .. N_new - 1 of X
 * (rows appended to the corpus) are added to every tree. A point descends a
 * tree by the rule of the search (query value below the split value: left
 * child 2v + 1, else right child 2v + 2) to a leaf and joins that leaf's
 * bucket after the points already there, the new points in index order. The
 * split dimensions and values do not change (the paper updates the forest per
 * point in O(log N), without rebuilding).
 *  perm_in [T][N_old] and ofs_in [T][2^h + 1] (each tree its own leaf offsets,
 *  as buckets differ once points are added) -> perm_out [T][N_new], ofs_out.
 */
int oracle_forest_insert(const float *X, int64_t N_old, int64_t N_new, int32_t D, int32_t T, int32_t h,
                         const int32_t *split_dim, const float *split_val, const int32_t *perm_in,
                         const int64_t *ofs_in, int32_t *perm_out, int64_t *ofs_out)
{
    if (!X || N_old < 0 || N_new < N_old || D < 1 || T < 1 || h < 0 || !perm_out || !ofs_out ||
        (N_old > 0 && (!perm_in || !ofs_in)) || (h > 0 && (!split_dim || !split_val)))
        return 1;
    const int64_t L = (int64_t)1 << h, n_int = L - 1, B = N_new - N_old;
    int64_t *leaf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(B > 0 ? B : 1));
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
    if (!leaf || !cur) {
        free(leaf);
        free(cur);
        return 2;
    }
    for (int32_t t = 0; t < T; ++t) {
        const int64_t *oi = ofs_in ? ofs_in + (int64_t)t * (L + 1) : NULL;
        int64_t *oo = ofs_out + (int64_t)t * (L + 1);
        for (int64_t b = 0; b < B; ++b) {
            const float *x = X + (N_old + b) * D;
            int64_t v = 0;
            while (v < n_int) {
                const int32_t dim = split_dim[(int64_t)t * n_int + v];
                v = x[dim] < split_val[(int64_t)t * n_int + v] ? 2 * v + 1 : 2 * v + 2;
            }
            leaf[b] = v - n_int;
        }
        for (int64_t m = 0; m <= L; ++m) oo[m] = 0;
        for (int64_t m = 0; m < L; ++m) oo[m + 1] = oi ? oi[m + 1] - oi[m] : 0;
        for (int64_t b = 0; b < B; ++b) oo[leaf[b] + 1]++;
        for (int64_t m = 0; m < L; ++m) oo[m + 1] += oo[m];
        int32_t *po = perm_out + (int64_t)t * N_new;
        for (int64_t m = 0; m < L; ++m) {
            cur[m] = oo[m];
            if (oi)
                for (int64_t q = oi[m]; q < oi[m + 1]; ++q) po[cur[m]++] = perm_in[(int64_t)t * N_old + q];
        }
        for (int64_t b = 0; b < B; ++b) po[cur[leaf[b]]++] = (int32_t)(N_old + b);
    }
    free(leaf);
    free(cur);
    return 0;
}

/*
 * Deletion from the forest, Sec. 5.3.2: the listed points (del [R], distinct,
 * in [0, N)) leave every bucket; the remaining points keep their order and are
 * renumbered as the corpus rows are (j becomes j minus the number of deleted
 * points below j). Split dimensions and values do not change.
 *  perm_in [T][N], ofs_in [T][2^h + 1] -> perm_out [T][N - R], ofs_out.
 */
int oracle_forest_delete(int64_t N, int32_t T, int32_t h, const int32_t *perm_in, const int64_t *ofs_in,
                         const int32_t *del, int64_t R, int32_t *perm_out, int64_t *ofs_out)
{
    if (N < 0 || T < 1 || h < 0 || R < 0 || R > N || !perm_in || !ofs_in || !perm_out || !ofs_out ||
        (R > 0 && !del))
        return 1;
    const int64_t L = (int64_t)1 << h, n = N - R;
    int64_t *before = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
    unsigned char *dead = (unsigned char *)calloc((size_t)(N > 0 ? N : 1), 1);
    if (!before || !dead) {
        free(before);
        free(dead);
        return 2;
    }
    int rc = 0;
    for (int64_t r = 0; r < R; ++r) {
        if (del[r] < 0 || del[r] >= N || dead[del[r]]) rc = 1;
        else dead[del[r]] = 1;
    }
    if (!rc) {
        for (int64_t j = 0; j < N; ++j) before[j + 1] = before[j] + dead[j];
        for (int32_t t = 0; t < T; ++t) {
            const int64_t *oi = ofs_in + (int64_t)t * (L + 1);
            int64_t *oo = ofs_out + (int64_t)t * (L + 1);
            const int32_t *pi = perm_in + (int64_t)t * N;
            int32_t *po = perm_out + (int64_t)t * n;
            int64_t w = 0;
            oo[0] = 0;
            for (int64_t m = 0; m < L; ++m) {
                for (int64_t q = oi[m]; q < oi[m + 1]; ++q) {
                    const int32_t p = pi[q];
                    if (!dead[p]) po[w++] = (int32_t)(p - before[p]);
                }
                oo[m + 1] = w;
            }
        }
    }
    free(before);
    free(dead);
    return rc;
}

/*
 * Refinement of a selected subset (Sec. 4.3, Sec. 5.1.1): for every listed
 * point the exact neighbourhood (Eq. 8) against all N points, its Gaussian
 * (Eq. 3, Eq. 4) and rho_i = 1; rows not listed are left unchanged. The
 * state arrays are [N][k] (idx, d2, P) and [N] (beta, rho). A point listed
 * twice is written twice with the same values.
 */
int oracle_refine(const float *X, int64_t N, int32_t D, const int32_t *subset, int64_t S, int32_t k,
                  double perplexity, double tol, int32_t max_iter, int32_t *idx, double *d2,
                  double *P, double *beta, double *rho)
{
    if (!subset || S < 0 || !idx || !d2 || !P) return 1;
    if (S == 0) return 0;
    int32_t *ti = (int32_t *)malloc(sizeof(int32_t) * (size_t)(S * k));
    double *td = (double *)malloc(sizeof(double) * (size_t)(S * k));
    double *tp = (double *)malloc(sizeof(double) * (size_t)(S * k));
    double *tb = (double *)malloc(sizeof(double) * (size_t)S);
    int rc = (!ti || !td || !tp || !tb) ? 2 : 0;
    if (!rc) rc = oracle_knn_exact(X, N, D, subset, S, k, ti, td);
    if (!rc) rc = oracle_calibrate(td, S, k, perplexity, tol, max_iter, tp, tb, NULL, NULL);
    if (!rc) {
        for (int64_t s = 0; s < S; ++s) {
            const int64_t i = subset[s];
            memcpy(idx + i * k, ti + s * k, sizeof(int32_t) * (size_t)k);
            memcpy(d2 + i * k, td + s * k, sizeof(double) * (size_t)k);
            memcpy(P + i * k, tp + s * k, sizeof(double) * (size_t)k);
            if (beta) beta[i] = tb[s];
            if (rho) rho[i] = 1.0;
        }
    }
    free(ti);
    free(td);
    free(tp);
    free(tb);
    return rc;
}


/*
 * Deletion of points, Sec. 5.3.2. Each point of del (R distinct rows in
 * [0, N)) leaves every neighbourhood that holds it: the row keeps its other
 * entries in their order and ends with an absent entry (index -1, distance
 * +inf) per point removed, and rho_i falls by 1/k per point removed (not
 * below 0; the paper ignores the missing (K+1)-th neighbour instead of
 * searching it). The deleted rows go away: the remaining points keep their
 * order and are numbered 0..N-R-1 (X's rows and every index follow). Reading:
 * P_{j|i} is defined over N_i (Eq. 3, Eq. 4), so every remaining row's
 * Gaussian is calibrated again over its remaining neighbours. Arrays are
 * updated in place; *N_out = N - R. Returns 1 on an index out of range or
 * listed twice.
 */
int oracle_delete(float *X, int64_t N, int32_t D, const int32_t *del, int64_t R, int32_t k,
                  double perplexity, double tol, int32_t max_iter, int32_t *idx, double *d2, double *P,
                  double *beta, double *rho, int64_t *N_out)
{
    if (!X || N < 1 || D < 1 || k < 1 || R < 0 || (R > 0 && !del) || !idx || !d2 || !P) return 1;
    unsigned char *dead = (unsigned char *)calloc((size_t)N, 1);
    int64_t *newid = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    if (!dead || !newid) {
        free(dead);
        free(newid);
        return 2;
    }
    int rc = 0;
    for (int64_t r = 0; r < R && !rc; ++r) {
        if (del[r] < 0 || del[r] >= N || dead[del[r]]) rc = 1;
        else dead[del[r]] = 1;
    }
    if (!rc) {
        int64_t n = 0;
        for (int64_t i = 0; i < N; ++i) newid[i] = dead[i] ? -1 : n++;
        for (int64_t i = 0; i < N; ++i) {  /* newid[i] <= i: rows move down in order */
            if (dead[i]) continue;
            const int64_t ni = newid[i];
            memmove(X + ni * D, X + i * D, sizeof(float) * (size_t)D);
            int32_t c = 0, removed = 0;
            for (int32_t a = 0; a < k; ++a) {
                const int32_t j = idx[i * k + a];
                if (j >= 0 && dead[j]) {
                    removed++;
                    continue;
                }
                if (j < 0) continue;  /* already absent */
                idx[ni * k + c] = (int32_t)newid[j];
                d2[ni * k + c] = d2[i * k + a];
                c++;
            }
            for (; c < k; ++c) {
                idx[ni * k + c] = -1;
                d2[ni * k + c] = INFINITY;
            }
            if (rho) {
                const double v = rho[i] - (double)removed / (double)k;
                rho[ni] = v > 0.0 ? v : 0.0;
            }
        }
        *N_out = n;
        rc = oracle_calibrate(d2, n, k, perplexity, tol, max_iter, P, beta, NULL, NULL);
    }
    free(dead);
    free(newid);
    return rc;
}

/*
 * Density view of a 2-D embedding and its approximation map (Sec. 5.2), per
 * pixel p (centre x0 + (x + 0.5) pixel, y0 + (y + 0.5) pixel, an FP32 value
 * like the embedding's coordinates: fma(x + 0.5, pixel, x0) rounded once), with
 * G(d, h) = exp(-d^2 / (2 h^2)) / (2 pi h^2), the zero-mean Gaussian of
 * standard deviation h in the plane:
 *   f(p, h) = (1/N) sum_i G(|p - y_i|, h)                  Eq. 12
 *   s(p, h) = sum_{i in S} G / sum_i G                     Eq. 13
 *   a(p, h) = sum_i rho_i G / sum_i G                      Sec. 5.2.2
 *   alpha   = 1 - a^k                                      Sec. 5.2.2 (Magic Lens)
 * Reading: Eq. 13 and a(p,h) carry the normalisers 1/|S| and 1/sum rho_i; as
 * printed a would exceed 1 wherever the local precision beats the mean, which
 * the text rules out (a is between zero and one), and the fixed threshold 0.5
 * on s would depend on |S|/N. Both normalisers are read as 1/N, f's own, so s
 * is the selected share and a the precision-weighted mean of the kernel.
 * Empty pixels (no point within reach): s = 0, a = 1. A point farther than
 * cutoff * h from p is left out (cutoff = 0: none is). That test decides a
 * membership, so it is taken in the GPU kernel's precision (FP32: centre
 * fma(x + 0.5, pixel, x0), squared distance fma(dx, dx, dy * dy) against
 * (cutoff * h)^2, each operation rounded once); the sums are FP64, in point
 * order.
 */
int oracle_kde(const float *Y, int64_t N, const float *rho, const uint8_t *sel, double x0, double y0,
               double pixel, int32_t W, int32_t H, double h, double cutoff, double k, double *f,
               double *s, double *a, double *alpha)
{
    if (N < 1 || W < 1 || H < 1 || !(h > 0.0) || !(pixel > 0.0) || cutoff < 0.0) return 1;
    const float rf = (float)cutoff * (float)h;
    const float r2f = rf * rf;
    const double norm = 1.0 / (2.0 * 3.14159265358979323846 * h * h);
#pragma omp parallel for schedule(dynamic, 4)
    for (int32_t y = 0; y < H; ++y) {
        for (int32_t x = 0; x < W; ++x) {
            const float pxf = fmaf((float)x + 0.5f, (float)pixel, (float)x0);
            const float pyf = fmaf((float)y + 0.5f, (float)pixel, (float)y0);
            const double px = (double)pxf, py = (double)pyf;
            double F = 0.0, S = 0.0, R = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                if (cutoff > 0.0) {
                    const float dxf = pxf - Y[2 * i], dyf = pyf - Y[2 * i + 1];
                    const float dyy = dyf * dyf;
                    if (fmaf(dxf, dxf, dyy) > r2f) continue;
                }
                const double dx = px - (double)Y[2 * i], dy = py - (double)Y[2 * i + 1];
                const double d2 = dx * dx + dy * dy;
                const double g = norm * exp(-d2 / (2.0 * h * h));
                F += g;
                if (sel && sel[i]) S += g;
                R += (rho ? (double)rho[i] : 1.0) * g;
            }
            const int64_t o = (int64_t)y * W + x;
            f[o] = F / (double)N;
            s[o] = F > 0.0 ? S / F : 0.0;
            a[o] = F > 0.0 ? R / F : 1.0;
            alpha[o] = 1.0 - pow(a[o], k);
        }
    }
    return 0;
}


/*
 * The k nearest rows of Xc for each row of Xq (Eq. 8 with the query set apart
 * from the corpus, as insertion needs in Sec. 5.3.1): FP64 direct differences,
 * no point excluded, order (d^2, index).
 */
int oracle_knn_cross(const float *Xq, int64_t Nq, const float *Xc, int64_t Nc, int32_t D, int32_t k,
                     int32_t *idx, double *d2)
{
    if (k < 1 || k > Nc) return 1;
#pragma omp parallel for schedule(dynamic, 2)
    for (int64_t q = 0; q < Nq; ++q) {
        double *bd = d2 + q * k;
        int32_t *bj = idx + q * k;
        int cnt = 0;
        for (int64_t j = 0; j < Nc; ++j)
            best_insert(bd, bj, k, &cnt, sq_dist(Xq + q * D, Xc + j * D, D), (int32_t)j);
    }
    return 0;
}

/*
 * Insertion of new points into the existing neighbourhoods, Eq. 11 (Sec. 5.3.1).
 * X holds N_new rows; rows 0..N_old-1 carry the neighbourhoods idx/d2
 * ([N_old][k], each sorted by (d2, index); absent entries, index -1 and
 * distance +inf, come last). For row i, d_i^Max is the largest distance among
 * its present entries. A new point j (N_old <= j < N_new) enters N_i exactly
 * when d(i, j) < d_i^Max, strictly, with d in FP64 by direct differences. The
 * row then holds the k smallest of its present entries and the entering points
 * in the (d2, index) order: an entering point fills an absent entry while one
 * is left, and otherwise the farthest neighbour leaves. A tie with a listed
 * point goes to the listed point, whose index is smaller. A row with no
 * present entry has no d_i^Max and takes no point. changed[i] = 1 when the
 * row's list changed. rho_i is not an argument: insertion leaves it as it is.
 */
int oracle_insert(const float *X, int64_t N_old, int64_t N_new, int32_t D, int32_t k, int32_t *idx,
                  double *d2, uint8_t *changed)
{
    if (!X || N_old < 0 || N_new < N_old || D < 1 || k < 1 || (N_old > 0 && (!idx || !d2))) return 1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < N_old; ++i) {
        int32_t *ri = idx + i * k;
        double *rd = d2 + i * k;
        int cnt = 0;
        double dmax = -1.0;
        while (cnt < k && ri[cnt] >= 0) {
            if (rd[cnt] > dmax) dmax = rd[cnt];
            ++cnt;
        }
        int ch = 0;
        if (cnt > 0) {
            const float *xi = X + i * (int64_t)D;
            for (int64_t j = N_old; j < N_new; ++j) {
                const double d = sq_dist(xi, X + j * (int64_t)D, D);
                if (d < dmax) {
                    best_insert(rd, ri, k, &cnt, d, (int32_t)j);
                    ch = 1;
                }
            }
            for (int t = cnt; t < k; ++t) {
                ri[t] = -1;
                rd[t] = INFINITY;
            }
        }
        if (changed) changed[i] = (uint8_t)ch;
    }
    return 0;
}
