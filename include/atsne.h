/*
 * atsne.h -- C ABI of the GB300 (sm_103a) library for A-tSNE's high-dimensional
 * similarity matrix P (Pezzotti et al., "Approximated and User Steerable tSNE
 * for Progressive Visual Analytics").
 *
 * Conventions shared by every entry point:
 *  - Pointers named X, idx, d2, P_cond, beta, rho, row_ptr, col, val, nnz_dev,
 *    queries, subset, workspace and forest are DEVICE pointers owned by the
 *    caller. Arrays are dense and row-major. The library allocates no device
 *    memory: temporary storage comes from the caller's workspace, whose size
 *    atsne_workspace_bytes() returns (256-byte aligned base required).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). All work is
 *    enqueued on it; calls return without synchronising, except where noted.
 *  - Point indices are int32 (N <= 2^31 - 1); CSR row offsets are int64.
 *  - Return value: ATSNE_OK, or an error code with a message available from
 *    atsne_last_error() (thread-local). Argument errors are detected on the
 *    host before anything is enqueued. Problems found on the device
 *    (non-finite input, an expired bounded wait) set a device status word
 *    that atsne_check() reads.
 *  - kNN lists: row i of idx/d2 holds the k neighbours j != i of query i in
 *    ascending (squared distance, index) order; d2 is the FP32 squared
 *    Euclidean distance.
 */
#ifndef ATSNE_H
#define ATSNE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ATSNE_OK = 0,
    ATSNE_EINVAL = 1,       /* bad argument, or non-finite input found on the device */
    ATSNE_ENOMEM = 2,       /* workspace or output buffer too small */
    ATSNE_ECUDA = 3,        /* a CUDA runtime/driver call failed */
    ATSNE_ETIMEOUT = 4,     /* a bounded device-side wait expired */
    ATSNE_EUNSUPPORTED = 5  /* a valid request the library does not handle */
} atsne_status;

typedef enum { ATSNE_KNN_EXACT = 0, ATSNE_KNN_FOREST = 1 } atsne_knn_method;

/* Arithmetic of the exact path's distance contraction. FP32, BF16_RERANK and
 * FP32_CUDA_CORES return the exact kNN under FP32 direct-difference distances:
 * the tensor-core variants re-rank their candidates in FP32 and certify each
 * row (rows that cannot be certified are recomputed on the CUDA cores). The
 * two *_RERANK variants without a certificate are approximate. */
typedef enum {
    ATSNE_FP32 = 0,            /* tensor cores, 3 BF16 passes (hi.hi + hi.lo + lo.hi) */
    ATSNE_BF16_RERANK = 1,     /* tensor cores, 1 BF16 pass, rerank_k candidates per row */
    ATSNE_FP32_CUDA_CORES = 2, /* FP32 direct differences on the CUDA cores */
    ATSNE_FP8_RERANK = 3,      /* tensor cores, 1 FP8 (E4M3, per-row scale) pass; the
                                  rerank_k (default 4k, at most 512) best keys per row
                                  re-ranked in FP32, the k best returned: approximate,
                                  no certificate (measure recall against FP32) */
    ATSNE_BF16_RERANK_APPROX = 4 /* tensor cores, 1 BF16 pass; the rerank_k (default 4k,
                                  at most 512) best keys per row re-ranked in FP32, the
                                  k best returned: approximate, no certificate (on data
                                  whose BF16 error bound exceeds the neighbourhood's
                                  margin, BF16_RERANK sends most rows to the CUDA cores) */
} atsne_precision;

/* Operation codes for atsne_workspace_bytes(). */
typedef enum {
    ATSNE_OP_KNN = 0,
    ATSNE_OP_CALIBRATE = 1,
    ATSNE_OP_SYMMETRIZE = 2,
    ATSNE_OP_REFINE = 3,
    ATSNE_OP_FOREST_BUILD = 4,
    ATSNE_OP_FOREST_QUERY = 5,
    ATSNE_OP_REFINE_BATCH = 6, /* S = total entries of the concatenated selections */
    ATSNE_OP_KNN_CROSS = 7,    /* N = corpus rows, S = query rows */
    ATSNE_OP_KNN_CROSS_RADIUS = 8, /* as KNN_CROSS, with per-row radii */
    ATSNE_OP_DELETE = 9,           /* N = rows before the deletion, D, k */
    ATSNE_OP_TUNE_KNN = 10,        /* as ATSNE_OP_KNN: the largest candidate's workspace */
    ATSNE_OP_FOREST_UPDATE = 11    /* N = points the forest was built on, S = rows after an
                                      insertion / before a deletion */
} atsne_op;

/* Options of the kNN step. atsne_knn_opts_default() fills the defaults. */
typedef struct {
    int32_t method;        /* atsne_knn_method */
    int32_t precision;     /* atsne_precision (exact method) */
    int32_t trees;         /* forest: number of randomized KD-trees T (Sec. 4.2), default 4 */
    int32_t top_var_dims;  /* forest: V, split among the V highest-spread dims, default 5 */
    int32_t checks;        /* forest: budget of evaluated points ("leaves" L, Sec. 4.2) */
    int32_t leaf_size;     /* forest: maximum points per leaf, default 1 */
    int32_t queue_cap;     /* forest: capacity of the per-query priority queue; 0 (default)
                              = checks/2 rounded up to a power of two, within [256, 4096] */
    int32_t rerank_k;      /* exact tensor path: candidates kept per row and column split
                              (0 = k + 38 for FP32, 2k for BF16; at most 4096) */
    uint64_t seed;         /* forest: seed of the counter-based split choice */
} atsne_knn_opts;

void atsne_knn_opts_default(atsne_knn_opts *opts);

/*
 * Bytes of workspace `op` needs. N = corpus rows, D = dimensions, k = neighbours,
 * S = number of listed queries/subset rows (0 = all N rows), opts may be NULL
 * (defaults) and is read for ATSNE_OP_KNN / FOREST_* / REFINE.
 */
size_t atsne_workspace_bytes(int32_t op, int64_t N, int32_t D, int32_t k, int64_t S,
                             const atsne_knn_opts *opts);

/*
 * k-nearest neighbours, Eq. 8 (Sec. 3.1); with method FOREST the approximate
 * neighbourhoods N^A_i of Sec. 4.1, found by the forest search of Sec. 4.2
 * (the forest is built in the workspace on every call; see atsne_forest_*).
 *  X        [N][D] fp32, finite.
 *  queries  NULL: every row i of X is a query, S ignored, outputs have N rows.
 *           else [S] int32 row indices into X; output row s belongs to
 *           queries[s]. A query never lists itself.
 *  k        1 <= k <= N - 1 (the paper uses k = floor(3 * perplexity)).
 *  idx_out  [rows][k] int32, d2_out [rows][k] fp32, sorted as described above.
 * The exact tensor path of all rows of a large set (N >= 65536, D <= 256) first
 * groups the points by nearest centroid and streams each row tile's own group
 * first; the workspace holds that order, and the lists are the same as without it.
 * Errors: EINVAL (sizes, NULLs, index out of range), ENOMEM (workspace), ECUDA.
 */
atsne_status atsne_knn(const float *X, int64_t N, int32_t D, const int32_t *queries, int64_t S,
                       int32_t k, const atsne_knn_opts *opts, int32_t *idx_out, float *d2_out,
                       void *workspace, size_t ws_bytes, void *stream);

/*
 * Gaussian bandwidths and conditional probabilities, Eq. 3 and Eq. 4 (Sec. 3)
 * over the kNN support of Eq. 8: for each row, beta = 1/(2 sigma^2) is found by
 * bisection so that exp(H) = perplexity (H in nats, equal to Eq. 4's base-2
 * form), and P_cond[r][j] = exp(-beta d2[r][j]) / sum_l exp(-beta d2[r][l]).
 *  d2         [rows][k] fp32 squared distances (any order; >= 0). +inf marks an
 *             absent neighbour (a row shortened by atsne_delete_rows): it takes
 *             no part in the sums and gets P 0. NaN or a negative value raises
 *             the device status.
 *  perplexity 0 < perplexity < k.   tol: stop when |H - ln perplexity| < tol
 *  (<= 0 selects 1e-5).  max_iter: bisection steps (<= 0 selects 200).
 *  P_cond_out [rows][k] fp32 (rows sum to 1), beta_out [rows] fp32 (may be NULL).
 * Rows whose target is unreachable (k equal distances, or at least
 * `perplexity` neighbours tied at the smallest distance) end at max_iter.
 * A row of n present neighbours with n <= perplexity (its entropy is at most
 * ln n, reached only at beta = 0) takes the bisection's limit: beta = 0 and
 * P = 1/n on the present entries; a row with none gets P 0 and beta 0.
 */
atsne_status atsne_calibrate_P(const float *d2, int64_t rows, int32_t k, float perplexity,
                               float tol, int32_t max_iter, float *P_cond_out, float *beta_out,
                               void *stream);

/*
 * Symmetrised joint probabilities, Eq. 2 in the split form of Eq. 10
 * (Sec. 4.3): p_ij = (p_{j|i} + p_{i|j}) / (2N) over the union of the kNN
 * patterns, as CSR with ascending columns and no diagonal.
 *  idx [N][k] int32 (row i: distinct j != i), P_cond [N][k] fp32.
 *  row_ptr [N+1] int64; col, val: capacity 2*N*k entries (the maximum nnz).
 *  nnz_dev: device int64 receiving nnz (= row_ptr[N]); may be NULL.
 * Errors: EINVAL, ENOMEM (workspace), ECUDA. Malformed idx (out of range or
 * self) sets the device status word (EINVAL from atsne_check()).
 */
atsne_status atsne_symmetrize(const int32_t *idx, const float *P_cond, int64_t N, int32_t k,
                              int64_t *row_ptr, int32_t *col, float *val, int64_t *nnz_dev,
                              void *workspace, size_t ws_bytes, void *stream);

/*
 * Refinement of a user selection, Sec. 4.3 and Sec. 5.1.1: for each listed
 * point the exact neighbourhood (Eq. 8, FP32 path) against all N points, its
 * Gaussian (Eq. 3-4) and rho_i = 1 (Sec. 4.3's per-point precision). Rows of
 * the state not listed are untouched; call atsne_symmetrize() afterwards to
 * rebuild P (Eq. 10 makes that a per-row update of the stored conditionals).
 *  subset [S] int32 in [0, N); duplicates allowed (same values written).
 *  idx/d2/P_cond [N][k], beta [N], rho [N] (beta and rho may be NULL): in/out.
 */
atsne_status atsne_refine_subset(const float *X, int64_t N, int32_t D, const int32_t *subset,
                                 int64_t S, int32_t k, float perplexity, int32_t *idx, float *d2,
                                 float *P_cond, float *beta, float *rho, void *workspace,
                                 size_t ws_bytes, void *stream);

/*
 * Refinement without device allocation. The paper has no counterpart: this is
 * atsne_refine_subset for callers that cannot allocate device memory when they
 * refine: a render or UI callback of an interactive view that must not stall
 * on cudaMalloc (which can synchronise the whole device), or a program whose
 * device-memory budget is fixed up front by another component. Instead of a
 * workspace it uses one fixed device array
 * inside the library (3 MiB + 8 KiB, held on every GPU that loads the library
 * until the process exits), so it accepts at most
 * ATSNE_REFINE_NOALLOC_MAX_ROWS selected rows and k <= ATSNE_REFINE_NOALLOC_MAX_K;
 * larger requests return ATSNE_ENOMEM with a message. Arguments, outputs and
 * results are those of atsne_refine_subset. The first call on a device (any
 * size, an empty selection included) looks up the array's address and the
 * library's status word (cudaGetSymbolAddress); make it before any stream
 * capture. All calls share the array: calls whose work may overlap on the GPU
 * race and must be ordered (one stream, or events).
 */
#define ATSNE_REFINE_NOALLOC_MAX_ROWS 2048
#define ATSNE_REFINE_NOALLOC_MAX_K 128
atsne_status atsne_refine_subset_noalloc(const float *X, int64_t N, int32_t D,
                                         const int32_t *subset, int64_t S, int32_t k,
                                         float perplexity, int32_t *idx, float *d2, float *P_cond,
                                         float *beta, float *rho, void *stream);

/*
 * Batched refinement, Sec. 4.3 and Sec. 5.1.1: many user selections (brushes,
 * lenses) refined at once. `lists` holds the selections concatenated, `total`
 * entries in [0, N) (device int32; duplicates within and across selections
 * allowed). A refined row depends only on X and its point, so this equals
 * atsne_refine_subset on every selection in any order, and each point of the
 * union is computed once: the union is formed on the device (bitmap, then an
 * ordered compaction) and refined by one exact kNN on the tensor cores, one
 * bisection and one row scatter.
 *  refined_count  device int64 receiving the size of the union (may be NULL).
 *  lists may be NULL when total is 0 (nothing is refined).
 * Stream-ordered, with no host synchronisation and no allocation: the call can
 * be recorded into a CUDA graph and replayed (its workspace and arguments are
 * then fixed). Workspace: atsne_workspace_bytes(ATSNE_OP_REFINE_BATCH, N, D, k,
 * total, NULL). Errors as atsne_refine_subset.
 */
atsne_status atsne_refine_batch(const float *X, int64_t N, int32_t D, const int32_t *lists,
                                int64_t total, int32_t k, float perplexity, int32_t *idx, float *d2,
                                float *P_cond, float *beta, float *rho, int64_t *refined_count,
                                void *workspace, size_t ws_bytes, void *stream);

/*
 * atsne_knn for listed rows (method EXACT) with optional per-row bounds:
 * hint_d2 [S] (device, or NULL) holds for each listed row an upper bound of
 * its k-th nearest squared distance, e.g. its current d2[i][k-1] when the row
 * lists k real points (Sec. 4.3's refinement of an approximate row). The
 * tensor-core filter starts from it instead of from +inf; the result is the
 * same exact neighbourhood whatever the bounds (a wrong one costs time only:
 * its rows fail the certificate and take the brute-force kernel).
 * Workspace: atsne_workspace_bytes(ATSNE_OP_KNN, N, D, k, S, opts).
 */
atsne_status atsne_knn_rows(const float *X, int64_t N, int32_t D, const int32_t *queries, int64_t S,
                            int32_t k, const atsne_knn_opts *opts, const float *hint_d2,
                            int32_t *idx_out, float *d2_out, void *workspace, size_t ws_bytes,
                            void *stream);

/*
 * Autotuner of the exact tensor-core kNN. Its tunable is the column split: the
 * corpus columns are cut into `splits` ranges, each (row tile, range) unit runs
 * its own streaming top-k, and the partial lists are merged. Fewer splits mean
 * fewer survivors to merge, more splits more units to fill the SMs with when
 * the rows are few. This call times the candidates (one split, and the counts
 * giving about 152 .. 8192 units) on the given problem (the kNN of
 * atsne_knn with method EXACT on the tensor cores: `queries` [S] or all N rows
 * when NULL), one warm-up and two timed runs each with CUDA events, and
 * records the fastest for the shape (N, D, rows, k, precision, rerank_k) in a
 * process-wide table. Every later call of that shape uses it: atsne_knn,
 * atsne_knn_rows, atsne_knn_cross (rows = query rows), atsne_refine_subset
 * (FP32, rows = S) and atsne_refine_batch (FP32, rows = min(N, total)). The
 * workspace such calls need depends on the recorded split, so size it after
 * tuning. Results do not depend on the split (every split yields the exact
 * neighbourhoods), only the time does.
 *  idx_out/d2_out [rows][k]: scratch, left holding the last run's result.
 *  splits_out, ms_out (host, may be NULL): the chosen split and its time.
 * Synchronises the stream (not for use inside a stream capture).
 * Workspace: atsne_workspace_bytes(ATSNE_OP_TUNE_KNN, N, D, k, S, opts).
 */
atsne_status atsne_tune_knn(const float *X, int64_t N, int32_t D, const int32_t *queries, int64_t S,
                            int32_t k, const atsne_knn_opts *opts, int32_t *idx_out, float *d2_out,
                            void *workspace, size_t ws_bytes, void *stream, int32_t *splits_out,
                            float *ms_out);
/* Forgets every split recorded by atsne_tune_knn (the rule applies again). */
atsne_status atsne_tune_clear(void);

/*
 * k nearest rows of Xc for each row of Xq, Eq. 8 across two point sets; no
 * point is excluded. Insertion (Sec. 5.3.1) uses it for the candidates of
 * the existing points among the inserted ones. Output row r belongs to
 * Xq[r], indices are rows of Xc, sorted by (d^2, index).
 *  Xq [Nq][D], Xc [Nc][D] fp32 (device, finite); 1 <= k <= Nc.
 *  opts: the exact method's precision (any atsne_precision). With radii the
 *        result is exact in every mode: the FP8 mode runs on the CUDA cores (its
 *        keys carry no error bound) and both BF16 modes certify every row.
 *  radius_d2  NULL, or [Nq] fp32 squared radii: row r then lists only the rows
 *             of Xc with d^2 < radius_d2[r] among its k nearest, the rest of
 *             the row (-1, +inf). With the radius of each existing point's
 *             farthest neighbour (its cached d_i^Max), this is Eq. 11's test
 *             (Sec. 5.3.1) in O(Nq * Nc) without a top-k per row; on the tensor
 *             cores it is exact (the filter is widened by the key error bound
 *             and every candidate is re-ranked in FP32).
 * Workspace: atsne_workspace_bytes(radius_d2 ? ATSNE_OP_KNN_CROSS_RADIUS :
 * ATSNE_OP_KNN_CROSS, Nc, D, k, Nq, opts).
 */
atsne_status atsne_knn_cross(const float *Xq, int64_t Nq, const float *Xc, int64_t Nc, int32_t D,
                             int32_t k, const atsne_knn_opts *opts, const float *radius_d2,
                             int32_t *idx_out, float *d2_out, void *workspace, size_t ws_bytes,
                             void *stream);

/*
 * Insertion of new points into existing neighbourhoods, Eq. 11 (Sec. 5.3.1),
 * for a batch: row i of idx/d2 ([rows][k], sorted by (d^2, index)) becomes the
 * k smallest of its list and its kc candidates (cand_idx + index_offset,
 * cand_d2: [rows][kc], sorted, e.g. atsne_knn_cross against the new points).
 * A candidate enters exactly when it is closer than the row's farthest
 * neighbour d_i^Max (ties go to the listed point, whose index is smaller), and
 * takes the place of the farthest ones. changed [rows] uint8 (may be NULL)
 * receives 1 for a row whose list changed. rho is not touched (insertion does
 * not lower the precision); re-run atsne_calibrate_P on the changed rows.
 */
/*
 * d_i^Max of Eq. 11 (Sec. 5.3.1) for each row: the squared distance of its
 * farthest neighbour in N_i as it stands, i.e. the largest finite entry of
 * d2[i] (entries of +inf are absent neighbours, left by atsne_delete_rows),
 * or +inf for a row with no neighbour left. With these radii
 * atsne_knn_cross finds the new points that enter each row.
 *  d2 [rows][k] fp32 (device), dmax_out [rows] fp32 (device).
 */
atsne_status atsne_row_dmax(const float *d2, int64_t rows, int32_t k, float *dmax_out, void *stream);

atsne_status atsne_merge_neighbors(int32_t *idx, float *d2, int64_t rows, int32_t k,
                                   const int32_t *cand_idx, const float *cand_d2, int32_t kc,
                                   int32_t index_offset, uint8_t *changed, void *stream);

/*
 * Deletion of points, Sec. 5.3.2, for a batch: rows ([R], distinct, in
 * [0, N)) leave the state. Every neighbourhood that holds one of them loses it:
 * the row keeps its other entries in order and ends with one absent entry
 * (index -1, distance +inf, P 0) per point removed, and rho falls by 1/k per
 * point removed (not below 0): the paper leaves the (K+1)-th neighbour
 * unsearched. The remaining points keep their order and become rows
 * 0..N-R-1: X ([N][D]), idx/d2/P_cond ([N][k]), beta and rho ([N]) are
 * compacted in place and every index renumbered. Every remaining row's Gaussian
 * is then calibrated again over its remaining neighbours (Eq. 3, Eq. 4 over
 * N_i; bisection as atsne_calibrate_P with its default tolerance), which the
 * absent entries do not enter. A later insertion fills an absent entry with a
 * new point closer than the row's farthest remaining neighbour (d_i^Max over
 * N_i as it stands, atsne_row_dmax). An index out of range or listed twice raises the device
 * status (ATSNE_EINVAL from atsne_check) and leaves the state unspecified.
 * Workspace: atsne_workspace_bytes(ATSNE_OP_DELETE, N, D, k, 0, NULL).
 */
atsne_status atsne_delete_rows(const int32_t *rows, int64_t R, float *X, int64_t N, int32_t D, int32_t k,
                               float perplexity, int32_t *idx, float *d2, float *P_cond, float *beta,
                               float *rho, void *workspace, size_t ws_bytes, void *stream);

/*
 * Writes S computed rows into the state: row rows[s] of idx/d2/P_cond ([N][k])
 * receives row s of ti/td/tp ([S][k]), beta[rows[s]] = tb[s] and rho[rows[s]] =
 * 1 (an exactly computed neighbourhood, Sec. 4.3). Entries of rows outside
 * [0, N) are skipped. beta, rho and tb may be NULL. This is the write step of a
 * refinement or an insertion, for callers that compute rows on one stream and
 * commit them on another.
 */
atsne_status atsne_commit_rows(const int32_t *rows, int64_t S, int64_t N, int32_t k, const int32_t *ti,
                               const float *td, const float *tp, const float *tb, int32_t *idx,
                               float *d2, float *P_cond, float *beta, float *rho, void *stream);

/*
 * Density-based view of a 2-D embedding and its approximation map, Sec. 5.2.
 * For each pixel p of a width x height image (pixel (x, y) centred at
 * (x0 + (x + 0.5) pixel, y0 + (y + 0.5) pixel), each an FP32 fused
 * multiply-add rounded once; rows y outermost) and the
 * Gaussian kernel G(d, h) = exp(-d^2 / (2 h^2)) / (2 pi h^2):
 *   f = (1/N) sum_i G(|p - y_i|, h)                 Eq. 12, kernel density
 *   s = sum_{i selected} G / sum_i G                Eq. 13, selected share
 *   a = sum_i rho_i G / sum_i G                     Sec. 5.2.2, approximation
 *   alpha = 1 - a^lens_k                            the Magic Lens (paper: k = 2)
 * Eq. 13 and a(p,h) are printed with the normalisers 1/|S| and 1/sum rho_i;
 * they are read as 1/N (the same as f's), which makes s and a the shares in
 * [0, 1] that the text describes. Where no point reaches a pixel, s = 0 and
 * a = 1. Points farther than cutoff * h from a pixel are left out of its sums;
 * cutoff = 0 keeps every point.
 *  Y         [N][2] fp32 embedding coordinates (device).
 *  rho       [N] fp32 per-point precision (Eq. 9), or NULL for all 1.
 *  selected  [N] uint8 (non-zero = selected), or NULL for none.
 *  f_out, s_out, a_out, alpha_out: [height][width] fp32 (device); any may be NULL.
 * No workspace. Errors: EINVAL (sizes, h <= 0, cutoff < 0, NULL Y), ECUDA.
 */
atsne_status atsne_kde_map(const float *Y, int64_t N, const float *rho, const uint8_t *selected,
                           float x0, float y0, float pixel, int32_t width, int32_t height, float h,
                           float cutoff, float lens_k, float *f_out, float *s_out, float *a_out,
                           float *alpha_out, void *stream);

/*
 * Precision of approximate neighbourhoods, Eq. 9 (Sec. 4.1):
 * rho_i = |N^A_i intersect N_i| / k. rho_i_out [rows] fp32; rho_sum_dev: device
 * double receiving sum_i rho_i (divide by rows for rho); either may be NULL.
 */
atsne_status atsne_knn_precision(const int32_t *idx_approx, const int32_t *idx_exact,
                                 int64_t rows, int32_t k, float *rho_i_out, double *rho_sum_dev,
                                 void *stream);

/*
 * Randomized KD-forest kept by the caller (Sec. 4.2), for building once and
 * searching many times. Layout of the `forest` buffer (all offsets in bytes
 * from its start, filled by atsne_forest_layout()):
 *   split_dim [trees][2^depth - 1] int32, split_val [trees][2^depth - 1] fp32,
 *   perm [trees][N] int32 (points in leaf order),
 *   leaf_ofs [2^depth + 1] int32 (leaf m holds perm[t][leaf_ofs[m] .. leaf_ofs[m+1])),
 *   leaf_pt [trees][2^depth] int32 (first point of each leaf, -1 if the leaf is empty).
 * Trees are level-ordered: node v has children 2v+1 and 2v+2.
 */
typedef struct {
    int32_t depth;
    int32_t trees;
    int64_t n_internal;
    size_t off_split_dim, off_split_val, off_perm, off_leaf_ofs, off_leaf_pt;
    size_t bytes;
} atsne_forest_layout_t;

atsne_status atsne_forest_layout(int64_t N, int32_t D, const atsne_knn_opts *opts,
                                 atsne_forest_layout_t *out);
atsne_status atsne_forest_build(const float *X, int64_t N, int32_t D, const atsne_knn_opts *opts,
                                void *forest, size_t forest_bytes, void *workspace,
                                size_t ws_bytes, void *stream);
/*
 * Adding and removing points, Sec. 5.3.1 and Sec. 5.3.2: the forest's trees
 * (split dimensions and values, as built on N_built points with `opts`) stay,
 * and its leaf buckets change. An updated set of buckets lives in a separate
 * caller buffer ("buckets") of atsne_forest_buckets_bytes(N, depth, trees)
 * bytes: perm [T][N] int32 (each tree's points in leaf order), then at a
 * 256-byte offset the per-tree leaf offsets [T][2^depth + 1] int32 (trees
 * differ once points are added). depth is atsne_forest_layout's for N_built.
 *
 * atsne_forest_insert: rows N_old .. N_new-1 of X join every tree. A new
 * point descends a tree by the search's rule (value below the split: left
 * child) to a leaf and joins its bucket after the points already there, the
 * new points in index order. buckets_in: NULL for the forest's own buckets
 * (then N_old = N_built), else the buckets of the first N_old rows.
 * atsne_forest_delete: the listed rows ([R], distinct, in [0, N)) leave every
 * bucket; the others keep their order and are renumbered as the corpus rows
 * are (j becomes j minus the deleted rows below j), as atsne_delete_rows
 * renumbers the state. A row out of range or listed twice raises the device
 * status; the buckets are then unspecified.
 * Both write buckets_out (no byte of it may overlap buckets_in) and return the largest
 * bucket in *max_bucket_out (host), which atsne_forest_query_buckets takes:
 * they synchronise the stream to read it. Workspace:
 * atsne_workspace_bytes(ATSNE_OP_FOREST_UPDATE, N_built, D, 0, S, opts), S the
 * rows after an insertion or before a deletion.
 */
size_t atsne_forest_buckets_bytes(int64_t N, int32_t depth, int32_t trees);
atsne_status atsne_forest_insert(const float *X, int64_t N_built, int64_t N_old, int64_t N_new, int32_t D,
                                 const atsne_knn_opts *opts, const void *forest, const void *buckets_in,
                                 void *buckets_out, size_t out_bytes, int32_t *max_bucket_out, void *workspace,
                                 size_t ws_bytes, void *stream);
atsne_status atsne_forest_delete(const int32_t *rows, int64_t R, int64_t N_built, int64_t N, int32_t D,
                                 const atsne_knn_opts *opts, const void *forest, const void *buckets_in,
                                 void *buckets_out, size_t out_bytes, int32_t *max_bucket_out, void *workspace,
                                 size_t ws_bytes, void *stream);
/*
 * atsne_forest_query over updated buckets: the search of Sec. 4.2 with the
 * trees of `forest` (built on N_built points) and the leaves' points from
 * `buckets` (N = the rows of X now). Every point of a reached leaf is
 * evaluated as in a forest built with larger leaves. Workspace:
 * atsne_workspace_bytes(ATSNE_OP_FOREST_QUERY, N, D, k, S, opts) with
 * opts->leaf_size = max_bucket. max_bucket must be at least the largest
 * bucket (the value the update returned): each query's point list is sized
 * by it. A bucket above max_bucket raises the device status (atsne_check
 * returns ATSNE_EINVAL); no list is written past its end, and the results
 * are then unspecified.
 */
atsne_status atsne_forest_query_buckets(const float *X, int64_t N, int32_t D, int64_t N_built, const void *forest,
                                        const void *buckets, int32_t max_bucket, const int32_t *queries, int64_t S,
                                        int32_t k, const atsne_knn_opts *opts, int32_t *idx_out, float *d2_out,
                                        int64_t *evaluated_out, void *workspace, size_t ws_bytes, void *stream);

atsne_status atsne_forest_query(const float *X, int64_t N, int32_t D, const void *forest,
                                const int32_t *queries, int64_t S, int32_t k,
                                const atsne_knn_opts *opts, int32_t *idx_out, float *d2_out,
                                int64_t *evaluated_out, void *workspace, size_t ws_bytes,
                                void *stream);

/* Synchronise `stream`, then read and clear the device status word
 * (ATSNE_OK, ATSNE_EINVAL for non-finite or malformed input, ATSNE_ETIMEOUT). */
atsne_status atsne_check(void *stream);

/*
 * Failure detection of the tensor-core kNN (the paper has no counterpart):
 * every wait of its copy -> MMA -> epilogue pipeline is bounded. A wait that
 * runs out makes the kernel stop issuing work, let its issued copies and MMAs
 * complete, release its tensor memory and raise the device status, which
 * atsne_check reports as ATSNE_ETIMEOUT; that call's results are then
 * unspecified and the library stays usable. This sets the limit of those
 * waits for later calls (process-wide), in nanoseconds; 0 restores the
 * default of one second. A very short limit makes a wait run out on purpose
 * (the timeout path's test). Always ATSNE_OK.
 */
atsne_status atsne_set_wait_limit(uint64_t ns);

/* Message of the last error on this thread ("" if none). */
const char *atsne_last_error(void);

/* Number of kernel launches this library has enqueued since it was loaded
 * (all threads, all devices). */
int64_t atsne_launch_count(void);

/*
 * Per-kernel timing: while enabled, every kernel launch is bracketed by CUDA
 * events recorded on the launching stream. atsne_profile_read() synchronises
 * those events and returns the launch count and summed milliseconds of every
 * kernel whose name equals `kernel` (or all, if kernel is NULL).
 */
atsne_status atsne_profile_enable(int32_t on);
atsne_status atsne_profile_reset(void);
atsne_status atsne_profile_read(const char *kernel, int64_t *launches, double *total_ms);

#ifdef __cplusplus
}
#endif

#endif /* ATSNE_H */
