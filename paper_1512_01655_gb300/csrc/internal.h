// Host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "atsne.h"
#include "common.cuh"

namespace atsne {

// ---- input checks (device side; they raise the status word) -----------------
atsne_status check_finite(const float *X, int64_t n, cudaStream_t stream);
atsne_status check_indices(const int32_t *list, int64_t n, int64_t N, cudaStream_t stream);

// ---- exact kNN ------------------------------------------------------------
atsne_status knn_bruteforce(const float *X, int64_t N, int D, const int32_t *qlist, int64_t nq,
                            int k, int32_t *idx_out, float *d2_out, cudaStream_t stream);
// The rows listed in rows_list[0 .. *rows_count) (device count, at most nq).
atsne_status knn_bruteforce_rows(const float *X, int64_t N, int D, const int32_t *qlist,
                                 const int32_t *rows_list, const int32_t *rows_count, int64_t nq,
                                 int k, int32_t *idx_out, float *d2_out, cudaStream_t stream,
                                 const float *Xq = nullptr);

// Tensor-core exact kNN: plan (tile split, candidate capacity) and workspace.
struct TcPlan {
    int passes = 1, Dp = 0, row_tiles = 0, splits = 1, cols_per_split = 0, ksel = 0, cap = 0;
    int halves = 1;  // candidate buffers per (row, split): one per column half of a tile
    bool certify = true;  // rows certified exact (else the ksel best keys re-ranked, approximate)
};
// Row and column order of a large self kNN (points grouped by nearest
// centroid; each row tile streams its own groups' column tiles first).
constexpr int64_t ORD_MIN_ROWS = 65536;
constexpr int ORD_MAX_DIM = 256;
struct OrderWs {
    float *cent = nullptr, *cn = nullptr, *sum = nullptr;
    int *cnt = nullptr;
    int32_t *label = nullptr, *lab_sorted = nullptr;
    int32_t *perm = nullptr;  // position in the order -> row
    int32_t *bcnt = nullptr, *coff = nullptr;
    int32_t *pro = nullptr;   // per row tile: first column tile of its groups, their count
};
struct TcWs {
    uint16_t *hi = nullptr, *lo = nullptr, *qhi = nullptr, *qlo = nullptr;
    float *nrm = nullptr, *stats = nullptr;
    unsigned *gmax = nullptr;
    char *cand = nullptr, *meta = nullptr;
    unsigned *row_hist = nullptr;
    float *scale = nullptr, *qscale = nullptr;  // FP8 row scales
    float *qnrm = nullptr, *qstats = nullptr;   // queries from another array: norms, error stats
    int32_t *flag_rows = nullptr, *flag_count = nullptr;
    uint16_t *bext = nullptr, *aext = nullptr;  // one-pass BF16: the norm slices
    bool ordered = false;                       // rows and columns in the order of OrderWs
    unsigned long long *clock = nullptr;        // one split: tiles issued by all CTAs
    OrderWs ord;
};
// Limit of the tensor kernel's pipeline waits (process-wide; default 1 s).
uint64_t pipeline_wait_ns();
void set_pipeline_wait_ns(uint64_t ns);
// splits > 0 forces the column split count; else the one atsne_tune_knn
// recorded for this shape, else the rule.
TcPlan tc_plan(int64_t N, int D, int64_t Q, int k, int precision, int rerank_k, int splits = 0);
int tuned_splits(int64_t N, int D, int64_t Q, int k, int precision, int rerank_k);
void set_tuned_splits(int64_t N, int D, int64_t Q, int k, int precision, int rerank_k, int splits);
void clear_tuned_splits();
// Distinct column split counts worth timing for a shape (at most max_out).
int tc_split_candidates(int64_t N, int D, int64_t Q, int k, int precision, int rerank_k, int *out, int max_out);
size_t tc_workspace(Carver &c, int64_t N, int D, int64_t Q, bool list, const TcPlan &pl, TcWs *ws);
bool knn_ordered(int64_t N, int D, bool list, const TcPlan &pl);
size_t order_workspace(Carver &c, int64_t N, int D, const TcPlan &pl, OrderWs *ws);
atsne_status knn_order_launch(const float *X, int64_t N, int D, const TcPlan &pl, int bm, int bn,
                              const OrderWs &w, cudaStream_t stream);
// Xq != nullptr: the Q queries are the rows of Xq (another array), none excluded.
// radius != nullptr (with Xq): only neighbours with d^2 < radius[row] are kept,
// the row padded with (-1, +inf); the plan's cap is then RADIUS_CAP.
constexpr int RADIUS_CAP = 256;
atsne_status radius_filter_launch(int32_t *idx, float *d2, int64_t rows, int k, const float *radius,
                                  cudaStream_t stream);
atsne_status knn_exact_tc(const float *X, int64_t N, int D, const int32_t *qlist, int64_t Q, int k,
                          const TcPlan &pl, const TcWs &w, int32_t *idx_out, float *d2_out,
                          cudaStream_t stream, const float *Xq = nullptr,
                          const float *radius = nullptr, const float *hint = nullptr);

// ---- calibrate ------------------------------------------------------------
size_t calibrate_smem_bytes(int k);
atsne_status calibrate_launch(const float *d2, int64_t rows, int k, float perplexity, float tol,
                              int max_iter, float *P, float *beta, cudaStream_t stream);

// ---- symmetrize -------------------------------------------------------------
struct SymWs {
    int32_t *scol = nullptr;   // [N][k] conditional rows sorted by column
    float *sval = nullptr;
    int32_t *rev_i = nullptr;  // reverse lists: source rows, [N * k]
    float *rev_p = nullptr;    // and their conditionals
    int32_t *rcnt = nullptr, *cursor = nullptr, *len = nullptr, *long_rows = nullptr, *n_long = nullptr,
            *own = nullptr;
    int64_t *roff = nullptr, *rtot = nullptr;  // reverse list offsets [N + 1], total
    int64_t *scan = nullptr;
};
size_t scan_partials_count(int64_t n);
atsne_status scan_rowlen(const int32_t *rev, int64_t n, int add, int64_t *out, int64_t *total,
                         int64_t *part, cudaStream_t stream);
size_t symmetrize_workspace(Carver &c, int64_t N, int k, SymWs *ws);
atsne_status symmetrize_launch(const int32_t *idx, const float *P, int64_t N, int k,
                               int64_t *row_ptr, int32_t *col, float *val, int64_t *nnz_dev,
                               const SymWs &w, cudaStream_t stream);

// ---- precision / refine -----------------------------------------------------
atsne_status precision_launch(const int32_t *a, const int32_t *e, int64_t rows, int k,
                              float *rho_i, double *rho_sum, cudaStream_t stream);
atsne_status kde_launch(const float *Y, int64_t N, const float *rho, const uint8_t *selected, float x0,
                        float y0, float pixel, int W, int H, float h, float cutoff, float lens_k,
                        float *f_out, float *s_out, float *a_out, float *alpha_out,
                        cudaStream_t stream);
atsne_status row_dmax_launch(const float *d2, int64_t rows, int k, float *dmax, cudaStream_t stream);
atsne_status gather_hint_launch(const int32_t *rows, int64_t S, int64_t N, int k, const float *d2,
                                float *hint, cudaStream_t stream);
atsne_status merge_neighbors_launch(int32_t *idx, float *d2, int64_t rows, int k, const int32_t *cidx,
                                    const float *cd2, int kc, int32_t offset, uint8_t *changed,
                                    cudaStream_t stream);
atsne_status union_launch(const int32_t *lists, int64_t total, int64_t N, uint32_t *bitmap,
                          int32_t *out, int64_t out_rows, int64_t *count, cudaStream_t stream);
// Deletion (Sec. 5.3.2): scratch of one call.
struct DeleteWs {
    int32_t *dead = nullptr;
    int64_t *before = nullptr, *total = nullptr, *scan = nullptr;
    float *X = nullptr, *d2 = nullptr, *beta = nullptr, *rho = nullptr;
    int32_t *idx = nullptr;
};
size_t delete_workspace(Carver &c, int64_t N, int D, int k, DeleteWs *ws);
atsne_status delete_launch(const int32_t *rows, int64_t R, float *X, int64_t N, int D, int k, float perplexity,
                           int32_t *idx, float *d2, float *P, float *beta, float *rho, const DeleteWs &w,
                           cudaStream_t stream);
// Byte copy xu8[N][Dp16] of X (zero padded) and, if nx8 is given, the rows'
// exact squared norms; *bad (cleared by the caller) is raised unless every value
// is an integer in [0, 255].
atsne_status u8_copy_launch(const char *name, const float *X, int64_t N, int D, int Dp16, uint8_t *xu8,
                            uint32_t *nx8, unsigned *bad, cudaStream_t stream);
atsne_status refine_scatter_launch(const int32_t *subset, int64_t S, int64_t N, int k, const int32_t *ti,
                                   const float *td, const float *tp, const float *tb, int32_t *idx,
                                   float *d2, float *P, float *beta, float *rho,
                                   cudaStream_t stream);

// ---- forest -------------------------------------------------------------------
struct ForestView {
    int64_t N;
    int D, trees, depth, leaf_size, top_var_dims;
    int64_t n_internal;
    uint64_t seed;
    int32_t *split_dim;
    float *split_val;
    int32_t *perm;
    int32_t *leaf_ofs;
    int32_t *leaf_pt;
    // 0: one leaf-offset array for all trees (a forest as built, leaf_pt valid);
    // else each tree's offsets (buckets after points were added or removed,
    // leaf_size = the largest bucket)
    int64_t ofs_stride = 0;
};
int forest_depth(int64_t N, int leaf_size);
size_t forest_layout(int64_t N, int trees, int leaf_size, atsne_forest_layout_t *out);
size_t forest_build_workspace(Carver &c, int64_t N, int D, int trees, int leaf_size, void *ws_out);
atsne_status forest_build_launch(const float *X, const ForestView &f, void *ws_base, size_t ws_bytes,
                                 cudaStream_t stream);
size_t forest_query_workspace(Carver &c, int64_t N, int D, int64_t nq, int k, int checks, int leaf_size,
                              void *ws_out);
// Buckets after points were added or removed (Sec. 5.3.1, 5.3.2): perm
// [T][N] and per-tree leaf offsets [T][2^h + 1], both int32, in one buffer.
struct BucketsView {
    int32_t *perm, *ofs;
};
size_t buckets_layout(int64_t N, int depth, int trees, size_t *off_ofs);
struct UpdateWs {
    int32_t *leaf = nullptr, *cursor = nullptr, *dead = nullptr, *bmax = nullptr;
    int64_t *before = nullptr, *total = nullptr, *scan = nullptr;
};
size_t update_workspace(Carver &c, int64_t N, int depth, int trees, UpdateWs *ws);
atsne_status forest_insert_launch(const float *X, int64_t N_old, int64_t N_new, int D, const ForestView &f,
                                  const int32_t *perm_in, const int32_t *ofs_in, int64_t stride_in,
                                  const BucketsView &out, const UpdateWs &w, cudaStream_t stream);
atsne_status forest_delete_launch(const int32_t *rows, int64_t R, int64_t N, const ForestView &f,
                                  const int32_t *perm_in, const int32_t *ofs_in, int64_t stride_in,
                                  const BucketsView &out, const UpdateWs &w, cudaStream_t stream);
// Flags (DEV_MALFORMED) any bucket of per-tree offsets ofs[trees][2^depth + 1]
// holding more than `bound` points.
atsne_status bucket_bound_check(const int32_t *ofs, int trees, int depth, int bound, cudaStream_t stream);
atsne_status forest_query_launch(const float *X, const ForestView &f, const int32_t *qlist,
                                 int64_t nq, int k, int checks, int qcap, int32_t *idx_out,
                                 float *d2_out, int64_t *evaluated_out, void *ws_base,
                                 size_t ws_bytes, cudaStream_t stream);

}  // namespace atsne
