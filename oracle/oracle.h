/*
 * oracle.h -- plain, slow CPU oracle for the DET-LSH hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code with the CUDA path and the CUDA path never calls it.
 *
 * Every function states the passage of the paper (DET-LSH / PDET-LSH,
 * arXiv 2603.24920) it follows.  Readings of passages the paper leaves open
 * are stated beside the function they shape.
 *
 * Precision: the projection is the correctly rounded FP32 value of the exact
 * real dot product (computed with exact big-integer arithmetic); breakpoints,
 * codes and trees are exact functions of those values; node lower bounds are
 * computed in FP32 in a fixed order (the precision the GPU takes the same
 * decision in); exact distances are FP64.
 */
#ifndef DETLSH_ORACLE_H
#define DETLSH_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), the counter-based
 * generator both sides implement from its published definition. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Eq. 1 (Sec. II-B): K*L Gaussian projection vectors, rows t = i*K + j.
 * A is (LK x d) row-major FP32.  Box-Muller in FP64 from Philox stream 2. */
void orc_projection_matrix(int LK, int64_t d, uint64_t seed, float *A);

/* Eq. 1: h(o) = a . o, returned as the FP32 value nearest (ties to even) to the
 * exact real dot product.  Exact zero is returned as +0. */
float orc_dot_rn32(const float *a, const float *x, int64_t d);

/* All projections P[p*LK + t] = h_t(X[p]) (Sec. III-A; cost term (1) of Sec. V-C). */
void orc_project(const float *X, int64_t n, int64_t d, const float *A, int LK, float *P);

/* Sample of ~frac*n points (Sec. III-A: n_s = 0.1 n).  Returns m and writes the
 * sampled ids in ascending order.  Falls back to all points when m < 2*N_r. */
int64_t orc_sample(int64_t n, uint64_t seed, double frac, int N_r, int64_t *ids);

/* Breakpoints (Sec. III-A, dynamic encoding scheme): B[t*(N_r+1) + z]. */
void orc_breakpoints(const float *P, int64_t n, int LK, const int64_t *sample, int64_t m,
                     int N_r, float *B);

/* Static encoding scheme (Sec. III-A): equal-mass N(0,1) breakpoints,
 * b_0 = -inf, b_{N_r} = +inf, every dimension alike. */
void orc_static_breakpoints(int LK, int N_r, float *B);
/* Alg. 1 (BinarySearch step): codes[p*LK + t] = region index of P[p*LK+t]. */
void orc_encode(const float *P, int64_t n, int LK, const float *B, int N_r, uint8_t *codes);

/* Eq. 2 / Lemma 3 (Sec. V-A): upper-quantile tail of chi^2(K) and eps^2. */
double orc_chi2_sf(double x, int K);
double orc_eps2(int K, int L);
/* Radius grid T(j) = fp32(eps^2 * c^(2j)), j = -127..127 (index j+127);
 * T(127) = +inf. */
void orc_level_table(double eps2, double c, float *T);
#define ORC_NLEV 255
#define ORC_JMIN (-127)

/* ---- index: encoding + L DE-Trees (Alg. 1, Alg. 2) ---- */
typedef struct orc_index orc_index;

/* box_mode 0 = prefix box (breakpoints dividing the node, Sec. IV-C),
 *          1 = tight min/max code box.
 * insertion_order 0 = canonical bulk build, 1 = literal Alg. 2 insertion.
 * encoding 0 = dynamic scheme (sampled equal-frequency breakpoints),
 *          1 = static scheme (N(0,1) equal-mass breakpoints). */
orc_index *orc_index_build(const float *X, int64_t n, int64_t d, int L, int K, int N_r,
                           uint64_t seed, double frac, int M, int box_mode,
                           int insertion_order, int encoding);
void orc_index_free(orc_index *ix);
int64_t orc_index_sample_size(const orc_index *ix);
int64_t orc_index_num_leaves(const orc_index *ix, int t);
void orc_index_export_arrays(const orc_index *ix, float *A, float *B, uint8_t *codes,
                             float *P, int64_t *sample);
/* Leaves of tree t in canonical order (first-layer key ascending, child 0
 * before child 1); members of a leaf in ascending id order. */
void orc_index_export_tree(const orc_index *ix, int t, int64_t *perm, int64_t *leaf_begin,
                           uint8_t *box_lo, uint8_t *box_hi, uint8_t *nbits,
                           int64_t *leaf_of);
void orc_index_level_table(const orc_index *ix, double c, float *T);

/* Alg. 5 (c^2-k-ANN) with the optimised range query of Sec. VI-B2 and the
 * "magic" r_min of Sec. V-B1.  Returns 0 on success.
 * S_out (capacity n, nullable) receives the candidate ids in arrival order. */
int orc_index_query(const orc_index *ix, const float *q, int k, double beta, double c,
                    int64_t *ids, double *dists, int64_t *S_out, int64_t *S_size,
                    int *jstar, int *istar);
/* Alg. 5 run literally from a fixed r_min (radii r_min c^i, i = 0, 1, ...;
 * radius index i uses T'(i) = fp32(eps^2 r_min^2 c^(2i)), the last +inf),
 * with condition 2 (at least k points of S within c*r, each distance compared
 * with c*r exactly) checked after each radius.  jstop = the stopping radius index, istop = the tree for
 * condition 1 or -1 for condition 2.  S_out (capacity n, nullable). */
/* Exact ||q - x|| <= R for FP32 rows and a double R (1 within, 0 beyond, -1 if
 * R cannot be cut into FP32 pieces; R >= 2^127 is within).  Condition 2 of
 * Alg. 5. */
int orc_dist2_le(const float *q, const float *x, int64_t d, double R);
int orc_index_query_fixed(const orc_index *ix, const float *q, int k, double beta, double c,
                          double r_min, int64_t *ids, double *dists, int64_t *S_out,
                          int64_t *S_size, int *jstop, int *istop);
/* Alg. 5 at the smallest continuous r_min (no radius grid): v* = the
 * (beta*n + k)-th smallest of the points' smallest leaf lower bound over the
 * trees; then Alg. 5's first round at that squared radius.  *vstar = v*,
 * istar as orc_index_query.  S_out (capacity n, nullable). */
int orc_index_query_magic_min(const orc_index *ix, const float *q, int k, double beta,
                              int64_t *ids, double *dists, int64_t *S_out, int64_t *S_size,
                              float *vstar, int *istar);
/* As orc_index_query; per_tree = 1 drops the priority queue: each tree's
 * range query joins S whole and |S| >= beta*n + k is checked after each tree
 * (Alg. 5 as printed). */
int orc_index_query_ex(const orc_index *ix, const float *q, int k, double beta, double c,
                       int per_tree, int64_t *ids, double *dists, int64_t *S_out,
                       int64_t *S_size, int *jstar, int *istar);
/* Same, over m queries, OpenMP over queries (nthreads <= 0: all cores). */
int orc_index_query_batch(const orc_index *ix, const float *Q, int64_t m, int k, double beta,
                          double c, int64_t *ids, double *dists, int64_t *S_sizes,
                          int nthreads);
/* Lower bound of every leaf of tree t to query q (FP32, Sec. IV-C). */
void orc_index_leaf_lb2(const orc_index *ix, int t, const float *q, float *lb2);

/* Alg. 3 as printed, without the optimisations of Sec. VI-B2: the points of
 * tree t within r' = eps*r of q' in the projected space (node lower bound
 * prunes, leaf upper bound within r' takes the leaf whole, otherwise each
 * point's projected distance is tested).  Squared comparisons in FP32 against
 * R2 = fp32(eps^2 r^2).  Writes the ids (capacity n), returns their count. */
int64_t orc_index_range_exact(const orc_index *ix, int t, const float *q, double r,
                              int64_t *out);
/* Upper bound of every leaf of tree t to query q (FP32, Sec. IV-C). */
void orc_index_leaf_ub2(const orc_index *ix, int t, const float *q, float *ub2);
/* Lower and upper bound (Sec. IV-C) of one box: B holds K rows of N_r + 1
 * breakpoints, lo/hi the box's first and last region per dimension. */
void orc_box_bounds(const float *B, int K, int N_r, const float *qp, const uint8_t *lo,
                    const uint8_t *hi, float *lb2, float *ub2);
/* Alg. 4, (r,c)-ANN: trees in order, S = union of the range queries (Alg. 3
 * as printed, or with optimised = 1 optimisation (1) of Sec. VI-B2: every
 * leaf whose lower bound is within r' whole);
 * once |S| >= beta*n + 1 the point of S closest to q is returned (tree_stop =
 * that tree); after all L trees, the closest point of S if it lies within
 * c*r, else id = -1 (tree_stop = -1).  FP64 distances, ties by smaller id.
 * S_out (capacity n, nullable) receives S in arrival order. */
int orc_index_rc_ann(const orc_index *ix, const float *q, double r, double beta, double c,
                     int optimised, int64_t *id, double *dist, int64_t *S_out,
                     int64_t *S_size, int *tree_stop);
/* Exact kNN by brute force, FP64 distances, ties by smaller id. */
void orc_bruteforce_knn(const float *X, int64_t n, int64_t d, const float *Q, int64_t m,
                        int k, int64_t *ids, double *dists, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
