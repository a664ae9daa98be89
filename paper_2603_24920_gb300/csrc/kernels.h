// kernels.h -- host-side launchers of the DET-LSH kernels (internal).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dl {

// ---- exact projection (project.cu) ----------------------------------------
struct ProjArgs {
  // modes 0 (row-major P[row][col]) and 1 (column-major P[col][row])
  float *P = nullptr;
  int64_t ldP = 0;
  // mode 2: encode into codes[tree][n][16] and track per-column min/max
  uint8_t *codes = nullptr;
  int64_t n = 0;
  const float *B = nullptr;  // [LK][N_r+1]
  int N_r = 0, K = 0;
  uint32_t *minmax = nullptr;  // [LK][2] order-preserving keys
  uint32_t *ubound = nullptr;    // [LK][2] running bounds of column min/max (mode 2)
  float gamma = 0.0f;            // encoder error factor (mode 2; set by project_rows)
  // outputs the compensated path cannot certify
  uint2 *fb_list = nullptr;
  uint32_t *fb_count = nullptr;
  uint32_t fb_cap = 0;
  unsigned long long *fb_total = nullptr;  // running count (device)
  int *err = nullptr;                      // device status word
};

// Tensor-core encoder of all n points (encode_tc.cu), mode 2 of project_rows
// for contiguous rows with d a multiple of 4 up to 128; *used = 0 when it
// does not apply (the CUDA-core encoder then runs).
int launch_encode_tc(const float *X, int64_t nrows, int d, const float *A, int LK, int W,
                     ProjArgs o, cudaStream_t st, int *used);

// rows == nullptr: rows 0..nrows-1 of X; else the listed row ids.
int project_rows(const float *X, int64_t ldx, const uint32_t *rows, int64_t nrows, int d,
                 const float *A, int LK, int mode, ProjArgs o, cudaStream_t st);

// ---- sorting and compaction (sort.cu) --------------------------------------
struct SortTemp {
  uint32_t *keys_alt = nullptr, *vals_alt = nullptr;
  uint32_t *counts = nullptr;  // [segs][256][tiles]
  uint32_t *digit_base = nullptr;
  size_t count_cap = 0;
};
size_t sort_tiles(int64_t len);
// Stable LSD radix sort of nseg equal-length segments (keys, optional values)
// on key bits [0, nbits).  Result ends in keys/vals.
int segmented_sort(uint32_t *keys, uint32_t *vals, int nseg, int64_t len, int nbits,
                   SortTemp &tmp, cudaStream_t st);

// Ids of the sampled points in ascending order (Philox stream 3); returns m.
int sample_ids(int64_t n, uint64_t seed, double frac, uint32_t *ids, uint32_t *block_counts,
               int64_t *m_out, cudaStream_t st);
size_t sample_blocks(int64_t n);

// Float sample columns -> order keys in place; breakpoint extraction.
int float_to_keys(float *v, int64_t count, cudaStream_t st);
int extract_breakpoints(const uint32_t *sorted_keys, int LK, int64_t m, int N_r, float *B,
                        cudaStream_t st);
int finish_breakpoint_ends(const uint32_t *minmax, int LK, int N_r, float *B, cudaStream_t st);

// ---- DE-Tree layout (tree.cu) ----------------------------------------------
struct TreeBuildArgs {
  int64_t n;
  int G;                   // trees built together: t0 .. t0 + G - 1
  int K, bbits, M, box_mode;
  const uint8_t *codes;    // codes of tree t0, then the next G - 1 trees: [G][n][16]
  // outputs
  uint32_t *perm;          // [G][n] point ids leaf by leaf (the trees' rows of perm)
  uint32_t *leaf_begin;    // [leaves + G]: each tree's starts (within the tree) and end n
  uint8_t *leaf_lo, *leaf_hi, *leaf_nb;  // [leaves][16], trees one after another
  uint32_t *leaf_of;       // [n][L] (columns t0 ..)
  uint32_t *scalars;       // [4 + G + 1] (device): first-layer nodes, leaves, error,
                           // largest leaf, first leaf of every tree and the total
  int L, t0;
};
struct TreeTemp {
  uint32_t *keys = nullptr, *vals = nullptr;
  uint4 *codesA = nullptr, *codesB = nullptr;
  uint32_t *idsB = nullptr;
  uint32_t *node_begin = nullptr, *block_counts = nullptr;
  uint32_t *tmp_begin = nullptr;  // [n] leaf start flags
  uint8_t *tmp_box = nullptr;  // [n][48]: lo, hi, nb of the leaf starting there
  uint4 *lists = nullptr;      // [2n][2]: the open nodes of two levels
  uint32_t *leaf_start = nullptr;  // [G n] first position of every leaf
  SortTemp sort;
};
// Enqueues the build of G trees (no host synchronisation); the counts land in
// a.scalars.  Temporaries hold G n entries; the leaf arrays G n (G n + G for
// leaf_begin).
int build_trees(const TreeBuildArgs &a, TreeTemp &tmp, cudaStream_t st);
// Hull boxes of runs of LEAF_BLOCK boxes, every tree in one launch: tree t's
// ceil(cnt[t]/LEAF_BLOCK) hulls ([16] lo and hi bytes each) start at out_off[t].
struct HullSet {
  int L;
  int64_t in_off[17];   // first input box of every tree; in_off[t] + cnt[t] ends it
  int64_t cnt[16];      // input boxes per tree
  int64_t out_off[17];  // first hull of every tree; out_off[L] = all hulls
};
int block_hulls(const uint8_t *lo, const uint8_t *hi, const HullSet &h, uint8_t *hlo, uint8_t *hhi,
                cudaStream_t st);

// ---- queries (query.cu) ----------------------------------------------------
struct QueryIndexView {
  int64_t n;
  int d, L, K, LK, N_r;
  const float *X;
  const __nv_bfloat16 *Xh;
  const float2 *Xn;          // [n] {||bf16(x)||^2, upper bound of ||x - bf16(x)||}
  const float *P;            // [n][LK] exact projections (null unless kept at build)
  const float *B;            // [LK][N_r+1]
  const uint32_t *perm;      // [L][n]
  const uint32_t *leaf_begin;  // concatenated, tree t at leaf_off[t] + t
  const uint8_t *leaf_lo, *leaf_hi;  // [total_leaves][16]
  const uint32_t *leaf_of;   // [n][L]
  const uint8_t *blk_lo, *blk_hi;  // [total_blocks][16] hulls of LEAF_BLOCK leaves
  int64_t leaf_off[17];      // leaf index offset of each tree (prefix)
  int64_t blk_off[17];       // block index offset of each tree (prefix)
  const uint8_t *sblk_lo, *sblk_hi;  // [total_sblocks][16] hulls of LEAF_BLOCK blocks
  int64_t sblk_off[17];      // super-block index offset of each tree (prefix)
  const uint8_t *tblk_lo, *tblk_hi;  // [total_tblocks][16] hulls of LEAF_BLOCK super-blocks
  int64_t tblk_off[17];      // top-block index offset of each tree (prefix)
  int64_t max_leaves;        // max leaves of one tree
  int64_t max_leaf_size;
  int bf16_exact;            // 1: every row equals its BF16 copy (no residuals)
};
// Query tables: T[256] squared-radius grid; for a fixed r_min also
// (c r_i)^2 rounded down [256] and up [256] and c r_i as three FP32 pieces
// [256][3] (the exact test of condition 2 near the sphere).
constexpr int TABLE_FLOATS = 256 * 6;
// Arrays of a query kernel's per-CTA scratch slot (query_slot_offsets).
constexpr int SLOT_ARRAYS = 14;
struct QueryArgs {
  const float *Q;            // [m][d]
  const __nv_bfloat16 *Qh;   // [m][d] (bf16 path)
  const float *Qp;           // [m][LK] exact projections
  int64_t m;
  const int32_t *kq;         // per-query k (nullable)
  int k_max;
  int64_t tau_base;          // ceil(beta * n)
  const float *T;            // [255] radius grid
  const float *Tc;           // fixed r_min, condition 2: the query tables from offset 256
                             // (rounded-down (c r_i)^2 [256], rounded-up [256], pieces [3][256])
  int policy;                // DETLSH_RMIN_MAGIC / DETLSH_RMIN_FIXED / _CONTINUOUS
  int per_tree;              // 1: whole trees join S (no priority queue)
  float lg_eps2, inv_2lg_c;  // log2(eps^2), 1/(2 log2 c): level estimate before the exact fix-up
  int precision, rerank_mult;
  int64_t *ids;              // [m][k_max]
  float *dists;              // [m][k_max]
  // optional candidate export
  int64_t *S_out;            // [m][S_cap] (device)
  int64_t S_cap;
  int64_t *S_size;
  int32_t *jstar, *istar;
  // scratch: one slot per CTA, offsets from query_slot_offsets
  uint8_t *scratch;
  int64_t slot_bytes;
  int64_t off[SLOT_ARRAYS + 1];
  int64_t cand_cap;
  unsigned long long *epoch_counter;  // leaf levels are tagged (epoch << 8 | level); each
                                      // query takes the next epoch from this device word
  int nslots;
  uint32_t *work_counter;
  int *err;
  unsigned long long *stats;  // [5]: candidates, leaves expanded, hull blocks, points visited,
                              // rows re-ranked
  // tuning knobs (detlsh_tuning; the defaults are the hand-picked values)
  int ctas_per_sm = 0;        // persistent CTAs per SM (0: as many as fit)
  int expand_runs = 4;        // leaf runs per warp per chunk of the level-ordered expansion, 1..8
  int visit_chunk = 512;      // listed leaves per chunk of a flattened visit, 64..512
  int top_min = 1024;         // super-hulls per tree above which pruning starts from top hulls
  int hash_kb = 0;  // shared memory (KiB) for the leaf-level hash; 0 = the LUT region
};
size_t query_slot_bytes(const QueryIndexView &ix, int64_t cand_cap, int rerank_cap);
void query_slot_offsets(const QueryIndexView &ix, int64_t cand_cap, int64_t off[SLOT_ARRAYS + 1]);
int query_slots(const QueryIndexView &ix);
int run_queries(const QueryIndexView &ix, const QueryArgs &qa, cudaStream_t st);

// (r,c)-ANN queries (Alg. 4) over the range query of Alg. 3 as printed.
struct RcArgs {
  const float *Q;            // [m][d]
  const float *Qp;           // [m][LK] exact projections
  int64_t m;
  float R2;                  // fp32((eps r)^2)
  float cr;                  // fp32(c r)
  int64_t need;              // ceil(beta n) + 1
  int optimised;             // 1: leaves whole by lower bound (Sec. VI-B2 (1))
  int64_t *ids;              // [m], -1 when nothing is returned
  float *dists;              // [m], +inf when nothing is returned
  int32_t *tree_stop;        // [m], tree where |S| reached need, -1 if none
  int64_t *S_size;           // [m]
  int64_t *S;                // [m][S_cap] (nullable)
  int64_t S_cap;
  uint8_t *scratch;          // nslots slots of rcann_slot_bytes
  int64_t slot_bytes;
  int nslots;
  uint32_t *work_counter;    // zeroed by run_rcann
};
size_t rcann_slot_bytes(const QueryIndexView &ix);
int rcann_slots(const QueryIndexView &ix);
int run_rcann(const QueryIndexView &ix, const RcArgs &a, cudaStream_t st);

// ---- misc (api.cu) ----------------------------------------------------------
int f32_to_bf16(const float *src, __nv_bfloat16 *dst, int64_t count, cudaStream_t st);

}  // namespace dl
