// query.cu -- batched c^2-k-ANN queries over the DE-Trees (Alg. 3-5) for
// sm_103a.  One persistent launch: each CTA takes queries from a global work
// counter and runs the whole query in its own scratch slot.
//
// Per query (q' = exact projections, computed beforehand by the projection
// kernel):
//  1. Range-query bounds (Alg. 3, Sec. IV-C): for every leaf of every tree,
//     LB^2 = sum_j gap_j^2 with gap_j the distance from q'_j to the leaf's
//     breakpoint interval [B(lo_j), B(hi_j + 1)], in FP32, dimensions in
//     order, from a per-tree lookup table g[j][z] = B_j[z] - q'_j held in
//     shared memory.  The leaf's level is the smallest radius index j with
//     LB^2 <= T(j) = fp32(eps^2 c^(2j)): the first radius of the grid whose
//     range query takes the whole leaf (optimisation (1) of Sec. VI-B2).
//  2. Magic r_min (Sec. V-B1): N(j) = |union over trees of points in leaves
//     of level <= j|; r_min = c^{j*}, j* = min{j : N(j) >= beta*n + k}.
//     Union counts need no per-query bitmaps: for every level j exactly one
//     tree counts a point of the union (the first tree holding it within j),
//     so N(j) is the sum over trees of per-tree difference arrays of new
//     points, each point looking up only its levels in earlier trees.
//  3. Alg. 5 at r_min: trees in order; a point is new in tree t if no earlier
//     tree holds it within level j*; i* = first tree where the running count
//     reaches beta*n + k; inside tree i* the leaves enter in ascending
//     (LB^2, leaf index) order -- the priority queue of Sec. VI-B2 -- until the
//     count is reached (a weighted radix select on LB^2).
//  4. Verification: exact distances of every candidate (FP32, or BF16 scores
//     with an FP32 re-rank of the best rerank_mult*k) and top-k by
//     (distance, id) via radix select.
#include "common.cuh"
#include "compact.cuh"
#include "kernels.h"
#include "lut.cuh"

#include <algorithm>

namespace dl {

constexpr int QT = 256;
constexpr int QW = QT / 32;
constexpr int KMAX = 1024;
constexpr int RR_MAX = 4096;  // re-rank pool of the BF16 path
constexpr int FLC = 512;      // largest chunk of listed leaves of a flattened visit
// (the chunk itself and the leaf runs per warp per expansion chunk are the
// tuning knobs qa.visit_chunk and qa.expand_runs)

struct Slot {
  unsigned long long *lev;  // [total_leaves] (epoch << 8) | level of expanded leaves
  uint8_t *blev;    // [total_blocks] block levels (255 = beyond the bound)
  uint32_t *border; // [total_blocks] block ids ordered by level
  uint32_t *lleaf;  // [total_leaves] per-tree lists of expanded leaves (at leaf_off[t])
  float *llb2;      // [total_leaves]
  uint8_t *llev;    // [total_leaves]
  uint32_t *cval;   // [max_leaves] new points per list entry of tree i*
  uint32_t *cand;   // [cap]
  uint32_t *key;    // [cap] order keys of distances
  uint32_t *rid;    // [RR_MAX] re-rank ids
  uint32_t *rkey;   // [RR_MAX]
  uint8_t *cm;      // [cap] smallest level of each candidate (fixed r_min)
  uint32_t *hkey;   // [cap] upper ends of the certified BF16 intervals
  uint32_t *guess;  // [1] this slot's last final bound + 1 (0: none), kept across launches
};

__host__ __device__ inline int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

static void slot_layout(const QueryIndexView &ix, int64_t cap, int64_t off[SLOT_ARRAYS + 1]) {
  const int64_t tl = ix.leaf_off[ix.L], tb = ix.blk_off[ix.L];
  const int64_t sz[SLOT_ARRAYS] = {8 * tl, tb, 4 * tb, 4 * tl, 4 * tl, tl, 4 * ix.max_leaves,
                                   4 * cap, 4 * cap, 4 * RR_MAX, 4 * RR_MAX, cap, 4 * cap, 4};
  int64_t o = 0;
  for (int i = 0; i < SLOT_ARRAYS; ++i) { off[i] = o; o = align_up(o + sz[i], 256); }
  off[SLOT_ARRAYS] = o;
}

size_t query_slot_bytes(const QueryIndexView &ix, int64_t cand_cap, int) {
  int64_t off[SLOT_ARRAYS + 1];
  slot_layout(ix, cand_cap, off);
  return (size_t)off[SLOT_ARRAYS];
}

void query_slot_offsets(const QueryIndexView &ix, int64_t cand_cap, int64_t off[SLOT_ARRAYS + 1]) {
  slot_layout(ix, cand_cap, off);
}

struct QShared {
  float T[256];
  uint32_t H[256];
  uint32_t rh[256];
  uint32_t bstart[256];
  uint32_t wt[32];
  uint32_t topk_key[KMAX];
  uint32_t topk_id[KMAX];
  uint32_t nlist[16];
  // scalars
  int64_t qi;
  int jhi, jstar, istar, jcur, stop;
  uint32_t need, ncand, sel_v, sel_below, sel_at, nres;
  unsigned long long epoch;  // this query's tag for the leaf levels in the slot
  uint64_t cum;
  unsigned long long n_blocks, n_leaves, n_visit;  // work counters of this CTA
  int use_hash;
  uint32_t hash_bits, hash_count;
  int sel_g;
  uint64_t sel_bf;
  int64_t newt[16];
  uint32_t cpos;
  int jchk;
  float qn;  // |q|^2 of the BF16 query
  float qr;  // upper bound of ||q - bf16(q)||
  int jguess, crossed;  // bound guessed from this CTA's previous query; tree crossed tau
};
static_assert(KMAX >= 1024, "the flattened visit borrows the top-k arrays");

__device__ __forceinline__ uint32_t byte_of(const uint4 &c, int j) {
  const uint32_t w = j < 4 ? c.x : j < 8 ? c.y : j < 12 ? c.z : c.w;
  return (w >> (8 * (j & 3))) & 255u;
}

// Smallest radius level with x <= T[level] (T is nondecreasing, T[254] = +inf).
// A log2 estimate of the level is corrected against T itself, so the result
// is exactly the table's answer whatever the estimate's rounding.
__device__ __forceinline__ uint32_t level_of(const float *T, float x, float lg_eps2,
                                             float inv_2lg_c) {
  if (!(x > 0.0f)) return 0u;
  int i = NLEV - 1;
  if (x <= 3.0e38f) {
    i = (int)ceilf((__log2f(x) - lg_eps2) * inv_2lg_c) - JMIN;
    i = max(0, min(NLEV - 1, i));
  }
  while (i > 0 && x <= T[i - 1]) --i;
  while (x > T[i]) ++i;
  return (uint32_t)i;
}

// Adds w to bins[v] once per distinct v among the active lanes of a warp
// (shared-memory atomics on a few hot bins would otherwise serialise).
__device__ __forceinline__ void warp_bin_add(uint32_t *bins, bool active, uint32_t v, uint32_t w) {
  unsigned act = __ballot_sync(FULL, active);
  const int lane = threadIdx.x & 31;
  while (act) {
    const int src = __ffs(act) - 1;
    const uint32_t key = __shfl_sync(FULL, v, src);
    const bool mine = active && v == key;
    const unsigned grp = __ballot_sync(FULL, mine);
    const uint32_t sum = __reduce_add_sync(FULL, mine ? w : 0u);
    if (lane == src) atomicAdd(&bins[key], sum);
    act &= ~grp;
  }
}

// Adds w to bins[v] for every active lane (w the same in every lane): lanes
// holding the same v are grouped in one step and the lowest lane of each
// group adds w times the group size.
__device__ __forceinline__ void warp_bin_count(uint32_t *bins, bool active, uint32_t v, uint32_t w) {
  const unsigned grp = __match_any_sync(FULL, active ? v : 0xffffffffu);
  if (active && __ffs(grp) - 1 == (int)(threadIdx.x & 31)) atomicAdd(&bins[v], w * (uint32_t)__popc(grp));
}

// Warp 0 finds, over 256 bins, the first bin g with
// below + sum(bins[0..g]) >= need, and writes g and the sum of the bins
// before it (plus below) to shared memory.  Every thread of the block calls
// it; only warp 0 works.  With no crossing it reports bin 255.
__device__ __forceinline__ void warp_first_crossing(const uint32_t *bins, uint64_t below,
                                                    uint64_t need, int *g_out, uint64_t *before) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  uint32_t v[8];
  uint64_t sum = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) { v[i] = bins[lane * 8 + i]; sum += v[i]; }
  uint64_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  const uint64_t excl = incl - sum;
  const bool mine = below + excl < need && below + incl >= need;
  const unsigned b = __ballot_sync(FULL, mine);
  const int src = b ? __ffs(b) - 1 : 31;
  if (lane == src) {
    uint64_t acc = below + excl;
    int g = lane * 8 + 7;
    if (mine) {
      for (int i = 0; i < 8; ++i) {
        if (acc + v[i] >= need) { g = lane * 8 + i; break; }
        acc += v[i];
      }
    } else {
      acc = below + incl - v[7];
    }
    *g_out = g;
    *before = acc;
  }
}

// Block-wide weighted radix select over 32-bit keys: finds the smallest key
// v with W(key <= v) >= need, where item i has (key_i, weight_i) from get(i)
// (weight 0 = absent).  Returns v in sm.sel_v, W(key < v) in sm.sel_below and
// W(key == v) in sm.sel_at.  With last_shift = 8 s > 0 it stops after the top
// 32 - 8 s bits: sel_v is then that prefix of v with the low bits zero.
template <class Get>
__device__ __forceinline__ void block_select(int64_t N, Get get, uint32_t need, QShared &sm,
                                             int last_shift = 0) {
  uint32_t prefix = 0, below = 0;
  for (int shift = 24; shift >= last_shift; shift -= 8) {
    sm.rh[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t hmask = (shift == 24) ? 0u : (0xffffffffu << (shift + 8));
    for (int64_t i = threadIdx.x; i < N; i += QT) {
      uint32_t k, w;
      get(i, k, w);
      if (w && (k & hmask) == (prefix & hmask)) atomicAdd(&sm.rh[(k >> shift) & 255u], w);
    }
    __syncthreads();    warp_first_crossing(sm.rh, below, need, &sm.sel_g, &sm.sel_bf);
    __syncthreads();
    prefix |= (uint32_t)sm.sel_g << shift;
    below = (uint32_t)sm.sel_bf;
    __syncthreads();
  }
  if (threadIdx.x == 0) { sm.sel_v = prefix; sm.sel_below = below; sm.sel_at = sm.rh[prefix & 255u]; }
  __syncthreads();
}

struct QCtx {
  const QueryIndexView &ix;
  const QueryArgs &qa;
  QShared &sm;
  float *lut;       // [LUT_ROWS][LUT_STRIDE]
  uint32_t *hist;   // [L][256] point counts of expanded leaves by level
  int32_t *D;       // [L][256] new-point difference arrays
  Slot s;
  int64_t qi;
  int64_t tau;
};

__device__ __forceinline__ uint32_t leaf_begin_of(const QueryIndexView &ix, int t, int64_t l) {
  return ix.leaf_begin[ix.leaf_off[t] + t + l];
}

// Level of leaf l of tree u for this query.  After the expansion, the levels
// of every listed leaf at or below the final bound sit in a shared-memory
// hash table (when they fit); otherwise they are read from the slot's
// epoch-tagged array.  Leaves absent from both are beyond the bound: 255.
__device__ __forceinline__ uint32_t leaf_level_h(const QueryIndexView &ix, const Slot &s,
                                                 const QShared &sm, const float *lut, int u,
                                                 uint32_t l) {
  if (sm.use_hash) {
    const uint32_t key = (uint32_t)(ix.leaf_off[u] + l) + 1u;
    const uint32_t *keys = reinterpret_cast<const uint32_t *>(lut);
    const uint8_t *levs = reinterpret_cast<const uint8_t *>(keys + (1u << sm.hash_bits));
    const uint32_t mask = (1u << sm.hash_bits) - 1u;
    uint32_t h = (key * 0x9E3779B1u) >> (32 - sm.hash_bits);
    while (true) {  // load factor <= 1/2: an empty slot always ends the probe
      const uint32_t k = keys[h];
      if (k == key) return levs[h];
      if (k == 0u) return 255u;
      h = (h + 1u) & mask;
    }
  }
  const unsigned long long v = s.lev[ix.leaf_off[u] + l];
  return (v >> 8) == sm.epoch ? (uint32_t)(v & 255u) : 255u;
}

// Leaf of point p in tree u.  With LC = 4 (four trees) the point's four
// leaf ids come from one 16-byte load; LC = 0 reads them one by one.
template <int LC>
struct PointLeaves {
  uint32_t v[LC ? LC : 1];
  const uint32_t *row;
  __device__ __forceinline__ PointLeaves(const QueryIndexView &ix, uint32_t p) {
    row = ix.leaf_of + (int64_t)p * ix.L;
    if (LC == 4) {
      const uint4 w = *reinterpret_cast<const uint4 *>(row);
      v[0] = w.x; v[LC > 1 ? 1 : 0] = w.y; v[LC > 2 ? 2 : 0] = w.z; v[LC > 3 ? 3 : 0] = w.w;
    }
  }
  __device__ __forceinline__ uint32_t operator[](int u) const { return LC == 4 ? v[u & 3] : row[u]; }
};

// Smallest level of point p over trees t' < tlim (255 if none).
template <int LC>
__device__ __forceinline__ uint32_t min_level_before(const QueryIndexView &ix, const Slot &s,
                                                     const QShared &sm, const float *lut,
                                                     uint32_t p, int tlim) {
  uint32_t f = 255u;
  const PointLeaves<LC> lf(ix, p);
  const int L = LC ? LC : ix.L;
#pragma unroll
  for (int u = 0; u < L; ++u)
    if (u < tlim) f = min(f, leaf_level_h(ix, s, sm, lut, u, lf[u]));
  return f;
}

// ---- step 1: range-query levels, expanding leaf blocks in level order ----
// For tree t: hull levels of every block; blocks at level <= the current
// bound J are bucketed by level and expanded in ascending order.  A leaf's
// level is never below its block's, so after expanding the blocks of level
// <= j the per-level point counts of tree t are complete up to j.  Expansion
// stops at the first j where tree t alone holds beta*n + k points (that j
// bounds j* from above) or at J; J shrinks to it.  Every leaf of level <= the
// final J therefore ends up expanded and listed.
__device__ __forceinline__ void expand_levels(QCtx &c) {
  const QueryIndexView &ix = c.ix;
  QShared &sm = c.sm;
  const int K = ix.K, NR1 = ix.N_r + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float *qp = c.qa.Qp + c.qi * ix.LK;
  // The first tree starts from a guessed bound (this CTA's previous final
  // bound plus a margin) so that the second hull level can prune its scan as
  // well.  If the tree does not reach beta*n + k within the guess, it is
  // expanded again without one; either way every leaf at or below its
  // crossing level is listed and counted, so the results do not depend on it.
  if (threadIdx.x == 0) sm.jhi = min(NLEV - 1, sm.jguess + 2);
  __syncthreads();
  for (int t = 0; t < ix.L; ++t) {
    build_lut(c.lut, ix.B, qp + t * K, t, K, NR1);
    sm.rh[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
      sm.nlist[t] = 0; sm.cum = 0; sm.stop = 0; sm.jcur = NLEV; sm.crossed = 0;
    }
    __syncthreads();
    const uint32_t J0 = (uint32_t)sm.jhi;
    const int64_t nb = ix.blk_off[t + 1] - ix.blk_off[t];
    const int64_t nl = ix.leaf_off[t + 1] - ix.leaf_off[t];
    const uint4 *hlo = reinterpret_cast<const uint4 *>(ix.blk_lo) + ix.blk_off[t];
    const uint4 *hhi = reinterpret_cast<const uint4 *>(ix.blk_hi) + ix.blk_off[t];
    uint8_t *blev = c.s.blev + ix.blk_off[t];
    // Once a bound J0 is known (every tree after the first), the hulls of
    // runs of LEAF_BLOCK hulls prune the hull scan: a run whose hull lies
    // beyond T[J0] holds no hull, leaf or point within it.  The scan then
    // covers the hulls of the listed runs (listed in the cut-count array,
    // free until the cut).
    const bool prune = J0 < (uint32_t)(NLEV - 1);
    uint32_t *slist = c.s.cval;
    int64_t nscan = nb;
    if (prune) {
      const int64_t ns = ix.sblk_off[t + 1] - ix.sblk_off[t];
      const uint4 *slo = reinterpret_cast<const uint4 *>(ix.sblk_lo) + ix.sblk_off[t];
      const uint4 *shi = reinterpret_cast<const uint4 *>(ix.sblk_hi) + ix.sblk_off[t];
      // With more than qa.top_min super-hulls (by default 1,024: about a
      // million leaves per tree) the top hulls (runs of LEAF_BLOCK
      // super-hulls) are tested first and only the super-hulls of the listed
      // ones follow; their list goes after the top list (both fit: nt + ns <=
      // 2 ns <= the tree's leaves once ns > 1; smaller trees skip this level).
      const bool two = ns > max((int64_t)c.qa.top_min, (int64_t)1);
      int64_t nsc = ns;
      uint32_t *tlist = c.s.cval;
      if (two) {
        const int64_t nt = ix.tblk_off[t + 1] - ix.tblk_off[t];
        const uint4 *tlo = reinterpret_cast<const uint4 *>(ix.tblk_lo) + ix.tblk_off[t];
        const uint4 *thi = reinterpret_cast<const uint4 *>(ix.tblk_hi) + ix.tblk_off[t];
        if (threadIdx.x == 0) { sm.cpos = 0; sm.n_blocks += (unsigned long long)nt; }
        __syncthreads();
        for (int64_t u = threadIdx.x; u < nt; u += QT)
          if (box_lb2(c.lut, tlo[u], thi[u]) <= sm.T[J0]) tlist[atomicAdd(&sm.cpos, 1u)] = (uint32_t)u;
        __syncthreads();
        nsc = (int64_t)sm.cpos * LEAF_BLOCK;
        slist = c.s.cval + nt;
        __syncthreads();  // every thread has read cpos
      }
      if (threadIdx.x == 0) { sm.cpos = 0; sm.n_blocks += (unsigned long long)nsc; }
      __syncthreads();
      for (int64_t i = threadIdx.x; i < nsc; i += QT) {
        const int64_t u = two ? (int64_t)tlist[i / LEAF_BLOCK] * LEAF_BLOCK + (i % LEAF_BLOCK) : i;
        if (u < ns && box_lb2(c.lut, slo[u], shi[u]) <= sm.T[J0]) slist[atomicAdd(&sm.cpos, 1u)] = (uint32_t)u;
      }
      __syncthreads();
      nscan = (int64_t)sm.cpos * LEAF_BLOCK;
    }
    auto blk = [&](int64_t i) -> int64_t {  // i-th hull of the scan
      return prune ? (int64_t)slist[i / LEAF_BLOCK] * LEAF_BLOCK + (i % LEAF_BLOCK) : i;
    };
    for (int64_t b0 = 0; b0 < nscan; b0 += QT) {  // uniform trip count for the warp collectives
      const int64_t i = b0 + threadIdx.x;
      const int64_t b = i < nscan ? blk(i) : nb;
      uint32_t lv = 255u;
      // level <= J0 exactly when LB^2 <= T[J0]; only those need their level.
      // Half the dimensions first: a warp whose hulls are all beyond T[J0]
      // by then skips the rest (partial sums only grow).
      const float thr0 = sm.T[J0];
      uint4 hl = make_uint4(0, 0, 0, 0), hh = make_uint4(0, 0, 0, 0);
      float lb = 0.0f;
      if (b < nb) { hl = hlo[b]; hh = hhi[b]; lb = box_lb2_part<0, LUT_ROWS / 2>(c.lut, hl, hh, 0.0f); }
      if (__any_sync(FULL, b < nb && lb <= thr0) && b < nb)
        lb = box_lb2_part<LUT_ROWS / 2, LUT_ROWS>(c.lut, hl, hh, lb);
      if (b < nb) {
        if (lb <= thr0) lv = level_of(sm.T, lb, c.qa.lg_eps2, c.qa.inv_2lg_c);
        blev[b] = (uint8_t)lv;
        if (lv <= J0) atomicMin(&sm.jcur, (int)lv);
      }
      const unsigned vm = __ballot_sync(FULL, b < nb);
      if ((threadIdx.x & 31) == 0) atomicAdd(&sm.n_blocks, (unsigned long long)__popc(vm));
      warp_bin_count(sm.rh, b < nb && lv <= J0, lv, 1u);
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive prefix of the per-level block counts
      uint32_t v[8], sum = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) { v[i] = sm.rh[lane * 8 + i]; sum += v[i]; }
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
      }
      uint32_t acc = incl - sum;
#pragma unroll
      for (int i = 0; i < 8; ++i) { sm.bstart[lane * 8 + i] = acc; acc += v[i]; }
    }
    __syncthreads();
    // bucket the scanned blocks by level (ids in border[bstart[lv] ...])
    for (int64_t i = threadIdx.x; i < nscan; i += QT) {
      const int64_t b = blk(i);
      if (b >= nb) continue;
      const uint32_t lv = blev[b];
      if (lv <= J0) {
        const uint32_t pos = atomicAdd(&sm.bstart[lv], 1u);
        c.s.border[ix.blk_off[t] + pos] = (uint32_t)b;
      }
    }
    __syncthreads();
    // bstart[j] now holds the end of bucket j; its start is end - count
    uint32_t *hist_t = c.hist + t * 256;
    const uint4 *llo = reinterpret_cast<const uint4 *>(ix.leaf_lo) + ix.leaf_off[t];
    const uint4 *lhi = reinterpret_cast<const uint4 *>(ix.leaf_hi) + ix.leaf_off[t];
    // Expand the level-sorted blocks in chunks.  After a chunk, every block
    // below the level of the next unexpanded block is done, so this tree's
    // point counts are complete for those levels: check them for beta*n + k.
    if (threadIdx.x == 0) { sm.cpos = 0; sm.jchk = sm.jcur; }
    __syncthreads();
    const uint32_t nsel = sm.bstart[255];
    while (true) {
      const uint32_t Jnow = (uint32_t)sm.jhi;
      const uint32_t p0c = sm.cpos, p1c = min(nsel, p0c + (uint32_t)(c.qa.expand_runs * QW));
      // the level of the first block after this chunk (thread 0 needs it
      // after the chunk)
      int jnext = NLEV;
      if (threadIdx.x == 0 && p1c < nsel) jnext = (int)blev[c.s.border[ix.blk_off[t] + p1c]];
      // This warp's runs of the chunk are p0c + warp + r QW, r < nr: their
      // block ids in one load, then each run's boxes and leaf offsets are
      // fetched one run ahead of the run being tested.
      const int nr = p1c > p0c + (uint32_t)warp ? (int)((p1c - p0c - warp + QW - 1) / QW) : 0;
      uint32_t myb = 0;
      if (lane < nr) myb = c.s.border[ix.blk_off[t] + p0c + warp + lane * QW];
      const float thr = sm.T[Jnow];
      const uint32_t *lbeg = ix.leaf_begin + ix.leaf_off[t] + t;
      uint4 nlo = make_uint4(0, 0, 0, 0), nhi = make_uint4(0, 0, 0, 0);
      uint32_t nb0 = 0, nb1 = 0, nl_id = 0;
      auto fetch = [&](int r) {  // run r into the "next" registers
        nl_id = __shfl_sync(FULL, myb, r) * LEAF_BLOCK + lane;
        if (nl_id < (uint32_t)nl) {
          nlo = llo[nl_id];
          nhi = lhi[nl_id];
          nb0 = lbeg[nl_id];
          nb1 = lbeg[nl_id + 1];
        }
      };
      if (nr > 0) fetch(0);
      for (int r = 0; r < nr; ++r) {
        const uint4 blo = nlo, bhi = nhi;
        const uint32_t l = nl_id, sz_all = nb1 - nb0;
        if (r + 1 < nr) fetch(r + 1);
        const bool valid = l < (uint32_t)nl;
        uint32_t lv = 255u;
        float lb = 0.0f;
        uint32_t sz = 0;
        // Half the dimensions first: when every leaf of the run is already
        // above T[Jnow] the rest is skipped (partial sums only grow).
        if (valid) lb = box_lb2_part<0, LUT_ROWS / 2>(c.lut, blo, bhi, 0.0f);
        const bool more = __any_sync(FULL, valid && lb <= thr);
        if (valid && more) lb = box_lb2_part<LUT_ROWS / 2, LUT_ROWS>(c.lut, blo, bhi, lb);
        if (valid && more) {
          // Leaves above Jnow are never needed again (every later test is
          // against a bound <= Jnow), so only the others get their level and
          // size and are listed; the rest read as level 255.
          if (lb <= thr) {
            lv = level_of(sm.T, lb, c.qa.lg_eps2, c.qa.inv_2lg_c);
            sz = sz_all;
          }
        }
        const bool keep = valid && lv <= Jnow;
        warp_bin_add(hist_t, keep, lv, sz);
        const unsigned km = __ballot_sync(FULL, keep);
        const unsigned vm = __ballot_sync(FULL, valid);
        if (lane == 0) atomicAdd(&sm.n_leaves, (unsigned long long)__popc(vm));
        uint32_t p0 = 0;
        if (lane == 0 && km) p0 = atomicAdd(&sm.nlist[t], (uint32_t)__popc(km));
        p0 = __shfl_sync(FULL, p0, 0);
        if (keep) {
          const uint32_t pos = (uint32_t)ix.leaf_off[t] + p0 + __popc(km & ((1u << lane) - 1u));
          c.s.lleaf[pos] = l;
          c.s.llb2[pos] = lb;
          c.s.llev[pos] = (uint8_t)lv;
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        int j = sm.jchk;
        for (; j < jnext && j <= sm.jhi; ++j) {
          sm.cum += hist_t[j];
          if (sm.cum >= (uint64_t)c.tau) { sm.jhi = j; sm.stop = 1; sm.crossed = 1; break; }
        }
        sm.jchk = j;  // first level not yet added
        if (jnext > sm.jhi || p1c >= nsel) sm.stop = 1;
        sm.cpos = p1c;
      }
      __syncthreads();
      if (sm.stop) break;
    }
    __syncthreads();
    if (t == 0 && !sm.crossed && J0 < (uint32_t)(NLEV - 1)) {
      // the guessed bound was too low: expand the first tree again without it
      for (int i = threadIdx.x; i < 256; i += QT) hist_t[i] = 0;
      if (threadIdx.x == 0) sm.jhi = NLEV - 1;
      __syncthreads();
      t = -1;
      continue;
    }
  }
  if (threadIdx.x == 0) sm.jguess = sm.jhi;
}

// ---- step 1b: shared-memory table of the levels at or below the bound ----
// Reuses the lookup table's space (no longer needed): keys (global leaf
// index + 1, 0 = empty) then one level byte per slot, linear probing.
// Floats of the shared region that holds the projection LUT during the
// expansion and the leaf-level hash after it: the LUT's size, or hash_kb KiB
// when that is larger (a larger hash keeps the levels of more listed leaves
// on chip, at the cost of fewer resident CTAs per SM).
__host__ __device__ __forceinline__ int lut_region_floats(int hash_kb) {
  return LUT_ROWS * LUT_STRIDE > hash_kb * 256 ? LUT_ROWS * LUT_STRIDE : hash_kb * 256;
}

__device__ __forceinline__ void build_level_hash(QCtx &c) {
  const QueryIndexView &ix = c.ix;
  QShared &sm = c.sm;
  const uint32_t jhi = (uint32_t)sm.jhi;
  const uint32_t bytes = (uint32_t)(lut_region_floats(c.qa.hash_kb) * sizeof(float));
  uint32_t bits = 0;
  while ((1u << (bits + 1)) * 5u <= bytes && bits + 1 <= 16) ++bits;
  if (threadIdx.x == 0) { sm.hash_count = 0; sm.hash_bits = bits; }
  __syncthreads();
  uint32_t cnt = 0;
  for (int t = 0; t < ix.L; ++t)
    for (int64_t e = threadIdx.x; e < sm.nlist[t]; e += QT)
      cnt += c.s.llev[ix.leaf_off[t] + e] <= jhi;
  atomicAdd(&sm.hash_count, cnt);
  __syncthreads();
  const uint32_t slots = 1u << bits;
  const bool use = bits >= 4 && sm.hash_count * 2u <= slots;
  if (!use) {  // the slot's epoch-tagged level array instead: every listed leaf
    const unsigned long long ep = sm.epoch;
    for (int t = 0; t < ix.L; ++t)
      for (int64_t e = threadIdx.x; e < sm.nlist[t]; e += QT)
        c.s.lev[ix.leaf_off[t] + c.s.lleaf[ix.leaf_off[t] + e]] = (ep << 8) | c.s.llev[ix.leaf_off[t] + e];
    if (threadIdx.x == 0) sm.use_hash = 0;
    __syncthreads();
    return;
  }
  uint32_t *keys = reinterpret_cast<uint32_t *>(c.lut);
  uint8_t *levs = reinterpret_cast<uint8_t *>(keys + slots);
  for (uint32_t i = threadIdx.x; i < slots; i += QT) keys[i] = 0u;
  __syncthreads();
  for (int t = 0; t < ix.L; ++t) {
    for (int64_t e = threadIdx.x; e < sm.nlist[t]; e += QT) {
      const uint32_t lv = c.s.llev[ix.leaf_off[t] + e];
      if (lv > jhi) continue;
      const uint32_t key = (uint32_t)(ix.leaf_off[t] + c.s.lleaf[ix.leaf_off[t] + e]) + 1u;
      uint32_t h = (key * 0x9E3779B1u) >> (32 - bits);
      while (true) {
        const uint32_t old = atomicCAS(&keys[h], 0u, key);
        if (old == 0u || old == key) { levs[h] = (uint8_t)lv; break; }
        h = (h + 1u) & (slots - 1u);
      }
    }
  }
  if (threadIdx.x == 0) sm.use_hash = 1;
  __syncthreads();
}

// ---- flattened visit of the points of listed leaves ------------------------
// Threads are spread over points rather than leaves (leaves hold ~20 points
// on average): per chunk of listed leaves, a block scan lays out the points of
// the leaves selected by pred, and each warp walks a run of consecutive
// points, a lane finding the leaf of its first point by a binary search in
// shared memory.  fn(valid, point, entry, level) is called
// by every thread with a uniform trip count, so it may use warp collectives.
// With count set, the points visited are added to the CTA's work counter.
template <class Pred, class Fn>
__device__ __forceinline__ void visit_points(QCtx &c, int t, Pred pred, Fn fn, bool count = false) {
  const QueryIndexView &ix = c.ix;
  QShared &sm = c.sm;
  const int64_t nlist = sm.nlist[t];
  const int64_t lo0 = ix.leaf_off[t];
  const uint32_t *permt = ix.perm + (int64_t)t * ix.n;
  // chunk layout in the top-k arrays (free until the top-k step of a query):
  // point prefix [FLC + 1], leaf level bytes [FLC]; perm begin, list entry [FLC] each
  uint32_t *fl_pre = sm.topk_key;
  uint8_t *fl_lev = reinterpret_cast<uint8_t *>(sm.topk_key + 520);
  uint32_t *fl_beg = sm.topk_id;
  uint32_t *fl_ent = sm.topk_id + FLC;
  const int fc = c.qa.visit_chunk;  // <= FLC
  for (int64_t e0 = 0; e0 < nlist; e0 += fc) {
    uint32_t q[2], sz[2], bg[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t e = e0 + threadIdx.x * 2 + u;
      q[u] = 0; sz[u] = 0; bg[u] = 0;
      if ((int)threadIdx.x * 2 + u < fc && e < nlist && pred(e)) {
        const uint32_t leaf = c.s.lleaf[lo0 + e];
        bg[u] = leaf_begin_of(ix, t, leaf);
        sz[u] = leaf_begin_of(ix, t, leaf + 1) - bg[u];
        q[u] = 1;
      }
    }
    uint32_t nq, np, qs, ps;
    if (ix.max_leaf_size < 8192) {  // one scan of (count << 22 | points): 512 leaves of < 8192 points fit
      uint32_t tot;
      const uint32_t ex = block_exclusive_scan(((q[0] + q[1]) << 22) | (sz[0] + sz[1]), sm.wt, &tot);
      qs = ex >> 22; ps = ex & 0x3fffffu; nq = tot >> 22; np = tot & 0x3fffffu;
    } else {
      qs = block_exclusive_scan(q[0] + q[1], sm.wt, &nq);
      ps = block_exclusive_scan(sz[0] + sz[1], sm.wt, &np);
    }
    {
      uint32_t slot = qs, pre = ps;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (q[u]) {
          const int64_t e = e0 + threadIdx.x * 2 + u;
          fl_pre[slot] = pre;
          fl_beg[slot] = bg[u];
          fl_ent[slot] = (uint32_t)e;
          fl_lev[slot] = c.s.llev[lo0 + e];
          ++slot;
          pre += sz[u];
        }
      }
    }
    if (threadIdx.x == 0) {
      fl_pre[nq] = np;
      if (count) sm.n_visit += np;
    }
    __syncthreads();
    // each warp walks a run of P * 32 consecutive points, lane-interleaved
    // (coalesced): one search for the leaf of a lane's first point, then
    // forward steps over leaf boundaries
    const uint32_t P = (np + QT - 1) / QT;
    const uint32_t i0 = (threadIdx.x >> 5) * P * 32u + (threadIdx.x & 31);
    int cur = 0;
    if (i0 < np) {
      int hi = (int)nq;  // last k with fl_pre[k] <= i0
      while (hi - cur > 1) {
        const int mid = (cur + hi) >> 1;
        if (fl_pre[mid] <= i0) cur = mid; else hi = mid;
      }
    }
    // Software pipeline: the point of step r + 1 is read from perm while
    // step r runs, and its leaf ids (leaf_of, read by every caller) are
    // prefetched into L1 after step r.
    auto locate = [&](uint32_t i, uint32_t &p, uint32_t &ent, uint32_t &lev) {
      while (fl_pre[cur + 1] <= i) ++cur;
      p = permt[fl_beg[cur] + (i - fl_pre[cur])];
      ent = fl_ent[cur];
      lev = fl_lev[cur];
    };
    uint32_t pn = 0, entn = 0, levn = 255u;
    bool validn = P > 0 && i0 < np;
    if (validn) locate(i0, pn, entn, levn);
    for (uint32_t r = 0; r < P; ++r) {
      const bool valid = validn;
      const uint32_t p = pn, ent = entn, lev = levn;
      const uint32_t inext = i0 + (r + 1) * 32u;
      validn = r + 1 < P && inext < np;
      if (validn) locate(inext, pn, entn, levn);
      fn(valid, p, ent, lev);
      if (validn) asm volatile("prefetch.global.L1 [%0];" ::"l"(ix.leaf_of + (int64_t)pn * ix.L));
    }
    __syncthreads();
  }
}

// ---- step 2: union counts and per-tree new-point counts ------------------
// A point of tree t's listed leaves at level lv_t is new in tree t for the
// levels in [lv_t, f_t), f_t = its smallest level in trees u < t: D_t gets +1
// at lv_t and -1 at f_t.  For every level j exactly one tree counts a point
// whose smallest level is <= j (the first tree reaching j), so the union
// increments are H[j] = sum_t D_t[j] and only the earlier trees' levels are
// looked up.  The fixed-r_min loop needs per-tree owner counts instead
// (owner = the tree of the point's smallest level): every tree's level.
template <int LC>
__device__ __forceinline__ void union_counts_t(QCtx &c) {
  const QueryIndexView &ix = c.ix;
  const uint32_t jhi = (uint32_t)c.sm.jhi;
  const bool fixed = c.qa.policy == DETLSH_RMIN_FIXED;
  const int L = LC ? LC : ix.L;
  for (int t = 0; t < L; ++t) {
    const int64_t lo0 = ix.leaf_off[t];
    uint32_t *Dt = reinterpret_cast<uint32_t *>(c.D + t * 256);
    if (fixed) {
      visit_points(
          c, t, [&](int64_t e) { return c.s.llev[lo0 + e] <= jhi; },
          [&](bool valid, uint32_t p, uint32_t, uint32_t lvt) {
            uint32_t m = 255u;
            int owner = -1;
            if (valid) {
              const PointLeaves<LC> lf(ix, p);
#pragma unroll
              for (int u = 0; u < L; ++u) {
                const uint32_t lv = (u == t) ? lvt : leaf_level_h(ix, c.s, c.sm, c.lut, u, lf[u]);
                if (lv < m) { m = lv; owner = u; }
              }
            }
            warp_bin_count(c.sm.H, valid && owner == t, m, 1u);
            warp_bin_count(Dt, valid && owner == t, m, 1u);  // owned by tree t, by smallest level
          },
          true);
    } else {
      visit_points(
          c, t, [&](int64_t e) { return c.s.llev[lo0 + e] <= jhi; },
          [&](bool valid, uint32_t p, uint32_t, uint32_t lvt) {
            uint32_t f = 255u;
            if (valid && t > 0) {
              const PointLeaves<LC> lf(ix, p);
#pragma unroll
              for (int u = 0; u < L; ++u)
                if (u < t) f = min(f, leaf_level_h(ix, c.s, c.sm, c.lut, u, lf[u]));
            }
            warp_bin_count(Dt, valid && f > lvt, lvt, 1u);
            warp_bin_count(Dt, valid && f > lvt && f <= jhi, f, 0xffffffffu);  // -1 (two's complement)
          },
          true);
    }
  }
  __syncthreads();
  if (!fixed) {
    for (int j = threadIdx.x; j < 256; j += QT) {
      int32_t h = 0;
      for (int t = 0; t < L; ++t) h += c.D[t * 256 + j];
      c.sm.H[j] = (uint32_t)h;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void union_counts(QCtx &c) {
  if (c.ix.L == 4) union_counts_t<4>(c);
  else union_counts_t<0>(c);
}

// ---- step 3: candidate cut inside tree i* and candidate list -------------
template <int LC>
__device__ __forceinline__ void cut_and_collect_t(QCtx &c) {
  const QueryIndexView &ix = c.ix;
  const uint32_t js = (uint32_t)c.sm.jstar;
  const int is = c.sm.istar;
  const int64_t li0 = ix.leaf_off[is];
  const int64_t nli = c.sm.nlist[is];
  // new points of every qualifying listed leaf of tree i*
  for (int64_t e = threadIdx.x; e < nli; e += QT) {
    uint32_t v = 0;
    if (is == 0 && c.s.llev[li0 + e] <= js) {
      const uint32_t leaf = c.s.lleaf[li0 + e];
      v = leaf_begin_of(ix, is, leaf + 1) - leaf_begin_of(ix, is, leaf);
    }
    c.s.cval[e] = v;
  }
  __syncthreads();
  if (is > 0) {
    visit_points(
        c, is, [&](int64_t e) { return c.s.llev[li0 + e] <= js; },
        [&](bool valid, uint32_t p, uint32_t ent, uint32_t) {
          const bool nw = valid && min_level_before<LC>(ix, c.s, c.sm, c.lut, p, is) > js;
          warp_bin_count(c.s.cval, nw, ent, 1u);
        });
  }
  __syncthreads();
  // priority order (LB^2, leaf index): smallest LB^2 value v reaching the
  // count still needed, then the smallest leaf index among LB^2 == v (with
  // whole trees joining S, tree i* is taken whole)
  const uint32_t need = c.sm.need;
  uint32_t v = 0xffffffffu, cut = 0xffffffffu;
  if (!c.qa.per_tree) {
    auto get_lb = [&](int64_t i, uint32_t &k, uint32_t &w) {
      w = (c.s.llev[li0 + i] <= js) ? c.s.cval[i] : 0u;
      k = __float_as_uint(c.s.llb2[li0 + i]);
    };
    block_select(nli, get_lb, need, c.sm);
    v = c.sm.sel_v;
    const uint32_t need2 = need - c.sm.sel_below;
    if (need2 < c.sm.sel_at) {  // else every leaf at LB^2 == v is needed
      auto get_id = [&](int64_t i, uint32_t &k, uint32_t &w) {
        const bool q = c.s.llev[li0 + i] <= js && __float_as_uint(c.s.llb2[li0 + i]) == v;
        w = q ? c.s.cval[i] : 0u;
        k = c.s.lleaf[li0 + i];
      };
      block_select(nli, get_id, need2, c.sm);
      cut = c.sm.sel_v;
    }
  }
  // collect S: trees before i* whole (new points only), tree i* up to the cut
  if (threadIdx.x == 0) c.sm.ncand = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int t = 0; t <= is; ++t) {
    const int64_t lo0 = ix.leaf_off[t];
    visit_points(
        c, t,
        [&](int64_t e) {
          if (c.s.llev[lo0 + e] > js) return false;
          if (t < is) return true;
          const uint32_t kb = __float_as_uint(c.s.llb2[lo0 + e]);
          return kb < v || (kb == v && c.s.lleaf[lo0 + e] <= cut);
        },
        [&](bool valid, uint32_t p, uint32_t, uint32_t) {
          const bool take = valid && (t == 0 || min_level_before<LC>(ix, c.s, c.sm, c.lut, p, t) > js);
          const unsigned tm = __ballot_sync(FULL, take);
          uint32_t pos0 = 0;
          if (lane == 0 && tm) pos0 = atomicAdd(&c.sm.ncand, (uint32_t)__popc(tm));
          pos0 = __shfl_sync(FULL, pos0, 0);
          const uint32_t pos = pos0 + __popc(tm & ((1u << lane) - 1u));
          if (take && pos < (uint32_t)c.qa.cand_cap) c.s.cand[pos] = p;
        });
  }
  __syncthreads();
}

__device__ __forceinline__ void cut_and_collect(QCtx &c) {
  if (c.ix.L == 4) cut_and_collect_t<4>(c);
  else cut_and_collect_t<0>(c);
}

// ---- step 4: distances ----------------------------------------------------
// Sums NV per-lane values over aligned groups of W lanes in log2(W) shuffle
// rounds: each round halves the values a lane holds by swapping half of them
// with its partner, then a butterfly finishes.  Afterwards every lane holds
// the group total of value index transpose_index<NV, W>(lane).
template <int NV, int W>
__device__ __forceinline__ float transpose_sum(float (&a)[NV], int lane) {
#pragma unroll
  for (int n = NV, off = W / 2; n > 1; n >>= 1, off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const float send = up ? a[i] : a[i + n / 2];
      const float keep = up ? a[i + n / 2] : a[i];
      a[i] = __fadd_rn(keep, __shfl_xor_sync(FULL, send, off));
    }
  }
  float v = a[0];
#pragma unroll
  for (int off = W / NV / 2; off > 0; off >>= 1) v = __fadd_rn(v, __shfl_xor_sync(FULL, v, off));
  return v;
}
template <int NV, int W>
__device__ __forceinline__ int transpose_index(int lane) {
  int idx = 0;
#pragma unroll
  for (int n = NV, off = W / 2; n > 1; n >>= 1, off >>= 1) idx = idx * 2 + ((lane & off) ? 1 : 0);
  return idx;
}

// FP32 squared distances sum((q - x)^2) of rows get_id(0..nrows) into out[]
// (as ordered uint32 keys).  A row is split over W lanes (float4 chunks when
// d % 4 == 0, else scalars); a warp keeps 4 * (32 / W) rows in flight.
template <int W, bool VEC, class GetId>
__device__ __forceinline__ void dist_fp32_rows(const QueryIndexView &ix, const float *q,
                                               int64_t nrows, GetId get_id, uint32_t *out) {
  constexpr int NV = 4, PER = 32 / W, RPI = NV * PER;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int h = lane / W, cl = lane % W;
  const int d = ix.d;
  const int nch = VEC ? d >> 2 : d;
  for (int64_t r0 = (int64_t)warp * RPI; r0 < nrows; r0 += QW * RPI) {
    uint32_t myid = 0;
    if (lane < RPI && r0 + lane < nrows) myid = get_id(r0 + lane);
    // row ids of the lane's rows (the shuffles stay outside the chunk loop,
    // whose trip count differs between lanes)
    uint32_t pid[NV];
#pragma unroll
    for (int u = 0; u < NV; ++u) pid[u] = __shfl_sync(FULL, myid, u * PER + h);
    float acc[NV];
#pragma unroll
    for (int u = 0; u < NV; ++u) acc[u] = 0.0f;
    for (int ch = cl; ch < nch; ch += W) {
      if (VEC) {
        const float4 qv = reinterpret_cast<const float4 *>(q)[ch];
        float4 xv[NV];
#pragma unroll
        for (int u = 0; u < NV; ++u)  // issue every row's load first
          xv[u] = r0 + u * PER + h < nrows
                      ? reinterpret_cast<const float4 *>(ix.X + (int64_t)pid[u] * d)[ch]
                      : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < NV; ++u) {
          const float t0 = __fsub_rn(qv.x, xv[u].x), t1 = __fsub_rn(qv.y, xv[u].y);
          const float t2 = __fsub_rn(qv.z, xv[u].z), t3 = __fsub_rn(qv.w, xv[u].w);
          acc[u] = __fmaf_rn(t0, t0, acc[u]);
          acc[u] = __fmaf_rn(t1, t1, acc[u]);
          acc[u] = __fmaf_rn(t2, t2, acc[u]);
          acc[u] = __fmaf_rn(t3, t3, acc[u]);
        }
      } else {
        const float qv = q[ch];
#pragma unroll
        for (int u = 0; u < NV; ++u) {
          const float xv = r0 + u * PER + h < nrows ? ix.X[(int64_t)pid[u] * d + ch] : qv;
          const float t0 = __fsub_rn(qv, xv);
          acc[u] = __fmaf_rn(t0, t0, acc[u]);
        }
      }
    }
    const float v = transpose_sum<NV, W>(acc, cl);
    const int64_t r = r0 + (int64_t)transpose_index<NV, W>(cl) * PER + h;
    if ((cl & (W / NV - 1)) == 0 && r < nrows) out[r] = __float_as_uint(v);
  }
}

// Rows ids[0..nrows) (ids == nullptr: rows 0..nrows) -- one instantiation
// for every caller keeps the kernel's code small.
__device__ __forceinline__ void dist_fp32(const QueryIndexView &ix, const float *q, int64_t nrows,
                                          const uint32_t *ids, uint32_t *out) {
  auto get_id = [ids](int64_t i) { return ids ? ids[i] : (uint32_t)i; };
  const int d = ix.d;
  if ((d & 3) == 0) {
    const int nch = d >> 2;
    if (nch >= 32) dist_fp32_rows<32, true>(ix, q, nrows, get_id, out);
    else if (nch >= 16) dist_fp32_rows<16, true>(ix, q, nrows, get_id, out);
    else dist_fp32_rows<8, true>(ix, q, nrows, get_id, out);
  } else {
    if (d >= 32) dist_fp32_rows<32, false>(ix, q, nrows, get_id, out);
    else if (d >= 16) dist_fp32_rows<16, false>(ix, q, nrows, get_id, out);
    else dist_fp32_rows<8, false>(ix, q, nrows, get_id, out);
  }
  __syncthreads();
}

// (key, id) of item i from two arrays (ids == nullptr: id = i).
struct ArrGet {
  const uint32_t *keys, *ids;
  __device__ void operator()(int64_t i, uint32_t &key, uint32_t &id) const {
    key = keys[i];
    id = ids ? ids[i] : (uint32_t)i;
  }
};
// key of item i from an array, weight 1.
struct ArrKey {
  const uint32_t *keys;
  __device__ void operator()(int64_t i, uint32_t &key, uint32_t &w) const {
    key = keys[i];
    w = 1u;
  }
};

// One m16n8k16 BF16 tensor-core product with FP32 accumulation (c += a b).
__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], uint32_t a0, uint32_t a1,
                                               uint32_t a2, uint32_t a3, uint32_t b0,
                                               uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Certified interval of the FP32 path's squared distance from a BF16 score.
// s = fl(fl(qn + xn) - 2 acc) estimates D~ = ||q~ - x~||^2 (q~, x~ the BF16
// rows): qn and xn are FMA sums of d non-negative terms (relative error at
// most d u each, u = 2^-24), the products of acc are exact (8-bit
// significands) and the tensor core's FP32 accumulation of the d products is
// taken to err by at most 2 ulps of 24 bits per addition (4 d u in all,
// relative to sum |q~_j x~_j| <= (|q~|^2 + |x~|^2) / 2), and the last two
// roundings add u each on magnitudes below 2 (|q~|^2 + |x~|^2).  Together
// |s - D~| <= (6d + 16) u (qn + xn) + d 2^-125 (the last term covers subnormal
// products flushed to zero).  The triangle inequality moves from D~ to the
// exact distance D of the FP32 rows: |sqrt(D) - sqrt(D~)| <= |q - q~| +
// |x - x~| (both bounded from above at build / here).  The FP32 path computes
// D with relative error at most (2d + 16) u plus d 2^-148 absolute.  Every
// step rounds outwards, so lo <= FP32 key <= hi; any NaN or overflow gives
// the empty information [0, inf].
__device__ __forceinline__ float nonneg_bits(float v) {  // -0 -> +0 (keys compare as uint)
  return __uint_as_float(__float_as_uint(v) & 0x7fffffffu);
}
__device__ __forceinline__ void bf16_interval(float s, float qn, float2 xn, float qr, int d,
                                              float &lo, float &hi) {
  const float fd = (float)d;  // the constants are recomputed here: no registers held across
  const float e = __fmaf_ru(__fmaf_ru(6.0f, fd, 16.0f) * 0x1p-24f, __fadd_ru(qn, xn.x), fd * 0x1p-125f);
  const float r = __fadd_ru(qr, xn.y);
  const float g = __fmaf_ru(2.0f, fd, 16.0f) * 0x1p-24f;
  const float dlo = fmaxf(__fsub_rd(__fsqrt_rd(fmaxf(__fsub_rd(s, e), 0.0f)), r), 0.0f);
  const float dhi = __fadd_ru(__fsqrt_ru(__fadd_ru(s, e)), r);
  lo = nonneg_bits(fmaxf(__fsub_rd(__fmul_rd(__fmul_rd(dlo, dlo), 1.0f - g), fd * 0x1p-148f), 0.0f));
  hi = __fadd_ru(__fmul_ru(__fmul_ru(dhi, dhi), __fadd_ru(1.0f, g)), fd * 0x1p-148f);
  if (!(lo <= hi)) { lo = 0.0f; hi = __int_as_float(0x7f800000); }
}

// BF16 scores on the tensor cores: score(x) = |q|^2 + |x|^2 - 2 q.x with the
// dot products of 16 candidate rows per warp and k-block of 16 from one
// m16n8k16 MMA (the query is column 0 of B; columns 1-7 are zero).  The dot
// product does not depend on the order of k, so each lane loads 4 consecutive
// elements per row and k-block (8 bytes) and the same 4 query elements are
// placed at the matching B positions: memory element 4t+{0,1,2,3} of a block
// is MMA k-index {2t, 2t+1, 2t+8, 2t+9} for lane t = lane % 4.
// cert: key[] and hkey[] get the certified interval of each candidate's FP32
// key (bf16_interval); otherwise key[] gets the score.
__device__ __forceinline__ void distances_bf16(QCtx &c, int64_t nc, bool allpts, bool cert) {
  const QueryIndexView &ix = c.ix;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int d = ix.d;  // d % 8 == 0 on this path
  const int g = lane >> 2, t = lane & 3;
  const __nv_bfloat16 *qh = c.qa.Qh + c.qi * d;
  // |q|^2 of the BF16 query and the bound of |q - bf16(q)|
  if (warp == 0) {
    const float *qf = c.qa.Q + c.qi * d;
    float a = 0.0f, r = 0.0f;
    for (int j = lane; j < d; j += 32) {
      const float f = __bfloat162float(qh[j]);
      a = __fmaf_rn(f, f, a);
      const float e = qf[j] - f;  // exact
      r = __fmaf_ru(e, e, r);
    }
    for (int o = 16; o > 0; o >>= 1) {
      a = __fadd_rn(a, __shfl_xor_sync(FULL, a, o));
      r = __fadd_ru(r, __shfl_xor_sync(FULL, r, o));
    }
    if (lane == 0) { c.sm.qn = a; c.sm.qr = __fsqrt_ru(r); }
  }
  // the query's B fragments come from shared memory (the top-k arrays are
  // free until the top-k step) when the row fits
  if (2 * d <= 4 * KMAX) {
    for (int i = threadIdx.x; i < d / 2; i += QT)
      c.sm.topk_key[i] = reinterpret_cast<const uint32_t *>(qh)[i];
    qh = reinterpret_cast<const __nv_bfloat16 *>(c.sm.topk_key);
  }
  __syncthreads();
  const float qn = c.sm.qn, qr = c.sm.qr;
  // exact BF16 rows and query: the interval needs no square roots and is
  // formed in the tile loop (constants as in bf16_interval)
  const bool fast = ix.bf16_exact && qr == 0.0f;
  const float fdd = (float)d;
  const float ecs = __fmaf_ru(6.0f, fdd, 16.0f) * 0x1p-24f, eabs = fdd * 0x1p-125f;
  const float gg = __fmaf_ru(2.0f, fdd, 16.0f) * 0x1p-24f;
  const float glo = 1.0f - gg, ghi = __fadd_ru(1.0f, gg), dabs = fdd * 0x1p-148f;
  const int nblk = (d + 15) >> 4;
  auto id_of = [&](int64_t r) -> uint32_t {
    return (lane < 16 && r + lane < nc) ? (allpts ? (uint32_t)(r + lane) : c.s.cand[r + lane]) : 0u;
  };
  uint32_t myid = id_of((int64_t)warp * 16);
  for (int64_t r0 = (int64_t)warp * 16; r0 < nc; r0 += QW * 16) {
    const uint32_t p0 = __shfl_sync(FULL, myid, g), p1 = __shfl_sync(FULL, myid, g + 8);
    const bool ok0 = r0 + g < nc, ok1 = r0 + g + 8 < nc;
    // norm terms and the next rows' ids go out with this tile's row loads
    float xn0 = 0.0f, xn1 = 0.0f;
    if (t == 0) {
      if (ok0) xn0 = ix.Xn[p0].x;
      if (ok1) xn1 = ix.Xn[p1].x;
    }
    myid = id_of(r0 + QW * 16);
    const __nv_bfloat16 *x0 = ix.Xh + (int64_t)p0 * d + 4 * t;
    const __nv_bfloat16 *x1 = ix.Xh + (int64_t)p1 * d + 4 * t;
    const __nv_bfloat16 *qt = qh + 4 * t;
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    int b = 0;
    // Pairs of k-blocks by 16-byte loads: in a 32-element chunk lane t holds
    // elements 8t..8t+7, the first four in the first block's positions
    // {2t, 2t+1, 2t+8, 2t+9}, the next four in the second block's (the same
    // bijection for the rows and the query), two chunks per step.
    const __nv_bfloat16 *x0w = ix.Xh + (int64_t)p0 * d + 8 * t;
    const __nv_bfloat16 *x1w = ix.Xh + (int64_t)p1 * d + 8 * t;
    const __nv_bfloat16 *qw = qh + 8 * t;
    for (; (b + 4) * 16 <= d; b += 4) {
      uint4 xa[2], xb[2], qv[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = (b + 2 * u) * 16;
        xa[u] = ok0 ? *reinterpret_cast<const uint4 *>(x0w + e) : make_uint4(0u, 0u, 0u, 0u);
        xb[u] = ok1 ? *reinterpret_cast<const uint4 *>(x1w + e) : make_uint4(0u, 0u, 0u, 0u);
        qv[u] = g == 0 ? *reinterpret_cast<const uint4 *>(qw + e) : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        mma_bf16_16816(acc, xa[u].x, xb[u].x, xa[u].y, xb[u].y, qv[u].x, qv[u].y);
        mma_bf16_16816(acc, xa[u].z, xb[u].z, xa[u].w, xb[u].w, qv[u].z, qv[u].w);
      }
    }
    for (; b < nblk; ++b) {
      const int e = b * 16;
      uint2 xa = make_uint2(0u, 0u), xb = make_uint2(0u, 0u), qv = make_uint2(0u, 0u);
      if (e + 4 * t < d) {  // d % 4 == 0: the 4 elements are all in range
        if (ok0) xa = *reinterpret_cast<const uint2 *>(x0 + e);
        if (ok1) xb = *reinterpret_cast<const uint2 *>(x1 + e);
        if (g == 0) qv = *reinterpret_cast<const uint2 *>(qt + e);
      }
      mma_bf16_16816(acc, xa.x, xb.x, xa.y, xb.y, qv.x, qv.y);
    }
    if (t == 0) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!(h ? ok1 : ok0)) continue;
        const float sc = __fadd_rn(__fadd_rn(qn, h ? xn1 : xn0), -2.0f * acc[2 * h]);
        const int64_t r = r0 + g + 8 * h;
        if (cert && fast) {
          // rows and query exact in BF16 (no residuals): the interval of
          // bf16_interval without its square roots
          const float e = __fmaf_ru(ecs, __fadd_ru(qn, h ? xn1 : xn0), eabs);
          const float lo = fmaxf(__fsub_rd(__fmul_rd(fmaxf(__fsub_rd(sc, e), 0.0f), glo), dabs), 0.0f);
          const float hi = __fadd_ru(__fmul_ru(__fadd_ru(sc, e), ghi), dabs);
          const bool okv = lo <= hi;  // false on NaN
          c.s.key[r] = okv ? __float_as_uint(nonneg_bits(lo)) : 0u;
          c.s.hkey[r] = okv ? __float_as_uint(hi) : 0x7f800000u;
        } else if (cert) {
          c.s.hkey[r] = __float_as_uint(sc);  // the interval follows below
        } else {
          c.s.key[r] = __float_as_uint(nonneg_bits(fmaxf(sc, 0.0f)));
        }
      }
    }
  }
  __syncthreads();
  if (cert && !fast) {  // a second pass keeps the tile loop's registers free
    for (int64_t i = threadIdx.x; i < nc; i += QT) {
      const uint32_t p = allpts ? (uint32_t)i : c.s.cand[i];
      float lo, hi;
      bf16_interval(__uint_as_float(c.s.hkey[i]), qn, ix.Xn[p], qr, d, lo, hi);
      c.s.key[i] = __float_as_uint(lo);
      c.s.hkey[i] = __float_as_uint(hi);
    }
    __syncthreads();
  }
}

// ---- step 5: top-k by (key, id) -------------------------------------------
// Selects the kk smallest (key, id) pairs among n items from get(i) and
// leaves them sorted in sm.topk_key / sm.topk_id[0..kk).
template <class Get>
__device__ __forceinline__ void topk_select(int64_t n, int kk, Get get, QShared &sm) {
  auto gk = [&](int64_t i, uint32_t &k, uint32_t &w) { uint32_t id; get(i, k, id); w = 1u; };
  block_select(n, gk, (uint32_t)kk, sm);
  const uint32_t vk = sm.sel_v;
  const uint32_t below = sm.sel_below;
  // ties at vk: the (kk - below) smallest ids, unless all of them are needed
  uint32_t idcut = 0xffffffffu;
  if ((uint32_t)kk - below < sm.sel_at) {
    auto gi = [&](int64_t i, uint32_t &k, uint32_t &w) {
      uint32_t key, id;
      get(i, key, id);
      k = id;
      w = key == vk ? 1u : 0u;
    };
    block_select(n, gi, (uint32_t)kk - below, sm);
    idcut = sm.sel_v;
  }
  if (threadIdx.x == 0) sm.nres = 0;
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += QT) {
    uint32_t key, id;
    get(i, key, id);
    if (key < vk || (key == vk && id <= idcut)) {
      const uint32_t pos = atomicAdd(&sm.nres, 1u);
      if (pos < KMAX) { sm.topk_key[pos] = key; sm.topk_id[pos] = id; }
    }
  }
  __syncthreads();
  // bitonic sort of the kk results by (key, id), padded to a power of two
  int np = 1;
  while (np < kk) np <<= 1;
  for (int i = kk + threadIdx.x; i < np; i += QT) {
    sm.topk_key[i] = 0xffffffffu;
    sm.topk_id[i] = 0xffffffffu;
  }
  __syncthreads();
  for (int size = 2; size <= np; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < np; i += QT) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const uint64_t a = ((uint64_t)sm.topk_key[i] << 32) | sm.topk_id[i];
          const uint64_t b = ((uint64_t)sm.topk_key[j] << 32) | sm.topk_id[j];
          if ((a > b) == up) {
            sm.topk_key[i] = (uint32_t)(b >> 32); sm.topk_id[i] = (uint32_t)b;
            sm.topk_key[j] = (uint32_t)(a >> 32); sm.topk_id[j] = (uint32_t)a;
          }
        }
      }
      __syncthreads();
    }
  }
}

// ---- exact test of condition 2 near the sphere ---------------------------
// ||q - x||^2 <= R^2 decided without rounding: the square expands into
// products of two floats, sum_j (q_j q_j + x_j x_j - 2 q_j x_j), and
// R = R0 + R1 + R2 (three FP32 pieces, exact) gives R^2 as nine products;
// every product is added exactly to a 640-bit fixed-point accumulator
// (digit i weighs 2^(32 i - 298)) and the sign of the sum decides.  Only
// candidates whose certified FP32 interval straddles a tested radius come
// here, one thread each.
struct Fixed640 {
  long long dig[20];
  __device__ void add(float a, float b, bool neg) {
    const uint32_t ab = __float_as_uint(a), bb = __float_as_uint(b);
    const uint32_t ae = (ab >> 23) & 0xffu, be = (bb >> 23) & 0xffu;
    const uint64_t am = (ab & 0x7fffffu) | (ae ? 0x800000u : 0u);
    const uint64_t bm = (bb & 0x7fffffu) | (be ? 0x800000u : 0u);
    if (am == 0 || bm == 0) return;
    const int pos = (int)(ae ? ae : 1u) + (int)(be ? be : 1u) - 2;  // weight of the product's bit 0: 2^(pos - 298)
    const uint64_t prod = am * bm;                                   // < 2^48, exact
    const int ci = pos >> 5, sh = pos & 31;
    const uint64_t lo = prod << sh;
    const uint64_t hi = sh ? (prod >> (64 - sh)) : 0ull;
    const long long p0 = (long long)(lo & 0xffffffffull), p1 = (long long)(lo >> 32), p2 = (long long)hi;
    if (neg != (((ab ^ bb) >> 31) != 0)) { dig[ci] -= p0; dig[ci + 1] -= p1; dig[ci + 2] -= p2; }
    else { dig[ci] += p0; dig[ci + 1] += p1; dig[ci + 2] += p2; }
  }
  // -1, 0 or +1: the sign of the accumulated value
  __device__ int sign() {
    for (int i = 0; i < 19; ++i) {
      const long long carry = dig[i] >> 32;  // floor division: digits end in [0, 2^32)
      dig[i] -= carry * 4294967296ll;
      dig[i + 1] += carry;
    }
    if (dig[19] < 0) return -1;
    for (int i = 0; i < 20; ++i)
      if (dig[i]) return 1;
    return 0;
  }
};

__device__ __noinline__ bool exact_within(const float *__restrict__ q, const float *__restrict__ x,
                                          int d, const float *__restrict__ Rp) {
  Fixed640 acc;
  for (int i = 0; i < 20; ++i) acc.dig[i] = 0;
  for (int j = 0; j < d; ++j) {
    const float a = q[j], b = x[j];
    acc.add(a, a, false);
    acc.add(b, b, false);
    acc.add(a, b, true);
    acc.add(a, b, true);
  }
  for (int u = 0; u < 3; ++u)
    for (int v = 0; v < 3; ++v) acc.add(Rp[u], Rp[v], true);
  return acc.sign() <= 0;
}

// First index i of a nondecreasing table with x <= tab[i] (tab[254] = +inf).
__device__ __forceinline__ int first_at_or_above(const float *tab, float x) {
  int lo = 0, hi = NLEV - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (x <= tab[mid]) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// ---- Alg. 5 from a fixed r_min, with condition 2 -------------------------
// Radius index i stands for r_min c^i.  j1 = the first radius whose union
// holds beta*n + k points (condition 1), if any.  Every radius before j1 is
// passed whole, so at radius j1 the loop starts from S(j1 - 1) = the points
// whose smallest level is below j1, and condition 2 can only stop it before
// j1: at the first j < j1 where k points of S(j) lie within c r_j, i.e. k
// points with max(smallest level, first radius covering their distance)
// <= j.  Otherwise at j1 the trees add, in order, the points whose smallest
// level is j1, each from the first tree attaining it; inside tree i* the
// leaves enter by (LB^2, leaf index) until the count is reached.

// Smallest level of p over trees u < t (fb) and over u > t (fa).
template <int LC>
__device__ __forceinline__ void levels_around(const QCtx &c, uint32_t p, int t, uint32_t &fb,
                                              uint32_t &fa) {
  const PointLeaves<LC> lf(c.ix, p);
  const int L = LC ? LC : c.ix.L;
  fb = 255u;
  fa = 255u;
#pragma unroll
  for (int u = 0; u < L; ++u) {
    if (u == t) continue;
    const uint32_t lv = leaf_level_h(c.ix, c.s, c.sm, c.lut, u, lf[u]);
    if (u < t) fb = min(fb, lv); else fa = min(fa, lv);
  }
}

// Appends to the candidate list, warp-aggregated.
__device__ __forceinline__ uint32_t warp_append(QCtx &c, bool take) {
  const int lane = threadIdx.x & 31;
  const unsigned tm = __ballot_sync(FULL, take);
  uint32_t pos0 = 0;
  if (lane == 0 && tm) pos0 = atomicAdd(&c.sm.ncand, (uint32_t)__popc(tm));
  pos0 = __shfl_sync(FULL, pos0, 0);
  return pos0 + __popc(tm & ((1u << lane) - 1u));
}

// S(js): every point whose smallest level is <= js, once (from the first
// tree where its level is <= js), with that smallest level in cm[].
template <int LC>
__device__ __forceinline__ void collect_below(QCtx &c, uint32_t js) {
  if (threadIdx.x == 0) c.sm.ncand = 0;
  __syncthreads();
  const int L = LC ? LC : c.ix.L;
  for (int t = 0; t < L; ++t) {
    const int64_t lo0 = c.ix.leaf_off[t];
    visit_points(
        c, t, [&](int64_t e) { return c.s.llev[lo0 + e] <= js; },
        [&](bool valid, uint32_t p, uint32_t, uint32_t lvt) {
          uint32_t fb = 0, fa = 0;
          if (valid) levels_around<LC>(c, p, t, fb, fa);
          const bool take = valid && fb > js;
          const uint32_t pos = warp_append(c, take);
          if (take && pos < (uint32_t)c.qa.cand_cap) {
            c.s.cand[pos] = p;
            c.s.cm[pos] = (uint8_t)min(lvt, fa);
          }
        });
  }
  __syncthreads();
}

// Condition 1 at radius j1 after S(j1 - 1): the cut in tree i* and the new
// points of trees <= i*, appended after the ncA points already listed.
template <int LC>
__device__ __forceinline__ void cut_and_collect_fixed(QCtx &c, uint32_t j1) {
  const QueryIndexView &ix = c.ix;
  const int is = c.sm.istar;
  const int64_t li0 = ix.leaf_off[is];
  const int64_t nli = c.sm.nlist[is];
  for (int64_t e = threadIdx.x; e < nli; e += QT) c.s.cval[e] = 0u;
  __syncthreads();
  // new points of tree i*'s leaves at level j1: smallest level j1, first tree
  visit_points(
      c, is, [&](int64_t e) { return c.s.llev[li0 + e] == j1; },
      [&](bool valid, uint32_t p, uint32_t ent, uint32_t) {
        uint32_t fb = 0, fa = 0;
        if (valid) levels_around<LC>(c, p, is, fb, fa);
        warp_bin_count(c.s.cval, valid && fb > j1 && fa >= j1, ent, 1u);
      });
  __syncthreads();
  const uint32_t need = c.sm.need;
  auto get_lb = [&](int64_t i, uint32_t &k, uint32_t &w) {
    w = (c.s.llev[li0 + i] <= j1) ? c.s.cval[i] : 0u;
    k = __float_as_uint(c.s.llb2[li0 + i]);
  };
  block_select(nli, get_lb, need, c.sm);
  const uint32_t v = c.sm.sel_v;
  const uint32_t need2 = need - c.sm.sel_below;
  uint32_t cut = 0xffffffffu;
  if (need2 < c.sm.sel_at) {
    auto get_id = [&](int64_t i, uint32_t &k, uint32_t &w) {
      const bool q = c.s.llev[li0 + i] <= j1 && __float_as_uint(c.s.llb2[li0 + i]) == v;
      w = q ? c.s.cval[i] : 0u;
      k = c.s.lleaf[li0 + i];
    };
    block_select(nli, get_id, need2, c.sm);
    cut = c.sm.sel_v;
  }
  for (int t = 0; t <= is; ++t) {
    const int64_t lo0 = ix.leaf_off[t];
    visit_points(
        c, t,
        [&](int64_t e) {
          if (c.s.llev[lo0 + e] != j1) return false;
          if (t < is) return true;
          const uint32_t kb = __float_as_uint(c.s.llb2[lo0 + e]);
          return kb < v || (kb == v && c.s.lleaf[lo0 + e] <= cut);
        },
        [&](bool valid, uint32_t p, uint32_t, uint32_t) {
          uint32_t fb = 0, fa = 0;
          if (valid) levels_around<LC>(c, p, t, fb, fa);
          const bool take = valid && fb > j1 && fa >= j1;
          const uint32_t pos = warp_append(c, take);
          if (take && pos < (uint32_t)c.qa.cand_cap) c.s.cand[pos] = p;
        });
  }
  __syncthreads();
}

// The whole fixed-r_min resolution after the union counts: fills S, j and
// the stopping tree (-1 = condition 2), and the top-k in sm.topk_*.
template <int LC>
__device__ __forceinline__ int64_t fixed_rmin_query(QCtx &c, int k) {
  const QueryIndexView &ix = c.ix;
  QShared &sm = c.sm;
  const int64_t tau = c.tau;
  const uint32_t j1 = (sm.sel_g <= sm.jhi) ? (uint32_t)sm.sel_g : (uint32_t)NLEV;
  // rounded-down and rounded-up (c r_i)^2 in shared memory (both arrays are
  // free after the expansion and the union counts)
  float *Tcl = reinterpret_cast<float *>(sm.bstart);
  float *Tch = reinterpret_cast<float *>(sm.H);
  for (int i = threadIdx.x; i < 256; i += QT) { Tcl[i] = c.qa.Tc[i]; Tch[i] = c.qa.Tc[256 + i]; }
  const float *Rp = c.qa.Tc + 512;
  const float *q = c.qa.Q + c.qi * ix.d;
  const uint32_t *cand = c.s.cand;
  int64_t ncA = 0;
  if (j1 > 0) {
    collect_below<LC>(c, j1 - 1);
    ncA = min((int64_t)sm.ncand, c.qa.cand_cap);
    dist_fp32(ix, q, ncA, cand, c.s.key);
    // condition 2: first j < j1 with k points of max(level, covering radius) <= j
    sm.rh[threadIdx.x] = 0;
    __syncthreads();
    // The covering radius of a candidate (first i with ||q - x|| <= c r_i):
    // the FP32 key is within (2d + 16) u relative plus d 2^-148 of the exact
    // squared distance, so from i1 (its upper end below the rounded-down
    // (c r_i)^2) it is certainly within and before i0 (its lower end above
    // the rounded-up one) certainly not; the radii in between are decided
    // exactly.  Only max(covering radius, smallest level) < j1 matters.
    const float fd = (float)ix.d;
    const float g = __fmaf_ru(2.0f, fd, 16.0f) * 0x1p-24f;
    for (int64_t i = threadIdx.x; i < ncA; i += QT) {
      const float d2 = __uint_as_float(c.s.key[i]);
      const float lo2 = fmaxf(__fsub_rd(__fmul_rd(d2, 1.0f - g), fd * 0x1p-148f), 0.0f);
      const float hi2 = __fadd_ru(__fmul_ru(d2, __fadd_ru(1.0f, g)), fd * 0x1p-148f);
      const int i1 = first_at_or_above(Tcl, hi2), i0 = first_at_or_above(Tch, lo2);
      const uint32_t cmv = c.s.cm[i];
      int cov = i1;
      if (i0 < i1 && (uint32_t)i0 < j1 && cmv < (uint32_t)i1) {
        const float *xp = ix.X + (int64_t)cand[i] * ix.d;
        for (int r = i0; r < i1; ++r)
          if (exact_within(q, xp, ix.d, Rp + 3 * r)) { cov = r; break; }
      }
      const uint32_t b = max((uint32_t)cov, cmv);
      if (b < j1) atomicAdd(&sm.rh[b], 1u);
    }
    __syncthreads();
    warp_first_crossing(sm.rh, 0, (uint64_t)k, &sm.sel_g, &sm.sel_bf);
    __syncthreads();
    const uint32_t j2 = (uint32_t)sm.sel_g;
    if (j2 < j1 && sm.sel_g < 255) {
      // stop by condition 2 at radius j2: S = S(j2), top-k of it
      if (threadIdx.x == 0) { sm.jstar = (int)j2; sm.istar = -1; sm.nres = 0; }
      __syncthreads();
      int64_t* Sout = c.qa.S_out;
      for (int64_t i = threadIdx.x; i < ncA; i += QT) {
        if (c.s.cm[i] <= j2) {
          const uint32_t pos = atomicAdd(&sm.nres, 1u);
          if (Sout && pos < c.qa.S_cap) Sout[c.qi * c.qa.S_cap + pos] = cand[i];
        }
      }
      __syncthreads();
      const int64_t ns = sm.nres;
      __syncthreads();
      auto get_s = [&](int64_t i, uint32_t &key, uint32_t &id) {
        key = c.s.cm[i] <= j2 ? c.s.key[i] : 0xffffffffu;
        id = cand[i];
      };
      topk_select(ncA, k, get_s, sm);
      return -ns - 1;  // negative: S was written here
    }
  }
  // condition 1 at radius j1 (j1 < NLEV here: tau <= n)
  if (threadIdx.x == 0) {
    int64_t cum = ncA, basev = ncA;
    int is = ix.L - 1;
    for (int t = 0; t < ix.L; ++t) {
      const int64_t nt = c.D[t * 256 + j1];
      if (cum + nt >= tau) { is = t; basev = cum; break; }
      cum += nt;
    }
    sm.jstar = (int)j1;
    sm.istar = is;
    sm.need = (uint32_t)(tau - basev);
    sm.ncand = (uint32_t)ncA;
  }
  __syncthreads();
  cut_and_collect_fixed<LC>(c, j1);
  const int64_t nc = min((int64_t)sm.ncand, c.qa.cand_cap);
  if (sm.ncand > c.qa.cand_cap && threadIdx.x == 0) atomicExch(c.qa.err, (int)DETLSH_ERR_CAPACITY);
  dist_fp32(ix, q, nc - ncA, cand + ncA, c.s.key + ncA);
  auto get_s = [&](int64_t i, uint32_t &key, uint32_t &id) { key = c.s.key[i]; id = cand[i]; };
  topk_select(nc, k, get_s, sm);
  return nc;
}

// ---- Alg. 5 at the smallest continuous r_min -----------------------------
// v* = the (beta*n + k)-th smallest of m(p) = min over trees of the lower
// bound of p's leaf: N(T(j*-1)) < beta*n + k <= N(T(j*)) on the grid, so v*
// lies in (T(j*-1), T(j*)] and is found among the points whose smallest level
// is j*.  A leaf of level < j* is within v*, one of level > j* is not; for
// level j* the exact lower bound decides.  Then Alg. 5's first round at v*.

// Lower bound of leaf l of tree u, from the breakpoints and q' in global
// memory: the same FP32 operations in the same order as box_lb2 on the table.
__device__ __forceinline__ float leaf_lb2_direct(const QueryIndexView &ix, const float *qp,
                                                 int u, uint32_t l) {
  const int64_t g = ix.leaf_off[u] + l;
  const uint4 lo = reinterpret_cast<const uint4 *>(ix.leaf_lo)[g];
  const uint4 hi = reinterpret_cast<const uint4 *>(ix.leaf_hi)[g];
  const uint32_t wl[4] = {lo.x, lo.y, lo.z, lo.w}, wh[4] = {hi.x, hi.y, hi.z, hi.w};
  const int NR1 = ix.N_r + 1;
  float acc = 0.0f;
  for (int j = 0; j < ix.K; ++j) {
    const uint32_t zl = (wl[j >> 2] >> (8 * (j & 3))) & 255u;
    const uint32_t zh = (wh[j >> 2] >> (8 * (j & 3))) & 255u;
    const float *Bj = ix.B + (int64_t)(u * ix.K + j) * NR1;
    const float q = qp[u * ix.K + j];
    const float a = __fsub_rn(Bj[zl], q);
    const float b = -__fsub_rn(Bj[zh + 1], q);
    const float gap = fmaxf(fmaxf(a, b), 0.0f);
    acc = __fadd_rn(acc, __fmul_rn(gap, gap));
  }
  return acc;
}

// Is p (visited in tree t's leaf of level lvt and lower bound lbt) within the
// squared radius v, and does no earlier tree hold it within v?  The smallest
// lower bound of p over all trees goes to *m (trees of level j* recomputed).
template <int LC>
__device__ __forceinline__ bool new_at_v(const QCtx &c, uint32_t p, int t, uint32_t js,
                                         float v, bool want_m, float lbt, float *m) {
  const PointLeaves<LC> lf(c.ix, p);
  const int L = LC ? LC : c.ix.L;
  const float *qp = c.qa.Qp + c.qi * c.ix.LK;
  bool blocked = false;
  float mm = lbt;
#pragma unroll
  for (int u = 0; u < L; ++u) {
    if (u == t || (u > t && !want_m)) continue;
    const uint32_t lv = leaf_level_h(c.ix, c.s, c.sm, c.lut, u, lf[u]);
    if (lv > js) continue;
    const float lb = (lv < js) ? 0.0f : leaf_lb2_direct(c.ix, qp, u, lf[u]);
    if (u < t && (lv < js || lb <= v)) blocked = true;
    if (lv == js) mm = fminf(mm, lb);
  }
  if (m) *m = mm;
  return !blocked;
}

template <int LC>
__device__ __forceinline__ void magic_min_resolve(QCtx &c) {
  const QueryIndexView &ix = c.ix;
  QShared &sm = c.sm;
  const int L = LC ? LC : ix.L;
  const uint32_t js = (uint32_t)min(sm.sel_g, sm.jhi);
  const uint32_t need0 = (uint32_t)(c.tau - (int64_t)sm.sel_bf);  // beyond N(j* - 1)
  // v*: radix select over m(p) of the points whose smallest level is j*,
  // each counted once (from the first tree at level j*)
  uint32_t prefix = 0, below = 0;
  for (int shift = 24; shift >= 0; shift -= 8) {
    sm.rh[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t hmask = (shift == 24) ? 0u : (0xffffffffu << (shift + 8));
    for (int t = 0; t < L; ++t) {
      const int64_t lo0 = ix.leaf_off[t];
      visit_points(
          c, t, [&](int64_t e) { return c.s.llev[lo0 + e] == js; },
          [&](bool valid, uint32_t p, uint32_t ent, uint32_t) {
            bool take = false;
            uint32_t key = 0;
            if (valid) {
              uint32_t fb = 0, fa = 0;
              levels_around<LC>(c, p, t, fb, fa);
              if (fb > js && fa >= js) {  // first tree at level j*, none below
                float m;
                new_at_v<LC>(c, p, t, js, 0.0f, true, c.s.llb2[lo0 + ent], &m);
                key = __float_as_uint(m);
                take = (key & hmask) == (prefix & hmask);
              }
            }
            warp_bin_count(sm.rh, take, (key >> shift) & 255u, 1u);
          });
    }
    __syncthreads();
    warp_first_crossing(sm.rh, below, need0, &sm.sel_g, &sm.sel_bf);
    __syncthreads();
    prefix |= (uint32_t)sm.sel_g << shift;
    below = (uint32_t)sm.sel_bf;
    __syncthreads();
  }
  const float v = __uint_as_float(prefix);
  // new points per tree at v, i*, the count still needed inside tree i*
  if (threadIdx.x < 16) sm.newt[threadIdx.x] = 0;
  __syncthreads();
  for (int t = 0; t < L; ++t) {
    const int64_t lo0 = ix.leaf_off[t];
    visit_points(
        c, t, [&](int64_t e) { return c.s.llev[lo0 + e] <= js && c.s.llb2[lo0 + e] <= v; },
        [&](bool valid, uint32_t p, uint32_t, uint32_t) {
          const bool nw = valid && new_at_v<LC>(c, p, t, js, v, false, 0.0f, nullptr);
          const unsigned bm = __ballot_sync(FULL, nw);
          if ((threadIdx.x & 31) == 0 && bm)
            atomicAdd(reinterpret_cast<unsigned long long *>(&sm.newt[t]), (unsigned long long)__popc(bm));
        });
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t cum = 0, basev = 0;
    int is = L - 1;
    for (int t = 0; t < L; ++t) {
      if (cum + sm.newt[t] >= c.tau) { is = t; basev = cum; break; }
      cum += sm.newt[t];
    }
    sm.jstar = (int)js;
    sm.istar = is;
    sm.need = (uint32_t)(c.tau - basev);
  }
  __syncthreads();
  const int is = sm.istar;
  const int64_t li0 = ix.leaf_off[is];
  const int64_t nli = sm.nlist[is];
  for (int64_t e = threadIdx.x; e < nli; e += QT) c.s.cval[e] = 0u;
  __syncthreads();
  auto inside = [&](int64_t lo0, int64_t e) {
    return c.s.llev[lo0 + e] <= js && c.s.llb2[lo0 + e] <= v;
  };
  visit_points(
      c, is, [&](int64_t e) { return inside(li0, e); },
      [&](bool valid, uint32_t p, uint32_t ent, uint32_t) {
        const bool nw = valid && new_at_v<LC>(c, p, is, js, v, false, 0.0f, nullptr);
        warp_bin_count(c.s.cval, nw, ent, 1u);
      });
  __syncthreads();
  const uint32_t need = sm.need;
  auto get_lb = [&](int64_t i, uint32_t &k, uint32_t &w) {
    w = inside(li0, i) ? c.s.cval[i] : 0u;
    k = __float_as_uint(c.s.llb2[li0 + i]);
  };
  block_select(nli, get_lb, need, sm);
  const uint32_t vb = sm.sel_v;
  const uint32_t need2 = need - sm.sel_below;
  uint32_t cut = 0xffffffffu;
  if (need2 < sm.sel_at) {
    auto get_id = [&](int64_t i, uint32_t &k, uint32_t &w) {
      const bool q = inside(li0, i) && __float_as_uint(c.s.llb2[li0 + i]) == vb;
      w = q ? c.s.cval[i] : 0u;
      k = c.s.lleaf[li0 + i];
    };
    block_select(nli, get_id, need2, sm);
    cut = sm.sel_v;
  }
  if (threadIdx.x == 0) sm.ncand = 0;
  __syncthreads();
  for (int t = 0; t <= is; ++t) {
    const int64_t lo0 = ix.leaf_off[t];
    visit_points(
        c, t,
        [&](int64_t e) {
          if (!inside(lo0, e)) return false;
          if (t < is) return true;
          const uint32_t kb = __float_as_uint(c.s.llb2[lo0 + e]);
          return kb < vb || (kb == vb && c.s.lleaf[lo0 + e] <= cut);
        },
        [&](bool valid, uint32_t p, uint32_t, uint32_t) {
          const bool take = valid && new_at_v<LC>(c, p, t, js, v, false, 0.0f, nullptr);
          const uint32_t pos = warp_append(c, take);
          if (take && pos < (uint32_t)c.qa.cand_cap) c.s.cand[pos] = p;
        });
  }
  __syncthreads();
}

// One instantiation per r_min policy, so the common (magic grid) kernel
// carries none of the other policies' code or register pressure.
template <int POL>
__global__ void __launch_bounds__(QT, 5) k_query(QueryIndexView ix, QueryArgs qa) {
  extern __shared__ __align__(16) uint8_t dsm[];
  QShared &sm = *reinterpret_cast<QShared *>(dsm);
  float *lut = reinterpret_cast<float *>(dsm + align_up(sizeof(QShared), 16));
  uint32_t *hist = reinterpret_cast<uint32_t *>(lut + lut_region_floats(qa.hash_kb));
  int32_t *D = reinterpret_cast<int32_t *>(hist + 256 * ix.L);

  uint8_t *base = qa.scratch + (int64_t)blockIdx.x * qa.slot_bytes;
  Slot s;
  s.lev = reinterpret_cast<unsigned long long *>(base + qa.off[0]);
  s.blev = base + qa.off[1];
  s.border = reinterpret_cast<uint32_t *>(base + qa.off[2]);
  s.lleaf = reinterpret_cast<uint32_t *>(base + qa.off[3]);
  s.llb2 = reinterpret_cast<float *>(base + qa.off[4]);
  s.llev = base + qa.off[5];
  s.cval = reinterpret_cast<uint32_t *>(base + qa.off[6]);
  s.cand = reinterpret_cast<uint32_t *>(base + qa.off[7]);
  s.key = reinterpret_cast<uint32_t *>(base + qa.off[8]);
  s.rid = reinterpret_cast<uint32_t *>(base + qa.off[9]);
  s.rkey = reinterpret_cast<uint32_t *>(base + qa.off[10]);
  s.cm = base + qa.off[11];
  s.hkey = reinterpret_cast<uint32_t *>(base + qa.off[12]);
  s.guess = reinterpret_cast<uint32_t *>(base + qa.off[13]);
  for (int i = threadIdx.x; i < 256; i += QT) sm.T[i] = i < NLEV ? qa.T[i] : __int_as_float(0x7f800000);
  if (threadIdx.x == 0) {
    // the bound guess survives launches in the slot (queries of later
    // batches start from it; any value gives the same results)
    const uint32_t g = *s.guess;
    sm.n_blocks = 0; sm.n_leaves = 0; sm.n_visit = 0;
    sm.jguess = (g >= 1u && g <= (uint32_t)NLEV) ? (int)g - 1 : NLEV - 1;
    // a status already set (a query projection found NaN/Inf) stops the
    // launch before any query: the caller reports it
    sm.stop = *(volatile int *)qa.err;
  }
  __syncthreads();
  if (sm.stop) return;

  while (true) {
    if (threadIdx.x == 0) sm.qi = atomicAdd(qa.work_counter, 1u);
    __syncthreads();
    const int64_t qi = sm.qi;
    if (qi >= qa.m) break;
    int k = qa.kq ? qa.kq[qi] : qa.k_max;
    if (k < 1 || k > qa.k_max) {  // per-query k outside [1, k_max]: report, clamp
      if (threadIdx.x == 0) atomicExch(qa.err, (int)DETLSH_ERR_INVALID_ARG);
      k = k < 1 ? 1 : qa.k_max;
    }
    const int64_t tau = qa.tau_base + k;
    QCtx c{ix, qa, sm, lut, hist, D, s, qi, tau};
    bool fixed_done = false, s_written = false;  // fixed r_min: top-k (and S) done
    // beta*n + k > n: with the magic r_min the budget is never met and S is
    // every point; a fixed r_min still runs its radius loop (condition 2)
    const bool allpts = tau > ix.n && qa.policy != DETLSH_RMIN_FIXED;
    int64_t nc;
    if (allpts) {
      // beta*n + k > n: the budget is never met; Alg. 5 stops through its
      // second condition with S = every point.
      nc = ix.n;
      if (threadIdx.x == 0) { sm.jstar = NLEV - 1; sm.istar = -1; }
    } else {
      for (int i = threadIdx.x; i < 256 * ix.L; i += QT) { hist[i] = 0; D[i] = 0; }
      sm.H[threadIdx.x] = 0;
      // a fresh tag from the slot area's counter: no tag left by an earlier
      // query (or an earlier launch) can match it
      if (threadIdx.x == 0) sm.epoch = atomicAdd(qa.epoch_counter, 1ull) + 1ull;
      __syncthreads();
      expand_levels(c);
      build_level_hash(c);
      union_counts(c);
      // j* = first level whose union count reaches tau (<= jhi by construction)
      warp_first_crossing(sm.H, 0, (uint64_t)tau, &sm.sel_g, &sm.sel_bf);
      __syncthreads();
      if constexpr (POL == DETLSH_RMIN_FIXED) {
        const int64_t r = ix.L == 4 ? fixed_rmin_query<4>(c, k) : fixed_rmin_query<0>(c, k);
        fixed_done = true;
        s_written = r < 0;
        nc = r < 0 ? -r - 1 : r;
      } else if constexpr (POL == DETLSH_RMIN_CONTINUOUS) {
        if (ix.L == 4) magic_min_resolve<4>(c); else magic_min_resolve<0>(c);
        nc = sm.ncand;
        if (nc > qa.cand_cap) {
          if (threadIdx.x == 0) atomicExch(qa.err, (int)DETLSH_ERR_CAPACITY);
          nc = qa.cand_cap;
        }
      } else {
        const int js = min(sm.sel_g, sm.jhi);
        {  // points new in each tree at level j*: one warp per tree
          const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
          for (int t = warp; t < ix.L; t += QW) {
            int64_t v = 0;
            for (int j = lane; j <= js; j += 32) v += D[t * 256 + j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
            if (lane == 0) sm.newt[t] = v;
          }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          int64_t cum = 0, basev = 0;
          int is = ix.L - 1;
          for (int t = 0; t < ix.L; ++t) {
            if (cum + sm.newt[t] >= tau) { is = t; basev = cum; break; }
            cum += sm.newt[t];
          }
          sm.jstar = js;
          sm.istar = is;
          sm.need = (uint32_t)(tau - basev);
        }
        __syncthreads();
        cut_and_collect(c);
        nc = sm.ncand;
        if (nc > qa.cand_cap) {
          // cannot happen for |S| < beta*n + k + largest leaf; report and skip
          if (threadIdx.x == 0) atomicExch(qa.err, (int)DETLSH_ERR_CAPACITY);
          nc = qa.cand_cap;
        }
      }
    }
    if (qa.S_out) {
      if (!s_written)
        for (int64_t i = threadIdx.x; i < nc && i < qa.S_cap; i += QT)
          qa.S_out[qi * qa.S_cap + i] = allpts ? i : (int64_t)s.cand[i];
      if (threadIdx.x == 0) {
        qa.S_size[qi] = nc;
        // grid index j of r_min = c^j, or the radius index i of r_min c^i
        qa.jstar[qi] = qa.policy == DETLSH_RMIN_FIXED ? sm.jstar : sm.jstar + JMIN;
        qa.istar[qi] = sm.istar;
        if (nc > qa.S_cap) atomicExch(qa.err, (int)DETLSH_ERR_CAPACITY);
      }
    }
    if (!fixed_done) {
      // verification and top-k
      // Every branch ends in one FP32 distance pass over (rows, ids) and one
      // top-k over its keys: single call sites keep the kernel's code small.
      const uint32_t *cid = allpts ? nullptr : s.cand;
      int64_t rows = nc;
      const uint32_t *rids = cid;
      uint32_t *rkeys = s.key;
      if (qa.precision == DETLSH_PREC_BF16_REFINE) {
        distances_bf16(c, nc, allpts, qa.rerank_mult == 0);
        uint32_t need;
        const uint32_t *selk;
        if (qa.rerank_mult == 0) {
          // certified pool: every candidate whose interval starts at or
          // below T, some bound at or above the k-th smallest interval end.
          // The k candidates with the smallest ends have FP32 keys <= T, so
          // each of the FP32 path's top k has key <= T and lies in the pool:
          // re-ranking the pool in FP32 gives the FP32 path's answer exactly.
          need = (uint32_t)k;
          selk = s.hkey;
        } else {  // the rerank_mult * k best scores
          int64_t R = min((int64_t)qa.rerank_mult * k, (int64_t)RR_MAX);
          need = (uint32_t)max(min(R, nc), (int64_t)k);
          selk = s.key;
        }
        // the certified pool only needs some T >= the k-th end: its top 24
        // bits (three radix passes) with the low byte all ones
        const bool cert = qa.rerank_mult == 0;
        block_select(nc, ArrKey{selk}, need, sm, cert ? 8 : 0);
        const uint32_t T = cert ? (sm.sel_v | 0xffu) : sm.sel_v;
        // fixed pool: ties at T by smaller id
        uint32_t idcut = 0xffffffffu;
        if (qa.rerank_mult != 0 && need - sm.sel_below < sm.sel_at) {
          auto gi = [&](int64_t i, uint32_t &kk2, uint32_t &w) {
            kk2 = cid ? cid[i] : (uint32_t)i;
            w = s.key[i] == T ? 1u : 0u;
          };
          block_select(nc, gi, need - sm.sel_below, sm);
          idcut = sm.sel_v;
        }
        if (threadIdx.x == 0) sm.nres = 0;
        __syncthreads();
        for (int64_t i0 = 0; i0 < nc; i0 += QT) {  // uniform trip count: warp collectives inside
          const int64_t i = i0 + threadIdx.x;
          bool in = false;
          uint32_t id = 0;
          if (i < nc) {
            const uint32_t kv = s.key[i];
            id = cid ? cid[i] : (uint32_t)i;
            in = kv < T || (kv == T && id <= idcut);
          }
          const unsigned bm = __ballot_sync(FULL, in);
          uint32_t pos0 = 0;
          if ((threadIdx.x & 31) == 0 && bm) pos0 = atomicAdd(&sm.nres, (uint32_t)__popc(bm));
          pos0 = __shfl_sync(FULL, pos0, 0) + __popc(bm & ((1u << (threadIdx.x & 31)) - 1u));
          if (in && pos0 < RR_MAX) s.rid[pos0] = id;
        }
        __syncthreads();
        const int64_t np = sm.nres;
        if (threadIdx.x == 0 && qa.stats) atomicAdd(&qa.stats[4], (unsigned long long)min(np, nc));
        if (np <= RR_MAX) { rows = np; rids = s.rid; rkeys = s.rkey; }
        // else a pool beyond the re-rank buffers: FP32 over every candidate
      }
      dist_fp32(ix, qa.Q + qi * ix.d, rows, rids, rkeys);
      topk_select(rows, k, ArrGet{rkeys, rids}, sm);
    }
    if (threadIdx.x == 0 && qa.stats) atomicAdd(&qa.stats[0], (unsigned long long)nc);
    for (int r = threadIdx.x; r < qa.k_max; r += QT) {
      if (r < k) {
        qa.ids[qi * qa.k_max + r] = (int64_t)sm.topk_id[r];
        qa.dists[qi * qa.k_max + r] = __fsqrt_rn(__uint_as_float(sm.topk_key[r]));
      } else {
        qa.ids[qi * qa.k_max + r] = -1;
        qa.dists[qi * qa.k_max + r] = __int_as_float(0x7f800000);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *s.guess = (uint32_t)sm.jguess + 1u;
  if (threadIdx.x == 0 && qa.stats) {
    atomicAdd(&qa.stats[1], sm.n_leaves);
    atomicAdd(&qa.stats[2], sm.n_blocks);
    atomicAdd(&qa.stats[3], sm.n_visit);
  }
}

static size_t query_smem(const QueryIndexView &ix, int hash_kb) {
  return (size_t)align_up(sizeof(QShared), 16) + sizeof(float) * lut_region_floats(hash_kb) +
         sizeof(uint32_t) * 256 * ix.L * 2;
}

int query_slots(const QueryIndexView &ix) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = query_smem(ix, 0);
  cudaFuncSetAttribute(k_query<DETLSH_RMIN_MAGIC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_query<DETLSH_RMIN_MAGIC>, QT, smem);
  if (per < 1) per = 1;
  return sms * per;
}

int run_queries(const QueryIndexView &ix, const QueryArgs &qa, cudaStream_t st) {
  if (qa.m <= 0) return DETLSH_OK;
  const size_t smem = query_smem(ix, qa.hash_kb);
  auto kern = qa.policy == DETLSH_RMIN_FIXED        ? k_query<DETLSH_RMIN_FIXED>
              : qa.policy == DETLSH_RMIN_CONTINUOUS ? k_query<DETLSH_RMIN_CONTINUOUS>
                                                    : k_query<DETLSH_RMIN_MAGIC>;
  DL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  DL_CUDA(cudaMemsetAsync(qa.work_counter, 0, sizeof(uint32_t), st));
  int grid = (int)std::min<int64_t>(qa.nslots, qa.m);
  if (qa.ctas_per_sm > 0) {  // tuned: at most this many CTAs per SM
    int dev = 0, sms = 0;
    DL_CUDA(cudaGetDevice(&dev));
    DL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    grid = std::max(1, std::min(grid, sms * qa.ctas_per_sm));
  }
  if (qa.hash_kb > 0) {  // a larger shared region: no more CTAs than fit at once
    int dev = 0, sms = 0, per = 0;
    DL_CUDA(cudaGetDevice(&dev));
    DL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, QT, smem));
    if (per < 1) return DETLSH_ERR_INVALID_ARG;
    grid = std::max(1, std::min(grid, sms * per));
  }
  kern<<<grid, QT, smem, st>>>(ix, qa);
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  return DETLSH_OK;
}

}  // namespace dl
