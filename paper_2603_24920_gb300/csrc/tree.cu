// tree.cu -- DE-Tree layout (Alg. 2, Sec. III-B) for sm_103a.
//
// A DE-Tree is stored as arrays: perm (point ids leaf by leaf), leaf_begin,
// per-leaf boxes (lo/hi region per dimension) and prefix lengths, and
// leaf_of (the leaf of every point).  Leaves are in canonical order: first-
// layer key ascending (dimension 0 is the most significant bit), then child 0
// before child 1; points inside a leaf in ascending id order.
//
// Build, for a group of G trees at once (every kernel runs over the G * n
// positions of the group; tree g owns positions [g n, (g + 1) n)): (1) stable
// radix sort of the point ids by their K-bit first-layer key (the root's 2^K
// children), one segment per tree; (2) the subtrees of the first-layer nodes,
// level by level: a CTA takes the first-layer nodes that start in its range
// of points (first-layer subtrees are independent, as the paper's parallel
// indexing phase notes in Sec. IV-B) and, at each level, its warps take the
// open nodes one each, choosing the dimension that splits a node most evenly
// and stably partitioning its range between two ping-pong buffers; a leaf is
// recorded at the position where its points start; (3) leaves are numbered
// by a compaction of those start flags: position order is depth-first order
// (child 0 holds the lower part of its parent's range), so a leaf's rank
// among the flags is its number and the records land in the final layout.
//
// Reading of Alg. 2 (insertion order and max_size are left open): a node is
// split iff it holds more than max_size points and some dimension has prefix
// bits left; the split dimension minimises |n0 - n1| (ties: smallest
// dimension); a split that leaves one side empty still refines the prefix;
// empty children are dropped.
#include "common.cuh"
#include "compact.cuh"
#include "kernels.h"

#include <algorithm>

namespace dl {


// keys and point ids of G trees: position i is point i % n of tree i / n
__global__ void k_first_keys(const uint8_t *__restrict__ codes, int64_t n, int64_t N, int K, int bbits,
                             uint32_t *keys, uint32_t *vals) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 c = reinterpret_cast<const uint4 *>(codes)[i];
    const uint32_t w[4] = {c.x, c.y, c.z, c.w};
    uint32_t key = 0;
    for (int j = 0; j < K; ++j) {
      const uint32_t byte = (w[j >> 2] >> (8 * (j & 3))) & 255u;
      key |= ((byte >> (bbits - 1)) & 1u) << (K - 1 - j);
    }
    keys[i] = key;
    vals[i] = (uint32_t)(i % n);
  }
}

__global__ void k_gather_codes(const uint4 *__restrict__ codes, const uint32_t *__restrict__ ids,
                               int64_t n, int64_t N, uint4 *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = codes[(i / n) * n + ids[i]];
}

// a first-layer node starts at every change of key and at every tree start
struct BoundaryFlag {
  const uint32_t *keys;
  int64_t n;
  __device__ bool operator()(int64_t i) const { return i % n == 0 || keys[i] != keys[i - 1]; }
};

__device__ __forceinline__ uint32_t code_byte(const uint4 &c, int j) {
  const uint32_t w = j < 4 ? c.x : j < 8 ? c.y : j < 12 ? c.z : c.w;
  return (w >> (8 * (j & 3))) & 255u;
}

struct NodeEntry {
  uint32_t b, e, par, f;  // range, buffer holding it, first-layer node
  uint4 nb;               // prefix length per dimension, one byte each
};

struct SubtreeArgs {
  int64_t n;
  int K, bbits, M, box_mode;
  const uint32_t *F;           // number of first-layer nodes (device)
  const uint32_t *node_begin;  // [F+1]
  uint4 *codesA, *codesB;
  uint32_t *idsA, *idsB;
  uint32_t *perm;
  uint32_t *leaf_flag;         // [n] 1 where a leaf starts (zeroed)
  uint8_t *tmp_box;            // [n][48] box of the leaf starting there
  NodeEntry *listA, *listB;    // [n] each: open nodes of a level
  int *err;
};

constexpr int TB_THREADS = 256;
constexpr int TB_WARPS = TB_THREADS / 32;
constexpr int TB_POINTS = 2048;  // first-layer nodes starting in a CTA's range of points

// four CTAs per SM (at most 64 registers): the levels are latency-bound
__global__ void __launch_bounds__(TB_THREADS, 4) k_subtree(SubtreeArgs a) {
  __shared__ uint32_t ncur, nnext, f_lo, f_hi;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int K = a.K, bb = a.bbits;
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t P0 = blockIdx.x * (uint32_t)TB_POINTS;
  if (threadIdx.x == 0) {  // first-layer nodes f with node_begin[f] in [P0, P0 + TB_POINTS)
    const uint32_t F = *a.F;
    uint32_t lo = 0, hi = F;
    while (lo < hi) { const uint32_t mid = (lo + hi) >> 1; if (a.node_begin[mid] < P0) lo = mid + 1; else hi = mid; }
    f_lo = lo;
    hi = F;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (a.node_begin[mid] < P0 + (uint32_t)TB_POINTS) lo = mid + 1; else hi = mid;
    }
    f_hi = lo;
    ncur = f_hi - f_lo;
  }
  __syncthreads();
  if (ncur == 0) return;
  // this CTA's lists live at the positions of its points: nodes of a level
  // are disjoint and non-empty, so a level never holds more of them
  const uint32_t lbase = a.node_begin[f_lo];
  NodeEntry *cur = a.listA + lbase, *nxt = a.listB + lbase;
  uint32_t root_nb[4] = {0u, 0u, 0u, 0u};
  for (int j = 0; j < 16; ++j) root_nb[j >> 2] |= (uint32_t)(j < K ? 1 : bb) << (8 * (j & 3));
  for (uint32_t f = f_lo + threadIdx.x; f < f_hi; f += TB_THREADS) {
    NodeEntry r;
    r.b = a.node_begin[f]; r.e = a.node_begin[f + 1]; r.par = 0; r.f = f;
    r.nb = make_uint4(root_nb[0], root_nb[1], root_nb[2], root_nb[3]);
    cur[f - f_lo] = r;
  }
  __syncthreads();
  while (ncur > 0) {  // one level per pass
    if (threadIdx.x == 0) nnext = 0;
    __syncthreads();
    const uint32_t nc = ncur;
    for (uint32_t i = w; i < nc; i += TB_WARPS) {
      const NodeEntry ent = cur[i];
      const uint32_t b = ent.b, e = ent.e, par = ent.par;
      const uint4 nbv = ent.nb;
      const uint32_t cnt = e - b;
      const uint4 *src = par ? a.codesB : a.codesA;
      const uint32_t *srcid = par ? a.idsB : a.idsA;
      bool eligible_any = false;
      for (int j = 0; j < K; ++j) eligible_any |= (int)code_byte(nbv, j) < bb;
      if (cnt > (uint32_t)a.M && eligible_any) {
        // Per-dimension counts of the next prefix bit.  The bit of dimension j
        // sits at bit bb-1-nb_j of code byte j: one mask per code word picks
        // it out of four bytes at once, and per-byte counters (flushed before
        // they can reach 256) accumulate four dimensions per add.  Loads run
        // four rounds ahead.
        uint32_t msk[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int nbj = (int)code_byte(nbv, j);
          if (j < K && nbj < bb) msk[j >> 2] |= (1u << (bb - 1 - nbj)) << (8 * (j & 3));
        }
        uint32_t c1[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) c1[j] = 0u;
        uint32_t pk[4] = {0u, 0u, 0u, 0u};
        int rounds = 0;
        auto flush = [&]() {
#pragma unroll
          for (int j = 0; j < 16; ++j) c1[j] += (pk[j >> 2] >> (8 * (j & 3))) & 255u;
#pragma unroll
          for (int q = 0; q < 4; ++q) pk[q] = 0u;
          rounds = 0;
        };
        for (uint32_t base = b; base < e; base += 128) {
          uint4 cv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const uint32_t x = base + u * 32 + lane;
            cv[u] = x < e ? src[x] : make_uint4(0u, 0u, 0u, 0u);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const uint32_t wd[4] = {cv[u].x, cv[u].y, cv[u].z, cv[u].w};
#pragma unroll
            for (int q = 0; q < 4; ++q) pk[q] += __vcmpne4(wd[q] & msk[q], 0u) & 0x01010101u;
          }
          if ((rounds += 4) > 250) flush();
        }
        flush();
        // most even split, ties to the smallest dimension
        int best = -1;
        int64_t bestd = 0;
        uint32_t n1 = 0;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const uint32_t v = __reduce_add_sync(FULL, c1[j]);
          if (j < K && (int)code_byte(nbv, j) < bb) {
            int64_t dd = (int64_t)cnt - 2 * (int64_t)v;
            if (dd < 0) dd = -dd;
            if (best < 0 || dd < bestd) { best = j; bestd = dd; n1 = v; }
          }
        }
        uint32_t wv[4] = {nbv.x, nbv.y, nbv.z, nbv.w};
        const uint32_t nbbest = code_byte(nbv, best);
        wv[best >> 2] += 1u << (8 * (best & 3));  // one more prefix bit in the split dimension
        const uint4 nbc = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        if (n1 == 0u || n1 == cnt) {
          // one side empty: the only child has the same points, one more bit
          if (lane == 0) {
            NodeEntry ch = ent;
            ch.nb = nbc;
            nxt[atomicAdd(&nnext, 1u)] = ch;
          }
          continue;
        }
        const uint32_t n0 = cnt - n1;
        const uint32_t sh = (uint32_t)(bb - 1) - nbbest;
        uint4 *dst = par ? a.codesA : a.codesB;
        uint32_t *dstid = par ? a.idsA : a.idsB;
        uint32_t zrun = 0, orun = 0;
        for (uint32_t base0 = b; base0 < e; base0 += 128) {
          uint4 cv[4];
          uint32_t idv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {  // loads four rounds ahead of the stores
            const uint32_t x = base0 + u * 32 + lane;
            cv[u] = make_uint4(0u, 0u, 0u, 0u);
            idv[u] = 0u;
            if (x < e) { cv[u] = src[x]; idv[u] = srcid[x]; }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const uint32_t x = base0 + u * 32 + lane;
            const bool valid = x < e;
            const uint32_t bit = valid ? (code_byte(cv[u], best) >> sh) & 1u : 0u;
            const unsigned ones = __ballot_sync(FULL, valid && bit);
            const unsigned zeros = __ballot_sync(FULL, valid && !bit);
            if (valid) {
              const uint32_t pos = bit ? (b + n0 + orun + __popc(ones & lt)) : (b + zrun + __popc(zeros & lt));
              dst[pos] = cv[u];
              dstid[pos] = idv[u];
            }
            zrun += __popc(zeros);
            orun += __popc(ones);
          }
        }
        if (lane == 0) {
          const uint32_t q = atomicAdd(&nnext, 2u);
          NodeEntry c0 = ent, c1e = ent;
          c0.nb = c1e.nb = nbc;
          c0.par = c1e.par = par ^ 1u;
          c0.e = b + n0;
          c1e.b = b + n0;
          nxt[q] = c0;
          nxt[q + 1] = c1e;
        }
        continue;
      }
      // ---- leaf: ids to perm, box and flag at the leaf's first position ----
      for (uint32_t x = b + lane; x < e; x += 32) a.perm[x] = srcid[x];
      uint32_t lo = 255u, hi = 0u;
      if (a.box_mode == DETLSH_BOX_TIGHT) {  // lane j < 16 gathers dimension j
        for (uint32_t x = b; x < e; ++x) {
          const uint32_t v = code_byte(src[x], lane & 15);
          lo = min(lo, v);
          hi = max(hi, v);
        }
      }
      if (lane < 16) {
        uint8_t blo = 0, bhi = 0;
        if (lane < K) {
          const uint32_t freeb = (uint32_t)bb - code_byte(nbv, lane);
          const uint32_t pre = code_byte(src[b], lane) >> freeb;
          blo = (uint8_t)(pre << freeb);
          bhi = (uint8_t)((pre << freeb) + (1u << freeb) - 1u);
          if (a.box_mode == DETLSH_BOX_TIGHT) { blo = (uint8_t)lo; bhi = (uint8_t)hi; }
        }
        a.tmp_box[(int64_t)b * 48 + lane] = blo;
        a.tmp_box[(int64_t)b * 48 + 16 + lane] = bhi;
        a.tmp_box[(int64_t)b * 48 + 32 + lane] = lane < K ? (uint8_t)code_byte(nbv, lane) : 0;
      }
      if (lane == 0) a.leaf_flag[b] = 1u;
    }
    __syncthreads();  // this level's partitions and children are complete
    if (threadIdx.x == 0) ncur = nnext;
    NodeEntry *t = cur; cur = nxt; nxt = t;
    __syncthreads();
  }
}

// ---- leaf records --------------------------------------------------------
// Leaves start at the flagged positions; in position order they are in
// canonical (depth-first) order, so a leaf's number in the group is its rank
// among the flags, and a tree's first leaf starts at the tree's first
// position.
struct LeafStart {
  const uint32_t *flag;
  __device__ bool operator()(int64_t i) const { return flag[i] != 0u; }
};

struct LeafWriteArgs {
  int64_t n, N;
  int L, t0;
  const uint32_t *starts;         // [leaves] first position of every leaf
  const uint32_t *total;          // number of leaves (device)
  const uint32_t *tree_leaf_off;  // [G+1] first leaf of every tree of the group
  const uint32_t *perm, *leaf_flag, *block_offsets;
  const uint8_t *tmp_box;
  uint32_t *leaf_begin;
  uint8_t *leaf_lo, *leaf_hi, *leaf_nb;
  uint32_t *leaf_of;
  uint32_t *max_leaf;
};

// One thread per leaf g (tree t = its start / n): box record g, leaf_begin
// entry g + t (each tree's leaf_begin has one end entry more), size.
__global__ void k_leaf_records(LeafWriteArgs a) {
  const uint32_t total = *a.total;
  uint32_t big = 0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < (int64_t)total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t lb = a.starts[g];
    const uint32_t t = (uint32_t)(lb / a.n);
    const uint32_t tend = (uint32_t)((t + 1) * a.n);
    const uint32_t le = g + 1 < total ? min(a.starts[g + 1], tend) : tend;
    const uint4 *src = reinterpret_cast<const uint4 *>(a.tmp_box + (int64_t)lb * 48);
    reinterpret_cast<uint4 *>(a.leaf_lo)[g] = src[0];
    reinterpret_cast<uint4 *>(a.leaf_hi)[g] = src[1];
    reinterpret_cast<uint4 *>(a.leaf_nb)[g] = src[2];
    a.leaf_begin[g + t] = lb - (uint32_t)(t * a.n);
    big = max(big, le - lb);
  }
  big = __reduce_max_sync(FULL, big);
  if ((threadIdx.x & 31) == 0 && big) atomicMax(a.max_leaf, big);
}

// One thread per position: the leaf holding it is (flags up to it) - 1, from
// the compaction's block offsets and an in-block scan; leaf_of gets the
// number within the tree.
__global__ void k_leaf_of(LeafWriteArgs a) {
  __shared__ uint32_t wt[32];
  const int64_t base = (int64_t)blockIdx.x * CP_TILE + (int64_t)threadIdx.x * CP_ITEMS;
  uint32_t flags = 0, c = 0;
  for (int i = 0; i < CP_ITEMS; ++i) {
    const int64_t idx = base + i;
    if (idx < a.N && a.leaf_flag[idx] != 0u) { flags |= 1u << i; ++c; }
  }
  uint32_t cur = a.block_offsets[blockIdx.x] + block_exclusive_scan(c, wt, nullptr);  // flags before base
  for (int i = 0; i < CP_ITEMS; ++i) {
    const int64_t idx = base + i;
    if (idx >= a.N) break;
    cur += (flags >> i) & 1u;
    const uint32_t t = (uint32_t)(idx / a.n);
    a.leaf_of[(int64_t)a.perm[idx] * a.L + a.t0 + t] = cur - 1u - a.tree_leaf_off[t];
  }
}

// base[*idx] = v, the index read on the device
__global__ void k_set_at(uint32_t *base, const uint32_t *idx, uint32_t v) { base[*idx] = v; }

// First leaf of every tree of the group (the leaf starting at position t n),
// the total, and each tree's end entry of leaf_begin.
__global__ void k_tree_leaf_offsets(const uint32_t *starts, const uint32_t *total, int64_t n, int G,
                                    uint32_t *off, uint32_t *leaf_begin) {
  const int t = threadIdx.x;
  if (t > G) return;
  const uint32_t tot = *total;
  uint32_t o = tot;
  if (t < G) {
    uint32_t lo = 0, hi = tot;
    const uint32_t key = (uint32_t)(t * n);
    while (lo < hi) { const uint32_t mid = (lo + hi) >> 1; if (starts[mid] < key) lo = mid + 1; else hi = mid; }
    o = lo;
  }
  off[t] = o;
  if (t > 0) leaf_begin[o + (uint32_t)t - 1] = (uint32_t)n;  // end of tree t - 1
}

// Hull boxes of consecutive runs of LEAF_BLOCK boxes (in canonical order),
// for every tree in one launch: per dimension the smallest lo and largest hi
// of the run (byte-wise SIMD min/max).  A hull contains every box of its run,
// so its lower bound bounds theirs from below.
__global__ void k_block_hulls(const uint4 *__restrict__ lo, const uint4 *__restrict__ hi, HullSet h,
                              uint4 *hlo, uint4 *hhi) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= h.out_off[h.L]) return;
  int t = 0;
  while (b >= h.out_off[t + 1]) ++t;
  const int64_t l0 = h.in_off[t] + (b - h.out_off[t]) * LEAF_BLOCK;
  const int64_t l1 = min(l0 + LEAF_BLOCK, h.in_off[t] + h.cnt[t]);
  uint4 mn = make_uint4(~0u, ~0u, ~0u, ~0u), mx = make_uint4(0u, 0u, 0u, 0u);
  for (int64_t l = l0; l < l1; ++l) {
    const uint4 a = lo[l], c = hi[l];
    mn.x = __vminu4(mn.x, a.x); mn.y = __vminu4(mn.y, a.y); mn.z = __vminu4(mn.z, a.z); mn.w = __vminu4(mn.w, a.w);
    mx.x = __vmaxu4(mx.x, c.x); mx.y = __vmaxu4(mx.y, c.y); mx.z = __vmaxu4(mx.z, c.z); mx.w = __vmaxu4(mx.w, c.w);
  }
  hlo[b] = mn;
  hhi[b] = mx;
}

int block_hulls(const uint8_t *lo, const uint8_t *hi, const HullSet &h, uint8_t *hlo, uint8_t *hhi,
                cudaStream_t st) {
  const int64_t nb = h.out_off[h.L];
  if (nb == 0) return DETLSH_OK;
  k_block_hulls<<<(unsigned)ceil_div(nb, 128), 128, 0, st>>>(
      reinterpret_cast<const uint4 *>(lo), reinterpret_cast<const uint4 *>(hi), h,
      reinterpret_cast<uint4 *>(hlo), reinterpret_cast<uint4 *>(hhi));
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  return DETLSH_OK;
}

int build_trees(const TreeBuildArgs &A, TreeTemp &T, cudaStream_t st) {
  const int64_t n = A.n, N = (int64_t)A.G * n;
  const int gs = (int)std::min<int64_t>(ceil_div(N, 256), 4096);
  // no host round trip: counts stay on the device, launches are sized by
  // their upper bounds
  uint32_t *S = A.scalars;  // [0] F, [1] leaves, [2] error, [3] largest leaf, [4..] tree offsets
  DL_CUDA(cudaMemsetAsync(S, 0, 4 * sizeof(uint32_t), st));
  k_first_keys<<<gs, 256, 0, st>>>(A.codes, n, N, A.K, A.bbits, T.keys, T.vals);
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  DL_TRY(segmented_sort(T.keys, T.vals, A.G, n, A.K, T.sort, st));
  k_gather_codes<<<gs, 256, 0, st>>>(reinterpret_cast<const uint4 *>(A.codes), T.vals, n, N,
                                     T.codesA);
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  // first-layer nodes = runs of equal keys within a tree
  DL_TRY(compact(N, BoundaryFlag{T.keys, n}, T.block_counts, T.node_begin, S + 0, st));
  k_set_at<<<1, 1, 0, st>>>(T.node_begin, S + 0, (uint32_t)N);
  dl_count_launch();
  SubtreeArgs sa;
  sa.n = N; sa.K = A.K; sa.bbits = A.bbits; sa.M = A.M; sa.box_mode = A.box_mode;
  sa.F = S + 0;
  sa.node_begin = T.node_begin;
  sa.codesA = T.codesA; sa.codesB = T.codesB;
  sa.idsA = T.vals; sa.idsB = T.idsB;
  sa.perm = A.perm;
  sa.leaf_flag = T.tmp_begin;
  sa.tmp_box = T.tmp_box;
  sa.listA = reinterpret_cast<NodeEntry *>(T.lists);
  sa.listB = reinterpret_cast<NodeEntry *>(T.lists) + N;
  sa.err = reinterpret_cast<int *>(S + 2);
  DL_CUDA(cudaMemsetAsync(T.tmp_begin, 0, sizeof(uint32_t) * (size_t)N, st));
  k_subtree<<<(unsigned)ceil_div(N, TB_POINTS), TB_THREADS, 0, st>>>(sa);
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  // leaf numbering: compaction of the leaf start flags (position order)
  uint32_t *starts = T.leaf_start;
  DL_TRY(compact(N, LeafStart{T.tmp_begin}, T.block_counts, starts, S + 1, st));
  k_tree_leaf_offsets<<<1, 32, 0, st>>>(starts, S + 1, n, A.G, S + 4, A.leaf_begin);
  dl_count_launch();
  LeafWriteArgs lw;
  lw.n = n; lw.N = N; lw.L = A.L; lw.t0 = A.t0;
  lw.starts = starts; lw.total = S + 1; lw.tree_leaf_off = S + 4;
  lw.perm = A.perm; lw.leaf_flag = T.tmp_begin; lw.block_offsets = T.block_counts;
  lw.tmp_box = T.tmp_box;
  lw.leaf_begin = A.leaf_begin; lw.leaf_lo = A.leaf_lo; lw.leaf_hi = A.leaf_hi;
  lw.leaf_nb = A.leaf_nb; lw.leaf_of = A.leaf_of; lw.max_leaf = S + 3;
  int dev = 0, sms = 0;
  DL_CUDA(cudaGetDevice(&dev));
  DL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  k_leaf_records<<<(unsigned)std::min<int64_t>(ceil_div(N, 256), (int64_t)sms * 8), 256, 0, st>>>(lw);
  dl_count_launch();
  k_leaf_of<<<(unsigned)compact_blocks(N), CP_THREADS, 0, st>>>(lw);
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  return DETLSH_OK;
}

}  // namespace dl
