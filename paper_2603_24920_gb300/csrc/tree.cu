// tree.cu -- DE-Tree layout (Alg. 2, Sec. III-B) for sm_103a.
//
// A DE-Tree is stored as arrays: perm (point ids leaf by leaf), leaf_begin,
// per-leaf boxes (lo/hi region per dimension) and prefix lengths, and
// leaf_of (the leaf of every point).  Leaves are in canonical order: first-
// layer key ascending (dimension 0 is the most significant bit), then child 0
// before child 1; points inside a leaf in ascending id order.
//
// Build: (1) stable radix sort of the point ids by their K-bit first-layer
// key (the root's 2^K children); (2) one CTA per non-empty first-layer node
// builds that node's binary subtree depth-first, choosing at every node the
// dimension that splits it most evenly and stably partitioning the node's
// range between two ping-pong buffers (first-layer subtrees are independent,
// as the paper's parallel indexing phase notes in Sec. IV-B); (3) leaves are
// numbered by a scan over first-layer nodes and written out in order.
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

constexpr int TB_THREADS = 256;
constexpr int TB_STACK = 128;  // > K * (bits - 1) + 1 for K <= 16, bits <= 8

__global__ void k_first_keys(const uint8_t *__restrict__ codes, int64_t n, int K, int bbits,
                             uint32_t *keys, uint32_t *vals) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 c = reinterpret_cast<const uint4 *>(codes)[i];
    const uint32_t w[4] = {c.x, c.y, c.z, c.w};
    uint32_t key = 0;
    for (int j = 0; j < K; ++j) {
      const uint32_t byte = (w[j >> 2] >> (8 * (j & 3))) & 255u;
      key |= ((byte >> (bbits - 1)) & 1u) << (K - 1 - j);
    }
    keys[i] = key;
    vals[i] = (uint32_t)i;
  }
}

__global__ void k_gather_codes(const uint4 *__restrict__ codes, const uint32_t *__restrict__ ids,
                               int64_t n, uint4 *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = codes[ids[i]];
}

struct BoundaryFlag {
  const uint32_t *keys;
  __device__ bool operator()(int64_t i) const { return i == 0 || keys[i] != keys[i - 1]; }
};

__device__ __forceinline__ uint32_t code_byte(const uint4 &c, int j) {
  const uint32_t w = j < 4 ? c.x : j < 8 ? c.y : j < 12 ? c.z : c.w;
  return (w >> (8 * (j & 3))) & 255u;
}

struct StackEntry {
  uint32_t b, e;
  uint8_t nb[16];
  uint32_t par;
};

struct SubtreeArgs {
  int64_t n;
  int K, bbits, M, box_mode;
  const uint32_t *node_begin;  // [F+1]
  uint4 *codesA, *codesB;
  uint32_t *idsA, *idsB;
  uint32_t *perm;
  uint32_t *node_count;        // leaves per first-layer node
  uint32_t *tmp_begin;         // [n] leaf begin by slot
  uint8_t *tmp_box;            // [n][48]
  int *err;
};

__global__ void __launch_bounds__(TB_THREADS) k_subtree(SubtreeArgs a) {
  __shared__ StackEntry stk[TB_STACK];
  __shared__ int sp;
  __shared__ uint32_t nleaf;
  __shared__ uint32_t wpart[TB_THREADS / 32][16];
  __shared__ uint32_t n1s[16];
  __shared__ int split_dim, degenerate;
  __shared__ StackEntry cur;
  __shared__ uint32_t wz[TB_THREADS / 32], wo[TB_THREADS / 32];
  __shared__ uint32_t boxv[2][16];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = a.K, bb = a.bbits;
  const uint32_t b0 = a.node_begin[blockIdx.x], e0 = a.node_begin[blockIdx.x + 1];

  if (tid == 0) {
    StackEntry r;
    r.b = b0; r.e = e0; r.par = 0;
    for (int j = 0; j < 16; ++j) r.nb[j] = j < K ? 1 : (uint8_t)bb;
    stk[0] = r;
    sp = 1;
    nleaf = 0;
  }
  __syncthreads();

  while (true) {
    if (tid == 0) {
      if (sp > 0) cur = stk[--sp];
      else cur.e = cur.b;  // signals done with b == e below (never a real node)
    }
    __syncthreads();
    const uint32_t b = cur.b, e = cur.e, par = cur.par;
    if (e <= b) break;  // uniform
    const uint32_t cnt = e - b;
    const uint4 *src = par ? a.codesB : a.codesA;
    const uint32_t *srcid = par ? a.idsB : a.idsA;

    bool eligible_any = false;
    for (int j = 0; j < K; ++j) eligible_any |= cur.nb[j] < bb;

    if (cnt > (uint32_t)a.M && eligible_any) {
      // count the next bit of every dimension with bits left
      uint32_t c1[16], shj[16];
      uint32_t elig = 0;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        c1[j] = 0;
        const bool el = j < K && cur.nb[j] < bb;
        elig |= (el ? 1u : 0u) << j;
        shj[j] = el ? (uint32_t)(bb - 1 - cur.nb[j]) : 0u;
      }
      for (uint32_t i = b + tid; i < e; i += TB_THREADS) {
        const uint4 c = src[i];
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (elig & (1u << j)) c1[j] += (code_byte(c, j) >> shj[j]) & 1u;
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        uint32_t v = c1[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        if (lane == 0) wpart[warp][j] = v;
      }
      __syncthreads();
      if (tid < 16) {
        uint32_t v = 0;
        for (int w = 0; w < TB_THREADS / 32; ++w) v += wpart[w][tid];
        n1s[tid] = v;
      }
      __syncthreads();
      if (tid == 0) {
        int best = -1;
        int64_t bestd = 0;
        for (int j = 0; j < K; ++j) {
          if (cur.nb[j] >= bb) continue;
          int64_t dd = (int64_t)cnt - 2 * (int64_t)n1s[j];
          if (dd < 0) dd = -dd;
          if (best < 0 || dd < bestd) { best = j; bestd = dd; }
        }
        split_dim = best;
        degenerate = (n1s[best] == 0u || n1s[best] == cnt);
        if (degenerate) {
          // one side empty: the only child has the same points, one more bit
          StackEntry ch = cur;
          ch.nb[best] = (uint8_t)(cur.nb[best] + 1);
          if (sp < TB_STACK) stk[sp++] = ch;
          else atomicExch(a.err, (int)DETLSH_ERR_CAPACITY);
        }
      }
      __syncthreads();
      if (degenerate) continue;
      const int js = split_dim;
      const uint32_t n0 = cnt - n1s[js];
      const uint32_t sh = (uint32_t)(bb - 1 - cur.nb[js]);
      uint4 *dst = par ? a.codesA : a.codesB;
      uint32_t *dstid = par ? a.idsA : a.idsB;
      uint32_t zrun = 0, orun = 0;
      const unsigned lt = (1u << lane) - 1u;
      for (uint32_t base = b; base < e; base += TB_THREADS) {
        const uint32_t i = base + tid;
        const bool valid = i < e;
        uint4 c = make_uint4(0, 0, 0, 0);
        uint32_t id = 0, bit = 0;
        if (valid) { c = src[i]; id = srcid[i]; bit = (code_byte(c, js) >> sh) & 1u; }
        const unsigned ones = __ballot_sync(FULL, valid && bit);
        const unsigned zeros = __ballot_sync(FULL, valid && !bit);
        if (lane == 0) { wz[warp] = __popc(zeros); wo[warp] = __popc(ones); }
        __syncthreads();
        uint32_t zb = 0, ob = 0, zt = 0, ot = 0;
        for (int w = 0; w < TB_THREADS / 32; ++w) {
          if (w < warp) { zb += wz[w]; ob += wo[w]; }
          zt += wz[w]; ot += wo[w];
        }
        if (valid) {
          const uint32_t pos = bit ? (b + n0 + orun + ob + __popc(ones & lt))
                                   : (b + zrun + zb + __popc(zeros & lt));
          dst[pos] = c;
          dstid[pos] = id;
        }
        zrun += zt;
        orun += ot;
        __syncthreads();
      }
      if (tid == 0) {
        StackEntry c0 = cur, c1e = cur;
        c0.nb[js] = c1e.nb[js] = (uint8_t)(cur.nb[js] + 1);
        c0.par = c1e.par = par ^ 1u;
        c0.e = b + n0;
        c1e.b = b + n0;
        // child 1 below child 0: DFS visits child 0 first.  Depth is bounded
        // by K*(bits-1)+1 < TB_STACK; the guard only reports, never overflows.
        if (sp + 2 > TB_STACK) {
          atomicExch(a.err, (int)DETLSH_ERR_CAPACITY);
        } else {
          if (c1e.e > c1e.b) stk[sp++] = c1e;
          if (c0.e > c0.b) stk[sp++] = c0;
        }
      }
      __syncthreads();
      continue;
    }

    // ---- leaf: ids to perm, box to the slot of this first-layer node ----
    for (uint32_t i = b + tid; i < e; i += TB_THREADS) a.perm[i] = srcid[i];
    const uint32_t slot = b0 + nleaf;
    __syncthreads();  // every thread has read nleaf before thread 0 advances it
    if (a.box_mode == DETLSH_BOX_TIGHT) {
      uint32_t mn[16], mx[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) { mn[j] = 255u; mx[j] = 0u; }
      for (uint32_t i = b + tid; i < e; i += TB_THREADS) {
        const uint4 c = src[i];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const uint32_t v = code_byte(c, j);
          mn[j] = min(mn[j], v);
          mx[j] = max(mx[j], v);
        }
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          mn[j] = min(mn[j], __shfl_xor_sync(FULL, mn[j], o));
          mx[j] = max(mx[j], __shfl_xor_sync(FULL, mx[j], o));
        }
      }
      if (tid < 16) { boxv[0][tid] = 255u; boxv[1][tid] = 0u; }
      __syncthreads();
      if (lane == 0) {
        for (int j = 0; j < 16; ++j) {
          atomicMin(&boxv[0][j], mn[j]);
          atomicMax(&boxv[1][j], mx[j]);
        }
      }
      __syncthreads();
    }
    if (tid < 16) {
      uint8_t lo = 0, hi = 0;
      if (tid < K) {
        const uint32_t freeb = (uint32_t)(bb - cur.nb[tid]);
        const uint32_t pre = code_byte(src[b], tid) >> freeb;
        lo = (uint8_t)(pre << freeb);
        hi = (uint8_t)((pre << freeb) + (1u << freeb) - 1u);
        if (a.box_mode == DETLSH_BOX_TIGHT) { lo = (uint8_t)boxv[0][tid]; hi = (uint8_t)boxv[1][tid]; }
      }
      a.tmp_box[(int64_t)slot * 48 + tid] = lo;
      a.tmp_box[(int64_t)slot * 48 + 16 + tid] = hi;
      a.tmp_box[(int64_t)slot * 48 + 32 + tid] = tid < K ? cur.nb[tid] : 0;
    }
    if (tid == 0) {
      a.tmp_begin[slot] = b;
      nleaf = nleaf + 1;
    }
    __syncthreads();
  }
  if (tid == 0) a.node_count[blockIdx.x] = nleaf;
}

struct LeafWriteArgs {
  int64_t n;
  int L, t;
  const uint32_t *node_begin, *node_count, *leaf_base, *tmp_begin, *perm;
  const uint8_t *tmp_box;
  uint32_t *leaf_begin;
  uint8_t *leaf_lo, *leaf_hi, *leaf_nb;
  uint32_t *leaf_of;
  uint32_t *max_leaf;
};

// One warp per first-layer node: number its leaves, copy their records and
// write leaf_of for their points.
__global__ void k_leaf_write(LeafWriteArgs a, int64_t F) {
  const int64_t f = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (f >= F) return;
  const uint32_t nb0 = a.node_begin[f], ne = a.node_begin[f + 1];
  const uint32_t cnt = a.node_count[f], base = a.leaf_base[f];
  for (uint32_t l = 0; l < cnt; ++l) {
    const uint32_t slot = nb0 + l;
    const uint32_t g = base + l;
    const uint32_t lb = a.tmp_begin[slot];
    const uint32_t le = (l + 1 < cnt) ? a.tmp_begin[slot + 1] : ne;
    if (lane < 16) {
      a.leaf_lo[(int64_t)g * 16 + lane] = a.tmp_box[(int64_t)slot * 48 + lane];
      a.leaf_hi[(int64_t)g * 16 + lane] = a.tmp_box[(int64_t)slot * 48 + 16 + lane];
      a.leaf_nb[(int64_t)g * 16 + lane] = a.tmp_box[(int64_t)slot * 48 + 32 + lane];
    }
    if (lane == 0) {
      a.leaf_begin[g] = lb;
      atomicMax(a.max_leaf, le - lb);
    }
    for (uint32_t i = lb + lane; i < le; i += 32)
      a.leaf_of[(int64_t)a.perm[i] * a.L + a.t] = g;
  }
}

__global__ void k_set_u32(uint32_t *p, uint32_t v) { *p = v; }

// Hull boxes of consecutive runs of LEAF_BLOCK leaves (in canonical order):
// per dimension the smallest lo and largest hi of the run.  A hull contains
// every leaf box of its run, so its lower bound bounds theirs from below.
__global__ void k_block_hulls(const uint8_t *__restrict__ lo, const uint8_t *__restrict__ hi,
                              int64_t nleaves, int64_t nblocks, uint8_t *hlo, uint8_t *hhi) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblocks) return;
  uint32_t mn[16], mx[16];
  for (int j = 0; j < 16; ++j) { mn[j] = 255u; mx[j] = 0u; }
  const int64_t l1 = nleaves < (b + 1) * LEAF_BLOCK ? nleaves : (b + 1) * LEAF_BLOCK;
  for (int64_t l = b * LEAF_BLOCK; l < l1; ++l) {
    const uint4 a = reinterpret_cast<const uint4 *>(lo)[l];
    const uint4 c = reinterpret_cast<const uint4 *>(hi)[l];
    for (int j = 0; j < 16; ++j) {
      mn[j] = min(mn[j], code_byte(a, j));
      mx[j] = max(mx[j], code_byte(c, j));
    }
  }
  uint32_t w0[4] = {0, 0, 0, 0}, w1[4] = {0, 0, 0, 0};
  for (int j = 0; j < 16; ++j) {
    w0[j >> 2] |= mn[j] << (8 * (j & 3));
    w1[j >> 2] |= mx[j] << (8 * (j & 3));
  }
  reinterpret_cast<uint4 *>(hlo)[b] = make_uint4(w0[0], w0[1], w0[2], w0[3]);
  reinterpret_cast<uint4 *>(hhi)[b] = make_uint4(w1[0], w1[1], w1[2], w1[3]);
}

int block_hulls(const uint8_t *lo, const uint8_t *hi, int64_t nleaves, uint8_t *hlo, uint8_t *hhi,
                cudaStream_t st) {
  const int64_t nb = ceil_div(nleaves, LEAF_BLOCK);
  if (nb == 0) return DETLSH_OK;
  k_block_hulls<<<(unsigned)ceil_div(nb, 128), 128, 0, st>>>(lo, hi, nleaves, nb, hlo, hhi);
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  return DETLSH_OK;
}

int build_tree(const TreeBuildArgs &A, TreeTemp &T, int64_t *nleaves, int64_t *max_leaf,
               cudaStream_t st) {
  const int64_t n = A.n;
  const int gs = (int)std::min<int64_t>(ceil_div(n, 256), 4096);
  DL_CUDA(cudaMemsetAsync(T.scalars, 0, 4 * sizeof(uint32_t), st));
  k_first_keys<<<gs, 256, 0, st>>>(A.codes_t, n, A.K, A.bbits, T.keys, T.vals);
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  DL_TRY(segmented_sort(T.keys, T.vals, 1, n, A.K, T.sort, st));
  k_gather_codes<<<gs, 256, 0, st>>>(reinterpret_cast<const uint4 *>(A.codes_t), T.vals, n,
                                     T.codesA);
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  // first-layer nodes = runs of equal keys
  uint32_t *F_dev = T.scalars;
  DL_TRY(compact(n, BoundaryFlag{T.keys}, T.block_counts, T.node_begin, F_dev, st));
  uint32_t F = 0;
  DL_CUDA(cudaMemcpyAsync(&F, F_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  DL_CUDA(cudaStreamSynchronize(st));
  k_set_u32<<<1, 1, 0, st>>>(T.node_begin + F, (uint32_t)n);
  dl_count_launch();
  SubtreeArgs sa;
  sa.n = n; sa.K = A.K; sa.bbits = A.bbits; sa.M = A.M; sa.box_mode = A.box_mode;
  sa.node_begin = T.node_begin;
  sa.codesA = T.codesA; sa.codesB = T.codesB;
  sa.idsA = T.vals; sa.idsB = T.idsB;
  sa.perm = A.perm;
  sa.node_count = T.node_count;
  sa.tmp_begin = T.tmp_begin;
  sa.tmp_box = T.tmp_box;
  sa.err = reinterpret_cast<int *>(T.scalars + 2);
  k_subtree<<<F, TB_THREADS, 0, st>>>(sa);
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  // leaf numbering
  DL_CUDA(cudaMemcpyAsync(T.leaf_base, T.node_count, sizeof(uint32_t) * F,
                          cudaMemcpyDeviceToDevice, st));
  k_scan_counts<<<1, 1024, 0, st>>>(T.leaf_base, F, T.scalars + 1);
  dl_count_launch();
  DL_CUDA(cudaMemsetAsync(T.scalars + 3, 0, sizeof(uint32_t), st));
  LeafWriteArgs lw;
  lw.n = n; lw.L = A.L; lw.t = A.t;
  lw.node_begin = T.node_begin; lw.node_count = T.node_count; lw.leaf_base = T.leaf_base;
  lw.tmp_begin = T.tmp_begin; lw.perm = A.perm; lw.tmp_box = T.tmp_box;
  lw.leaf_begin = A.leaf_begin; lw.leaf_lo = A.leaf_lo; lw.leaf_hi = A.leaf_hi;
  lw.leaf_nb = A.leaf_nb; lw.leaf_of = A.leaf_of; lw.max_leaf = T.scalars + 3;
  k_leaf_write<<<(unsigned)ceil_div((int64_t)F * 32, 256), 256, 0, st>>>(lw, F);
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  uint32_t hs[4];
  DL_CUDA(cudaMemcpyAsync(hs, T.scalars, sizeof(hs), cudaMemcpyDeviceToHost, st));
  DL_CUDA(cudaStreamSynchronize(st));
  if (hs[2] != 0) return (int)hs[2];
  k_set_u32<<<1, 1, 0, st>>>(A.leaf_begin + hs[1], (uint32_t)n);
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  *nleaves = hs[1];
  *max_leaf = hs[3];
  return DETLSH_OK;
}

}  // namespace dl
