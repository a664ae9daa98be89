// rcann.cu -- (r,c)-ANN queries (Alg. 4) over the DE-Trees with the range
// query of Alg. 3 as printed (Sec. IV-C pruning), or with optimisation (1)
// of Sec. VI-B2 (every leaf whose lower bound is within r' taken whole).
//
// One persistent launch, one CTA per query at a time.  For each tree in
// order: the leaf-run hulls and then the leaves whose lower bound is within
// r' = eps r are listed; a leaf whose upper bound is within r' gives all its
// points, any other listed leaf gives the points whose projection lies within
// r' of q' (FP32, dimensions in order).  A point is new when no earlier tree
// returned it, i.e. its projected distance in every earlier tree exceeds r'
// (the bounds only accelerate that test: LB <= distance <= UB).  New points
// are counted, written to S and folded into the running nearest point; once
// |S| >= beta n + 1 the query stops (Alg. 4, first condition); after all L
// trees the nearest point of S is returned only if it lies within c r (its
// second condition).
#include "common.cuh"
#include "compact.cuh"
#include "kernels.h"
#include "lut.cuh"

#include <algorithm>

namespace dl {

constexpr int RT = 256;
constexpr int RW = RT / 32;
constexpr int RFLC = 512;  // listed leaves per chunk of the point visit

struct RcShared {
  float qp[256];
  uint32_t wt[32];
  uint32_t fl_pre[RFLC + 1], fl_beg[RFLC];
  uint64_t best;       // (squared distance bits << 32) | id of the nearest new point
  unsigned long long count;
  int64_t qi;
  uint32_t nblist, nllist;
  int stop;
};

size_t rcann_slot_bytes(const QueryIndexView &ix) {
  const int64_t tb = ix.blk_off[ix.L], tl = ix.leaf_off[ix.L];
  return (size_t)(4 * (tb + tl) + 512);
}

// Squared distance between point p's projection and q' in tree u (FP32,
// dimensions in order, no fused multiply-add).
__device__ __forceinline__ float proj_d2(const QueryIndexView &ix, const float *qp, uint32_t p,
                                         int u) {
  const float *po = ix.P + (int64_t)p * ix.LK + u * ix.K;
  const float *qu = qp + u * ix.K;
  float acc = 0.0f;
  for (int j = 0; j < ix.K; ++j) {
    const float dj = __fsub_rn(po[j], qu[j]);
    acc = __fadd_rn(acc, __fmul_rn(dj, dj));
  }
  return acc;
}

// Squared FP32 distance between q and x_p (one thread).
__device__ __forceinline__ float point_d2(const QueryIndexView &ix, const float *q, uint32_t p) {
  const int d = ix.d;
  const float *x = ix.X + (int64_t)p * d;
  float acc = 0.0f;
  if ((d & 3) == 0) {
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    const float4 *q4 = reinterpret_cast<const float4 *>(q);
    for (int c = 0; c < (d >> 2); ++c) {
      const float4 a = q4[c], b = x4[c];
      const float t0 = __fsub_rn(a.x, b.x), t1 = __fsub_rn(a.y, b.y);
      const float t2 = __fsub_rn(a.z, b.z), t3 = __fsub_rn(a.w, b.w);
      acc = __fmaf_rn(t0, t0, acc);
      acc = __fmaf_rn(t1, t1, acc);
      acc = __fmaf_rn(t2, t2, acc);
      acc = __fmaf_rn(t3, t3, acc);
    }
  } else {
    for (int c = 0; c < d; ++c) {
      const float t0 = __fsub_rn(q[c], x[c]);
      acc = __fmaf_rn(t0, t0, acc);
    }
  }
  return acc;
}

// Lower bound of leaf l of tree u from the breakpoints and q' (the table's
// operations in the table's order, so it equals box_lb2 on the table).
__device__ __forceinline__ float leaf_lb2_of(const QueryIndexView &ix, const float *qp, int u,
                                             uint32_t l) {
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
    const float gap = fmaxf(fmaxf(__fsub_rn(Bj[zl], q), -__fsub_rn(Bj[zh + 1], q)), 0.0f);
    acc = __fadd_rn(acc, __fmul_rn(gap, gap));
  }
  return acc;
}

__global__ void __launch_bounds__(RT) k_rcann(QueryIndexView ix, RcArgs a) {
  extern __shared__ __align__(16) uint8_t dsm[];
  float *lut = reinterpret_cast<float *>(dsm);
  __shared__ RcShared sm;
  uint8_t *base = a.scratch + (int64_t)blockIdx.x * a.slot_bytes;
  uint32_t *blist = reinterpret_cast<uint32_t *>(base);
  uint32_t *llist = blist + ix.blk_off[ix.L];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int NR1 = ix.N_r + 1;

  while (true) {
    if (threadIdx.x == 0) sm.qi = atomicAdd(a.work_counter, 1u);
    __syncthreads();
    const int64_t qi = sm.qi;
    if (qi >= a.m) break;
    for (int i = threadIdx.x; i < ix.LK; i += RT) sm.qp[i] = a.Qp[qi * ix.LK + i];
    if (threadIdx.x == 0) { sm.count = 0; sm.best = ~0ull; sm.stop = -1; }
    const float *q = a.Q + qi * ix.d;
    __syncthreads();
    for (int t = 0; t < ix.L; ++t) {
      build_lut(lut, ix.B, sm.qp + t * ix.K, t, ix.K, NR1);
      if (threadIdx.x == 0) { sm.nblist = 0; sm.nllist = 0; }
      __syncthreads();
      // hulls of leaf runs within r'
      const int64_t nb = ix.blk_off[t + 1] - ix.blk_off[t];
      const int64_t nl = ix.leaf_off[t + 1] - ix.leaf_off[t];
      const uint4 *hlo = reinterpret_cast<const uint4 *>(ix.blk_lo) + ix.blk_off[t];
      const uint4 *hhi = reinterpret_cast<const uint4 *>(ix.blk_hi) + ix.blk_off[t];
      for (int64_t b = threadIdx.x; b < nb; b += RT)
        if (box_lb2(lut, hlo[b], hhi[b]) <= a.R2) blist[atomicAdd(&sm.nblist, 1u)] = (uint32_t)b;
      __syncthreads();
      // leaves within r' (whole when the upper bound is within r' too)
      const uint4 *llo = reinterpret_cast<const uint4 *>(ix.leaf_lo) + ix.leaf_off[t];
      const uint4 *lhi = reinterpret_cast<const uint4 *>(ix.leaf_hi) + ix.leaf_off[t];
      const uint32_t nbl = sm.nblist;
      for (uint32_t i = warp; i < nbl; i += RW) {
        const int64_t l = (int64_t)blist[i] * LEAF_BLOCK + lane;
        bool keep = false, whole = false;
        if (l < nl) {
          keep = box_lb2(lut, llo[l], lhi[l]) <= a.R2;
          whole = keep && (a.optimised || box_ub2(lut, llo[l], lhi[l]) <= a.R2);
        }
        const unsigned km = __ballot_sync(FULL, keep);
        uint32_t p0 = 0;
        if (lane == 0 && km) p0 = atomicAdd(&sm.nllist, (uint32_t)__popc(km));
        p0 = __shfl_sync(FULL, p0, 0);
        if (keep) llist[p0 + __popc(km & ((1u << lane) - 1u))] = (uint32_t)l | (whole ? 0x80000000u : 0u);
      }
      __syncthreads();
      // points of the listed leaves, in chunks laid out by a block scan
      const uint32_t nll = sm.nllist;
      const uint32_t *permt = ix.perm + (int64_t)t * ix.n;
      for (uint32_t e0 = 0; e0 < nll; e0 += RFLC) {
        uint32_t sz[2], bg[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const uint32_t e = e0 + threadIdx.x * 2 + u;
          sz[u] = 0; bg[u] = 0;
          if (e < nll) {
            const uint32_t l = llist[e] & 0x7fffffffu;
            bg[u] = ix.leaf_begin[ix.leaf_off[t] + t + l];
            sz[u] = ix.leaf_begin[ix.leaf_off[t] + t + l + 1] - bg[u];
          }
        }
        uint32_t np;
        const uint32_t ps = block_exclusive_scan(sz[0] + sz[1], sm.wt, &np);
        const uint32_t nq = min((uint32_t)RFLC, nll - e0);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const uint32_t k = threadIdx.x * 2 + u;
          if (k < nq) {
            sm.fl_pre[k] = ps + (u ? sz[0] : 0u);
            // the whole-leaf flag rides in the top bit of the perm offset
            sm.fl_beg[k] = bg[u] | (llist[e0 + k] & 0x80000000u);
          }
        }
        if (threadIdx.x == 0) sm.fl_pre[nq] = np;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < np; i += RT) {
          int lo = 0, hi = (int)nq;  // last k with fl_pre[k] <= i
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (sm.fl_pre[mid] <= i) lo = mid; else hi = mid;
          }
          const uint32_t fb = sm.fl_beg[lo];
          const uint32_t p = permt[(fb & 0x7fffffffu) + (i - sm.fl_pre[lo])];
          bool in = (fb >> 31) || proj_d2(ix, sm.qp, p, t) <= a.R2;
          for (int u = 0; in && u < t; ++u) {  // returned by an earlier tree?
            if (a.optimised) {
              if (leaf_lb2_of(ix, sm.qp, u, ix.leaf_of[(int64_t)p * ix.L + u]) <= a.R2) in = false;
            } else if (proj_d2(ix, sm.qp, p, u) <= a.R2) {
              in = false;
            }
          }
          if (in) {
            const unsigned long long pos = atomicAdd(&sm.count, 1ull);
            if (a.S && (int64_t)pos < a.S_cap) a.S[qi * a.S_cap + (int64_t)pos] = p;
            const float d2 = point_d2(ix, q, p);
            atomicMin(reinterpret_cast<unsigned long long *>(&sm.best),
                      ((unsigned long long)__float_as_uint(d2) << 32) | p);
          }
        }
        __syncthreads();
      }
      __syncthreads();
      const bool done = (int64_t)sm.count >= a.need;
      if (done) {
        if (threadIdx.x == 0) sm.stop = t;
        break;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t id = -1;
      float dist = __int_as_float(0x7f800000);
      if (sm.best != ~0ull) {
        const float dd = __fsqrt_rn(__uint_as_float((uint32_t)(sm.best >> 32)));
        if (sm.stop >= 0 || dd <= a.cr) { id = (int64_t)(uint32_t)sm.best; dist = dd; }
      }
      a.ids[qi] = id;
      a.dists[qi] = dist;
      a.tree_stop[qi] = sm.stop;
      a.S_size[qi] = (int64_t)sm.count;
    }
    __syncthreads();
  }
}

static size_t rcann_smem() { return sizeof(float) * LUT_ROWS * LUT_STRIDE; }

int rcann_slots(const QueryIndexView &) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_rcann, RT, rcann_smem());
  if (per < 1) per = 1;
  return sms * per;
}

int run_rcann(const QueryIndexView &ix, const RcArgs &a, cudaStream_t st) {
  if (a.m <= 0) return DETLSH_OK;
  DL_CUDA(cudaMemsetAsync(a.work_counter, 0, sizeof(uint32_t), st));
  const int grid = (int)std::min<int64_t>(a.nslots, a.m);
  k_rcann<<<grid, RT, rcann_smem(), st>>>(ix, a);
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  return DETLSH_OK;
}

}  // namespace dl
