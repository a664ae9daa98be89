// compact.cuh -- order-preserving stream compaction of flagged indices.
#pragma once
#include "common.cuh"

namespace dl {

constexpr int CP_THREADS = 256;
constexpr int CP_ITEMS = 16;
constexpr int CP_TILE = CP_THREADS * CP_ITEMS;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_tot,
                                                          uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t w = lane < nw ? warp_tot[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) warp_tot[lane] = w;  // inclusive
  }
  __syncthreads();
  const uint32_t before = (warp ? warp_tot[warp - 1] : 0u) + x - v;
  if (total) *total = warp_tot[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

template <class Flag>
__global__ void k_compact_count(int64_t n, Flag f, uint32_t *block_counts) {
  __shared__ uint32_t wt[32];
  const int64_t base = (int64_t)blockIdx.x * CP_TILE + (int64_t)threadIdx.x * CP_ITEMS;
  uint32_t c = 0;
  for (int i = 0; i < CP_ITEMS; ++i) {
    const int64_t idx = base + i;
    if (idx < n && f(idx)) ++c;
  }
  uint32_t tot;
  block_exclusive_scan(c, wt, &tot);
  if (threadIdx.x == 0) block_counts[blockIdx.x] = tot;
}

// Exclusive scan of counts[0 .. nb) in place (nb read from *nb_dev when that
// is given); *total (optional) receives the sum.
__global__ void k_scan_counts(uint32_t *counts, int64_t nb, const uint32_t *nb_dev, uint32_t *total);

template <class Flag>
__global__ void k_compact_write(int64_t n, Flag f, const uint32_t *block_offsets, uint32_t *out) {
  __shared__ uint32_t wt[32];
  const int64_t base = (int64_t)blockIdx.x * CP_TILE + (int64_t)threadIdx.x * CP_ITEMS;
  uint32_t flags = 0, c = 0;
  for (int i = 0; i < CP_ITEMS; ++i) {
    const int64_t idx = base + i;
    if (idx < n && f(idx)) { flags |= 1u << i; ++c; }
  }
  uint32_t pos = block_offsets[blockIdx.x] + block_exclusive_scan(c, wt, nullptr);
  for (int i = 0; i < CP_ITEMS; ++i)
    if (flags & (1u << i)) out[pos++] = (uint32_t)(base + i);
}

inline int64_t compact_blocks(int64_t n) { return ceil_div(n, CP_TILE); }

// out receives the flagged indices in ascending order; *count (device) the total.
template <class Flag>
int compact(int64_t n, Flag f, uint32_t *block_counts, uint32_t *out, uint32_t *count,
            cudaStream_t st) {
  const int64_t nb = compact_blocks(n);
  if (nb == 0) {
    DL_CUDA(cudaMemsetAsync(count, 0, sizeof(uint32_t), st));
    return DETLSH_OK;
  }
  k_compact_count<<<(unsigned)nb, CP_THREADS, 0, st>>>(n, f, block_counts);
  dl_count_launch();
  k_scan_counts<<<1, 1024, 0, st>>>(block_counts, nb, nullptr, count);
  dl_count_launch();
  k_compact_write<<<(unsigned)nb, CP_THREADS, 0, st>>>(n, f, block_counts, out);
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  return DETLSH_OK;
}

}  // namespace dl
