// sort.cu -- segmented stable radix sort, Bernoulli sampling and breakpoint
// extraction for the encoding phase (Sec. III-A).
//
// The paper selects the N_r+1 breakpoints of every projected dimension with
// rounds of QuickSelect on a 0.1 n sample.  Those are order statistics of
// the sample; on the GPU all L*K sample columns are sorted at once by a
// stable LSD radix sort (one launch per 8-bit digit covers every column) and
// the order statistics are read off the sorted columns.
#include "common.cuh"
#include "compact.cuh"
#include "kernels.h"

#include <algorithm>
#include <cmath>
#include <utility>

namespace dl {

constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;

size_t sort_tiles(int64_t len) { return (size_t)ceil_div(len, SORT_TILE); }

// counts[(seg*256 + digit)*tiles + tile] = digit histogram of one tile.
__global__ void __launch_bounds__(SORT_THREADS)
k_radix_hist(const uint32_t *__restrict__ keys, int64_t len, int shift, uint32_t *counts,
             int tiles) {
  __shared__ uint32_t h[256];
  const int seg = blockIdx.y, tile = blockIdx.x;
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t *k = keys + (int64_t)seg * len;
  const int64_t base = (int64_t)tile * SORT_TILE;
  for (int i = threadIdx.x; i < SORT_TILE; i += SORT_THREADS) {
    const int64_t idx = base + i;
    if (idx < len) atomicAdd(&h[(k[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[((int64_t)seg * 256 + threadIdx.x) * tiles + tile] = h[threadIdx.x];
}

// Exclusive scan across tiles of one (segment, digit); digit totals out.
__global__ void __launch_bounds__(SORT_THREADS)
k_radix_scan_digit(uint32_t *counts, int tiles, uint32_t *digit_total) {
  __shared__ uint32_t wt[32];
  const int seg = blockIdx.y, digit = blockIdx.x;
  uint32_t *c = counts + ((int64_t)seg * 256 + digit) * tiles;
  uint32_t carry = 0;
  for (int base = 0; base < tiles; base += SORT_THREADS) {
    const int i = base + threadIdx.x;
    const uint32_t v = i < tiles ? c[i] : 0u;
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan(v, wt, &tot);
    if (i < tiles) c[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) digit_total[seg * 256 + digit] = carry;
}

// digit_total -> exclusive digit base, per segment.
__global__ void __launch_bounds__(256) k_radix_scan_totals(uint32_t *digit_total) {
  __shared__ uint32_t wt[32];
  uint32_t *t = digit_total + blockIdx.x * 256;
  const uint32_t v = t[threadIdx.x];
  const uint32_t ex = block_exclusive_scan(v, wt, nullptr);
  t[threadIdx.x] = ex;
}

// Stable scatter of one tile.  Warp w owns elements [512 w, 512 w + 512) of
// the tile and ranks them in index order against its own digit counters
// (lanes with equal digits found by one ballot per digit bit); one block
// scan then turns the per-warp counts into positions in a digit-sorted copy
// of the tile in shared memory, which is written out in order, so the
// elements of one digit leave as one contiguous run.
// FUSED: counts holds the raw per-tile histograms (few tiles per segment);
// each tile sums the earlier tiles' counts and scans the segment's digit
// totals itself.  Otherwise counts and digit_base come scanned.
template <bool FUSED>
__global__ void __launch_bounds__(SORT_THREADS)
k_radix_scatter(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                uint32_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t len, int shift,
                const uint32_t *__restrict__ counts, const uint32_t *__restrict__ digit_base,
                int tiles) {
  constexpr int NW = SORT_THREADS / 32;
  constexpr int PER_WARP = SORT_TILE / NW;  // = 32 * SORT_ITEMS
  __shared__ uint32_t sk[SORT_TILE], sv[SORT_TILE];
  __shared__ uint32_t wh[NW][256];    // per-warp digit counters, then per-warp digit starts
  __shared__ uint32_t gshift[256];    // global position - local position, per digit
  __shared__ uint32_t wt[32];
  const int seg = blockIdx.y, tile = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t soff = (int64_t)seg * len;
  const int64_t t0 = (int64_t)tile * SORT_TILE;
  const int nvalid = (int)(len - t0 < SORT_TILE ? len - t0 : (int64_t)SORT_TILE);
  for (int w = 0; w < NW; ++w) wh[w][threadIdx.x] = 0;
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  uint32_t key[SORT_ITEMS], val[SORT_ITEMS], rk[SORT_ITEMS];
#pragma unroll
  for (int r = 0; r < SORT_ITEMS; ++r) {
    const int i = warp * PER_WARP + r * 32 + lane;
    const bool valid = i < nvalid;
    key[r] = valid ? kin[soff + t0 + i] : 0u;
    val[r] = (valid && vin) ? vin[soff + t0 + i] : 0u;
    const uint32_t digit = (key[r] >> shift) & 255u;
    unsigned peers = __ballot_sync(FULL, valid);
#pragma unroll
    for (int bt = 0; bt < 8; ++bt) {
      const bool set = (digit >> bt) & 1u;
      const unsigned bb = __ballot_sync(FULL, set);
      peers &= set ? bb : ~bb;
    }
    const int rank = __popc(peers & lt);
    const uint32_t base = wh[warp][digit];
    rk[r] = base + rank;
    __syncwarp();
    if (valid && rank == 0) wh[warp][digit] = base + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {  // digit d: local start, per-warp starts, global shift
    const int d = threadIdx.x;
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) cnt += wh[w][d];
    const uint32_t ls = block_exclusive_scan(cnt, wt, nullptr);
    uint32_t acc = ls;
#pragma unroll
    for (int w = 0; w < NW; ++w) { const uint32_t v = wh[w][d]; wh[w][d] = acc; acc += v; }
    const uint32_t *cd = counts + ((int64_t)seg * 256 + d) * tiles;
    if (FUSED) {
      uint32_t pre = 0, tot = 0;
      for (int t = 0; t < tiles; ++t) {
        const uint32_t v = cd[t];
        if (t < tile) pre += v;
        tot += v;
      }
      const uint32_t db = block_exclusive_scan(tot, wt, nullptr);
      gshift[d] = db + pre - ls;
    } else {
      gshift[d] = digit_base[seg * 256 + d] + cd[tile] - ls;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < SORT_ITEMS; ++r) {
    const int i = warp * PER_WARP + r * 32 + lane;
    if (i < nvalid) {
      const uint32_t pos = wh[warp][(key[r] >> shift) & 255u] + rk[r];
      sk[pos] = key[r];
      sv[pos] = val[r];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nvalid; i += SORT_THREADS) {
    const uint32_t k = sk[i];
    const uint32_t pos = gshift[(k >> shift) & 255u] + (uint32_t)i;
    kout[soff + pos] = k;
    if (vin) vout[soff + pos] = sv[i];
  }
}

int segmented_sort(uint32_t *keys, uint32_t *vals, int nseg, int64_t len, int nbits,
                   SortTemp &tmp, cudaStream_t st) {
  if (len <= 0 || nseg <= 0 || nbits <= 0) return DETLSH_OK;
  const int tiles = (int)sort_tiles(len);
  if ((size_t)nseg * 256 * tiles > tmp.count_cap) return DETLSH_ERR_CAPACITY;
  uint32_t *kin = keys, *vin = vals, *kout = tmp.keys_alt, *vout = vals ? tmp.vals_alt : nullptr;
  int passes = 0;
  for (int shift = 0; shift < nbits; shift += 8, ++passes) {
    dim3 g((unsigned)tiles, (unsigned)nseg);
    k_radix_hist<<<g, SORT_THREADS, 0, st>>>(kin, len, shift, tmp.counts, tiles);
    dl_count_launch();
    if (tiles <= 64) {  // few tiles per segment: the scatter scans the counts itself
      k_radix_scatter<true><<<g, SORT_THREADS, 0, st>>>(kin, vin, kout, vout, len, shift,
                                                        tmp.counts, tmp.digit_base, tiles);
      dl_count_launch();
    } else {
      k_radix_scan_digit<<<dim3(256, nseg), SORT_THREADS, 0, st>>>(tmp.counts, tiles, tmp.digit_base);
      dl_count_launch();
      k_radix_scan_totals<<<nseg, 256, 0, st>>>(tmp.digit_base);
      dl_count_launch();
      k_radix_scatter<false><<<g, SORT_THREADS, 0, st>>>(kin, vin, kout, vout, len, shift,
                                                         tmp.counts, tmp.digit_base, tiles);
      dl_count_launch();
    }
    DL_CUDA(cudaGetLastError());
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  if (passes & 1) {
    DL_CUDA(cudaMemcpyAsync(keys, kin, sizeof(uint32_t) * (size_t)nseg * len,
                            cudaMemcpyDeviceToDevice, st));
    if (vals)
      DL_CUDA(cudaMemcpyAsync(vals, vin, sizeof(uint32_t) * (size_t)nseg * len,
                              cudaMemcpyDeviceToDevice, st));
  }
  return DETLSH_OK;
}

// ---- compaction scan ----------------------------------------------------------
__global__ void k_scan_counts(uint32_t *counts, int64_t nb, const uint32_t *nb_dev, uint32_t *total) {
  __shared__ uint32_t wt[32];
  if (nb_dev) nb = *nb_dev;  // the count lives on the device (no host round trip)
  uint32_t carry = 0;
  for (int64_t base = 0; base < nb; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const uint32_t v = i < nb ? counts[i] : 0u;
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan(v, wt, &tot);
    if (i < nb) counts[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

// ---- Bernoulli sample (Sec. III-A, n_s = 0.1 n) -------------------------------
struct SampleFlag {
  uint32_t k0, k1, thr;
  int all;
  __device__ bool operator()(int64_t p) const {
    if (all) return true;
    const U4 r = philox4x32_10(U4{(uint32_t)p, (uint32_t)((uint64_t)p >> 32), STREAM_SAMPLE, 0u},
                               k0, k1);
    return r.x < thr;
  }
};

struct AllFlag {
  __device__ bool operator()(int64_t) const { return true; }
};

size_t sample_blocks(int64_t n) { return (size_t)compact_blocks(n); }

int sample_ids(int64_t n, uint64_t seed, double frac, uint32_t *ids, uint32_t *block_counts,
               int64_t *m_out, cudaStream_t st) {
  // threshold floor(frac * 2^32); frac >= 1 takes every point
  const double scaled = floor(frac * 4294967296.0);
  SampleFlag f{(uint32_t)seed, (uint32_t)(seed >> 32),
               scaled >= 4294967296.0 ? 0u : (uint32_t)scaled, scaled >= 4294967296.0};
  uint32_t *count = block_counts + compact_blocks(n) + 1;
  DL_TRY(compact(n, f, block_counts, ids, count, st));
  uint32_t m = 0;
  DL_CUDA(cudaMemcpyAsync(&m, count, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  DL_CUDA(cudaStreamSynchronize(st));
  *m_out = m;
  return DETLSH_OK;
}

// ---- breakpoints -------------------------------------------------------------
__global__ void k_float_to_keys(float *v, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t *u = reinterpret_cast<uint32_t *>(v);
    u[i] = fkey(v[i] + 0.0f);
  }
}

int float_to_keys(float *v, int64_t count, cudaStream_t st) {
  if (count <= 0) return DETLSH_OK;
  const int64_t blocks = std::min<int64_t>(ceil_div(count, 256), 65535);
  k_float_to_keys<<<(unsigned)blocks, 256, 0, st>>>(v, count);
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  return DETLSH_OK;
}

// Interior breakpoints B[t][b] = S_t[q*b - 1], q = max(1, floor(m/N_r)),
// index clamped to m-1 (Sec. III-A, breakpoint rule on the sorted sample).
__global__ void k_extract_breakpoints(const uint32_t *__restrict__ sorted, int LK, int64_t m,
                                      int N_r, float *B) {
  const int t = blockIdx.x;
  int64_t q = m / N_r;
  if (q < 1) q = 1;
  for (int b = 1 + threadIdx.x; b < N_r; b += blockDim.x) {
    int64_t idx = q * b - 1;
    if (idx > m - 1) idx = m - 1;
    B[(int64_t)t * (N_r + 1) + b] = funkey(sorted[(int64_t)t * m + idx]);
  }
}

int extract_breakpoints(const uint32_t *sorted_keys, int LK, int64_t m, int N_r, float *B,
                        cudaStream_t st) {
  k_extract_breakpoints<<<LK, 256, 0, st>>>(sorted_keys, LK, m, N_r, B);
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  return DETLSH_OK;
}

// End breakpoints: the minimum and maximum of each column over all n points.
__global__ void k_finish_ends(const uint32_t *minmax, int LK, int N_r, float *B) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= LK) return;
  B[(int64_t)t * (N_r + 1)] = funkey(minmax[2 * t]);
  B[(int64_t)t * (N_r + 1) + N_r] = funkey(minmax[2 * t + 1]);
}

int finish_breakpoint_ends(const uint32_t *minmax, int LK, int N_r, float *B, cudaStream_t st) {
  k_finish_ends<<<(unsigned)ceil_div(LK, 128), 128, 0, st>>>(minmax, LK, N_r, B);
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  return DETLSH_OK;
}

}  // namespace dl
