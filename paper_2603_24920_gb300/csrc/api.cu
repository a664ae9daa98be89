// api.cu -- C-ABI of the DET-LSH hot path (include/detlsh.h): argument
// checks, device memory of the index, and the order of the kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"

// ---------------------------------------------------------------------------
#include <atomic>

static thread_local char g_last_cuda[256];
static std::atomic<long long> g_launches{0};

void dl_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void dl_set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
  snprintf(g_last_cuda, sizeof g_last_cuda, "%s: %s (%s:%d)", cudaGetErrorString(e), what, file,
           line);
}

struct detlsh_index {
  int device = 0;
  int64_t n = 0;
  int d = 0, L = 0, K = 0, LK = 0, N_r = 0, bbits = 0, M = 0, box_mode = 0, encoding = 0, tree_group = 0;
  uint64_t seed = 0;
  double frac = 0.1, eps2 = 0.0;
  int64_t m_sample = 0;
  int64_t nleaves[16] = {0}, leaf_off[17] = {0};
  int64_t max_leaf = 0, max_leaves = 0;
  int64_t device_bytes = 0;
  int64_t fb_total = 0;
  // device arrays
  float *X = nullptr;
  __nv_bfloat16 *Xh = nullptr;
  float2 *Xn = nullptr;  // per row {||bf16(x)||^2, upper bound of ||x - bf16(x)||}
  int bf16_exact = 0;    // every row equals its BF16 copy
  float *A = nullptr, *B = nullptr, *P = nullptr;
  uint8_t *codes = nullptr;
  uint32_t *sample = nullptr;
  uint32_t *perm = nullptr, *leaf_begin = nullptr, *leaf_of = nullptr;
  uint8_t *leaf_lo = nullptr, *leaf_hi = nullptr, *leaf_nb = nullptr;
  uint8_t *blk_lo = nullptr, *blk_hi = nullptr;  // hulls of LEAF_BLOCK-leaf runs
  int64_t blk_off[17] = {0};
  uint8_t *sblk_lo = nullptr, *sblk_hi = nullptr;  // hulls of LEAF_BLOCK-hull runs
  int64_t sblk_off[17] = {0};
  uint8_t *tblk_lo = nullptr, *tblk_hi = nullptr;  // hulls of LEAF_BLOCK super-hull runs
  int64_t tblk_off[17] = {0};
  cudaEvent_t ev[8] = {nullptr};
  detlsh_timings timings{};
  detlsh_tuning tuning{0, 4, 512, 1024, 0, 0};  // query kernel knobs (detlsh_set_tuning / detlsh_autotune)
  std::vector<void *> owned;
  // per-index query buffers, reused across calls (guarded by qmu)
  std::mutex qmu;
  struct QBuf {
    void *p = nullptr;
    size_t bytes = 0;
  };
  QBuf qQ, qQh, qQp, qk, qids, qdists, qT, qscratch, qstat, qS, qfb, qrc, qrcs;
  // detlsh_query_reserve / detlsh_query_async: buffers of their own, so that a
  // captured graph's pointers stay valid whatever other calls do
  struct AsyncPlan {
    bool ready = false;
    detlsh_query_params qp{};
    int64_t m_max = 0;
    int32_t k_max = 0;
    int slots = 0;
    int64_t cap = 0, tau_base = 0;
    int64_t off[dl::SLOT_ARRAYS + 1] = {0};
  } plan;
  QBuf aQp, aQh, afb, aT, astat, ascratch;
};

namespace {

using namespace dl;

// Device memory comes from a library-owned stream-ordered pool per device
// that keeps freed blocks for reuse: repeated builds and growing query
// buffers then allocate without synchronising the device.
constexpr int kPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kPoolDevices] = {};

int pool_get(cudaMemPool_t *out) {
  int dev = 0;
  DL_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kPoolDevices) return DETLSH_ERR_NO_DEVICE;
  std::lock_guard<std::mutex> g(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    DL_CUDA(cudaMemPoolCreate(&pool, &props));
    uint64_t keep = UINT64_MAX;
    DL_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    g_pool[dev] = pool;
  }
  *out = g_pool[dev];
  return DETLSH_OK;
}

int pool_alloc(void **p, size_t bytes, cudaStream_t st) {
  cudaMemPool_t pool;
  DL_TRY(pool_get(&pool));
  DL_CUDA(cudaMallocFromPoolAsync(p, bytes ? bytes : 1, pool, st));
  return DETLSH_OK;
}

// Query scratch outlives its index: a freed index hands its slots to the
// next index on the same device, so rebuilding an index does not clear the
// slots again.  The scratch starts with a device word that hands out the
// per-query epochs its level tags carry; epochs only grow (56 bits), so tags
// left by earlier queries never match a later one.
constexpr size_t kScratchHeader = 256;
struct ScratchCache {
  void *p = nullptr;
  size_t bytes = 0;
};
std::mutex g_scratch_mu;
ScratchCache g_scratch[kPoolDevices];

template <class T>
int dalloc(detlsh_index *ix, T **p, size_t count, cudaStream_t st) {
  *p = nullptr;
  if (count == 0) count = 1;
  void *q = nullptr;
  DL_TRY(pool_alloc(&q, sizeof(T) * count, st));
  *p = static_cast<T *>(q);
  ix->owned.push_back(q);
  ix->device_bytes += (int64_t)(sizeof(T) * count);
  return DETLSH_OK;
}

struct TempPool {
  cudaStream_t st;
  std::vector<void *> ptrs;
  explicit TempPool(cudaStream_t s) : st(s) {}
  template <class T>
  int get(T **p, size_t count) {
    *p = nullptr;
    void *q = nullptr;
    DL_TRY(pool_alloc(&q, sizeof(T) * (count ? count : 1), st));
    ptrs.push_back(q);
    *p = static_cast<T *>(q);
    return DETLSH_OK;
  }
  ~TempPool() {
    for (void *q : ptrs) cudaFreeAsync(q, st);
  }
};

int grow(detlsh_index::QBuf &b, size_t bytes, cudaStream_t st, bool *fresh = nullptr) {
  if (fresh) *fresh = false;
  if (b.bytes >= bytes && b.p) return DETLSH_OK;
  if (b.p) cudaFreeAsync(b.p, st);
  b.p = nullptr;
  b.bytes = 0;
  DL_TRY(pool_alloc(&b.p, bytes, st));
  b.bytes = bytes;
  if (fresh) *fresh = true;
  return DETLSH_OK;
}

// Scratch slots for the query kernel.  `want` is capped by a set budget
// (tuning.query_scratch_mb MiB) and served from the scratch already `held`
// when it fits there (no driver call).  Otherwise the budget is the set one,
// or by default a quarter of the free device memory plus the held scratch,
// never above 90% of the two together; a larger scratch replaces the held
// block only for a clear gain (over a quarter more slots), since the new
// block is a separate allocation.  At least one slot.
int slots_within_budget(const detlsh_index *ix, int want, size_t slot_bytes, size_t held,
                        int *out) {
  const int64_t mb = ix->tuning.query_scratch_mb;
  const int64_t have =
      (slot_bytes && held > kScratchHeader) ? (int64_t)((held - kScratchHeader) / slot_bytes) : 0;
  int64_t cap = want;
  if (mb > 0 && slot_bytes) cap = std::min<int64_t>(cap, (int64_t)(((size_t)mb << 20) / slot_bytes));
  cap = std::max<int64_t>(cap, 1);
  if (cap <= have) {
    *out = (int)cap;
    return DETLSH_OK;
  }
  size_t freeb = 0, totb = 0;
  DL_CUDA(cudaMemGetInfo(&freeb, &totb));
  size_t budget = mb > 0 ? (size_t)mb << 20 : freeb / 4 + held;
  budget = std::min(budget, (freeb + held) / 10 * 9);
  int64_t s = slot_bytes ? std::min<int64_t>(cap, (int64_t)(budget / slot_bytes)) : cap;
  if (have > 0 && s <= have + have / 4) s = std::min<int64_t>(cap, have);
  *out = (int)std::max<int64_t>(1, s);
  return DETLSH_OK;
}

// Grows a query scratch to hold *slots slots.  The larger block is a new
// allocation that the pool may be unable to assemble from the block it
// replaces: when it fails, the scratch falls back to the slots it held
// before, then to halves of that (the failed allocation's error is cleared),
// so the call runs with fewer queries in flight instead of failing.
int grow_scratch(detlsh_index::QBuf &b, int *slots, size_t slot_bytes, cudaStream_t st,
                 bool *fresh) {
  int64_t held = (slot_bytes && b.bytes > kScratchHeader) ? (int64_t)((b.bytes - kScratchHeader) / slot_bytes) : 0;
  int64_t s = *slots;
  while (true) {
    const int rc = grow(b, kScratchHeader + (size_t)s * slot_bytes, st, fresh);
    if (rc == DETLSH_OK) {
      *slots = (int)s;
      return DETLSH_OK;
    }
    if (rc != DETLSH_ERR_OOM || s <= 1) return rc;
    cudaGetLastError();
    s = (held > 0 && held < s) ? held : s / 2;
    held = 0;
  }
}

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int copy_in(void *dst, const void *src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return DETLSH_OK;
  DL_CUDA(cudaMemcpyAsync(dst, src, bytes,
                          is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  return DETLSH_OK;
}

int copy_out(void *dst, const void *src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return DETLSH_OK;
  DL_CUDA(cudaMemcpyAsync(dst, src, bytes,
                          is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  return DETLSH_OK;
}

// Eq. 1: entries of the K*L projection vectors are N(0,1).  Pair (2u, 2u+1)
// of row t comes from Philox4x32-10 block (u, t, stream 2, 0) keyed by the
// seed, through Box-Muller in FP64, rounded to FP32.
void projection_matrix(int LK, int d, uint64_t seed, float *A) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int t = 0; t < LK; ++t) {
    for (int u = 0; 2 * u < d; ++u) {
      const U4 r = philox4x32_10(U4{(uint32_t)u, (uint32_t)t, STREAM_PROJ, 0u}, k0, k1);
      const double u1 = ((double)r.x + 1.0) * 0x1p-32;
      const double u2 = (double)r.y * 0x1p-32;
      const double rad = std::sqrt(-2.0 * std::log(u1));
      const double th = 6.283185307179586 * u2;
      const float z0 = (float)(rad * std::cos(th)) + 0.0f;
      const float z1 = (float)(rad * std::sin(th)) + 0.0f;
      A[(int64_t)t * d + 2 * u] = z0;
      if (2 * u + 1 < d) A[(int64_t)t * d + 2 * u + 1] = z1;
    }
  }
}

// Pr[chi^2(K) > x] (Lemma 2), closed forms for even and odd K.
double chi2_tail(double x, int K) {
  if (x <= 0.0) return 1.0;
  const double h = 0.5 * x;
  if ((K & 1) == 0) {
    double term = 1.0, sum = 1.0;
    for (int i = 1; i < K / 2; ++i) {
      term *= h / i;
      sum += term;
    }
    return std::exp(-h) * sum;
  }
  double term = 1.0, sum = 0.0;
  for (int i = 1; i <= (K - 1) / 2; ++i) {
    if (i > 1) term *= x / (2 * i - 1);
    sum += term;
  }
  return std::erfc(std::sqrt(h)) + std::exp(-h) * std::sqrt(2.0 * x / 3.141592653589793) * sum;
}

// Eq. 2 with L = -1/ln(alpha1): eps^2 is the upper alpha1 quantile of chi^2(K).
double eps2_of(int K, int L) {
  const double a1 = std::exp(-1.0 / L);
  double lo = 0.0, hi = 1.0;
  while (chi2_tail(hi, K) > a1) hi *= 2.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (chi2_tail(mid, K) > a1) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

// Squared-radius grid of the magic r_min (Sec. V-B1): r_j = c^j.
void level_table(double eps2, double c, float *T) {
  for (int i = 0; i < NLEV; ++i) T[i] = (float)(eps2 * std::pow(c, 2.0 * (double)(i + JMIN)));
  T[NLEV - 1] = INFINITY;
}

// Static encoding scheme (Sec. III-A): the N(0,1) quantiles z/N_r.  Start
// from the Abramowitz-Stegun 26.2.22 rational approximation (error < 3e-3)
// and polish with Newton steps on Phi(x) = erfc(-x/sqrt 2)/2 to full double
// precision; the upper half by symmetry, the median exactly 0.
double normal_quantile(double p) {
  if (p == 0.5) return 0.0;
  if (p > 0.5) return -normal_quantile(1.0 - p);
  const double t = std::sqrt(-2.0 * std::log(p));
  double x = -(t - (2.30753 + 0.27061 * t) / (1.0 + t * (0.99229 + 0.04481 * t)));
  for (int it = 0; it < 100; ++it) {
    const double f = 0.5 * std::erfc(-x / std::sqrt(2.0)) - p;
    const double dens = std::exp(-0.5 * x * x) / 2.5066282746310002;  // sqrt(2 pi)
    const double step = f / dens;
    x -= step;
    if (std::fabs(step) <= 1e-17 * std::fabs(x)) break;
  }
  return x;
}

void static_breakpoints(int LK, int N_r, float *B) {
  for (int t = 0; t < LK; ++t) {
    float *Bt = B + (int64_t)t * (N_r + 1);
    for (int z = 1; z < N_r; ++z) Bt[z] = (float)normal_quantile((double)z / (double)N_r);
    Bt[0] = -INFINITY;
    Bt[N_r] = INFINITY;
  }
}

uint32_t host_fkey(float f) {
  uint32_t b;
  memcpy(&b, &f, sizeof b);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__global__ void k_fill_minmax(uint32_t *mm, int LK, const float *B, int N_r) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < LK) {
    mm[2 * t] = fkey(B[(int64_t)t * (N_r + 1) + 1] + 0.0f);
    mm[2 * t + 1] = fkey(B[(int64_t)t * (N_r + 1) + N_r - 1] + 0.0f);
  }
}

__global__ void k_iota(uint32_t *p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (uint32_t)i;
}

// BF16 copy of the rows, a warp per row, with two FP32 terms per row for the
// certified BF16 scores: ||bf16(x)||^2 (round to nearest, the norm term of
// the tensor-core scores) and an upper bound of ||x - bf16(x)|| (each
// difference is exact, the squares and their sum round up, then a rounded-up
// square root).  Rows with d a multiple of 4 go by 16-byte loads and 8-byte
// stores, two rows at a time.
__device__ __forceinline__ void bf16_row_terms(float x, __nv_bfloat16 b, float &nsq, float &res) {
  const float f = __bfloat162float(b);
  nsq = __fmaf_rn(f, f, nsq);
  const float e = x - f;  // exact: bf16(x) is within a factor 2 of x
  res = __fmaf_ru(e, e, res);
}

__global__ void k_rows_to_bf16(const float *s, __nv_bfloat16 *h, float2 *nrm, int64_t n, int d,
                               uint32_t *inexact) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if ((d & 3) == 0) {
    const int d4 = d >> 2;
    for (int64_t r0 = 2 * w0; r0 < n; r0 += 2 * warps) {
      float acc[2] = {0.0f, 0.0f}, res[2] = {0.0f, 0.0f};
      for (int j = lane; j < d4; j += 32) {
        float4 v[2];
#pragma unroll
        for (int u = 0; u < 2; ++u)
          v[u] = r0 + u < n ? reinterpret_cast<const float4 *>(s + (r0 + u) * d)[j] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          if (r0 + u >= n) continue;
          const __nv_bfloat162 a = __floats2bfloat162_rn(v[u].x, v[u].y);
          const __nv_bfloat162 b = __floats2bfloat162_rn(v[u].z, v[u].w);
          uint2 pk;
          pk.x = *reinterpret_cast<const uint32_t *>(&a);
          pk.y = *reinterpret_cast<const uint32_t *>(&b);
          reinterpret_cast<uint2 *>(h + (r0 + u) * d)[j] = pk;
          bf16_row_terms(v[u].x, a.x, acc[u], res[u]);
          bf16_row_terms(v[u].y, a.y, acc[u], res[u]);
          bf16_row_terms(v[u].z, b.x, acc[u], res[u]);
          bf16_row_terms(v[u].w, b.y, acc[u], res[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        for (int o = 16; o > 0; o >>= 1) {
          acc[u] = __fadd_rn(acc[u], __shfl_xor_sync(0xffffffffu, acc[u], o));
          res[u] = __fadd_ru(res[u], __shfl_xor_sync(0xffffffffu, res[u], o));
        }
        if (lane == 0 && r0 + u < n) {
          nrm[r0 + u] = make_float2(acc[u], __fsqrt_ru(res[u]));
          // one atomic per row would serialise on the flag: set it once
          if (res[u] != 0.0f && *(volatile uint32_t *)inexact == 0u) atomicOr(inexact, 1u);
        }
      }
    }
    return;
  }
  for (int64_t r = w0; r < n; r += warps) {
    float acc = 0.0f, res = 0.0f;
    for (int j = lane; j < d; j += 32) {
      const float x = s[r * d + j];
      const __nv_bfloat16 v = __float2bfloat16_rn(x);
      h[r * d + j] = v;
      bf16_row_terms(x, v, acc, res);
    }
    for (int o = 16; o > 0; o >>= 1) {
      acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
      res = __fadd_ru(res, __shfl_xor_sync(0xffffffffu, res, o));
    }
    if (lane == 0) {
      nrm[r] = make_float2(acc, __fsqrt_ru(res));
      if (res != 0.0f && *(volatile uint32_t *)inexact == 0u) atomicOr(inexact, 1u);
    }
  }
}

__global__ void k_f32_to_bf16(const float *s, __nv_bfloat16 *d, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    d[i] = __float2bfloat16_rn(s[i]);
}

int ensure_events(detlsh_index *ix) {
  for (auto &e : ix->ev)
    if (!e) DL_CUDA(cudaEventCreate(&e));
  return DETLSH_OK;
}

float ev_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.0f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
    cudaGetLastError();
    return -1.0f;
  }
  return ms;
}

int check_err(int *err_dev, cudaStream_t st) {
  int h = 0;
  DL_CUDA(cudaMemcpyAsync(&h, err_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  DL_CUDA(cudaStreamSynchronize(st));
  return h;
}

int validate_build(int64_t n, int32_t d, const detlsh_build_params *p) {
  if (!p) return DETLSH_ERR_INVALID_ARG;
  if (n < 1 || n >= (int64_t)0x7fffffff) return DETLSH_ERR_INVALID_ARG;
  if (d < 1 || d > 65536) return DETLSH_ERR_INVALID_ARG;
  if (p->L < 1 || p->L > 16 || p->K < 1 || p->K > 16 || p->L * p->K > 256)
    return DETLSH_ERR_INVALID_ARG;
  if (p->N_r < 2 || p->N_r > 256 || (p->N_r & (p->N_r - 1))) return DETLSH_ERR_INVALID_ARG;
  if (p->max_size < 1) return DETLSH_ERR_INVALID_ARG;
  if (!(p->sample_frac > 0.0 && p->sample_frac <= 1.0)) return DETLSH_ERR_INVALID_ARG;
  if (p->encoding != DETLSH_ENC_DYNAMIC && p->encoding != DETLSH_ENC_STATIC)
    return DETLSH_ERR_INVALID_ARG;
  if (p->tree_group < 0 || p->tree_group > p->L) return DETLSH_ERR_INVALID_ARG;
  if (p->box_mode != DETLSH_BOX_PREFIX && p->box_mode != DETLSH_BOX_TIGHT)
    return DETLSH_ERR_INVALID_ARG;
  return DETLSH_OK;
}

// Third hull level: hulls of runs of LEAF_BLOCK super-hulls (LEAF_BLOCK^3
// leaves each), so that the range query's pruned scan starts from n/32768
// boxes per tree.  Derived from the super-hulls, so a loaded index rebuilds it.
int build_top_hulls(detlsh_index *ix, cudaStream_t st) {
  const int L = ix->L;
  int64_t tt = 0;
  for (int t = 0; t < L; ++t) {
    ix->tblk_off[t] = tt;
    tt += ceil_div(ix->sblk_off[t + 1] - ix->sblk_off[t], LEAF_BLOCK);
  }
  for (int t = L; t <= 16; ++t) ix->tblk_off[t] = tt;
  DL_TRY(dalloc(ix, &ix->tblk_lo, (size_t)tt * 16, st));
  DL_TRY(dalloc(ix, &ix->tblk_hi, (size_t)tt * 16, st));
  HullSet h;
  h.L = L;
  for (int t = 0; t <= L; ++t) { h.in_off[t] = ix->sblk_off[t]; h.out_off[t] = ix->tblk_off[t]; }
  for (int t = 0; t < L; ++t) h.cnt[t] = ix->sblk_off[t + 1] - ix->sblk_off[t];
  return block_hulls(ix->sblk_lo, ix->sblk_hi, h, ix->tblk_lo, ix->tblk_hi, st);
}

int build_impl(detlsh_index *ix, const float *data, cudaStream_t st, const detlsh_build_params *p) {
  const int64_t n = ix->n;
  const int d = ix->d, L = ix->L, K = ix->K, LK = ix->LK, N_r = ix->N_r;
  TempPool tp(st);
  DL_TRY(ensure_events(ix));
  const long long launches0 = g_launches.load();
  DL_CUDA(cudaEventRecord(ix->ev[0], st));
  // data copy (the index keeps its own FP32 rows for verification)
  DL_TRY(dalloc(ix, &ix->X, (size_t)n * d, st));
  DL_TRY(copy_in(ix->X, data, sizeof(float) * (size_t)n * d, st));
  const float *src = ix->X;
  // projection vectors (Eq. 1)
  std::vector<float> Ah((size_t)LK * d);
  projection_matrix(LK, d, ix->seed, Ah.data());
  DL_TRY(dalloc(ix, &ix->A, (size_t)LK * d, st));
  DL_CUDA(cudaMemcpyAsync(ix->A, Ah.data(), sizeof(float) * Ah.size(), cudaMemcpyHostToDevice, st));
  // status words and the exact-path list
  int *err = nullptr;
  uint32_t *fb_count = nullptr;
  unsigned long long *fb_total = nullptr;
  uint2 *fb_list = nullptr;
  const uint32_t fb_cap = (uint32_t)std::min<int64_t>(std::max<int64_t>(n * LK / 256, 65536), 1 << 24);
  DL_TRY(tp.get(&err, 1));
  DL_TRY(tp.get(&fb_count, 1));
  DL_TRY(tp.get(&fb_total, 1));
  DL_TRY(tp.get(&fb_list, fb_cap));
  DL_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  DL_CUDA(cudaMemsetAsync(fb_total, 0, sizeof(unsigned long long), st));
  ProjArgs pa;
  pa.fb_list = fb_list; pa.fb_count = fb_count; pa.fb_cap = fb_cap;
  pa.fb_total = fb_total; pa.err = err;

  const bool stat = ix->encoding == DETLSH_ENC_STATIC;
  SortTemp srt;  // the sample-column sort
  if (stat) {
    // ---- static scheme: fixed N(0,1) breakpoints, no sample ----
    DL_TRY(dalloc(ix, &ix->sample, 1, st));
    ix->m_sample = 0;
    std::vector<float> Bh((size_t)LK * (N_r + 1));
    static_breakpoints(LK, N_r, Bh.data());
    DL_TRY(dalloc(ix, &ix->B, Bh.size(), st));
    DL_CUDA(cudaMemcpyAsync(ix->B, Bh.data(), sizeof(float) * Bh.size(), cudaMemcpyHostToDevice, st));
    DL_CUDA(cudaEventRecord(ix->ev[1], st));
  } else {
    // ---- sample (Sec. III-A) ----
    DL_TRY(dalloc(ix, &ix->sample, (size_t)n, st));
    uint32_t *blk = nullptr;
    DL_TRY(tp.get(&blk, sample_blocks(n) + 4));
    int64_t m = 0;
    DL_TRY(sample_ids(n, ix->seed, ix->frac, ix->sample, blk, &m, st));
    if (m < 2 * (int64_t)N_r) {
      k_iota<<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 4096), 256, 0, st>>>(ix->sample, n);
      dl_count_launch();
      DL_CUDA(cudaGetLastError());
      m = n;
    }
    ix->m_sample = m;

    // ---- breakpoints: sample projections, sorted per column ----
    float *Ps = nullptr;
    DL_TRY(tp.get(&Ps, (size_t)LK * m));
    ProjArgs ps = pa;
    ps.P = Ps;
    ps.ldP = m;
    DL_TRY(project_rows(src, d, ix->sample, m, d, ix->A, LK, 1, ps, st));
    DL_CUDA(cudaEventRecord(ix->ev[1], st));
    DL_TRY(float_to_keys(Ps, (int64_t)LK * m, st));
    const size_t cnt_cap = (size_t)LK * 256 * sort_tiles(m);
    DL_TRY(tp.get(&srt.counts, cnt_cap));
    srt.count_cap = cnt_cap;
    DL_TRY(tp.get(&srt.keys_alt, (size_t)LK * m));
    DL_TRY(tp.get(&srt.digit_base, (size_t)LK * 256));
    DL_TRY(segmented_sort(reinterpret_cast<uint32_t *>(Ps), nullptr, LK, m, 32, srt, st));
    DL_TRY(dalloc(ix, &ix->B, (size_t)LK * (N_r + 1), st));
    DL_TRY(extract_breakpoints(reinterpret_cast<uint32_t *>(Ps), LK, m, N_r, ix->B, st));
  }
  DL_CUDA(cudaEventRecord(ix->ev[2], st));
  // ---- all projections, encoded (Alg. 1), and column min/max ----
  DL_TRY(dalloc(ix, &ix->codes, (size_t)L * n * CODE_STRIDE, st));
  DL_CUDA(cudaMemsetAsync(ix->codes, 0, (size_t)L * n * CODE_STRIDE, st));
  uint32_t *minmax = nullptr;
  DL_TRY(tp.get(&minmax, (size_t)2 * LK));
  // The column minimum is at most B[1] and the maximum at least B[N_r-1]
  // (both are data values); points beyond them lie in the outer regions,
  // which the encoder always recomputes exactly.
  k_fill_minmax<<<(unsigned)ceil_div(LK, 128), 128, 0, st>>>(minmax, LK, ix->B, N_r);
  dl_count_launch();
  // running bounds of the column extremes (same start as the extremes)
  uint32_t *ubound = nullptr;
  DL_TRY(tp.get(&ubound, (size_t)2 * LK));
  if (stat) {  // fixed infinite ends: no column extreme is tracked
    std::vector<uint32_t> ub((size_t)2 * LK);
    for (int t = 0; t < LK; ++t) { ub[2 * t] = host_fkey(-INFINITY); ub[2 * t + 1] = host_fkey(INFINITY); }
    DL_CUDA(cudaMemcpyAsync(ubound, ub.data(), sizeof(uint32_t) * ub.size(), cudaMemcpyHostToDevice, st));
    DL_CUDA(cudaStreamSynchronize(st));  // ub is a host temporary
  } else {
    DL_CUDA(cudaMemcpyAsync(ubound, minmax, sizeof(uint32_t) * 2 * LK, cudaMemcpyDeviceToDevice, st));
  }
  ProjArgs pe = pa;
  pe.codes = ix->codes; pe.n = n; pe.B = ix->B; pe.N_r = N_r; pe.K = K; pe.minmax = minmax;
  pe.ubound = ubound;
  // uncertain or outer-region coordinates: a few per cent of n*LK
  uint2 *fb_enc = nullptr;
  const uint32_t fb_enc_cap = (uint32_t)std::min<int64_t>(std::max<int64_t>(n * LK / 16, 65536), 1 << 26);
  DL_TRY(tp.get(&fb_enc, fb_enc_cap));
  pe.fb_list = fb_enc;
  pe.fb_cap = fb_enc_cap;
  // a non-finite input (flagged by the exact path) is reported after the
  // trees' single host wait: the kernels in between stay in bounds on any
  // values, and the index is not returned
  DL_TRY(project_rows(src, d, nullptr, n, d, ix->A, LK, 2, pe, st));
  if (!stat) DL_TRY(finish_breakpoint_ends(minmax, LK, N_r, ix->B, st));
  DL_CUDA(cudaEventRecord(ix->ev[3], st));
  if (p->keep_projections) {
    DL_TRY(dalloc(ix, &ix->P, (size_t)n * LK, st));
    ProjArgs pp = pa;
    pp.P = ix->P;
    pp.ldP = LK;
    DL_TRY(project_rows(src, d, nullptr, n, d, ix->A, LK, 0, pp, st));
  }
  uint32_t *inexact = nullptr;  // set when some row differs from its BF16 copy
  DL_TRY(tp.get(&inexact, 1));
  DL_CUDA(cudaMemsetAsync(inexact, 0, sizeof(uint32_t), st));
  if (p->keep_bf16) {
    DL_TRY(dalloc(ix, &ix->Xh, (size_t)n * d, st));
    DL_TRY(dalloc(ix, &ix->Xn, (size_t)n, st));
    k_rows_to_bf16<<<(unsigned)std::min<int64_t>(ceil_div(n, 8), 8192), 256, 0, st>>>(
        src, ix->Xh, ix->Xn, n, d, inexact);
    dl_count_launch();
    DL_CUDA(cudaGetLastError());
  }
  unsigned long long fbt = 0;
  DL_CUDA(cudaMemcpyAsync(&fbt, fb_total, sizeof fbt, cudaMemcpyDeviceToHost, st));
  uint32_t hinexact = 1;
  DL_CUDA(cudaMemcpyAsync(&hinexact, inexact, sizeof hinexact, cudaMemcpyDeviceToHost, st));

  // ---- DE-Trees (Alg. 2) ----
  // Trees are built G at a time (every kernel runs over G * n positions);
  // G is L unless the temporaries would crowd the device or the positions
  // would overflow 32 bits.  Each group writes its leaves to its own
  // worst-case region, so all groups are enqueued back to back and the host
  // waits once.
  DL_TRY(dalloc(ix, &ix->perm, (size_t)L * n, st));
  DL_TRY(dalloc(ix, &ix->leaf_of, (size_t)L * n, st));
  int G = ix->tree_group > 0 ? ix->tree_group : L;
  if (ix->tree_group == 0) {
    size_t freeb = 0, totb = 0;
    DL_CUDA(cudaMemGetInfo(&freeb, &totb));
    const size_t per_tree = (size_t)n * 240;  // group temporaries per tree, bytes
    while (G > 1 && (size_t)G * per_tree > freeb / 2) --G;
  }
  while (G > 1 && (int64_t)G * n + G > (int64_t)UINT32_MAX) --G;
  const int ngroups = (L + G - 1) / G;
  const int64_t N = (int64_t)G * n;
  TreeTemp tt;
  DL_TRY(tp.get(&tt.keys, (size_t)N));
  DL_TRY(tp.get(&tt.vals, (size_t)N));
  DL_TRY(tp.get(&tt.codesA, (size_t)N));
  DL_TRY(tp.get(&tt.codesB, (size_t)N));
  DL_TRY(tp.get(&tt.idsB, (size_t)N));
  DL_TRY(tp.get(&tt.node_begin, (size_t)N + 1));
  DL_TRY(tp.get(&tt.block_counts, sample_blocks(N) + 4));
  DL_TRY(tp.get(&tt.tmp_begin, (size_t)N));
  DL_TRY(tp.get(&tt.tmp_box, (size_t)N * 48));
  DL_TRY(tp.get(&tt.lists, (size_t)N * 4));
  DL_TRY(tp.get(&tt.leaf_start, (size_t)N));
  {
    const size_t cnt_cap = (size_t)G * 256 * sort_tiles(n);
    DL_TRY(tp.get(&tt.sort.counts, cnt_cap));
    tt.sort.count_cap = cnt_cap;
    DL_TRY(tp.get(&tt.sort.keys_alt, (size_t)N));
    DL_TRY(tp.get(&tt.sort.vals_alt, (size_t)N));
    DL_TRY(tp.get(&tt.sort.digit_base, (size_t)G * 256));
  }
  constexpr int SCAL = 32;  // scalars per group: 4 counts + up to 17 tree offsets
  uint32_t *scal = nullptr;
  DL_TRY(tp.get(&scal, (size_t)SCAL * ngroups));
  std::vector<uint32_t *> g_begin(ngroups);
  std::vector<uint8_t *> g_box(ngroups);
  for (int g = 0; g < ngroups; ++g) {
    const int t0 = g * G, Gg = std::min(G, L - t0);
    DL_TRY(tp.get(&g_begin[g], (size_t)Gg * (n + 1)));
    DL_TRY(tp.get(&g_box[g], (size_t)Gg * n * 48));
    TreeBuildArgs a;
    a.n = n; a.G = Gg; a.K = K; a.bbits = ix->bbits; a.M = ix->M; a.box_mode = ix->box_mode;
    a.codes = ix->codes + (size_t)t0 * n * CODE_STRIDE;
    a.perm = ix->perm + (size_t)t0 * n;
    a.leaf_begin = g_begin[g];
    a.leaf_lo = g_box[g];
    a.leaf_hi = a.leaf_lo + (size_t)Gg * n * 16;
    a.leaf_nb = a.leaf_lo + (size_t)Gg * n * 32;
    a.leaf_of = ix->leaf_of; a.L = L; a.t0 = t0;
    a.scalars = scal + SCAL * g;
    DL_TRY(build_trees(a, tt, st));
  }
  std::vector<uint32_t> hs((size_t)SCAL * ngroups);
  DL_CUDA(cudaMemcpyAsync(hs.data(), scal, sizeof(uint32_t) * hs.size(), cudaMemcpyDeviceToHost, st));
  int herr = 0;
  DL_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  DL_CUDA(cudaStreamSynchronize(st));
  if (herr) return herr;
  for (int g = 0; g < ngroups; ++g) {
    const uint32_t *h = hs.data() + SCAL * g;
    if (h[2] != 0) return (int)h[2];
    const int t0 = g * G, Gg = std::min(G, L - t0);
    for (int u = 0; u < Gg; ++u) {
      ix->nleaves[t0 + u] = (int64_t)h[4 + u + 1] - h[4 + u];
      ix->max_leaves = std::max(ix->max_leaves, ix->nleaves[t0 + u]);
    }
    ix->max_leaf = std::max<int64_t>(ix->max_leaf, h[3]);
  }
  int64_t tl = 0;
  for (int t = 0; t < L; ++t) { ix->leaf_off[t] = tl; tl += ix->nleaves[t]; }
  ix->leaf_off[L] = tl;
  DL_TRY(dalloc(ix, &ix->leaf_begin, (size_t)tl + L, st));
  DL_TRY(dalloc(ix, &ix->leaf_lo, (size_t)tl * 16, st));
  DL_TRY(dalloc(ix, &ix->leaf_hi, (size_t)tl * 16, st));
  DL_TRY(dalloc(ix, &ix->leaf_nb, (size_t)tl * 16, st));
  for (int g = 0; g < ngroups; ++g) {  // a group's leaves are contiguous in the final layout
    const int t0 = g * G, Gg = std::min(G, L - t0);
    const int64_t nl = ix->leaf_off[t0 + Gg] - ix->leaf_off[t0], o = ix->leaf_off[t0];
    const uint8_t *bx = g_box[g];
    DL_CUDA(cudaMemcpyAsync(ix->leaf_begin + o + t0, g_begin[g], sizeof(uint32_t) * (nl + Gg),
                            cudaMemcpyDeviceToDevice, st));
    DL_CUDA(cudaMemcpyAsync(ix->leaf_lo + o * 16, bx, (size_t)nl * 16, cudaMemcpyDeviceToDevice, st));
    DL_CUDA(cudaMemcpyAsync(ix->leaf_hi + o * 16, bx + (size_t)Gg * n * 16, (size_t)nl * 16,
                            cudaMemcpyDeviceToDevice, st));
    DL_CUDA(cudaMemcpyAsync(ix->leaf_nb + o * 16, bx + (size_t)Gg * n * 32, (size_t)nl * 16,
                            cudaMemcpyDeviceToDevice, st));
  }
  // hulls of runs of LEAF_BLOCK leaves, the coarse level of the range query
  int64_t tb = 0;
  for (int t = 0; t < L; ++t) { ix->blk_off[t] = tb; tb += ceil_div(ix->nleaves[t], LEAF_BLOCK); }
  ix->blk_off[L] = tb;
  for (int t = L + 1; t <= 16; ++t) ix->blk_off[t] = tb;
  DL_TRY(dalloc(ix, &ix->blk_lo, (size_t)tb * 16, st));
  DL_TRY(dalloc(ix, &ix->blk_hi, (size_t)tb * 16, st));
  {
    HullSet h;
    h.L = L;
    for (int t = 0; t <= L; ++t) { h.in_off[t] = ix->leaf_off[t]; h.out_off[t] = ix->blk_off[t]; }
    for (int t = 0; t < L; ++t) h.cnt[t] = ix->nleaves[t];
    DL_TRY(block_hulls(ix->leaf_lo, ix->leaf_hi, h, ix->blk_lo, ix->blk_hi, st));
  }
  // and hulls of runs of LEAF_BLOCK hulls (LEAF_BLOCK^2 leaves)
  int64_t ts = 0;
  for (int t = 0; t < L; ++t) {
    ix->sblk_off[t] = ts;
    ts += ceil_div(ix->blk_off[t + 1] - ix->blk_off[t], LEAF_BLOCK);
  }
  for (int t = L; t <= 16; ++t) ix->sblk_off[t] = ts;
  DL_TRY(dalloc(ix, &ix->sblk_lo, (size_t)ts * 16, st));
  DL_TRY(dalloc(ix, &ix->sblk_hi, (size_t)ts * 16, st));
  {
    HullSet h;
    h.L = L;
    for (int t = 0; t <= L; ++t) { h.in_off[t] = ix->blk_off[t]; h.out_off[t] = ix->sblk_off[t]; }
    for (int t = 0; t < L; ++t) h.cnt[t] = ix->blk_off[t + 1] - ix->blk_off[t];
    DL_TRY(block_hulls(ix->blk_lo, ix->blk_hi, h, ix->sblk_lo, ix->sblk_hi, st));
  }
  DL_TRY(build_top_hulls(ix, st));
  DL_CUDA(cudaEventRecord(ix->ev[4], st));
  DL_CUDA(cudaStreamSynchronize(st));
  ix->fb_total = (int64_t)fbt;
  ix->bf16_exact = (ix->Xh != nullptr && hinexact == 0) ? 1 : 0;
  ix->eps2 = eps2_of(K, L);
  ix->timings.build_ms = ev_ms(ix->ev[0], ix->ev[4]);
  ix->timings.sample_ms = ev_ms(ix->ev[0], ix->ev[1]);
  ix->timings.breakpoints_ms = ev_ms(ix->ev[1], ix->ev[2]);
  ix->timings.encode_ms = ev_ms(ix->ev[2], ix->ev[3]);
  ix->timings.trees_ms = ev_ms(ix->ev[3], ix->ev[4]);
  ix->timings.build_launches = g_launches.load() - launches0;
  return DETLSH_OK;
}

void free_index(detlsh_index *ix) {
  if (!ix) return;
  cudaDeviceSynchronize();  // no kernel of this index may still be running
  for (void *q : ix->owned) cudaFreeAsync(q, 0);
  for (auto &e : ix->ev)
    if (e) cudaEventDestroy(e);
  for (auto *b : {&ix->qQ, &ix->qQh, &ix->qQp, &ix->qk, &ix->qids, &ix->qdists, &ix->qT,
                  &ix->qstat, &ix->qS, &ix->qfb, &ix->qrc, &ix->qrcs, &ix->aQp, &ix->aQh,
                  &ix->afb, &ix->aT, &ix->astat, &ix->ascratch})
    if (b->p) cudaFreeAsync(b->p, 0);
  if (ix->qscratch.p) {  // keep the larger of this and the cached scratch
    void *drop = ix->qscratch.p;
    if (ix->device >= 0 && ix->device < kPoolDevices) {
      std::lock_guard<std::mutex> g(g_scratch_mu);
      ScratchCache &c = g_scratch[ix->device];
      if (ix->qscratch.bytes >= c.bytes) {
        drop = c.p;
        c.p = ix->qscratch.p;
        c.bytes = ix->qscratch.bytes;
      }
    }
    if (drop) cudaFreeAsync(drop, 0);
  }
  delete ix;
}

QueryIndexView view_of(const detlsh_index *ix) {
  QueryIndexView v;
  v.n = ix->n; v.d = ix->d; v.L = ix->L; v.K = ix->K; v.LK = ix->LK; v.N_r = ix->N_r;
  v.X = ix->X; v.Xh = ix->Xh; v.Xn = ix->Xn; v.P = ix->P; v.B = ix->B; v.perm = ix->perm; v.leaf_begin = ix->leaf_begin;
  v.leaf_lo = ix->leaf_lo; v.leaf_hi = ix->leaf_hi; v.leaf_of = ix->leaf_of;
  v.blk_lo = ix->blk_lo; v.blk_hi = ix->blk_hi;
  for (int t = 0; t <= 16; ++t) v.blk_off[t] = ix->blk_off[t];
  v.sblk_lo = ix->sblk_lo; v.sblk_hi = ix->sblk_hi;
  for (int t = 0; t <= 16; ++t) v.sblk_off[t] = ix->sblk_off[t];
  v.tblk_lo = ix->tblk_lo; v.tblk_hi = ix->tblk_hi;
  for (int t = 0; t <= 16; ++t) v.tblk_off[t] = ix->tblk_off[t];
  for (int t = 0; t <= 16; ++t) v.leaf_off[t] = t <= ix->L ? ix->leaf_off[t] : ix->leaf_off[ix->L];
  v.max_leaves = ix->max_leaves;
  v.max_leaf_size = ix->max_leaf;
  v.bf16_exact = ix->bf16_exact;
  return v;
}

int validate_query(const detlsh_index *ix, int64_t m, int32_t k_max, const detlsh_query_params *qp) {
  if (!ix || !qp || m < 0) return DETLSH_ERR_INVALID_ARG;
  if (k_max < 1 || k_max > 1024 || k_max > ix->n) return DETLSH_ERR_INVALID_ARG;
  if (!(qp->c >= 1.1 && qp->c <= 16.0)) return DETLSH_ERR_INVALID_ARG;
  if (!(qp->beta >= 0.0 && std::isfinite(qp->beta))) return DETLSH_ERR_INVALID_ARG;
  if (qp->precision != DETLSH_PREC_FP32 && qp->precision != DETLSH_PREC_BF16_REFINE)
    return DETLSH_ERR_INVALID_ARG;
  if (qp->precision == DETLSH_PREC_BF16_REFINE &&
      (!ix->Xh || (ix->d % 8) != 0 || qp->rerank_mult < 0))
    return DETLSH_ERR_INVALID_ARG;
  if (qp->rmin_policy != DETLSH_RMIN_MAGIC && qp->rmin_policy != DETLSH_RMIN_FIXED &&
      qp->rmin_policy != DETLSH_RMIN_CONTINUOUS)
    return DETLSH_ERR_INVALID_ARG;
  if (qp->per_tree != 0 && qp->per_tree != 1) return DETLSH_ERR_INVALID_ARG;
  if (qp->per_tree && qp->rmin_policy != DETLSH_RMIN_MAGIC) return DETLSH_ERR_INVALID_ARG;
  // a fixed r_min: c r_min >= 2^-60 keeps the radii of condition 2 exactly
  // representable as three FP32 pieces
  if (qp->rmin_policy == DETLSH_RMIN_FIXED &&
      (!(qp->r_min > 0.0) || !std::isfinite(qp->r_min) || qp->precision != DETLSH_PREC_FP32 ||
       !(qp->c * qp->r_min >= 0x1p-60)))
    return DETLSH_ERR_INVALID_ARG;
  return DETLSH_OK;
}

// Shared body of detlsh_query_ex and detlsh_query_candidates (qmu held).
// Float round-down / round-up of a double.
float f32_down(double x) {
  float f = (float)x;
  if ((double)f > x) f = std::nextafter(f, -INFINITY);
  return f;
}
float f32_up(double x) {
  float f = (float)x;
  if ((double)f < x) f = std::nextafter(f, INFINITY);
  return f;
}

// Query tables (TABLE_FLOATS floats, layout in kernels.h): the squared-radius
// grid of the range queries and, for a fixed r_min, the radii c r_i of
// condition 2 of Alg. 5 (c r_i = c (r_min c^i) in FP64): a rounded-down and
// a rounded-up FP32 copy of (c r_i)^2 for the certified FP32 test, and c r_i
// cut exactly into three FP32 pieces for the exact test near the sphere.  A
// radius of 2^127 or more (beyond FP32) takes every point.
void query_tables(const detlsh_index *ix, const detlsh_query_params *qp, float *Th) {
  float *T = Th, *Tcl = Th + 256, *Tch = Th + 512, *Rp = Th + 768;
  for (int i = 0; i < TABLE_FLOATS; ++i) Th[i] = INFINITY;
  if (qp->rmin_policy == DETLSH_RMIN_FIXED) {
    const double r0 = qp->r_min, c = qp->c;
    for (int i = 0; i < NLEV - 1; ++i) {
      T[i] = (float)(ix->eps2 * r0 * r0 * std::pow(c, 2.0 * (double)i));
      const double cr = c * (r0 * std::pow(c, (double)i));
      if (cr >= 0x1p127) continue;  // every point within: the tables stay +inf
      const double r2 = cr * cr;    // relative error <= 2^-53
      Tcl[i] = f32_down(r2 * (1.0 - 0x1p-52));
      Tch[i] = f32_up(r2 * (1.0 + 0x1p-52));
      double rest = cr;  // cr >= 2^-60 (checked): three pieces are exact
      for (int p = 0; p < 3; ++p) {
        Rp[3 * i + p] = (float)rest;
        rest -= (double)Rp[3 * i + p];
      }
    }
  } else {
    level_table(ix->eps2, qp->c, T);
  }
  T[255] = INFINITY;
}

int query_impl(detlsh_index *ix, const float *queries, int64_t m, const int32_t *kq,
               int32_t k_max, const detlsh_query_params *qp, cudaStream_t st, int64_t *ids,
               float *dists, int64_t S_cap, int64_t *S, int64_t *S_size, int32_t *jstar,
               int32_t *istar) {
  const int d = ix->d, LK = ix->LK;
  DL_TRY(ensure_events(ix));
  const long long launches0 = g_launches.load();
  std::vector<int32_t> kh;
  if (kq) {
    kh.resize((size_t)m);
    if (is_device_ptr(kq)) DL_CUDA(cudaMemcpy(kh.data(), kq, sizeof(int32_t) * m, cudaMemcpyDeviceToHost));
    else memcpy(kh.data(), kq, sizeof(int32_t) * m);
    for (int32_t v : kh)
      if (v < 1 || v > k_max) return DETLSH_ERR_INVALID_ARG;
  }
  DL_TRY(grow(ix->qQ, sizeof(float) * (size_t)m * d, st));
  DL_TRY(grow(ix->qQp, sizeof(float) * (size_t)m * LK, st));
  DL_TRY(grow(ix->qids, sizeof(int64_t) * (size_t)m * k_max, st));
  DL_TRY(grow(ix->qdists, sizeof(float) * (size_t)m * k_max, st));
  DL_TRY(grow(ix->qT, sizeof(float) * TABLE_FLOATS, st));
  DL_TRY(grow(ix->qstat, 256, st));
  float *Q = static_cast<float *>(ix->qQ.p);
  float *Qp = static_cast<float *>(ix->qQp.p);
  int *err = static_cast<int *>(ix->qstat.p);
  uint32_t *fb_count = reinterpret_cast<uint32_t *>(static_cast<char *>(ix->qstat.p) + 16);
  uint32_t *counter = reinterpret_cast<uint32_t *>(static_cast<char *>(ix->qstat.p) + 32);
  DL_CUDA(cudaMemsetAsync(ix->qstat.p, 0, 256, st));
  unsigned long long *stats = reinterpret_cast<unsigned long long *>(static_cast<char *>(ix->qstat.p) + 64);
  DL_CUDA(cudaEventRecord(ix->ev[5], st));
  DL_TRY(copy_in(Q, queries, sizeof(float) * (size_t)m * d, st));
  // exact query projections q'_i = H_i(q) (Alg. 5)
  const uint32_t fb_cap = (uint32_t)std::max<int64_t>(1024, m * LK / 64);
  DL_TRY(grow(ix->qfb, sizeof(uint2) * fb_cap, st));
  ProjArgs pa;
  pa.P = Qp; pa.ldP = LK; pa.fb_count = fb_count; pa.fb_cap = fb_cap; pa.err = err;
  pa.fb_list = static_cast<uint2 *>(ix->qfb.p);
  DL_TRY(project_rows(Q, d, nullptr, m, d, ix->A, LK, 0, pa, st));
  const __nv_bfloat16 *Qh = nullptr;
  if (qp->precision == DETLSH_PREC_BF16_REFINE) {
    DL_TRY(grow(ix->qQh, sizeof(__nv_bfloat16) * (size_t)m * d, st));
    DL_TRY(dl::f32_to_bf16(Q, static_cast<__nv_bfloat16 *>(ix->qQh.p), m * (int64_t)d, st));
    Qh = static_cast<const __nv_bfloat16 *>(ix->qQh.p);
  }
  // radius grid (and for a fixed r_min the condition-2 radii)
  const bool fixed = qp->rmin_policy == DETLSH_RMIN_FIXED;
  float Th[TABLE_FLOATS];
  query_tables(ix, qp, Th);
  DL_CUDA(cudaMemcpyAsync(ix->qT.p, Th, sizeof Th, cudaMemcpyHostToDevice, st));
  int32_t *kd = nullptr;
  if (kq) {
    DL_TRY(grow(ix->qk, sizeof(int32_t) * (size_t)m, st));
    kd = static_cast<int32_t *>(ix->qk.p);
    DL_CUDA(cudaMemcpyAsync(kd, kh.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
  }
  const double tb = std::ceil(qp->beta * (double)ix->n);
  const int64_t tau_base = tb > (double)ix->n ? ix->n + 1 : (int64_t)tb;
  int64_t cap = (tau_base + k_max > ix->n || qp->per_tree)
                    ? ix->n
                    : std::min<int64_t>(ix->n, tau_base + k_max + ix->max_leaf);
  QueryIndexView v = view_of(ix);
  QueryArgs qa{};
  qa.Q = Q; qa.Qh = Qh; qa.Qp = Qp; qa.m = m; qa.kq = kd; qa.k_max = k_max;
  qa.tau_base = tau_base; qa.T = static_cast<const float *>(ix->qT.p);
  qa.Tc = static_cast<const float *>(ix->qT.p) + 256;
  qa.policy = qp->rmin_policy;
  // level estimate log2(T) -> index: grid c^j from j = -127, or r_min c^i from i = 0
  qa.lg_eps2 = fixed ? (float)(std::log2(ix->eps2 * qp->r_min * qp->r_min) +
                               254.0 * std::log2(qp->c))
                     : (float)std::log2(ix->eps2);
  qa.inv_2lg_c = (float)(1.0 / (2.0 * std::log2(qp->c)));
  qa.precision = qp->precision; qa.rerank_mult = qp->rerank_mult;
  qa.ctas_per_sm = ix->tuning.query_ctas_per_sm;
  qa.expand_runs = ix->tuning.expand_runs;
  qa.visit_chunk = ix->tuning.visit_chunk;
  qa.top_min = ix->tuning.top_hull_min;
  qa.hash_kb = ix->tuning.hash_kb;
  qa.per_tree = qp->per_tree;
  qa.ids = static_cast<int64_t *>(ix->qids.p);
  qa.dists = static_cast<float *>(ix->qdists.p);
  if (S) {
    DL_TRY(grow(ix->qS, sizeof(int64_t) * (size_t)m * S_cap + 3 * 8 * (size_t)m, st));
    qa.S_out = static_cast<int64_t *>(ix->qS.p);
    qa.S_cap = S_cap;
    qa.S_size = qa.S_out + (size_t)m * S_cap;
    qa.jstar = reinterpret_cast<int32_t *>(qa.S_size + m);
    qa.istar = qa.jstar + m;
  }
  qa.cand_cap = cap;
  query_slot_offsets(v, cap, qa.off);
  qa.slot_bytes = qa.off[SLOT_ARRAYS];  // total bytes of one slot
  int slots = query_slots(v);
  slots = (int)std::min<int64_t>(slots, std::max<int64_t>(m, 1));
  // keep the scratch within its budget (a quarter of the free memory by default)
  DL_TRY(slots_within_budget(ix, slots, (size_t)qa.slot_bytes, ix->qscratch.bytes, &slots));
  const size_t need_bytes = kScratchHeader + (size_t)slots * qa.slot_bytes;
  if (!ix->qscratch.p && ix->device >= 0 && ix->device < kPoolDevices) {
    std::lock_guard<std::mutex> g(g_scratch_mu);
    ScratchCache &c = g_scratch[ix->device];
    if (c.p && c.bytes >= need_bytes) {  // adopt a freed index's slots
      ix->qscratch.p = c.p;
      ix->qscratch.bytes = c.bytes;
      c = ScratchCache{};
    }
  }
  bool fresh = false;
  DL_TRY(grow_scratch(ix->qscratch, &slots, (size_t)qa.slot_bytes, st, &fresh));
  // new scratch: zero tags and epoch counter (epochs then start at 1)
  if (fresh) DL_CUDA(cudaMemsetAsync(ix->qscratch.p, 0, ix->qscratch.bytes, st));
  qa.epoch_counter = static_cast<unsigned long long *>(ix->qscratch.p);
  qa.scratch = static_cast<uint8_t *>(ix->qscratch.p) + kScratchHeader;
  qa.nslots = slots;
  qa.work_counter = counter;
  qa.err = err;
  qa.stats = stats;
  // No host wait between the projections and the query kernel: a status set
  // by the projections (NaN/Inf in a query) makes the kernel return at once,
  // and one read of the status block after it reports either.
  DL_CUDA(cudaEventRecord(ix->ev[6], st));
  DL_TRY(run_queries(v, qa, st));
  DL_CUDA(cudaEventRecord(ix->ev[7], st));
  unsigned long long hblk[32];  // the 256-byte status block: err at 0, stats from byte 64
  DL_CUDA(cudaMemcpyAsync(hblk, ix->qstat.p, sizeof hblk, cudaMemcpyDeviceToHost, st));
  DL_CUDA(cudaStreamSynchronize(st));
  int e = 0;
  memcpy(&e, hblk, sizeof e);
  if (e) return e;
  const unsigned long long *hs = hblk + 8;
  ix->timings.query_project_ms = ev_ms(ix->ev[5], ix->ev[6]);
  ix->timings.query_kernel_ms = ev_ms(ix->ev[6], ix->ev[7]);
  ix->timings.query_ms = ev_ms(ix->ev[5], ix->ev[7]);
  ix->timings.query_launches = g_launches.load() - launches0;
  ix->timings.query_count = m;
  ix->timings.query_candidates = (int64_t)hs[0];
  ix->timings.query_leaves = (int64_t)hs[1];
  ix->timings.query_blocks = (int64_t)hs[2];
  ix->timings.query_points_visited = (int64_t)hs[3];
  ix->timings.query_reranked = (int64_t)hs[4];
  if (ids) DL_TRY(copy_out(ids, qa.ids, sizeof(int64_t) * (size_t)m * k_max, st));
  if (dists) DL_TRY(copy_out(dists, qa.dists, sizeof(float) * (size_t)m * k_max, st));
  if (S) {
    DL_CUDA(cudaMemcpyAsync(S, qa.S_out, sizeof(int64_t) * (size_t)m * S_cap, cudaMemcpyDeviceToHost, st));
    DL_CUDA(cudaMemcpyAsync(S_size, qa.S_size, sizeof(int64_t) * (size_t)m, cudaMemcpyDeviceToHost, st));
    DL_CUDA(cudaMemcpyAsync(jstar, qa.jstar, sizeof(int32_t) * (size_t)m, cudaMemcpyDeviceToHost, st));
    DL_CUDA(cudaMemcpyAsync(istar, qa.istar, sizeof(int32_t) * (size_t)m, cudaMemcpyDeviceToHost, st));
  }
  DL_CUDA(cudaStreamSynchronize(st));
  return DETLSH_OK;
}

// ---- index files ------------------------------------------------------------
// A file holds everything the queries and the accessors read, so a process can
// serve an index without rebuilding it: a fixed header (magic, format version,
// byte-order mark, build parameters, eps^2, per-tree leaf counts and offsets),
// then the arrays in a fixed order, each behind its tag and byte count, then a
// 64-bit checksum of all of it.  Arrays are written in the host's byte order;
// the byte-order mark rejects a file from a machine of the other order.
constexpr char kFileMagic[8] = {'D', 'E', 'T', 'L', 'S', 'H', 'I', 'X'};
constexpr uint32_t kFileVersion = 1;
constexpr uint32_t kByteOrderMark = 0x01020304u;
constexpr size_t kFileChunk = (size_t)64 << 20;  // staging chunk (a multiple of 8)

struct FileHeader {
  char magic[8];
  uint32_t version, bom, header_bytes, nsections;
  int64_t n;
  int32_t d, L, K, N_r, bbits, M, box_mode, encoding, tree_group, has_bf16, has_proj, bf16_exact;
  uint64_t seed;
  double frac, eps2;
  int64_t m_sample, max_leaf, max_leaves, fb_total;
  int64_t nleaves[16], leaf_off[17], blk_off[17], sblk_off[17];
};
static_assert(sizeof(FileHeader) == 672, "the header size include/detlsh.h documents");

struct SectionHead {
  uint32_t tag, reserved;
  uint64_t bytes;
};

// Order-dependent 64-bit checksum over 8-byte words (a multiply-rotate mix);
// a block's last partial word is zero-padded.  Callers feed blocks whose
// lengths are multiples of 8 except the last block of an array.
struct Checksum {
  uint64_t h = 0x9e3779b97f4a7c15ull;
  void word(uint64_t w) {
    h ^= w * 0xff51afd7ed558ccdull;
    h = (h << 29) | (h >> 35);
    h *= 0xc4ceb9fe1a85ec53ull;
  }
  void bytes(const void *p, size_t nb) {
    const uint8_t *b = static_cast<const uint8_t *>(p);
    size_t i = 0;
    for (; i + 8 <= nb; i += 8) {
      uint64_t w;
      memcpy(&w, b + i, 8);
      word(w);
    }
    if (i < nb) {
      uint64_t w = 0;
      memcpy(&w, b + i, nb - i);
      word(w);
    }
  }
};

struct Section {
  uint32_t tag;
  void *dev;
  uint64_t bytes;
};

// The arrays of an index file, in file order.  Sizes follow from the header
// alone, so the loader knows every section's length before reading it.
std::vector<Section> file_sections(const detlsh_index *ix) {
  const int64_t n = ix->n, L = ix->L, LK = ix->LK, d = ix->d;
  const int64_t tl = ix->leaf_off[ix->L], tb = ix->blk_off[ix->L], ts = ix->sblk_off[ix->L];
  std::vector<Section> s = {
      {1, ix->X, (uint64_t)(n * d * 4)},
      {2, ix->A, (uint64_t)(LK * d * 4)},
      {3, ix->B, (uint64_t)(LK * (ix->N_r + 1) * 4)},
      {4, ix->sample, (uint64_t)(ix->m_sample * 4)},
      {5, ix->codes, (uint64_t)(L * n * CODE_STRIDE)},
      {6, ix->perm, (uint64_t)(L * n * 4)},
      {7, ix->leaf_of, (uint64_t)(L * n * 4)},
      {8, ix->leaf_begin, (uint64_t)((tl + L) * 4)},
      {9, ix->leaf_lo, (uint64_t)(tl * 16)},
      {10, ix->leaf_hi, (uint64_t)(tl * 16)},
      {11, ix->leaf_nb, (uint64_t)(tl * 16)},
      {12, ix->blk_lo, (uint64_t)(tb * 16)},
      {13, ix->blk_hi, (uint64_t)(tb * 16)},
      {14, ix->sblk_lo, (uint64_t)(ts * 16)},
      {15, ix->sblk_hi, (uint64_t)(ts * 16)}};
  if (ix->Xh) {
    s.push_back({16, ix->Xh, (uint64_t)(n * d * 2)});
    s.push_back({17, ix->Xn, (uint64_t)(n * 8)});
  }
  if (ix->P) s.push_back({18, ix->P, (uint64_t)(n * LK * 4)});
  return s;
}

// Pinned staging buffer for the host side of the copies.
struct Staging {
  void *p = nullptr;
  ~Staging() {
    if (p) cudaFreeHost(p);
  }
};

struct File {
  FILE *f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

// Header checks that need no device: the format, and offsets consistent with
// the leaf counts (the loader trusts nothing else it has not checked).
int check_header(const FileHeader &h) {
  if (memcmp(h.magic, kFileMagic, 8) != 0 || h.version != kFileVersion ||
      h.bom != kByteOrderMark || h.header_bytes != sizeof(FileHeader))
    return DETLSH_ERR_FORMAT;
  detlsh_build_params p;
  detlsh_default_build_params(&p);
  p.L = h.L; p.K = h.K; p.N_r = h.N_r; p.max_size = h.M; p.sample_frac = h.frac;
  p.box_mode = h.box_mode; p.encoding = h.encoding; p.tree_group = h.tree_group;
  if (validate_build(h.n, h.d, &p) != DETLSH_OK) return DETLSH_ERR_FORMAT;
  if ((1 << h.bbits) != h.N_r) return DETLSH_ERR_FORMAT;
  if (h.has_bf16 != 0 && h.has_bf16 != 1) return DETLSH_ERR_FORMAT;
  if (h.has_proj != 0 && h.has_proj != 1) return DETLSH_ERR_FORMAT;
  if (h.bf16_exact != 0 && h.bf16_exact != h.has_bf16) return DETLSH_ERR_FORMAT;
  if (h.m_sample < 0 || h.m_sample > h.n || (h.encoding == DETLSH_ENC_STATIC && h.m_sample != 0))
    return DETLSH_ERR_FORMAT;
  if (!(h.eps2 > 0.0) || !std::isfinite(h.eps2)) return DETLSH_ERR_FORMAT;
  int64_t tl = 0, tb = 0, ts = 0, mx = 0;
  for (int t = 0; t < 16; ++t) {
    const int64_t nl = t < h.L ? h.nleaves[t] : 0;
    if (nl < 0 || nl > h.n || (t < h.L && nl < 1)) return DETLSH_ERR_FORMAT;
    if (h.leaf_off[t] != tl || h.blk_off[t] != tb || h.sblk_off[t] != ts) return DETLSH_ERR_FORMAT;
    const int64_t nb = ceil_div(nl, LEAF_BLOCK);
    tl += nl;
    tb += nb;
    ts += ceil_div(nb, LEAF_BLOCK);
    mx = std::max(mx, nl);
  }
  if (h.leaf_off[16] != tl || h.blk_off[16] != tb || h.sblk_off[16] != ts) return DETLSH_ERR_FORMAT;
  if (h.max_leaves != mx || h.max_leaf < 1 || h.max_leaf > h.n) return DETLSH_ERR_FORMAT;
  return DETLSH_OK;
}

int save_impl(const detlsh_index *ix, const char *path, cudaStream_t st) {
  FileHeader h;
  memset(&h, 0, sizeof h);
  memcpy(h.magic, kFileMagic, 8);
  h.version = kFileVersion;
  h.bom = kByteOrderMark;
  h.header_bytes = sizeof(FileHeader);
  const std::vector<Section> secs = file_sections(ix);
  h.nsections = (uint32_t)secs.size();
  h.n = ix->n; h.d = ix->d; h.L = ix->L; h.K = ix->K; h.N_r = ix->N_r; h.bbits = ix->bbits;
  h.M = ix->M; h.box_mode = ix->box_mode; h.encoding = ix->encoding; h.tree_group = ix->tree_group;
  h.has_bf16 = ix->Xh != nullptr; h.has_proj = ix->P != nullptr; h.bf16_exact = ix->bf16_exact;
  h.seed = ix->seed; h.frac = ix->frac; h.eps2 = ix->eps2;
  h.m_sample = ix->m_sample; h.max_leaf = ix->max_leaf; h.max_leaves = ix->max_leaves;
  h.fb_total = ix->fb_total;
  for (int t = 0; t < 16; ++t) h.nleaves[t] = ix->nleaves[t];
  for (int t = 0; t <= 16; ++t) {
    h.leaf_off[t] = ix->leaf_off[std::min(t, ix->L)];
    h.blk_off[t] = ix->blk_off[t];
    h.sblk_off[t] = ix->sblk_off[t];
  }
  // written to path.tmp and renamed at the end, so a failed save leaves no
  // partial file under the name
  const std::string tmp = std::string(path) + ".tmp";
  File f;
  f.f = fopen(tmp.c_str(), "wb");
  if (!f.f) return DETLSH_ERR_IO;
  Checksum cs;
  bool ok = fwrite(&h, sizeof h, 1, f.f) == 1;
  cs.bytes(&h, sizeof h);
  Staging buf;
  DL_CUDA(cudaMallocHost(&buf.p, kFileChunk));
  for (const Section &s : secs) {
    if (!ok) break;
    const SectionHead sh{s.tag, 0u, s.bytes};
    ok = fwrite(&sh, sizeof sh, 1, f.f) == 1;
    cs.bytes(&sh, sizeof sh);
    for (uint64_t o = 0; ok && o < s.bytes; o += kFileChunk) {
      const size_t nb = (size_t)std::min<uint64_t>(kFileChunk, s.bytes - o);
      DL_CUDA(cudaMemcpyAsync(buf.p, static_cast<const char *>(s.dev) + o, nb,
                              cudaMemcpyDeviceToHost, st));
      DL_CUDA(cudaStreamSynchronize(st));
      ok = fwrite(buf.p, 1, nb, f.f) == nb;
      cs.bytes(buf.p, nb);
    }
  }
  if (ok) ok = fwrite(&cs.h, sizeof cs.h, 1, f.f) == 1;
  if (fclose(f.f) != 0) ok = false;
  f.f = nullptr;
  if (!ok || rename(tmp.c_str(), path) != 0) {
    remove(tmp.c_str());
    return DETLSH_ERR_IO;
  }
  return DETLSH_OK;
}

int load_impl(const char *path, cudaStream_t st, detlsh_index **out) {
  File f;
  f.f = fopen(path, "rb");
  if (!f.f) return DETLSH_ERR_IO;
  FileHeader h;
  if (fread(&h, sizeof h, 1, f.f) != 1) return DETLSH_ERR_FORMAT;
  DL_TRY(check_header(h));
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return DETLSH_ERR_NO_DEVICE;
  }
  detlsh_index *ix = new (std::nothrow) detlsh_index();
  if (!ix) return DETLSH_ERR_OOM;
  struct Guard {  // frees the index unless it is handed out
    detlsh_index *ix;
    cudaStream_t st;
    ~Guard() {
      if (ix) {
        cudaStreamSynchronize(st);
        free_index(ix);
      }
    }
  } guard{ix, st};
  cudaGetDevice(&ix->device);
  ix->n = h.n; ix->d = h.d; ix->L = h.L; ix->K = h.K; ix->LK = h.L * h.K; ix->N_r = h.N_r;
  ix->bbits = h.bbits; ix->M = h.M; ix->box_mode = h.box_mode; ix->encoding = h.encoding;
  ix->tree_group = h.tree_group; ix->seed = h.seed; ix->frac = h.frac; ix->eps2 = h.eps2;
  ix->m_sample = h.m_sample; ix->max_leaf = h.max_leaf; ix->max_leaves = h.max_leaves;
  ix->fb_total = h.fb_total;
  ix->bf16_exact = h.bf16_exact;
  for (int t = 0; t < 16; ++t) ix->nleaves[t] = h.nleaves[t];
  for (int t = 0; t <= 16; ++t) {
    ix->leaf_off[t] = h.leaf_off[t];
    ix->blk_off[t] = h.blk_off[t];
    ix->sblk_off[t] = h.sblk_off[t];
  }
  const int64_t n = ix->n, d = ix->d, L = ix->L, LK = ix->LK;
  const int64_t tl = ix->leaf_off[L], tb = ix->blk_off[L], ts = ix->sblk_off[L];
  DL_TRY(dalloc(ix, &ix->X, (size_t)(n * d), st));
  DL_TRY(dalloc(ix, &ix->A, (size_t)(LK * d), st));
  DL_TRY(dalloc(ix, &ix->B, (size_t)(LK * (ix->N_r + 1)), st));
  DL_TRY(dalloc(ix, &ix->sample, (size_t)std::max<int64_t>(ix->m_sample, 1), st));
  DL_TRY(dalloc(ix, &ix->codes, (size_t)(L * n * CODE_STRIDE), st));
  DL_TRY(dalloc(ix, &ix->perm, (size_t)(L * n), st));
  DL_TRY(dalloc(ix, &ix->leaf_of, (size_t)(L * n), st));
  DL_TRY(dalloc(ix, &ix->leaf_begin, (size_t)(tl + L), st));
  DL_TRY(dalloc(ix, &ix->leaf_lo, (size_t)(tl * 16), st));
  DL_TRY(dalloc(ix, &ix->leaf_hi, (size_t)(tl * 16), st));
  DL_TRY(dalloc(ix, &ix->leaf_nb, (size_t)(tl * 16), st));
  DL_TRY(dalloc(ix, &ix->blk_lo, (size_t)(tb * 16), st));
  DL_TRY(dalloc(ix, &ix->blk_hi, (size_t)(tb * 16), st));
  DL_TRY(dalloc(ix, &ix->sblk_lo, (size_t)(ts * 16), st));
  DL_TRY(dalloc(ix, &ix->sblk_hi, (size_t)(ts * 16), st));
  if (h.has_bf16) {
    DL_TRY(dalloc(ix, &ix->Xh, (size_t)(n * d), st));
    DL_TRY(dalloc(ix, &ix->Xn, (size_t)n, st));
  }
  if (h.has_proj) DL_TRY(dalloc(ix, &ix->P, (size_t)(n * LK), st));
  const std::vector<Section> secs = file_sections(ix);
  if (h.nsections != secs.size()) return DETLSH_ERR_FORMAT;
  Checksum cs;
  cs.bytes(&h, sizeof h);
  Staging buf;
  DL_CUDA(cudaMallocHost(&buf.p, kFileChunk));
  for (const Section &s : secs) {
    SectionHead sh;
    if (fread(&sh, sizeof sh, 1, f.f) != 1) return DETLSH_ERR_FORMAT;
    if (sh.tag != s.tag || sh.reserved != 0 || sh.bytes != s.bytes) return DETLSH_ERR_FORMAT;
    cs.bytes(&sh, sizeof sh);
    for (uint64_t o = 0; o < s.bytes; o += kFileChunk) {
      const size_t nb = (size_t)std::min<uint64_t>(kFileChunk, s.bytes - o);
      DL_CUDA(cudaStreamSynchronize(st));  // the previous chunk has left the buffer
      if (fread(buf.p, 1, nb, f.f) != nb) return DETLSH_ERR_FORMAT;
      cs.bytes(buf.p, nb);
      DL_CUDA(cudaMemcpyAsync(static_cast<char *>(s.dev) + o, buf.p, nb, cudaMemcpyHostToDevice, st));
    }
  }
  uint64_t want = 0;
  if (fread(&want, sizeof want, 1, f.f) != 1 || want != cs.h) return DETLSH_ERR_FORMAT;
  if (fgetc(f.f) != EOF) return DETLSH_ERR_FORMAT;  // trailing bytes
  DL_TRY(build_top_hulls(ix, st));
  DL_CUDA(cudaStreamSynchronize(st));
  DL_TRY(ensure_events(ix));
  guard.ix = nullptr;
  *out = ix;
  return DETLSH_OK;
}

// ---- tuning -----------------------------------------------------------------
int check_tuning(const detlsh_tuning *t) {
  if (!t) return DETLSH_ERR_INVALID_ARG;
  if (t->query_ctas_per_sm < 0 || t->query_ctas_per_sm > 5) return DETLSH_ERR_INVALID_ARG;
  if (t->expand_runs < 1 || t->expand_runs > 8) return DETLSH_ERR_INVALID_ARG;
  if (t->visit_chunk < 64 || t->visit_chunk > 512 || (t->visit_chunk & 63)) return DETLSH_ERR_INVALID_ARG;
  if (t->top_hull_min < 1) return DETLSH_ERR_INVALID_ARG;
  if (t->hash_kb < 0 || t->hash_kb > 160) return DETLSH_ERR_INVALID_ARG;
  if (t->query_scratch_mb < 0) return DETLSH_ERR_INVALID_ARG;
  return DETLSH_OK;
}

// The cache key of a tuning: the device's name and the index and query shape
// it was measured on (d, L, K, N_r, n and beta*n + k to the nearest power of
// two, k, precision, r_min policy).
std::string tuning_key(const detlsh_index *ix, int32_t k, const detlsh_query_params *qp) {
  cudaDeviceProp prop;
  std::string name = "device";
  if (cudaGetDeviceProperties(&prop, ix->device) == cudaSuccess) name = prop.name;
  else cudaGetLastError();
  for (char &ch : name)
    if (ch == ' ' || ch == '\t' || ch == '|') ch = '_';
  const double tau = std::ceil(qp->beta * (double)ix->n) + k;
  char buf[512];
  snprintf(buf, sizeof buf, "%s|d%d|L%d|K%d|Nr%d|n2^%d|tau2^%d|k%d|p%d|r%d|v2", name.c_str(), ix->d, ix->L,
           ix->K, ix->N_r, (int)std::lround(std::log2((double)ix->n)),
           (int)std::lround(std::log2(std::max(tau, 1.0))), k, qp->precision, qp->rmin_policy);
  return buf;
}

// One text line per key: "<key> <ctas_per_sm> <expand_runs> <visit_chunk> <hash_kb> <ms>"
// (the key ends in "|v2", so lines of the older four-number format never match).
bool tuning_lookup(const char *path, const std::string &key, detlsh_tuning *t) {
  const int32_t ix_top_min = t->top_hull_min;  // not part of a cache line
  const int32_t ix_scratch = t->query_scratch_mb;  // nor is this
  FILE *f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    char k[600];
    detlsh_tuning c{0, 4, 512, ix_top_min, 0, ix_scratch};
    double ms = 0.0;
    if (sscanf(line, "%599s %d %d %d %d %lf", k, &c.query_ctas_per_sm, &c.expand_runs,
               &c.visit_chunk, &c.hash_kb, &ms) == 6 &&
        key == k && check_tuning(&c) == DETLSH_OK) {
      *t = c;  // the last matching line wins
      found = true;
    }
  }
  fclose(f);
  return found;
}

int autotune_impl(detlsh_index *ix, const float *queries, int64_t m, int32_t k,
                  const detlsh_query_params *qp, const char *cache_path, cudaStream_t st,
                  detlsh_tuning *out, int32_t *from_cache) {
  DL_TRY(validate_query(ix, m, k, qp));
  if (m < 1) return DETLSH_ERR_INVALID_ARG;
  const std::string key = tuning_key(ix, k, qp);
  detlsh_tuning best = ix->tuning;
  if (from_cache) *from_cache = 0;
  if (cache_path && tuning_lookup(cache_path, key, &best)) {
    ix->tuning = best;
    if (out) *out = best;
    if (from_cache) *from_cache = 1;
    return DETLSH_OK;
  }
  // Coordinate descent from the hand-picked defaults: each knob in turn
  // takes the value with the smallest query-kernel time (CUDA events, the
  // better of two runs after a warm-up run) on the sample, the others fixed.
  auto measure = [&](const detlsh_tuning &t, float *ms) -> int {
    ix->tuning = t;
    float b = INFINITY;
    for (int rep = 0; rep < 3; ++rep) {
      DL_TRY(query_impl(ix, queries, m, nullptr, k, qp, st, nullptr, nullptr, 0, nullptr, nullptr,
                        nullptr, nullptr));
      if (rep > 0) b = std::min(b, ix->timings.query_kernel_ms);
    }
    *ms = b;
    return DETLSH_OK;
  };
  detlsh_tuning cur{0, 4, 512, ix->tuning.top_hull_min, 0, ix->tuning.query_scratch_mb};
  float cur_ms = 0.0f;
  DL_TRY(measure(cur, &cur_ms));
  const int ctas[] = {3, 4, 0};
  const int runs[] = {2, 3, 4, 6, 8};
  const int chunks[] = {128, 256, 512};
  const int hashes[] = {0, 20, 40, 80};  // hash regions for 5 / 4 / 3 / 2 CTAs per SM
  for (int knob = 0; knob < 4; ++knob) {
    const int *vals = knob == 0 ? ctas : knob == 1 ? runs : knob == 2 ? chunks : hashes;
    const int nv = knob == 0 ? 3 : knob == 1 ? 5 : knob == 2 ? 3 : 4;
    for (int i = 0; i < nv; ++i) {
      detlsh_tuning t = cur;
      int &slot = knob == 0   ? t.query_ctas_per_sm
                  : knob == 1 ? t.expand_runs
                  : knob == 2 ? t.visit_chunk
                              : t.hash_kb;
      if (slot == vals[i]) continue;
      slot = vals[i];
      float ms = 0.0f;
      DL_TRY(measure(t, &ms));
      if (ms < cur_ms) { cur = t; cur_ms = ms; }
    }
  }
  ix->tuning = cur;
  if (out) *out = cur;
  if (cache_path) {
    FILE *f = fopen(cache_path, "a");
    if (!f) return DETLSH_ERR_IO;
    fprintf(f, "%s %d %d %d %d %.4f\n", key.c_str(), cur.query_ctas_per_sm, cur.expand_runs,
            cur.visit_chunk, cur.hash_kb, cur_ms);
    if (fclose(f) != 0) return DETLSH_ERR_IO;
  }
  return DETLSH_OK;
}

}  // namespace

namespace dl {
// Read-only view of an index for entry points in other translation units.
int index_query_view(const detlsh_index *ix, QueryIndexView *v, const float **A, int *has_bf16) {
  if (!ix) return DETLSH_ERR_INVALID_ARG;
  *v = view_of(ix);
  *A = ix->A;
  *has_bf16 = ix->Xh != nullptr;
  return DETLSH_OK;
}

// Device that holds the index's memory (-1 for a null index).
int index_device(const detlsh_index *ix) { return ix ? ix->device : -1; }

// Argument checks shared with detlsh_query_ex, and the radius grid.
int check_query_args(const detlsh_index *ix, int64_t m, int32_t k, const detlsh_query_params *qp) {
  return validate_query(ix, m, k, qp);
}

void radius_grid(const detlsh_index *ix, double c, float T[256]) {
  level_table(ix->eps2, c, T);
  T[255] = INFINITY;
}

int f32_to_bf16(const float *src, __nv_bfloat16 *dst, int64_t count, cudaStream_t st) {
  if (count <= 0) return DETLSH_OK;
  k_f32_to_bf16<<<(unsigned)std::min<int64_t>(ceil_div(count, 256), 8192), 256, 0, st>>>(src, dst, count);
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  return DETLSH_OK;
}
}  // namespace dl

// ===========================================================================
// C-ABI
// ===========================================================================
extern "C" {

int detlsh_default_build_params(detlsh_build_params *p) {
  if (!p) return DETLSH_ERR_INVALID_ARG;
  p->L = 4;
  p->K = 16;
  p->N_r = 256;
  p->max_size = 64;
  p->seed = 0;
  p->sample_frac = 0.1;
  p->box_mode = DETLSH_BOX_PREFIX;
  p->keep_bf16 = 1;
  p->keep_projections = 0;
  p->encoding = DETLSH_ENC_DYNAMIC;
  p->tree_group = 0;
  return DETLSH_OK;
}

int detlsh_default_query_params(detlsh_query_params *p) {
  if (!p) return DETLSH_ERR_INVALID_ARG;
  p->beta = 0.1;
  p->c = 1.5;
  p->precision = DETLSH_PREC_FP32;
  p->rerank_mult = 0;
  p->rmin_policy = DETLSH_RMIN_MAGIC;
  p->r_min = 1.0;
  p->per_tree = 0;
  return DETLSH_OK;
}

const char *detlsh_status_string(int s) {
  switch (s) {
    case DETLSH_OK: return "ok";
    case DETLSH_ERR_INVALID_ARG: return "invalid argument";
    case DETLSH_ERR_NONFINITE_INPUT: return "non-finite input or projection overflow";
    case DETLSH_ERR_OOM: return "out of memory";
    case DETLSH_ERR_CUDA: return g_last_cuda[0] ? g_last_cuda : "CUDA error";
    case DETLSH_ERR_CAPACITY: return "internal work list capacity exceeded";
    case DETLSH_ERR_NO_DEVICE: return "no CUDA device";
    case DETLSH_ERR_SCRATCH_LIMIT:
      return "request does not fit the fixed 32 MiB scratch of detlsh_query_noalloc";
    case DETLSH_ERR_TIMEOUT: return "a device-side wait ran past its limit";
    case DETLSH_ERR_IO: return "index file could not be opened, read or written";
    case DETLSH_ERR_FORMAT: return "not a valid index file (format, version, size or checksum)";
  }
  return "unknown status";
}

int detlsh_build_ex(const float *data, int64_t n, int32_t d, const detlsh_build_params *p,
                    void *stream, detlsh_index **out) {
  if (!out || !data) return DETLSH_ERR_INVALID_ARG;
  *out = nullptr;
  const int v = validate_build(n, d, p);
  if (v) return v;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return DETLSH_ERR_NO_DEVICE;
  }
  detlsh_index *ix = new (std::nothrow) detlsh_index();
  if (!ix) return DETLSH_ERR_OOM;
  cudaGetDevice(&ix->device);
  ix->n = n; ix->d = d; ix->L = p->L; ix->K = p->K; ix->LK = p->L * p->K; ix->N_r = p->N_r;
  ix->M = p->max_size; ix->box_mode = p->box_mode; ix->encoding = p->encoding; ix->tree_group = p->tree_group; ix->seed = p->seed; ix->frac = p->sample_frac;
  while ((1 << ix->bbits) < ix->N_r) ++ix->bbits;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int s = build_impl(ix, data, st, p);
  if (s != DETLSH_OK) {
    cudaStreamSynchronize(st);
    free_index(ix);
    return s;
  }
  *out = ix;
  return DETLSH_OK;
}

int detlsh_build(const float *data, int64_t n, int32_t d, int32_t L, int32_t K, int32_t N_r,
                 uint64_t seed, detlsh_index **out) {
  detlsh_build_params p;
  detlsh_default_build_params(&p);
  p.L = L; p.K = K; p.N_r = N_r; p.seed = seed;
  return detlsh_build_ex(data, n, d, &p, nullptr, out);
}

int detlsh_free(detlsh_index *ix) {
  free_index(ix);
  return DETLSH_OK;
}

int detlsh_query_ex(const detlsh_index *cix, const float *queries, int64_t m,
                    const int32_t *k_per_query, int32_t k_max, const detlsh_query_params *qp,
                    void *stream, int64_t *ids, float *dists) {
  detlsh_query_params def;
  detlsh_default_query_params(&def);
  if (!qp) qp = &def;
  const int v = validate_query(cix, m, k_max, qp);
  if (v) return v;
  if (m == 0) return DETLSH_OK;
  if (!queries || !ids || !dists) return DETLSH_ERR_INVALID_ARG;
  detlsh_index *ix = const_cast<detlsh_index *>(cix);
  std::lock_guard<std::mutex> g(ix->qmu);
  return query_impl(ix, queries, m, k_per_query, k_max, qp, static_cast<cudaStream_t>(stream), ids,
                    dists, 0, nullptr, nullptr, nullptr, nullptr);
}

int detlsh_query(const detlsh_index *ix, const float *queries, int64_t m, int32_t k, double c,
                 int64_t *ids, float *dists) {
  detlsh_query_params qp;
  detlsh_default_query_params(&qp);
  qp.c = c;
  return detlsh_query_ex(ix, queries, m, nullptr, k, &qp, nullptr, ids, dists);
}


int detlsh_query_reserve(detlsh_index *ix, int64_t m_max, int32_t k_max,
                         const detlsh_query_params *qp) {
  detlsh_query_params def;
  detlsh_default_query_params(&def);
  if (!qp) qp = &def;
  if (m_max < 1) return DETLSH_ERR_INVALID_ARG;
  const int v = validate_query(ix, m_max, k_max, qp);
  if (v) return v;
  std::lock_guard<std::mutex> g(ix->qmu);
  cudaStream_t st = nullptr;
  auto &P = ix->plan;
  P.ready = false;
  const int d = ix->d, LK = ix->LK;
  DL_TRY(grow(ix->aQp, sizeof(float) * (size_t)m_max * LK, st));
  if (qp->precision == DETLSH_PREC_BF16_REFINE)
    DL_TRY(grow(ix->aQh, sizeof(__nv_bfloat16) * (size_t)m_max * d, st));
  const uint32_t fb_cap = (uint32_t)std::max<int64_t>(1024, m_max * LK / 64);
  DL_TRY(grow(ix->afb, sizeof(uint2) * fb_cap, st));
  DL_TRY(grow(ix->aT, sizeof(float) * TABLE_FLOATS, st));
  DL_TRY(grow(ix->astat, 256, st));
  float Th[TABLE_FLOATS];
  query_tables(ix, qp, Th);
  DL_CUDA(cudaMemcpyAsync(ix->aT.p, Th, sizeof Th, cudaMemcpyHostToDevice, st));
  const double tb = std::ceil(qp->beta * (double)ix->n);
  P.tau_base = tb > (double)ix->n ? ix->n + 1 : (int64_t)tb;
  P.cap = (P.tau_base + k_max > ix->n || qp->per_tree)
              ? ix->n
              : std::min<int64_t>(ix->n, P.tau_base + k_max + ix->max_leaf);
  QueryIndexView vw = view_of(ix);
  query_slot_offsets(vw, P.cap, P.off);
  int slots = (int)std::min<int64_t>(query_slots(vw), m_max);
  DL_TRY(slots_within_budget(ix, slots, (size_t)P.off[SLOT_ARRAYS], ix->ascratch.bytes, &slots));
  bool fresh = false;
  DL_TRY(grow_scratch(ix->ascratch, &slots, (size_t)P.off[SLOT_ARRAYS], st, &fresh));
  if (fresh) DL_CUDA(cudaMemsetAsync(ix->ascratch.p, 0, ix->ascratch.bytes, st));
  DL_CUDA(cudaStreamSynchronize(st));
  P.qp = *qp;
  P.m_max = m_max;
  P.k_max = k_max;
  P.slots = slots;
  P.ready = true;
  return DETLSH_OK;
}

int detlsh_query_async(const detlsh_index *cix, const float *queries, int64_t m,
                       const int32_t *k_per_query, int32_t k_max, void *stream, int64_t *ids,
                       float *dists, int32_t *status) {
  if (!cix || !queries || !ids || !dists || !status) return DETLSH_ERR_INVALID_ARG;
  detlsh_index *ix = const_cast<detlsh_index *>(cix);
  std::lock_guard<std::mutex> g(ix->qmu);
  const auto &P = ix->plan;
  if (!P.ready || m < 0 || m > P.m_max || k_max < 1 || k_max > P.k_max)
    return DETLSH_ERR_INVALID_ARG;
  if (!is_device_ptr(queries) || !is_device_ptr(ids) || !is_device_ptr(dists) ||
      !is_device_ptr(status) || (k_per_query && !is_device_ptr(k_per_query)))
    return DETLSH_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int *err = static_cast<int *>(ix->astat.p);
  DL_CUDA(cudaMemsetAsync(ix->astat.p, 0, 256, st));
  if (m > 0) {
    const int d = ix->d, LK = ix->LK;
    float *Qp = static_cast<float *>(ix->aQp.p);
    ProjArgs pa;
    pa.P = Qp; pa.ldP = LK;
    pa.fb_count = reinterpret_cast<uint32_t *>(static_cast<char *>(ix->astat.p) + 16);
    pa.fb_cap = (uint32_t)(ix->afb.bytes / sizeof(uint2));
    pa.fb_list = static_cast<uint2 *>(ix->afb.p);
    pa.err = err;
    DL_TRY(project_rows(queries, d, nullptr, m, d, ix->A, LK, 0, pa, st));
    const __nv_bfloat16 *Qh = nullptr;
    if (P.qp.precision == DETLSH_PREC_BF16_REFINE) {
      DL_TRY(dl::f32_to_bf16(queries, static_cast<__nv_bfloat16 *>(ix->aQh.p), m * (int64_t)d, st));
      Qh = static_cast<const __nv_bfloat16 *>(ix->aQh.p);
    }
    QueryIndexView v = view_of(ix);
    QueryArgs qa{};
    qa.Q = queries; qa.Qh = Qh; qa.Qp = Qp; qa.m = m; qa.kq = k_per_query; qa.k_max = k_max;
    qa.tau_base = P.tau_base;
    qa.T = static_cast<const float *>(ix->aT.p);
    qa.Tc = qa.T + 256;
    qa.policy = P.qp.rmin_policy;
    const bool fixed = P.qp.rmin_policy == DETLSH_RMIN_FIXED;
    qa.lg_eps2 = fixed ? (float)(std::log2(ix->eps2 * P.qp.r_min * P.qp.r_min) +
                                 254.0 * std::log2(P.qp.c))
                       : (float)std::log2(ix->eps2);
    qa.inv_2lg_c = (float)(1.0 / (2.0 * std::log2(P.qp.c)));
    qa.precision = P.qp.precision; qa.rerank_mult = P.qp.rerank_mult;
    qa.ctas_per_sm = ix->tuning.query_ctas_per_sm;
    qa.expand_runs = ix->tuning.expand_runs;
    qa.visit_chunk = ix->tuning.visit_chunk;
    qa.top_min = ix->tuning.top_hull_min;
    qa.hash_kb = ix->tuning.hash_kb;
    qa.per_tree = P.qp.per_tree;
    qa.ids = ids; qa.dists = dists;
    qa.cand_cap = P.cap;
    for (int i = 0; i <= SLOT_ARRAYS; ++i) qa.off[i] = P.off[i];
    qa.slot_bytes = P.off[SLOT_ARRAYS];
    qa.epoch_counter = static_cast<unsigned long long *>(ix->ascratch.p);
    qa.scratch = static_cast<uint8_t *>(ix->ascratch.p) + kScratchHeader;
    qa.nslots = P.slots;
    qa.work_counter = reinterpret_cast<uint32_t *>(static_cast<char *>(ix->astat.p) + 32);
    qa.err = err;
    qa.stats = reinterpret_cast<unsigned long long *>(static_cast<char *>(ix->astat.p) + 64);
    DL_TRY(run_queries(v, qa, st));
  }
  DL_CUDA(cudaMemcpyAsync(status, err, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  return DETLSH_OK;
}

int detlsh_rc_ann(const detlsh_index *cix, const float *queries, int64_t m, double r,
                  double beta, double c, int32_t optimised, void *stream, int64_t *ids,
                  float *dists, int32_t *tree_stop, int64_t S_cap, int64_t *S,
                  int64_t *S_size) {
  if (!cix || m < 0) return DETLSH_ERR_INVALID_ARG;
  if (!(r > 0.0) || !std::isfinite(r) || !(beta >= 0.0) || !std::isfinite(beta) ||
      !(c > 1.0) || !std::isfinite(c))
    return DETLSH_ERR_INVALID_ARG;
  if (S && S_cap < 1) return DETLSH_ERR_INVALID_ARG;
  if (optimised != 0 && optimised != 1) return DETLSH_ERR_INVALID_ARG;
  if (!optimised && !cix->P) return DETLSH_ERR_INVALID_ARG;  // per-point tests read P
  if (m == 0) return DETLSH_OK;
  if (!queries || !ids || !dists) return DETLSH_ERR_INVALID_ARG;
  detlsh_index *ix = const_cast<detlsh_index *>(cix);
  std::lock_guard<std::mutex> g(ix->qmu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int d = ix->d, LK = ix->LK;
  DL_TRY(ensure_events(ix));
  const long long launches0 = g_launches.load();
  DL_TRY(grow(ix->qQ, sizeof(float) * (size_t)m * d, st));
  DL_TRY(grow(ix->qQp, sizeof(float) * (size_t)m * LK, st));
  DL_TRY(grow(ix->qstat, 256, st));
  const int64_t scap = S ? S_cap : 0;
  const size_t out_bytes = (size_t)m * (8 + 4 + 4 + 8) + (size_t)m * scap * 8 + 64;
  DL_TRY(grow(ix->qrc, out_bytes, st));
  float *Q = static_cast<float *>(ix->qQ.p);
  float *Qp = static_cast<float *>(ix->qQp.p);
  int *err = static_cast<int *>(ix->qstat.p);
  uint32_t *fb_count = reinterpret_cast<uint32_t *>(static_cast<char *>(ix->qstat.p) + 16);
  uint32_t *counter = reinterpret_cast<uint32_t *>(static_cast<char *>(ix->qstat.p) + 32);
  DL_CUDA(cudaMemsetAsync(ix->qstat.p, 0, 256, st));
  DL_CUDA(cudaEventRecord(ix->ev[5], st));
  DL_TRY(copy_in(Q, queries, sizeof(float) * (size_t)m * d, st));
  const uint32_t fb_cap = (uint32_t)std::max<int64_t>(1024, m * LK / 64);
  DL_TRY(grow(ix->qfb, sizeof(uint2) * fb_cap, st));
  ProjArgs pa;
  pa.P = Qp; pa.ldP = LK; pa.fb_count = fb_count; pa.fb_cap = fb_cap; pa.err = err;
  pa.fb_list = static_cast<uint2 *>(ix->qfb.p);
  DL_TRY(project_rows(Q, d, nullptr, m, d, ix->A, LK, 0, pa, st));
  int e = check_err(err, st);  // non-finite queries
  if (e) return e;
  QueryIndexView v = view_of(ix);
  RcArgs a{};
  a.Q = Q; a.Qp = Qp; a.m = m; a.optimised = optimised;
  a.R2 = (float)(ix->eps2 * r * r);  // (eps r)^2 rounded once, as the radius grid
  a.cr = (float)(c * r);
  const double nb = std::ceil(beta * (double)ix->n);
  a.need = nb > (double)ix->n ? ix->n + 1 : (int64_t)nb + 1;
  char *ob = static_cast<char *>(ix->qrc.p);
  a.ids = reinterpret_cast<int64_t *>(ob);
  a.S_size = a.ids + m;
  a.S = scap ? a.S_size + m : nullptr;
  a.S_cap = scap;
  a.dists = reinterpret_cast<float *>(ob + (size_t)m * 16 + (size_t)m * scap * 8);
  a.tree_stop = reinterpret_cast<int32_t *>(a.dists + m);
  a.slot_bytes = (int64_t)rcann_slot_bytes(v);
  int slots = (int)std::min<int64_t>(rcann_slots(v), m);
  size_t freeb = 0, totb = 0;
  DL_CUDA(cudaMemGetInfo(&freeb, &totb));
  while (slots > 1 && (size_t)slots * a.slot_bytes > freeb / 4 + ix->qrcs.bytes) slots /= 2;
  DL_TRY(grow(ix->qrcs, (size_t)slots * a.slot_bytes, st));
  a.scratch = static_cast<uint8_t *>(ix->qrcs.p);
  a.nslots = slots;
  a.work_counter = counter;
  DL_CUDA(cudaEventRecord(ix->ev[6], st));
  DL_TRY(run_rcann(v, a, st));
  DL_CUDA(cudaEventRecord(ix->ev[7], st));
  DL_TRY(copy_out(ids, a.ids, sizeof(int64_t) * (size_t)m, st));
  DL_TRY(copy_out(dists, a.dists, sizeof(float) * (size_t)m, st));
  if (tree_stop) DL_TRY(copy_out(tree_stop, a.tree_stop, sizeof(int32_t) * (size_t)m, st));
  if (S_size) DL_TRY(copy_out(S_size, a.S_size, sizeof(int64_t) * (size_t)m, st));
  if (S) DL_TRY(copy_out(S, a.S, sizeof(int64_t) * (size_t)m * scap, st));
  DL_CUDA(cudaStreamSynchronize(st));
  ix->timings.query_project_ms = ev_ms(ix->ev[5], ix->ev[6]);
  ix->timings.query_kernel_ms = ev_ms(ix->ev[6], ix->ev[7]);
  ix->timings.query_ms = ev_ms(ix->ev[5], ix->ev[7]);
  ix->timings.query_launches = g_launches.load() - launches0;
  ix->timings.query_count = m;
  return DETLSH_OK;
}

int detlsh_query_candidates(const detlsh_index *cix, const float *queries, int64_t m, int32_t k,
                            const detlsh_query_params *qp, int64_t cap, int64_t *S,
                            int64_t *S_size, int32_t *jstar, int32_t *istar) {
  detlsh_query_params def;
  detlsh_default_query_params(&def);
  if (!qp) qp = &def;
  const int v = validate_query(cix, m, k, qp);
  if (v) return v;
  if (m == 0) return DETLSH_OK;
  if (!queries || !S || !S_size || !jstar || !istar || cap < 1) return DETLSH_ERR_INVALID_ARG;
  detlsh_index *ix = const_cast<detlsh_index *>(cix);
  std::lock_guard<std::mutex> g(ix->qmu);
  return query_impl(ix, queries, m, nullptr, k, qp, nullptr, nullptr, nullptr, cap, S, S_size,
                    jstar, istar);
}

int detlsh_get_info(const detlsh_index *ix, detlsh_info *info) {
  if (!ix || !info) return DETLSH_ERR_INVALID_ARG;
  memset(info, 0, sizeof *info);
  info->n = ix->n; info->d = ix->d; info->L = ix->L; info->K = ix->K; info->N_r = ix->N_r;
  info->max_size = ix->M; info->box_mode = ix->box_mode; info->has_bf16 = ix->Xh != nullptr;
  info->encoding = ix->encoding;
  info->sample_size = ix->m_sample;
  for (int t = 0; t < ix->L; ++t) info->num_leaves[t] = ix->nleaves[t];
  info->max_leaf_size = ix->max_leaf;
  info->eps2 = ix->eps2;
  info->device_bytes = ix->device_bytes;
  info->projection_fallbacks = ix->fb_total;
  return DETLSH_OK;
}

int detlsh_get_projection_matrix(const detlsh_index *ix, float *A) {
  if (!ix || !A) return DETLSH_ERR_INVALID_ARG;
  DL_CUDA(cudaMemcpy(A, ix->A, sizeof(float) * (size_t)ix->LK * ix->d, cudaMemcpyDeviceToHost));
  return DETLSH_OK;
}

int detlsh_get_sample(const detlsh_index *ix, int64_t *ids) {
  if (!ix || !ids) return DETLSH_ERR_INVALID_ARG;
  std::vector<uint32_t> h((size_t)ix->m_sample);
  DL_CUDA(cudaMemcpy(h.data(), ix->sample, sizeof(uint32_t) * h.size(), cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < h.size(); ++i) ids[i] = h[i];
  return DETLSH_OK;
}

int detlsh_get_breakpoints(const detlsh_index *ix, float *B) {
  if (!ix || !B) return DETLSH_ERR_INVALID_ARG;
  DL_CUDA(cudaMemcpy(B, ix->B, sizeof(float) * (size_t)ix->LK * (ix->N_r + 1), cudaMemcpyDeviceToHost));
  return DETLSH_OK;
}

int detlsh_get_codes(const detlsh_index *ix, uint8_t *codes) {
  if (!ix || !codes) return DETLSH_ERR_INVALID_ARG;
  std::vector<uint8_t> h((size_t)ix->L * ix->n * CODE_STRIDE);
  DL_CUDA(cudaMemcpy(h.data(), ix->codes, h.size(), cudaMemcpyDeviceToHost));
  for (int64_t p = 0; p < ix->n; ++p)
    for (int t = 0; t < ix->L; ++t)
      for (int j = 0; j < ix->K; ++j)
        codes[p * ix->LK + t * ix->K + j] = h[((size_t)t * ix->n + p) * CODE_STRIDE + j];
  return DETLSH_OK;
}

int detlsh_get_projections(const detlsh_index *ix, float *P) {
  if (!ix || !P || !ix->P) return DETLSH_ERR_INVALID_ARG;
  DL_CUDA(cudaMemcpy(P, ix->P, sizeof(float) * (size_t)ix->n * ix->LK, cudaMemcpyDeviceToHost));
  return DETLSH_OK;
}

int detlsh_get_tree(const detlsh_index *ix, int32_t t, int64_t *perm, int64_t *leaf_begin,
                    uint8_t *box_lo, uint8_t *box_hi, uint8_t *nbits, int64_t *leaf_of) {
  if (!ix || t < 0 || t >= ix->L) return DETLSH_ERR_INVALID_ARG;
  const int64_t n = ix->n, nl = ix->nleaves[t], o = ix->leaf_off[t];
  const int K = ix->K;
  if (perm) {
    std::vector<uint32_t> h((size_t)n);
    DL_CUDA(cudaMemcpy(h.data(), ix->perm + (size_t)t * n, 4 * h.size(), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i) perm[i] = h[i];
  }
  if (leaf_begin) {
    std::vector<uint32_t> h((size_t)nl + 1);
    DL_CUDA(cudaMemcpy(h.data(), ix->leaf_begin + o + t, 4 * h.size(), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i <= nl; ++i) leaf_begin[i] = h[i];
  }
  const uint8_t *src[3] = {ix->leaf_lo, ix->leaf_hi, ix->leaf_nb};
  uint8_t *dst[3] = {box_lo, box_hi, nbits};
  for (int a = 0; a < 3; ++a) {
    if (!dst[a]) continue;
    std::vector<uint8_t> h((size_t)nl * 16);
    DL_CUDA(cudaMemcpy(h.data(), src[a] + o * 16, h.size(), cudaMemcpyDeviceToHost));
    for (int64_t l = 0; l < nl; ++l)
      for (int j = 0; j < K; ++j) dst[a][l * K + j] = h[(size_t)l * 16 + j];
  }
  if (leaf_of) {
    std::vector<uint32_t> h((size_t)n * ix->L);
    DL_CUDA(cudaMemcpy(h.data(), ix->leaf_of, 4 * h.size(), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i) leaf_of[i] = h[(size_t)i * ix->L + t];
  }
  return DETLSH_OK;
}

int detlsh_get_timings(const detlsh_index *ix, detlsh_timings *t) {
  if (!ix || !t) return DETLSH_ERR_INVALID_ARG;
  *t = ix->timings;
  return DETLSH_OK;
}

int detlsh_get_level_table(const detlsh_index *ix, double c, float *T) {
  if (!ix || !T || !(c > 1.0)) return DETLSH_ERR_INVALID_ARG;
  level_table(ix->eps2, c, T);
  return DETLSH_OK;
}

int detlsh_project(const detlsh_index *cix, const float *rows, int64_t m, float *out, void *stream) {
  if (!cix || m < 0) return DETLSH_ERR_INVALID_ARG;
  if (m == 0) return DETLSH_OK;
  if (!rows || !out) return DETLSH_ERR_INVALID_ARG;
  detlsh_index *ix = const_cast<detlsh_index *>(cix);
  std::lock_guard<std::mutex> g(ix->qmu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DL_TRY(grow(ix->qQ, sizeof(float) * (size_t)m * ix->d, st));
  DL_TRY(grow(ix->qQp, sizeof(float) * (size_t)m * ix->LK, st));
  DL_TRY(grow(ix->qstat, 256, st));
  DL_CUDA(cudaMemsetAsync(ix->qstat.p, 0, 256, st));
  float *Q = static_cast<float *>(ix->qQ.p);
  DL_TRY(copy_in(Q, rows, sizeof(float) * (size_t)m * ix->d, st));
  ProjArgs pa;
  pa.P = static_cast<float *>(ix->qQp.p);
  pa.ldP = ix->LK;
  pa.err = static_cast<int *>(ix->qstat.p);
  pa.fb_count = reinterpret_cast<uint32_t *>(static_cast<char *>(ix->qstat.p) + 16);
  pa.fb_cap = (uint32_t)std::max<int64_t>(1024, m * ix->LK / 64);
  DL_TRY(grow(ix->qfb, sizeof(uint2) * pa.fb_cap, st));
  pa.fb_list = static_cast<uint2 *>(ix->qfb.p);
  DL_TRY(project_rows(Q, ix->d, nullptr, m, ix->d, ix->A, ix->LK, 0, pa, st));
  const int e = check_err(pa.err, st);
  if (e) return e;
  DL_TRY(copy_out(out, ix->qQp.p, sizeof(float) * (size_t)m * ix->LK, st));
  DL_CUDA(cudaStreamSynchronize(st));
  return DETLSH_OK;
}

int detlsh_save(const detlsh_index *ix, const char *path, void *stream) {
  if (!ix || !path) return DETLSH_ERR_INVALID_ARG;
  return save_impl(ix, path, static_cast<cudaStream_t>(stream));
}

int detlsh_load(const char *path, void *stream, detlsh_index **out) {
  if (!path || !out) return DETLSH_ERR_INVALID_ARG;
  *out = nullptr;
  return load_impl(path, static_cast<cudaStream_t>(stream), out);
}

int detlsh_get_tuning(const detlsh_index *ix, detlsh_tuning *t) {
  if (!ix || !t) return DETLSH_ERR_INVALID_ARG;
  *t = ix->tuning;
  return DETLSH_OK;
}

int detlsh_set_tuning(detlsh_index *ix, const detlsh_tuning *t) {
  if (!ix) return DETLSH_ERR_INVALID_ARG;
  DL_TRY(check_tuning(t));
  std::lock_guard<std::mutex> g(ix->qmu);
  ix->tuning = *t;
  return DETLSH_OK;
}

int detlsh_autotune(detlsh_index *ix, const float *queries, int64_t m, int32_t k,
                    const detlsh_query_params *qp, const char *cache_path, void *stream,
                    detlsh_tuning *out, int32_t *from_cache) {
  if (!ix || !queries) return DETLSH_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(ix->qmu);
  const detlsh_tuning keep = ix->tuning;
  const int s = autotune_impl(ix, queries, m, k, qp, cache_path, static_cast<cudaStream_t>(stream),
                              out, from_cache);
  if (s != DETLSH_OK) ix->tuning = keep;
  return s;
}

}  // extern "C"
