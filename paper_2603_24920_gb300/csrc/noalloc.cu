// noalloc.cu -- detlsh_query_noalloc: c^2-k-ANN queries that allocate nothing.
//
// Some callers cannot allocate device memory at query time: a serving process
// whose framework has already reserved (nearly) all device memory for its own
// pool, a latency-critical path where a cudaMalloc/cudaFree would stall every
// stream on the device, or an embedded deployment that forbids allocation
// after start-up.  This entry point runs the same projection and query
// kernels as detlsh_query_ex, but every piece of scratch memory they need
// comes from one fixed array compiled into this library, so the call itself
// never allocates.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace dl {
int index_query_view(const detlsh_index *ix, QueryIndexView *v, const float **A, int *has_bf16);
int index_device(const detlsh_index *ix);
int check_query_args(const detlsh_index *ix, int64_t m, int32_t k, const detlsh_query_params *qp);
void radius_grid(const detlsh_index *ix, double c, float T[256]);
}  // namespace dl

namespace {

using namespace dl;

// The fixed scratch: 32 MiB of device memory that every GPU which loads this
// library holds until the process exits.
constexpr size_t kScratchBytes = size_t(32) << 20;
static __device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the fixed scratch on the current device (looked up once
// per device, with that device current; the host-side name of the array is
// not a device address and must never be handed to a kernel).
int scratch_address(void **out) {
  int dev = 0;
  DL_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return DETLSH_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    DL_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return DETLSH_OK;
}

// True when p is device (or managed) memory of device `dev` and its address
// is a multiple of `align` bytes.
bool on_device(const void *p, int dev, uintptr_t align) {
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return false;
  if (at.type == cudaMemoryTypeDevice && at.device != dev) return false;
  return (reinterpret_cast<uintptr_t>(p) & (align - 1)) == 0;
}

int64_t up256(int64_t v) { return (v + 255) / 256 * 256; }

}  // namespace

extern "C" int detlsh_query_noalloc(const detlsh_index *ix, const float *queries, int64_t m,
                                    int32_t k, const detlsh_query_params *qp, void *stream,
                                    int64_t *ids, float *dists) {
  detlsh_query_params def;
  detlsh_default_query_params(&def);
  if (!qp) qp = &def;
  DL_TRY(check_query_args(ix, m, k, qp));
  if (qp->rmin_policy != DETLSH_RMIN_MAGIC) return DETLSH_ERR_INVALID_ARG;  // magic r_min only
  if (m == 0) return DETLSH_OK;
  QueryIndexView v;
  const float *A = nullptr;
  int has_bf16 = 0;
  DL_TRY(index_query_view(ix, &v, &A, &has_bf16));
  // The caller's buffers go straight to the kernels (no staging copy), so
  // they must live on the index's device, which must be the current one, and
  // meet the kernels' vector-load alignment: 16 bytes for query rows read as
  // float4 (d a multiple of 4), 8 for ids, 4 for dists.
  int dev = -1;
  DL_CUDA(cudaGetDevice(&dev));
  if (index_device(ix) != dev) return DETLSH_ERR_INVALID_ARG;
  const uintptr_t q_align = (v.d % 4 == 0) ? 16 : 4;
  if (!on_device(queries, dev, q_align) || !on_device(ids, dev, 8) || !on_device(dists, dev, 4))
    return DETLSH_ERR_INVALID_ARG;
  const bool bf16 = qp->precision == DETLSH_PREC_BF16_REFINE;

  // Carve the fixed scratch: status words, radius grid, projection fallback
  // list, query projections (and BF16 queries), then one slot per CTA.
  const double tb = std::ceil(qp->beta * (double)v.n);
  const int64_t tau_base = tb > (double)v.n ? v.n + 1 : (int64_t)tb;
  // per_tree (Alg. 5 with whole trees joining S) can take up to every point
  const int64_t cap = (tau_base + k > v.n || qp->per_tree)
                          ? v.n
                          : std::min<int64_t>(v.n, tau_base + k + v.max_leaf_size);
  const uint32_t fb_cap = 4096;
  const int64_t o_status = 0, o_T = 256, o_fb = o_T + 1024;
  const int64_t o_qp = up256(o_fb + 8 * (int64_t)fb_cap);
  const int64_t o_qh = up256(o_qp + 4 * m * v.LK);
  const int64_t o_slots = up256(o_qh + (bf16 ? 2 * m * v.d : 0));
  QueryArgs qa{};
  query_slot_offsets(v, cap, qa.off);
  const int64_t slot = qa.off[SLOT_ARRAYS];
  if (o_slots + slot > (int64_t)kScratchBytes) return DETLSH_ERR_SCRATCH_LIMIT;
  int slots = query_slots(v);
  slots = (int)std::min<int64_t>({(int64_t)slots, m, ((int64_t)kScratchBytes - o_slots) / slot});

  uint8_t *base = nullptr;
  DL_TRY(scratch_address(reinterpret_cast<void **>(&base)));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Every call reuses the same bytes: clear the part this call uses (status
  // words, counters, level tags) so nothing from the previous call leaks in.
  DL_CUDA(cudaMemsetAsync(base, 0, (size_t)(o_slots + (int64_t)slots * slot), st));
  int *err = reinterpret_cast<int *>(base + o_status);
  uint32_t *fb_count = reinterpret_cast<uint32_t *>(base + o_status + 16);
  uint32_t *counter = reinterpret_cast<uint32_t *>(base + o_status + 32);
  unsigned long long *stats = reinterpret_cast<unsigned long long *>(base + o_status + 64);
  float Th[256];
  radius_grid(ix, qp->c, Th);
  DL_CUDA(cudaMemcpyAsync(base + o_T, Th, sizeof Th, cudaMemcpyHostToDevice, st));

  ProjArgs pa;
  pa.P = reinterpret_cast<float *>(base + o_qp);
  pa.ldP = v.LK;
  pa.fb_list = reinterpret_cast<uint2 *>(base + o_fb);
  pa.fb_count = fb_count;
  pa.fb_cap = fb_cap;
  pa.err = err;
  DL_TRY(project_rows(queries, v.d, nullptr, m, v.d, A, v.LK, 0, pa, st));
  // a query holding NaN/Inf stops the call here, before the query kernel
  int h = 0;
  DL_CUDA(cudaMemcpyAsync(&h, err, sizeof h, cudaMemcpyDeviceToHost, st));
  DL_CUDA(cudaStreamSynchronize(st));
  if (h) return h;
  const __nv_bfloat16 *Qh = nullptr;
  if (bf16) {
    __nv_bfloat16 *qh = reinterpret_cast<__nv_bfloat16 *>(base + o_qh);
    DL_TRY(f32_to_bf16(queries, qh, m * (int64_t)v.d, st));
    Qh = qh;
  }
  qa.Q = queries; qa.Qh = Qh; qa.Qp = pa.P; qa.m = m; qa.kq = nullptr; qa.k_max = k;
  qa.tau_base = tau_base; qa.T = reinterpret_cast<const float *>(base + o_T);
  qa.lg_eps2 = (float)std::log2((double)Th[127]);  // T(0) = eps^2 seeds the level estimate
  qa.inv_2lg_c = (float)(1.0 / (2.0 * std::log2(qp->c)));
  qa.precision = qp->precision; qa.rerank_mult = qp->rerank_mult;
  qa.per_tree = qp->per_tree;
  qa.ids = ids; qa.dists = dists;
  qa.cand_cap = cap;
  qa.slot_bytes = slot;
  qa.scratch = base + o_slots;
  qa.nslots = slots;
  qa.work_counter = counter;
  qa.err = err;
  qa.stats = stats;
  qa.epoch_counter = reinterpret_cast<unsigned long long *>(base + o_status + 128);  // cleared above
  DL_TRY(run_queries(v, qa, st));
  DL_CUDA(cudaMemcpyAsync(&h, err, sizeof h, cudaMemcpyDeviceToHost, st));
  DL_CUDA(cudaStreamSynchronize(st));
  return h;
}
