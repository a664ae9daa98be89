// common.cuh -- helpers shared by the DET-LSH CUDA kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/detlsh.h"

namespace dl {

constexpr unsigned FULL = 0xffffffffu;

// Philox stream ids (third counter word) used by the index.
constexpr uint32_t STREAM_PROJ = 2u;
constexpr uint32_t STREAM_SAMPLE = 3u;

// Radius grid for the magic r_min: levels j = -127..127 stored as 0..254.
constexpr int NLEV = 255;
constexpr int JMIN = -127;

// Codes are stored 16 bytes per (tree, point): K <= 16.
constexpr int CODE_STRIDE = 16;

// Leaves are grouped in runs of this many (canonical order) under a hull box.
constexpr int LEAF_BLOCK = 32;

struct U4 {
  uint32_t x, y, z, w;
};

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// multiply-xor S-box, key advanced by the Weyl increments between rounds.
__host__ __device__ inline U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t m0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t m1 = (uint64_t)0xCD9E8D57u * c.z;
    U4 n;
    n.x = (uint32_t)(m1 >> 32) ^ c.y ^ k0;
    n.y = (uint32_t)m1;
    n.z = (uint32_t)(m0 >> 32) ^ c.w ^ k1;
    n.w = (uint32_t)m0;
    c = n;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Order-preserving map between FP32 and uint32 (total order, -0 < +0).
__device__ __forceinline__ uint32_t fkey(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float funkey(uint32_t k) {
  const uint32_t b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(b);
}

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace dl

// Error plumbing for host code: returns a detlsh_status from the caller.
#define DL_CUDA(call)                                   \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) {                            \
      dl_set_last_cuda_error(_e, #call, __FILE__, __LINE__); \
      return (_e == cudaErrorMemoryAllocation) ? DETLSH_ERR_OOM : DETLSH_ERR_CUDA; \
    }                                                   \
  } while (0)

#define DL_TRY(expr)                 \
  do {                               \
    int _s = (expr);                 \
    if (_s != DETLSH_OK) return _s;  \
  } while (0)

void dl_set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line);

// Counts kernel launches made by the library (reported by detlsh_get_timings).
void dl_count_launch();
