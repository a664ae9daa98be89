// lut.cuh -- per-tree lower/upper-bound lookup table for box bounds
// (Sec. IV-C).  Shared by the query kernels.
#pragma once
#include "common.cuh"

namespace dl {

// The per-tree lookup table has 16 rows of LUT_STRIDE entries whatever K and
// N_r are: rows j >= K are zero, so the padded code bytes (zero) add an exact
// 0 to the sums, and every table offset is a compile-time constant.
// lut[j][z] = B_j[z] - q'_j.
constexpr int LUT_STRIDE = 257;
constexpr int LUT_ROWS = 16;

// Fills the table of tree t (whole block; the caller synchronises).  A
// thread takes table columns z (one region boundary, all rows): coalesced
// reads of B along z, no index division, eight loads in flight.
__device__ __forceinline__ void build_lut(float *lut, const float *B, const float *qpt, int t,
                                          int K, int NR1) {
  for (int z = threadIdx.x; z < LUT_STRIDE; z += blockDim.x) {
#pragma unroll
    for (int j0 = 0; j0 < LUT_ROWS; j0 += 8) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + u;
        v[u] = (j < K && z < NR1) ? __fsub_rn(B[(int64_t)(t * K + j) * NR1 + z], qpt[j]) : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) lut[(j0 + u) * LUT_STRIDE + z] = v[u];
    }
  }
}

// Squared lower bound of a box (Sec. IV-C) from the table: per dimension
// gap = max(0, B(lo) - q, q - B(hi+1)), summed in FP32 over dimensions in order.
__device__ __forceinline__ float box_lb2(const float *lut, const uint4 &lo, const uint4 &hi) {
  const uint32_t wl[4] = {lo.x, lo.y, lo.z, lo.w};
  const uint32_t wh[4] = {hi.x, hi.y, hi.z, hi.w};
  float acc = 0.0f;
#pragma unroll
  for (int j = 0; j < LUT_ROWS; ++j) {
    const uint32_t zl = (wl[j >> 2] >> (8 * (j & 3))) & 255u;
    const uint32_t zh = (wh[j >> 2] >> (8 * (j & 3))) & 255u;
    const float a = lut[j * LUT_STRIDE + zl];
    const float b = -lut[j * LUT_STRIDE + zh + 1];
    const float gap = fmaxf(fmaxf(a, b), 0.0f);
    acc = __fadd_rn(acc, __fmul_rn(gap, gap));
  }
  return acc;
}

// The same sum over dimensions [J0, J1) only, continuing from acc (the
// terms are non-negative and FP32 addition is monotone, so a partial sum
// above a threshold shows the whole sum is above it too).
template <int J0, int J1>
__device__ __forceinline__ float box_lb2_part(const float *lut, const uint4 &lo, const uint4 &hi,
                                              float acc) {
  const uint32_t wl[4] = {lo.x, lo.y, lo.z, lo.w};
  const uint32_t wh[4] = {hi.x, hi.y, hi.z, hi.w};
#pragma unroll
  for (int j = J0; j < J1; ++j) {
    const uint32_t zl = (wl[j >> 2] >> (8 * (j & 3))) & 255u;
    const uint32_t zh = (wh[j >> 2] >> (8 * (j & 3))) & 255u;
    const float a = lut[j * LUT_STRIDE + zl];
    const float b = -lut[j * LUT_STRIDE + zh + 1];
    const float gap = fmaxf(fmaxf(a, b), 0.0f);
    acc = __fadd_rn(acc, __fmul_rn(gap, gap));
  }
  return acc;
}

// Squared upper bound of a box (Sec. IV-C, Fig. 6): per dimension the
// distance to the farther edge, max(|B(lo) - q|, |B(hi+1) - q|), summed in
// FP32 over dimensions in order.
__device__ __forceinline__ float box_ub2(const float *lut, const uint4 &lo, const uint4 &hi) {
  const uint32_t wl[4] = {lo.x, lo.y, lo.z, lo.w};
  const uint32_t wh[4] = {hi.x, hi.y, hi.z, hi.w};
  float acc = 0.0f;
#pragma unroll
  for (int j = 0; j < LUT_ROWS; ++j) {
    const uint32_t zl = (wl[j >> 2] >> (8 * (j & 3))) & 255u;
    const uint32_t zh = (wh[j >> 2] >> (8 * (j & 3))) & 255u;
    const float far = fmaxf(fabsf(lut[j * LUT_STRIDE + zl]), fabsf(lut[j * LUT_STRIDE + zh + 1]));
    acc = __fadd_rn(acc, __fmul_rn(far, far));
  }
  return acc;
}

}  // namespace dl
