// encode_tc.cu -- projections of all n points (Eq. 1) and their region codes
// (Alg. 1) on the 5th-generation tensor cores of sm_103a.
//
// The codes must equal those of the exact projection (the real dot product
// rounded once to FP32), so the kernel needs a value together with a
// rigorous bound on its distance from the exact one; a coordinate whose
// interval holds no breakpoint keeps its region, the others go to the exact
// recomputation kernel (k_project_exact<2>) exactly as with the CUDA-core
// encoder.
//
// Error-free slicing (the scheme of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012, with
// BF16 slices as in the tensor-core variants of Ootomo, Ozaki and Yokota,
// 2024).  Each row x is scaled by a power of two to x^ = x 2^-E with
// |x^| < 1 (E from the row's largest magnitude) and cut, by round-to-nearest
// on fixed grids, into
//     x^ = h0 + h1 + h2 + rho,   h0 in 2^-8 Z, |h0| <= 1,
//                                h1 in 2^-16 Z, |h1| <= 2^-9,
//                                h2 in 2^-24 Z, |h2| <= 2^-17, |rho| <= 2^-25.
// Each slice has at most 8 significant bits, so it is exact in BF16, and a
// product of two slices is exact in FP32.  The rows of the projection matrix
// A are cut the same way (a^ = a0 + a1 + a2 + rho').  The three accumulators
//     S_g = sum over s + t = g of  sum_k  h_s[k] a_t[k],   g = 0, 1, 2,
// hold sums of terms that are all integer multiples of 2^-(16 + 8g) and whose
// magnitudes add up to below 2^24 of those units for d <= 256 (at most 1,
// 2^-8 and 5 2^-19 per term): every partial sum is then exactly
// representable, so the tensor core's FP32 accumulation is exact whatever
// its order or internal rounding, as long as it keeps 24 significant bits.
// What the three sums leave out is bounded per column of A alone:
//     |x^.a^ - (S_0 + S_1 + S_2)| <= ||rho'||_1 + 2^-25 ||a0+a1+a2||_1
//                                   + (2^-9 + 2^-17) ||a2||_1 + 2^-17 ||a1||_1,
// using |x^_k| < 1, |h1| <= 2^-9, |h2| <= 2^-17, |rho| <= 2^-25.  The sums
// are combined as z = fl(fl(S_0 + S_1) + S_2) (error at most u(|s| + |z|)),
// and y = z 2^(E_x + E_a) is exact scaling.
//
// Pipeline of one CTA (one per SM, persistent over 128-row tiles, 16 warps):
//   warp 0       TMA: the FP32 tile, boxes of 128 rows x 32 floats, 128-byte
//                swizzle, into shared memory;
//   warp 1       tcgen05.mma issue into TMEM (M = 128 rows, K = 16): per
//                k-step x0 [a0 a1 a2] (N = 192), x1 [a0 a1] (N = 128) and
//                x2 a0 (N = 64), the A slices stacked as one B operand, so
//                that the three products land on S_0 S_1 S_2, S_1 S_2 and S_2;
//                owns the TMEM allocation (512 columns: two buffers of 3 x 64);
//   warps 4-7    slicing, one thread per row: the row's largest magnitude,
//                then per k-step the three BF16 slices in the canonical
//                K-major layout, into a ring of three k-step slots;
//   warps 8-15   epilogue, one thread per (row, 32 columns): tcgen05.ld of the
//                three sums, the estimate and its bound, the region by a
//                branch-free search of the breakpoints (Eytzinger order in
//                shared memory), the certificate, codes, the exact-path list
//                and the running bounds of the column extremes.
// Every wait on an mbarrier has a time limit; on expiry the kernel records
// DETLSH_ERR_TIMEOUT, lets its copies and MMAs drain, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace dl {
namespace {

constexpr int TC_ROWS = 128;     // rows per tile (MMA M)
constexpr int TC_N = 64;         // projection columns per tile (MMA N)
constexpr int TC_DMAX = 128;     // largest d taken by this path (shared memory)
constexpr int TC_NSLOT = 3;      // k-step slots of the slice ring
constexpr int TC_THREADS = 512;
constexpr int TC_BOXW = 32;      // floats per TMA box row (128 bytes)

// shared memory map, bytes from a 1024-aligned base
constexpr int SM_X = 0;                                 // FP32 tile: boxes of 128 x 128 B
constexpr int SM_XBYTES = TC_ROWS * TC_DMAX * 4;        // 64 KB
constexpr int SM_A = SM_X + SM_XBYTES;                  // A slices [kstep][kh][rg 24][8][16 B]
constexpr int SM_AKSTEP = 3 * TC_N * 16 * 2;            // one k-step of the three stacked slices
constexpr int SM_ABYTES = (TC_DMAX / 16) * SM_AKSTEP;   // 48 KB
constexpr int SM_RING = SM_A + SM_ABYTES;               // x slices [slot][s][kh][rg][8][16 B]
constexpr int SM_SLOT = 3 * 4096;
constexpr int SM_B = SM_RING + TC_NSLOT * SM_SLOT;      // breakpoints [64][256] Eytzinger
constexpr int SM_ROWSC = SM_B + TC_N * 256 * 4;         // row scales [2][128]
constexpr int SM_COLSC = SM_ROWSC + 2 * TC_ROWS * 4;    // column scales [64]
constexpr int SM_COLC = SM_COLSC + TC_N * 4;            // column truncation bounds [64]
constexpr int SM_UB = SM_COLC + TC_N * 4;               // running bounds of the column extremes [64][2]
constexpr int SM_BAR = SM_UB + TC_N * 8;                // mbarriers
constexpr int NBAR = 16;
constexpr int SM_FLAGS = SM_BAR + NBAR * 8;             // TMEM address, abort flag
constexpr int SM_TOTAL = SM_FLAGS + 16;
constexpr size_t TC_SMEM = SM_TOTAL + 1024;             // slack to align the base

// barrier indices
constexpr int B_XFULL = 0, B_XEMPTY = 1, B_SFULL = 2, B_SEMPTY = 5, B_AFULL = 8,
              B_AEMPTY = 10, B_DRAIN = 12, B_RFULL = 13;
constexpr int TMEM_COLS = 512;   // two accumulator buffers of 3 x 64 columns

// 1 s: the whole encode normally takes well under a millisecond
constexpr unsigned long long WAIT_LIMIT_NS = 1000000000ull;

__device__ __forceinline__ uint32_t saddr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of `parity` to complete.  Gives up (false) when another
// role has aborted, or after WAIT_LIMIT_NS, in which case it raises the abort
// flag and records DETLSH_ERR_TIMEOUT.
// Polls back off with __nanosleep so that waiting warps leave the issue
// slots to the warps doing work.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          int *err) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_test(bar, parity)) return true;
    __nanosleep(it < 8 ? 32u : 256u);
    if ((it & 63u) == 0u) {
      if (*abort_flag) return false;
      if (now_ns() - t0 > WAIT_LIMIT_NS) {
        *abort_flag = 1;
        atomicExch(err, (int)DETLSH_ERR_TIMEOUT);
        return false;
      }
    }
  }
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor, canonical K-major layout without swizzle:
// core matrices of 8 rows x 16 bytes, `lbo` bytes apart along K and `sbo`
// bytes apart along M (or N); bits 46-47 hold the descriptor version (1).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(TC_ROWS >> 4) << 24);
}

template <int N>
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc_n(N)), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Round-to-nearest cut of v (|v| < 1) into h0 + h1 + h2 + rho on the grids
// 2^-8, 2^-16 and 2^-24: adding 1.5 2^(23-g) rounds to the grid 2^-g
// (the sum stays in one binade) and subtracting it back is exact, as is
// each remainder.  Intrinsics keep the compiler from fusing or reassociating.
__device__ __forceinline__ void slice3(float v, float &h0, float &h1, float &h2, float &rho) {
  h0 = __fsub_rn(__fadd_rn(v, 49152.0f), 49152.0f);  // 1.5 * 2^15
  const float r0 = __fsub_rn(v, h0);
  h1 = __fsub_rn(__fadd_rn(r0, 192.0f), 192.0f);     // 1.5 * 2^7
  const float r1 = __fsub_rn(r0, h1);
  h2 = __fsub_rn(__fadd_rn(r1, 0.75f), 0.75f);       // 1.5 * 2^-1
  rho = __fsub_rn(r1, h2);
}

// 2^(126 - me) for the biased exponent me of a row's largest magnitude: the
// factor that maps the row into (-1, 1).  Subnormal for me >= 253.
__device__ __forceinline__ float inv_scale_of(uint32_t me) {
  const int f = 253 - (int)me;
  return f >= 1 ? __uint_as_float((uint32_t)f << 23) : __uint_as_float(1u << (f + 22));
}
// 2^(me - 126), the factor back; +inf beyond FP32 (the outputs are then listed).
__device__ __forceinline__ float scale_of(uint32_t me) {
  return me <= 253u ? __uint_as_float((me + 1u) << 23) : INFINITY;
}
__device__ __forceinline__ float max_abs4(float4 v, float m) {
  return fmaxf(fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))), m);
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);  // exact: at most 8 significant bits
  return *reinterpret_cast<const uint32_t *>(&p);
}
__device__ __forceinline__ float warp_sum_ru(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = __fadd_ru(v, __shfl_xor_sync(FULL, v, off));
  return v;
}

__global__ void __launch_bounds__(TC_THREADS, 1)
k_encode_tc(const __grid_constant__ CUtensorMap tmx, int64_t nrows, int d,
            const float *__restrict__ A, int LK, int W, ProjArgs o) {
  extern __shared__ uint8_t smraw[];
  // 1024-byte aligned base (128-byte swizzled TMA boxes); offsetting the
  // array itself keeps every access below a shared-memory access
  uint8_t *sm = smraw + ((1024u - (saddr(smraw) & 1023u)) & 1023u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int col0 = blockIdx.y * W;
  const int ncol = min(LK, col0 + W) - col0;
  const int K = o.K, t0 = col0 / K, nint = o.N_r - 1;
  const int DK = (d + 15) & ~15;  // reduction length padded to whole k-steps
  const int nks = DK / 16;
  const int nbox = (d + TC_BOXW - 1) / TC_BOXW;
  const int64_t ntiles = ceil_div(nrows, TC_ROWS);
  float *rowsc = reinterpret_cast<float *>(sm + SM_ROWSC);
  float *colsc = reinterpret_cast<float *>(sm + SM_COLSC);
  float *colC = reinterpret_cast<float *>(sm + SM_COLC);
  float *Bsm = reinterpret_cast<float *>(sm + SM_B);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + SM_FLAGS);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + SM_FLAGS + 4);
  const uint32_t bar0 = saddr(sm + SM_BAR);
  auto bar = [&](int i) { return bar0 + 8u * (uint32_t)i; };

  // ---- set-up: barriers, TMEM, A slices, breakpoints ----
  if (tid == 0) {
    mbar_init(bar(B_XFULL), 1);
    mbar_init(bar(B_XEMPTY), 4);  // the four slicing warps
    for (int s = 0; s < TC_NSLOT; ++s) {
      mbar_init(bar(B_SFULL + s), 4);
      mbar_init(bar(B_SEMPTY + s), 1);  // tcgen05.commit
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar(B_AFULL + b), 1);   // tcgen05.commit
      mbar_init(bar(B_AEMPTY + b), 8);  // the eight epilogue warps
    }
    mbar_init(bar(B_DRAIN), 1);
    for (int b = 0; b < 2; ++b) mbar_init(bar(B_RFULL + b), 4);  // row scales, slicing warps
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(tmem_slot)),
                 "r"((uint32_t)TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // A slices (the B operand: N = 64 projection rows, K-major), one warp per
  // projection row, and the per-row truncation bound of the header comment
  for (int c = warp; c < TC_N; c += TC_THREADS / 32) {
    const bool colok = c < ncol;
    const float *ar = A + (int64_t)(col0 + (colok ? c : 0)) * d;
    float m = 0.0f;
    for (int k = lane; k < d; k += 32) m = colok ? fmaxf(m, fabsf(ar[k])) : 0.0f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL, m, off));
    const uint32_t me = __float_as_uint(m) >> 23;
    const float sin = inv_scale_of(me);
    float S1 = 0.0f, S2 = 0.0f, Sa = 0.0f, Sr = 0.0f;
    for (int k = lane; k < DK; k += 32) {
      const float a = (colok && k < d) ? ar[k] : 0.0f;
      float h[3], rho;
      slice3(__fmul_rn(a, sin), h[0], h[1], h[2], rho);
      const int off = (k >> 4) * SM_AKSTEP + ((k >> 3) & 1) * (SM_AKSTEP / 2) + (c >> 3) * 128 +
                      (c & 7) * 16 + (k & 7) * 2;
#pragma unroll
      for (int t = 0; t < 3; ++t)
        *reinterpret_cast<__nv_bfloat16 *>(sm + SM_A + t * (TC_N / 8) * 128 + off) =
            __float2bfloat16_rn(h[t]);
      S1 = __fadd_ru(S1, fabsf(h[1]));
      S2 = __fadd_ru(S2, fabsf(h[2]));
      Sa = __fadd_ru(Sa, __fadd_ru(fabsf(h[0]), __fadd_ru(fabsf(h[1]), fabsf(h[2]))));
      Sr = __fadd_ru(Sr, fabsf(rho));
    }
    S1 = warp_sum_ru(S1);
    S2 = warp_sum_ru(S2);
    Sa = warp_sum_ru(Sa);
    Sr = warp_sum_ru(Sr);
    if (lane == 0) {
      // ||rho'||_1 + 2^-25 ||a~||_1 + (2^-9 + 2^-17) ||a2||_1 + 2^-17 ||a1||_1, plus
      // DK 2^-148 for the scalings x 2^-E, a 2^-E that may round in the subnormal range
      const float tiny = __fmul_ru((float)DK, 0x1p-148f);
      const float C = __fadd_ru(
          Sr, __fmaf_ru(0x1p-25f, Sa,
                        __fmaf_ru(0x1.01p-9f, S2, __fmaf_ru(0x1p-17f, S1, tiny))));
      colC[c] = colok ? C : 0.0f;
      colsc[c] = colok ? scale_of(me) : 0.0f;
    }
  }
  // interior breakpoints of each column in Eytzinger order (node h at level
  // l, position p holds sorted entry (2p + 1) 2^(7 - l) - 1), +inf padded
  for (int idx = tid; idx < TC_N * 256; idx += TC_THREADS) {
    const int c = idx >> 8, h = idx & 255;
    float v = INFINITY;
    if (h >= 1 && c < ncol) {
      const int l = 31 - __clz(h), p = h - (1 << l);
      const int rank = ((2 * p + 1) << (7 - l)) - 1;
      if (rank < nint) v = o.B[(int64_t)(col0 + c) * (o.N_r + 1) + 1 + rank];
    }
    Bsm[idx] = v;
  }
  // running bounds of the column extremes, cached for the epilogue
  if (tid < 2 * TC_N)
    reinterpret_cast<uint32_t *>(sm + SM_UB)[tid] = tid < 2 * ncol ? o.ubound[2 * col0 + tid] : 0u;
  fence_async_smem();  // the A slices are read by the tensor cores
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---- TMA producer: one 128-row FP32 tile per step ----
    if (lane == 0) {
      int it = 0, last = -1;
      for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        if (!mbar_wait(bar(B_XEMPTY), (uint32_t)(it & 1) ^ 1u, abort_flag, o.err)) break;
        mbar_expect_tx(bar(B_XFULL), (uint32_t)(nbox * TC_ROWS * 128));
        for (int j = 0; j < nbox; ++j)
          tma_load_2d(saddr(sm + SM_X + j * TC_ROWS * 128), &tmx, j * TC_BOXW,
                      (int)(tile * TC_ROWS), bar(B_XFULL));
        last = it;
      }
      // let the last copy land before the CTA exits (normally already consumed)
      if (last >= 0) {
        const unsigned long long t0 = now_ns();
        while (!mbar_test(bar(B_XFULL), (uint32_t)(last & 1)) && now_ns() - t0 < WAIT_LIMIT_NS) {
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issue: per k-step the six slice pairs s + t <= 2, in three MMAs ----
    if (lane == 0) {
      uint32_t gk = 0;
      int it = 0;
      bool issued = false;
      const uint32_t abase = saddr(sm + SM_A);
      for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int b = it & 1;
        if (!mbar_wait(bar(B_AEMPTY + b), (uint32_t)((it >> 1) & 1) ^ 1u, abort_flag, o.err)) break;
        tc_fence_after();
        const uint32_t dacc = tmem + (uint32_t)b * 192u;
        bool ok = true;
        for (int k = 0; k < nks; ++k, ++gk) {
          const uint32_t slot = gk % TC_NSLOT, use = gk / TC_NSLOT;
          if (!mbar_wait(bar(B_SFULL + slot), use & 1u, abort_flag, o.err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t xs = saddr(sm + SM_RING + slot * SM_SLOT);
          // x slices: k-halves 2048 B apart (LBO), 8-row groups 128 B apart (SBO);
          // A slices a0, a1, a2 stacked as B-operand rows 0-63, 64-127,
          // 128-191: k-halves SM_AKSTEP / 2 apart, 8-row groups 128 B apart
          const uint64_t x0 = smem_desc(xs, 2048, 128), x1 = smem_desc(xs + 4096, 2048, 128),
                         x2 = smem_desc(xs + 8192, 2048, 128);
          const uint64_t av = smem_desc(abase + (uint32_t)(k * SM_AKSTEP), SM_AKSTEP / 2, 128);
          // x0 [a0 a1 a2] -> S_0 S_1 S_2;  x1 [a0 a1] -> S_1 S_2;  x2 a0 -> S_2
          mma_bf16<3 * TC_N>(dacc, x0, av, k > 0 ? 1u : 0u);
          mma_bf16<2 * TC_N>(dacc + TC_N, x1, av, 1u);
          mma_bf16<TC_N>(dacc + 2 * TC_N, x2, av, 1u);
          mma_commit(bar(B_SEMPTY + slot));      // the slot is free once these are done
          issued = true;
        }
        if (!ok) break;
        mma_commit(bar(B_AFULL + b));
      }
      // every MMA has completed before TMEM is released
      if (issued) {
        mma_commit(bar(B_DRAIN));
        const unsigned long long t0 = now_ns();
        while (!mbar_test(bar(B_DRAIN), 0u) && now_ns() - t0 < WAIT_LIMIT_NS) {
        }
      }
    }
  } else if (warp >= 4 && warp < 8) {
    // ---- slicing, one thread per row of the tile ----
    const int r = tid - 128;
    const int sw = r & 7;  // 128-byte swizzle of the TMA boxes: chunk c sits at c ^ (row & 7)
    uint32_t gk = 0;
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
      if (!__all_sync(FULL, mbar_wait(bar(B_XFULL), (uint32_t)(it & 1), abort_flag, o.err))) break;
      float m = 0.0f;
      for (int j = 0; j < nbox; ++j) {
        const uint8_t *rp = sm + SM_X + j * TC_ROWS * 128 + r * 128;
#pragma unroll
        for (int c = 0; c < 8; ++c) m = max_abs4(*reinterpret_cast<const float4 *>(rp + ((c ^ sw) << 4)), m);
      }
      const uint32_t me = __float_as_uint(m) >> 23;  // NaN elements do not raise m; they poison their outputs
      const float sin = inv_scale_of(me);
      const int b = it & 1;
      // the row scale buffer is free once the epilogue of the tile two back is done
      if (!__all_sync(FULL, mbar_wait(bar(B_AEMPTY + b), (uint32_t)((it >> 1) & 1) ^ 1u, abort_flag,
                                      o.err)))
        break;
      rowsc[b * TC_ROWS + r] = scale_of(me);
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_RFULL + b));
      bool ok = true;
      for (int k = 0; k < nks; ++k, ++gk) {
        const uint32_t slot = gk % TC_NSLOT, use = gk / TC_NSLOT;
        if (!__all_sync(FULL, mbar_wait(bar(B_SEMPTY + slot), (use & 1u) ^ 1u, abort_flag, o.err))) {
          ok = false;
          break;
        }
        const uint8_t *rp = sm + SM_X + (k >> 1) * TC_ROWS * 128 + r * 128;
        float xv[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 v = *reinterpret_cast<const float4 *>(rp + ((((k & 1) * 4 + q) ^ sw) << 4));
          xv[4 * q] = v.x; xv[4 * q + 1] = v.y; xv[4 * q + 2] = v.z; xv[4 * q + 3] = v.w;
        }
        uint32_t w[3][8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          float p[3], q[3], rho;
          slice3(__fmul_rn(xv[2 * e], sin), p[0], p[1], p[2], rho);
          slice3(__fmul_rn(xv[2 * e + 1], sin), q[0], q[1], q[2], rho);
#pragma unroll
          for (int s = 0; s < 3; ++s) w[s][e] = pack_bf16(p[s], q[s]);
        }
        uint8_t *dst = sm + SM_RING + slot * SM_SLOT + (r >> 3) * 128 + (r & 7) * 16;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
          *reinterpret_cast<uint4 *>(dst + s * 4096) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
          *reinterpret_cast<uint4 *>(dst + s * 4096 + 2048) =
              make_uint4(w[s][4], w[s][5], w[s][6], w[s][7]);
        }
        fence_async_smem();  // generic-proxy stores, read by the tensor cores
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(B_SFULL + slot));
      }
      if (!ok) break;
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_XEMPTY));  // done with this FP32 tile
    }
  } else if (warp >= 8) {
    // ---- epilogue: one thread per (row, 32 columns); warp w reads TMEM lanes 32 (w % 4) .. ----
    const int q = warp & 3, half = (warp - 8) >> 2;
    const int r = q * 32 + lane;
    const int et = tid - 256;  // 0..255
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    uint32_t *ubs = reinterpret_cast<uint32_t *>(sm + SM_UB);
    // Exchange of the column-extreme bounds with global memory, one bound per
    // thread for et < 2 * ncol: the shared copy is pushed with an atomic whose
    // returned global value is folded in one tile later (its latency hides
    // behind the tile).  Any older value is a valid, looser bound.
    const bool ub_owner = et < 2 * ncol;
    uint32_t *ub_g = o.ubound + 2 * col0 + et;
    uint32_t ub_pend = ub_owner ? ubs[et] : 0u;
    // List reservations: a warp takes LIST_CHUNK entries at a time with one
    // atomicAdd and writes padding entries (row 0xffffffff, skipped by the
    // exact kernel) over what it leaves unused.
    constexpr uint32_t LIST_CHUNK = 64;
    uint32_t res_base = 0, res_left = 0;
    auto pad_rest = [&]() {
      for (uint32_t i = lane; i < res_left; i += 32)
        if (res_base + i < o.fb_cap) o.fb_list[res_base + i] = make_uint2(0xffffffffu, 0u);
      // the exact kernel adds the whole list length to the fallback count
      if (lane == 0 && res_left && o.fb_total)
        atomicAdd(o.fb_total, (unsigned long long)(-(long long)res_left));
      res_left = 0;
    };
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
      const int b = it & 1;
      const uint32_t par = (uint32_t)((it >> 1) & 1);
      if (!__all_sync(FULL, mbar_wait(bar(B_AFULL + b), par, abort_flag, o.err))) break;
      if (!__all_sync(FULL, mbar_wait(bar(B_RFULL + b), par, abort_flag, o.err))) break;
      tc_fence_after();
      const int64_t rr = tile * TC_ROWS + r;
      const bool row_ok = rr < nrows;
      const float rs = rowsc[b * TC_ROWS + r];
      for (int hh = 0; hh < 2; ++hh) {
        const int c0 = half * 32 + hh * 16;
        float lo[16], hi[16];
        uint32_t fin = 0;
        {
          float s0[16], s1[16], s2[16];
          const uint32_t ta = tmem + lane_off + (uint32_t)b * 192u + (uint32_t)c0;
          tmem_ld16(ta, s0);
          tmem_ld16(ta + 64, s1);
          tmem_ld16(ta + 128, s2);
          tmem_ld_wait();
          if (hh == 1) {  // the accumulators and the row scale of buffer b may be reused
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(B_AEMPTY + b));
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            // estimate and bound (header comment), in output units
            const float s = __fadd_rn(s0[j], s1[j]);
            const float z = __fadd_rn(s, s2[j]);
            const float e = __fmaf_ru(__fadd_ru(fabsf(s), fabsf(z)), 0x1p-24f, colC[c0 + j]);
            const float cs = colsc[c0 + j];
            const float y = __fmul_rn(__fmul_rn(z, cs), rs);
            const float dlt = __fmul_ru(__fmul_ru(e, cs), rs);
            // widened by the final rounding of the exact value to FP32 and by
            // the underflow of the two scalings
            const float dl2 =
                __fadd_ru(dlt, __fmaf_ru(__fadd_ru(fabsf(y), dlt), 1.2e-7f, 0x1p-148f));
            lo[j] = __fsub_rd(y, dl2);
            hi[j] = __fadd_ru(y, dl2);
            fin |= (isfinite(y) ? 1u : 0u) << j;
          }
        }
        // #breakpoints < lo (h - 256 after eight levels), sixteen independent
        // searches advanced level by level; hi[j] becomes the certificate:
        // the smallest breakpoint >= lo must not be below it
        uint32_t h[16];
        float succ[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) { h[j] = 1u; succ[j] = INFINITY; }
#pragma unroll
        for (int l = 0; l < 8; ++l) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float key = Bsm[(c0 + j) * 256 + (int)h[j]];
            const bool go = key < lo[j];
            succ[j] = go ? succ[j] : key;
            h[j] = 2u * h[j] + (go ? 1u : 0u);
          }
        }
        uint32_t cw[4] = {0u, 0u, 0u, 0u}, f16 = 0u, o16 = 0u;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const uint32_t cnt = h[j] - 256u;
          cw[j >> 2] |= cnt << (8 * (j & 3));
          const bool fj = (fin >> j) & 1u;
          const bool valid = row_ok && c0 + j < ncol;
          if (!(fj && succ[j] >= hi[j]) && valid) f16 |= 1u << j;
          if (fj && valid && (cnt == 0u || cnt == (uint32_t)nint)) o16 |= 1u << j;
        }
        if (o16) {
          // outer regions (rare): possibly a column extreme, listed while the
          // bound says so; the bound is tightened
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            if ((o16 >> j) & 1u) {
              const uint32_t cnt = h[j] - 256u;
              uint32_t *ub = ubs + 2 * (c0 + j);
              if (cnt == 0u) {
                if (lo[j] <= funkey(ub[0])) f16 |= 1u << j;
                atomicMin(&ub[0], fkey(hi[j]));
              }
              if (cnt == (uint32_t)nint) {
                if (hi[j] >= funkey(ub[1])) f16 |= 1u << j;
                atomicMax(&ub[1], fkey(lo[j]));
              }
            }
          }
        }
        // codes (exact for certain coordinates, hints for listed ones)
        if (row_ok) {
          if (K == 16) {
            if (c0 < ncol)
              *reinterpret_cast<uint4 *>(o.codes + ((int64_t)(t0 + c0 / 16) * o.n + rr) * CODE_STRIDE) =
                  make_uint4(cw[0], cw[1], cw[2], cw[3]);
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int c = c0 + j;
              if (c < ncol)
                o.codes[((int64_t)(t0 + c / K) * o.n + rr) * CODE_STRIDE + c % K] =
                    (uint8_t)(cw[j >> 2] >> (8 * (j & 3)));
            }
          }
        }
        // the listed coordinates, from the warp's reservation
        const uint32_t nf = __popc(f16);
        uint32_t incl = nf;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const uint32_t v = __shfl_up_sync(FULL, incl, off);
          if (lane >= off) incl += v;
        }
        const uint32_t total = __shfl_sync(FULL, incl, 31);
        if (total) {
          if (total > res_left) {
            pad_rest();
            uint32_t nb = 0;
            const uint32_t take = total > LIST_CHUNK ? total : LIST_CHUNK;
            if (lane == 0) nb = atomicAdd(o.fb_count, take);
            res_base = __shfl_sync(FULL, nb, 0);
            res_left = take;
          }
          uint32_t pos = res_base + incl - nf;
          if (f16) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              if ((f16 >> j) & 1u) {
                const uint32_t hv = (cw[j >> 2] >> (8 * (j & 3))) & 255u;
                if (pos < o.fb_cap)
                  o.fb_list[pos] = make_uint2((uint32_t)rr, ((uint32_t)(col0 + c0 + j) << 8) | hv);
                ++pos;
              }
            }
          }
          res_base += total;
          res_left -= total;
        }
      }
      // exchange of the bounds (see above)
      if (ub_owner) {
        const uint32_t mine = ubs[et];
        if (et & 1) {
          atomicMax(&ubs[et], ub_pend);
          ub_pend = atomicMax(ub_g, mine);
        } else {
          atomicMin(&ubs[et], ub_pend);
          ub_pend = atomicMin(ub_g, mine);
        }
      }
    }
    pad_rest();
    if (ub_owner) {
      if (et & 1) atomicMax(ub_g, ubs[et]);
      else atomicMin(ub_g, ubs[et]);
    }
  }

  // ---- teardown: every role has left its loop ----
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)TMEM_COLS)
                 : "memory");
  }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, looked up once (no link against libcuda)
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

}  // namespace

int launch_encode_tc(const float *X, int64_t nrows, int d, const float *A, int LK, int W,
                     ProjArgs o, cudaStream_t st, int *used) {
  *used = 0;
  // the path: row-major rows whose length is a multiple of 16 bytes (TMA
  // strides), at most TC_DMAX long (shared memory), 16-byte aligned base
  if (d < 4 || d > TC_DMAX || (d & 3) || (reinterpret_cast<uintptr_t>(X) & 15) || W > TC_N ||
      nrows < 1 || nrows >= (int64_t)1 << 31)
    return DETLSH_OK;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return DETLSH_OK;
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)nrows};
  const cuuint64_t strides[1] = {(cuuint64_t)d * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)TC_BOXW, (cuuint32_t)TC_ROWS};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(X), dims, strides, box,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return DETLSH_OK;  // the CUDA-core encoder takes it
  DL_CUDA(cudaFuncSetAttribute(k_encode_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)TC_SMEM));
  int dev = 0, sms = 0;
  DL_CUDA(cudaGetDevice(&dev));
  DL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t ny = ceil_div(LK, W), tiles = ceil_div(nrows, TC_ROWS);
  const int64_t gx = std::min<int64_t>(tiles, std::max<int64_t>(sms / ny, 1));
  k_encode_tc<<<dim3((unsigned)gx, (unsigned)ny), TC_THREADS, TC_SMEM, st>>>(map, nrows, d, A, LK,
                                                                           W, o);
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  *used = 1;
  return DETLSH_OK;
}

}  // namespace dl
