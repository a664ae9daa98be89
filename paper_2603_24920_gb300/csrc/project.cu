// project.cu -- exact FP32 projection h_t(o) = a_t . o (Eq. 1) and the
// fused region encoding of Alg. 1, for sm_103a.
//
// Definition: the projection is the exact real dot product of the FP32
// operands, rounded once to the nearest FP32 (ties to even).  That value does
// not depend on summation order, so breakpoints, codes and trees built on it
// are reproducible bit for bit.
//
// Fast path (CUDA cores): the compensated dot product of Ogita, Rump and
// Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 26(6), 2005):
// each product is split exactly with an FMA (TwoProduct), the running sum
// with Knuth's TwoSum, and the exact error terms are summed separately.  The
// kernel also accumulates a rigorous bound E on what that separate sum lost;
// the result y = fl(p + s) is the correctly rounded value whenever
// |TwoSum error of (p + s)| + E stays below half the FP32 spacing at y.
// Uncertified outputs (about 1e-5 of them) go to a list that an exact
// big-integer kernel recomputes.
//
// Encoding (Alg. 1) needs only each coordinate's region, not its exact
// value.  k_encode computes a plain FP32 FMA dot product y and a rigorous
// bound on its distance to the exact value (a running chunked term plus a
// Cauchy-Schwarz term, detailed at the kernel), widened by one unit in the
// last place for the final rounding of the exact value.  When no breakpoint
// lies in that interval the region is certain; otherwise -- and for the two
// outer regions, which hold the column minimum and maximum -- the coordinate
// is listed and recomputed exactly.
#include "common.cuh"
#include "kernels.h"

#include <algorithm>
#include <cmath>

namespace dl {

constexpr int PJ_ROWS = 64;
constexpr int PJ_COLS = 64;
constexpr int PJ_KC = 32;
constexpr int PJ_THREADS = 256;

// u * (1 + 2^-6) rounded up, u = 2^-24: covers the rounding of the error
// accumulator for d <= 65536.
__device__ __forceinline__ float err_factor() { return 6.0536e-08f; }

__device__ __forceinline__ void dot2_step(float &p, float &s, float &e, float x, float a) {
  const float h = __fmul_rn(x, a);
  const float r = __fmaf_rn(x, a, -h);              // x*a = h + r exactly
  const float t = __fadd_rn(p, h);
  const float z = __fsub_rn(t, p);
  const float q = __fadd_rn(__fsub_rn(p, __fsub_rn(t, z)), __fsub_rn(h, z));  // p+h = t+q
  p = t;
  const float w = __fadd_rn(q, r);
  s = __fadd_rn(s, w);
  e = __fadd_rn(e, __fadd_rn(fabsf(w), fabsf(s)));   // rounding of w and s
}

// Returns true when y is certified to be the correctly rounded value.
__device__ __forceinline__ bool dot2_finish(float p, float s, float e, int d, float &y) {
  y = __fadd_rn(p, s);
  const float bv = __fsub_rn(y, p);
  const float zz = __fadd_rn(__fsub_rn(p, __fsub_rn(y, bv)), __fsub_rn(s, bv));
  // E >= u*(sum |w_i| + |s_i|) + underflow allowance d * 2^-148.
  const float tiny = __fmul_rn((float)d, __uint_as_float(2u));
  const float E = __fmaf_ru(e, err_factor(), tiny);
  const uint32_t yb = __float_as_uint(y);
  const uint32_t ex = (yb >> 23) & 0xffu;
  if (ex == 0xffu || ex < 32u) return false;        // non-finite or tiny: exact path
  float hb = __uint_as_float((ex - 24u) << 23);     // half the spacing above |y|
  if ((yb & 0x7fffffu) == 0u) hb = __fmul_rn(hb, 0.5f);  // power of two: spacing below halves
  const float lhs = __fadd_ru(fabsf(zz), E);
  return lhs < hb;
}

// Exact dot product rounded once to FP32, with a 640-bit fixed-point
// accumulator (value = sum dig[i] * 2^(32 i - 298)).  Used for the rare
// outputs the compensated path cannot certify.  Sets *bad on a non-finite
// operand or an FP32 overflow of the result.
__device__ float exact_dot_rn(const float *__restrict__ a, const float *__restrict__ x, int d,
                              bool *bad) {
  long long dig[20];
#pragma unroll
  for (int i = 0; i < 20; ++i) dig[i] = 0;
  for (int i = 0; i < d; ++i) {
    const uint32_t ab = __float_as_uint(a[i]), xb = __float_as_uint(x[i]);
    const uint32_t ae = (ab >> 23) & 0xffu, xe = (xb >> 23) & 0xffu;
    if (ae == 0xffu || xe == 0xffu) { *bad = true; return 0.0f; }
    const uint64_t am = (ab & 0x7fffffu) | (ae ? 0x800000u : 0u);
    const uint64_t xm = (xb & 0x7fffffu) | (xe ? 0x800000u : 0u);
    if (am == 0 || xm == 0) continue;
    const int pos = (int)(ae ? ae : 1u) + (int)(xe ? xe : 1u) - 2;  // bit offset of the product
    const uint64_t prod = am * xm;                                    // < 2^48
    const int c = pos >> 5, b = pos & 31;
    const uint64_t lo = prod << b;
    const uint64_t hi = b ? (prod >> (64 - b)) : 0ull;
    const long long p0 = (long long)(lo & 0xffffffffull);
    const long long p1 = (long long)(lo >> 32);
    const long long p2 = (long long)hi;
    if ((ab ^ xb) >> 31) { dig[c] -= p0; dig[c + 1] -= p1; dig[c + 2] -= p2; }
    else                 { dig[c] += p0; dig[c + 1] += p1; dig[c + 2] += p2; }
  }
  // carry-propagate into 32-bit digits, top digit signed
  for (int i = 0; i < 19; ++i) {
    const long long carry = dig[i] >> 32;
    dig[i] -= carry * 4294967296ll;
    dig[i + 1] += carry;
  }
  const bool neg = dig[19] < 0;
  if (neg) {
    for (int i = 0; i < 20; ++i) dig[i] = -dig[i];
    for (int i = 0; i < 19; ++i) {
      const long long carry = dig[i] >> 32;
      dig[i] -= carry * 4294967296ll;
      dig[i + 1] += carry;
    }
  }
  int top = -1;
  for (int i = 19; i >= 0; --i) {
    if (dig[i]) { top = 32 * i + 63 - __clzll(dig[i]); break; }  // digits are < 2^32
  }
  if (top < 0) return 0.0f;
  auto bit = [&](int q) -> uint32_t {
    return q < 0 ? 0u : (uint32_t)((dig[q >> 5] >> (q & 31)) & 1);
  };
  int lsb = top - 23;
  if (lsb < 149) lsb = 149;  // 2^-149 = FP32 subnormal spacing
  uint32_t mant = 0;
  for (int q = top; q >= lsb; --q) mant = (mant << 1) | bit(q);
  const uint32_t rb = bit(lsb - 1);
  uint32_t sticky = 0;
  for (int q = lsb - 2; q >= 0 && !sticky; --q) sticky = bit(q);
  if (rb && (sticky || (mant & 1u))) ++mant;
  if (mant == (1u << 24)) { mant >>= 1; ++lsb; }
  if (mant == 0) return 0.0f;
  const int e2 = lsb - 298;  // value = mant * 2^e2
  if (e2 + 24 > 128) { *bad = true; return 0.0f; }
  const float v = scalbnf((float)mant, e2);
  return neg ? -v : v;
}

// ---------------------------------------------------------------------------
// Epilogues.
// ---------------------------------------------------------------------------
// Interior breakpoints of a tile's columns are staged with a row stride of
// 257 floats so that the 16 columns a warp searches fall in distinct banks.
constexpr int BSTRIDE = 257;

// Number of interior breakpoints strictly below y (Alg. 1, lowest region on
// ties), from a column staged in shared memory and padded with +inf up to 255
// entries: eight power-of-two steps, branch-free.
__device__ __forceinline__ uint32_t region_smem(const float *Bs, float y) {
  uint32_t pos = 0;
#pragma unroll
  for (int s = 7; s >= 0; --s)
    if (Bs[pos + (1u << s) - 1] < y) pos += 1u << s;
  return pos;
}

// RI = rows per thread (16 RI rows per tile): RI = 1 gives small batches
// (queries) four times as many CTAs.
template <int MODE, int RI>
__global__ void __launch_bounds__(PJ_THREADS)
k_project(const float *__restrict__ X, int64_t ldx, const uint32_t *__restrict__ rows,
          int64_t nrows, int d, const float *__restrict__ A, int LK, int W, ProjArgs o) {
  // W = columns per tile, a multiple of K so that a tile never splits a tree
  constexpr int ROWS = 16 * RI;
  __shared__ float Xs[ROWS][PJ_KC + 1];
  __shared__ float As[PJ_COLS][PJ_KC + 1];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t row0 = (int64_t)blockIdx.x * ROWS;
  const int col0 = blockIdx.y * W;
  const int LKt = min(LK, col0 + W);  // end of this tile's columns

  float p[RI][4], s[RI][4], e[RI][4];
#pragma unroll
  for (int i = 0; i < RI; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) p[i][j] = s[i][j] = e[i][j] = 0.0f;

  for (int kc = 0; kc < d; kc += PJ_KC) {
    const int kmax = min(PJ_KC, d - kc);
    __syncthreads();
    for (int idx = tid; idx < PJ_COLS * PJ_KC; idx += PJ_THREADS) {
      const int r = idx / PJ_KC, c = idx % PJ_KC;
      if (r < ROWS) {
        const int64_t rr = row0 + r;
        float v = 0.0f;
        if (rr < nrows && c < kmax) {
          const int64_t src = rows ? (int64_t)rows[rr] : rr;
          v = X[src * ldx + kc + c];
        }
        Xs[r][c] = v;
      }
      const int oc = col0 + r;
      As[r][c] = (oc < LKt && c < kmax) ? A[(int64_t)oc * d + kc + c] : 0.0f;
    }
    __syncthreads();
#pragma unroll 2
    for (int kk = 0; kk < kmax; ++kk) {
      float xv[RI], av[4];
#pragma unroll
      for (int i = 0; i < RI; ++i) xv[i] = Xs[ty + 16 * i][kk];
#pragma unroll
      for (int j = 0; j < 4; ++j) av[j] = As[tx + 16 * j][kk];
#pragma unroll
      for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) dot2_step(p[i][j], s[i][j], e[i][j], xv[i], av[j]);
    }
  }

#pragma unroll
  for (int i = 0; i < RI; ++i) {
    const int64_t rr = row0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int oc = col0 + tx + 16 * j;
      float y;
      const bool ok = dot2_finish(p[i][j], s[i][j], e[i][j], d, y);
      if (rr < nrows && oc < LKt) {
        if (!ok) {
          const uint32_t slot = atomicAdd(o.fb_count, 1u);
          if (slot < o.fb_cap) o.fb_list[slot] = make_uint2((uint32_t)rr, (uint32_t)oc);
          y = 0.0f;
        }
        if (MODE == 0) o.P[rr * o.ldP + oc] = y + 0.0f;
        else o.P[(int64_t)oc * o.ldP + rr] = y + 0.0f;
      }
    }
  }
}

// Certified encoding: FP32 FMA estimate + rigorous a-posteriori bound.
//
// Each FMA s_k = fl(x_k a_k + s_{k-1}) errs by at most u |s_k| (+ an
// underflow allowance), so the estimate is within u * sum_k |s_k| of the
// exact product.  That sum is bounded in chunks of EN_CH terms: inside a
// chunk c that starts from s_c, |s_k| <= (|s_c| + T_c) / (1 - EN_CH u) with
// T_c = sum_{i in c} |x_i a_i|, so a chunk adds at most
// EN_CH (|s_c| + T_c) / (1 - EN_CH u); and sum_c T_c <= ||x|| ||a||
// (Cauchy-Schwarz).  The kernel therefore keeps one running term per output,
// E = sum_c EN_CH |s_c| (rounded up), and the bound is
//   gamma * (E + EN_CH ||x|| ||a||) + d 2^-148,  gamma >= u / (1 - EN_CH u),
// with ||x||, ||a|| upper bounds from round-up arithmetic.  A coordinate
// keeps its region when no breakpoint lies within that bound widened by one
// unit in the last place (the rounding of the exact value); otherwise it is
// listed.  Lowest- and highest-region coordinates are listed only while they
// can still be the column minimum or maximum, tested against running
// per-column bounds (init: B[1] and B[N_r-1], which are data values).
//
// Tiling: a CTA of 512 threads owns one column tile (<= 64 columns) and
// walks 256-row tiles; a thread accumulates 8 rows x 4 columns.  Chunks of 32
// terms are staged in shared memory k-major by cp.async (double-buffered), so
// the inner step is three 16-byte shared loads and 32 FMAs.  Row r of term k
// sits at float (k, ((r >> 2) ^ (k & 7)) * 4 + (r & 3)), which makes the
// copies' shared stores bank-conflict-free and keeps every 16-byte read whole.
constexpr int EN_ROWS = 256;
constexpr int EN_COLS = 64;
constexpr int EN_KC = 32;
constexpr int EN_CH = 8;
constexpr int EN_THREADS = 512;
constexpr int EN_CST = 18;  // codes: words per staged row (conflict-free stores)

__host__ __device__ constexpr size_t encode_smem_bytes() {
  return sizeof(float) * (2 * EN_KC * EN_ROWS + 2 * EN_KC * EN_COLS + EN_COLS * BSTRIDE +
                          EN_ROWS + EN_COLS) +
         sizeof(uint32_t) * (EN_ROWS * EN_CST + 2 * EN_COLS);
}

__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// EN_CH terms (k = kb .. kb + EN_CH - 1, kb a multiple of 8) of a thread's
// 8 x 4 outputs, after adding the chunk's EN_CH |s_c| to E.
__device__ __forceinline__ void encode_terms(float (&s)[8][4], float (&E)[8][4], const float *xs,
                                             const float *as, int kb, int ty, int tx) {
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) E[i][j] = __fmaf_ru((float)EN_CH, fabsf(s[i][j]), E[i][j]);
#pragma unroll
  for (int u = 0; u < EN_CH; ++u) {
    const int k = kb + u;
    const float4 x0 = *reinterpret_cast<const float4 *>(xs + k * EN_ROWS + (((2 * ty) ^ u) << 2));
    const float4 x1 = *reinterpret_cast<const float4 *>(xs + k * EN_ROWS + (((2 * ty + 1) ^ u) << 2));
    const float4 a4 = *reinterpret_cast<const float4 *>(as + k * EN_COLS + ((tx ^ u) << 2));
    const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
    const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) s[i][j] = __fmaf_rn(xv[i], av[j], s[i][j]);
  }
}

__global__ void __launch_bounds__(EN_THREADS, 1)
k_encode(const float *__restrict__ X, int64_t ldx, int64_t nrows, int d,
         const float *__restrict__ A, int LK, int W, ProjArgs o) {
  extern __shared__ float dyn[];
  float *Xs = dyn;                                  // [2][EN_KC][EN_ROWS], swizzled
  float *As = Xs + 2 * EN_KC * EN_ROWS;             // [2][EN_KC][EN_COLS], swizzled
  float *Bs = As + 2 * EN_KC * EN_COLS;             // [64 slots][BSTRIDE] interior breakpoints
  float *nxs = Bs + EN_COLS * BSTRIDE;              // [EN_ROWS] row norms (rounded up)
  float *nas = nxs + EN_ROWS;                       // [EN_COLS] column norms (rounded up)
  uint32_t *cst = reinterpret_cast<uint32_t *>(nas + EN_COLS);  // [EN_ROWS][EN_CST] codes
  uint32_t *cmin = cst + EN_ROWS * EN_CST, *cmax = cmin + EN_COLS;
  const uint8_t *cst8 = reinterpret_cast<const uint8_t *>(cst);

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int tx = tid & 15, ty = tid >> 4;           // columns 4tx.., rows 8ty..
  const int col0 = blockIdx.y * W;
  const int LKt = min(LK, col0 + W);
  const int ncol = LKt - col0;
  const int nint = o.N_r - 1;
  const float gam = o.gamma;                        // >= u / (1 - EN_CH u), rounded up
  const float tiny = __fmul_rn((float)d, __uint_as_float(2u));  // d * 2^-148
  const int K = o.K;
  const int ntree = ncol / K;
  const int t0 = col0 / K;
  const int64_t ntiles = ceil_div(nrows, EN_ROWS);
  const int nchunk = (d + EN_KC - 1) / EN_KC;
  // breakpoint slot of column c: columns 4tx + j of a warp land in 16 consecutive slots
  auto bslot = [](int c) { return (c & 3) * 16 + (c >> 2); };

  for (int idx = tid; idx < ncol * BSTRIDE; idx += EN_THREADS) {
    const int c = idx / BSTRIDE, z = idx % BSTRIDE;
    Bs[bslot(c) * BSTRIDE + z] = z < nint ? o.B[(int64_t)(col0 + c) * (o.N_r + 1) + 1 + z] : INFINITY;
  }
  if (tid < EN_COLS) {  // ||a|| per column, rounded up
    float s2 = 0.0f;
    if (tid < ncol) {
      const float *ar = A + (int64_t)(col0 + tid) * d;
      for (int k = 0; k < d; ++k) s2 = __fmaf_ru(ar[k], ar[k], s2);
    }
    nas[tid] = __fsqrt_ru(s2);
  }

  // cp.async of one chunk (tile, kc) into stage st: 16 X and 4 A words per thread
  auto load = [&](int64_t tile, int kc, int st) {
    const int64_t row0 = tile * EN_ROWS;
    const int kmax = min(EN_KC, d - kc);
    const int r3 = lane & 3, kq = lane >> 2;
    float *xs = Xs + st * EN_KC * EN_ROWS;
#pragma unroll
    for (int it = 0; it < 16; ++it) {
      const int cell = warp * 16 + it;              // 64 row groups x 4 k groups
      const int rg = cell >> 2, k = (cell & 3) * 8 + kq;
      const int r = rg * 4 + r3;
      const int64_t rr = row0 + r;
      const bool v = rr < nrows && k < kmax;
      cp_async4(xs + k * EN_ROWS + ((rg ^ kq) << 2) + r3, v ? X + rr * ldx + kc + k : X, v);
    }
    float *as = As + st * EN_KC * EN_COLS;
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int cell = warp * 4 + it;               // 16 column groups x 4 k groups
      const int cg = cell >> 2, k = (cell & 3) * 8 + kq;
      const int c = cg * 4 + r3;
      const bool v = c < ncol && k < kmax;
      cp_async4(as + k * EN_COLS + ((cg ^ kq) << 2) + r3, v ? A + (int64_t)(col0 + c) * d + kc + k : A, v);
    }
  };

  int64_t tile = blockIdx.x;
  int st = 0;
  if (tile < ntiles) load(tile, 0, 0);
  cp_async_commit();
  for (; tile < ntiles; tile += gridDim.x) {
    const int64_t row0 = tile * EN_ROWS;
    float s[8][4], E[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) s[i][j] = E[i][j] = 0.0f;
    // row norm^2 of row tid >> 1: this thread takes the terms with bit 2 of
    // k equal to tid & 1 (the pair's loads then fall in distinct banks)
    float nx2 = 0.0f;
    for (int q = 0; q < nchunk; ++q) {
      const int kc = q * EN_KC;
      __syncthreads();  // stage st ^ 1 is free
      if (q + 1 < nchunk) load(tile, kc + EN_KC, st ^ 1);
      else if (tile + gridDim.x < ntiles) load(tile + gridDim.x, 0, st ^ 1);
      cp_async_commit();
      cp_async_wait1();
      __syncthreads();  // stage st is visible
      const float *xs = Xs + st * EN_KC * EN_ROWS;
      const float *as = As + st * EN_KC * EN_COLS;
      {
        const int r = tid >> 1, h = tid & 1;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int k = (e >> 2) * 8 + h * 4 + (e & 3);
          const float v = xs[k * EN_ROWS + (((r >> 2) ^ (k & 7)) << 2) + (r & 3)];
          nx2 = __fmaf_ru(v, v, nx2);
        }
      }
      if (d - kc >= EN_KC) {  // a full chunk: every address is a constant offset
#pragma unroll
        for (int kb = 0; kb < EN_KC; kb += EN_CH) encode_terms(s, E, xs, as, kb, ty, tx);
      } else {
        const int kpad = (d - kc + EN_CH - 1) & ~(EN_CH - 1);
        for (int kb = 0; kb < kpad; kb += EN_CH) encode_terms(s, E, xs, as, kb, ty, tx);
      }
      st ^= 1;
    }
    nx2 = __fadd_ru(nx2, __shfl_xor_sync(FULL, nx2, 1));
    if ((tid & 1) == 0) nxs[tid >> 1] = __fsqrt_ru(nx2);
    if (tid < EN_COLS) { cmin[tid] = 0xffffffffu; cmax[tid] = 0u; }
    __syncthreads();
    uint32_t flags = 0;  // bit i*4+j: output (row 8ty+i, column 4tx+j) goes to the exact list
    float na[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) na[j] = nas[4 * tx + j];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = 8 * ty + i;
      const bool rowok = row0 + r < nrows;
      const float nx = nxs[r];
      // the row's four regions first (independent searches), then the certificates
      uint32_t word = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) word |= region_smem(Bs + bslot(4 * tx + j) * BSTRIDE, s[i][j]) << (8 * j);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = 4 * tx + j;
        const float y = s[i][j];
        const uint32_t reg = (word >> (8 * j)) & 255u;
        const float tot = __fmaf_ru((float)EN_CH, __fmul_ru(nx, na[j]), E[i][j]);
        const float dlt = __fmaf_ru(gam, tot, tiny);
        const float dl2 = __fadd_ru(dlt, __fmul_ru(__fadd_ru(fabsf(y), dlt), 1.2e-7f));
        const float lo = __fsub_rd(y, dl2), hi = __fadd_ru(y, dl2);
        const float *Bc = Bs + bslot(c) * BSTRIDE;
        const bool finite = isfinite(y);  // dl2 = +inf lists the output through lo = -inf
        const float below = reg == 0 ? -INFINITY : Bc[reg - 1];
        const float above = reg == (uint32_t)nint ? INFINITY : Bc[reg];
        bool list = !(finite && below < lo && above >= hi);
        if (finite && (reg == 0 || reg == (uint32_t)nint) && rowok && c < ncol) {
          if (reg == 0) {  // may be the column minimum?
            list |= lo <= funkey(*(volatile uint32_t *)&o.ubound[(col0 + c) * 2 + 0]);
            atomicMin(&cmin[c], fkey(hi));
          }
          if (reg == (uint32_t)nint) {  // may be the column maximum?
            list |= hi >= funkey(*(volatile uint32_t *)&o.ubound[(col0 + c) * 2 + 1]);
            atomicMax(&cmax[c], fkey(lo));
          }
        }
        if (list && rowok && c < ncol) flags |= 1u << (i * 4 + j);
      }
      cst[r * EN_CST + tx] = word;  // exact for sure coordinates; hints for listed ones
    }
    // one list reservation per warp: exclusive scan of the lanes' counts
    {
      const uint32_t cnt = __popc(flags);
      uint32_t incl = cnt;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, incl, off);
        if (lane >= off) incl += y;
      }
      uint32_t base = 0;
      if (lane == 31 && incl) base = atomicAdd(o.fb_count, incl);
      base = __shfl_sync(FULL, base, 31) + incl - cnt;
      while (flags) {
        const int b = __ffs(flags) - 1;
        flags &= flags - 1;
        const int r = 8 * ty + (b >> 2), c = 4 * tx + (b & 3);
        const uint32_t hint = cst8[r * EN_CST * 4 + c];
        if (base < o.fb_cap) o.fb_list[base] = make_uint2((uint32_t)(row0 + r), ((uint32_t)(col0 + c) << 8) | hint);
        ++base;
      }
    }
    __syncthreads();
    // tighten the running bounds: the column minimum is <= every hi seen in
    // its lowest region, the maximum >= every lo seen in its highest region
    if (tid < ncol) {
      if (cmin[tid] != 0xffffffffu) atomicMin(&o.ubound[(col0 + tid) * 2 + 0], cmin[tid]);
      if (cmax[tid] != 0u) atomicMax(&o.ubound[(col0 + tid) * 2 + 1], cmax[tid]);
    }
    for (int idx = tid; idx < EN_ROWS * ntree; idx += EN_THREADS) {
      const int r = idx / ntree, tt = idx % ntree;
      const int64_t rr = row0 + r;
      if (rr >= nrows) continue;
      uint4 w;
      if (K == 16) {
        const uint32_t *src = cst + r * EN_CST + tt * 4;
        w = make_uint4(src[0], src[1], src[2], src[3]);
      } else {
        const uint8_t *src = cst8 + r * EN_CST * 4 + tt * K;
        auto pack = [&](int j0) {
          uint32_t v = 0;
#pragma unroll
          for (int b = 0; b < 4; ++b)
            if (j0 + b < K) v |= (uint32_t)src[j0 + b] << (8 * b);
          return v;
        };
        w = make_uint4(pack(0), pack(4), pack(8), pack(12));
      }
      *reinterpret_cast<uint4 *>(o.codes + ((int64_t)(t0 + tt) * o.n + rr) * CODE_STRIDE) = w;
    }
  }
  cp_async_wait0();  // only empty groups can remain; drain them before exit
}

// Exact recomputation of the listed outputs, EX_GL lanes per output (eight
// outputs per warp).  The lanes split the row and run the compensated
// recurrence on their terms; the group folds its partial states
// (p_l, s_l, e_l) with the same error-free TwoSum step, so the certificate
// of dot2_finish still bounds the total error.  Uncertified outputs take the
// big-integer path.  The count is read on the device (no host
// synchronisation); if the list overflowed, every output is recomputed.
constexpr int EX_GL = 4;

template <int MODE>
__global__ void __launch_bounds__(256)
k_project_exact(const float *__restrict__ X, int64_t ldx, const uint32_t *__restrict__ rows,
                int64_t nrows, int d, const float *__restrict__ A, int LK, ProjArgs o) {
  const uint32_t cnt = *o.fb_count;
  if (cnt == 0) return;
  const bool all = cnt > o.fb_cap;
  if (blockIdx.x == 0 && threadIdx.x == 0 && o.fb_total)
    atomicAdd(o.fb_total, (unsigned long long)(all ? nrows * (int64_t)LK : (int64_t)cnt));
  const int64_t total = all ? nrows * (int64_t)LK : (int64_t)cnt;
  const int lane = threadIdx.x & 31, gl = lane & (EX_GL - 1);
  constexpr int PER_WARP = 32 / EX_GL;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  // warp-uniform trip count: every lane takes part in the group shuffles
  for (int64_t i0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * PER_WARP; i0 < total;
       i0 += warps * PER_WARP) {
    const int64_t i = i0 + lane / EX_GL;
    bool valid = i < total;
    int64_t rr = 0;
    int oc = 0;
    uint32_t hint = 0;
    if (valid) {
      if (all) { rr = i / LK; oc = (int)(i % LK); }
      else {
        const uint2 f = o.fb_list[i];
        if (f.x == 0xffffffffu) valid = false;  // padding of a list reservation
        rr = valid ? f.x : 0;
        oc = valid ? (MODE == 2 ? (int)(f.y >> 8) : (int)f.y) : 0;
        hint = MODE == 2 ? (f.y & 255u) : 0u;
      }
    }
    const int64_t src = valid ? (rows ? (int64_t)rows[rr] : rr) : 0;
    const float *ar = A + (int64_t)oc * d;
    const float *xr = X + src * ldx;
    float p = 0.0f, sc = 0.0f, ec = 0.0f;
    if (valid)
      for (int k2 = gl; k2 < d; k2 += EX_GL) dot2_step(p, sc, ec, xr[k2], ar[k2]);
    // butterfly fold: (Pa,Sa,Ea) + (Pb,Sb,Eb) -> P = fl(Pa+Pb) with its exact
    // TwoSum error q, S = fl(fl(Sa+Sb) + q), E gathers both bounds and the
    // two new roundings; the true sum stays within u*E of P + S.
    float P = p, S = sc, E = ec;
#pragma unroll
    for (int off = EX_GL / 2; off > 0; off >>= 1) {
      const float pb = __shfl_xor_sync(FULL, P, off), sb = __shfl_xor_sync(FULL, S, off);
      const float eb = __shfl_xor_sync(FULL, E, off);
      const float t = __fadd_rn(P, pb);
      const float z = __fsub_rn(t, P);
      const float q = __fadd_rn(__fsub_rn(P, __fsub_rn(t, z)), __fsub_rn(pb, z));
      const float w = __fadd_rn(S, sb);
      const float s2 = __fadd_rn(w, q);
      E = __fadd_rn(__fadd_rn(E, eb), __fadd_rn(fabsf(w), fabsf(s2)));
      P = t;
      S = s2;
    }
    if (gl != 0 || !valid) continue;
    float y;
    bool bad = false;
    if (!dot2_finish(P, S, E, d + 32, y)) y = exact_dot_rn(ar, xr, d, &bad);
    if (bad) { atomicExch(o.err, (int)DETLSH_ERR_NONFINITE_INPUT); continue; }
    y = y + 0.0f;  // exact zero is +0
    if (MODE == 0) { o.P[rr * o.ldP + oc] = y; continue; }
    if (MODE == 1) { o.P[(int64_t)oc * o.ldP + rr] = y; continue; }
    const float *Bint = o.B + (int64_t)oc * (o.N_r + 1) + 1;
    // walk from the estimated region to the exact one (#breakpoints < y)
    uint32_t code = min(hint, (uint32_t)(o.N_r - 1));
    while (code > 0 && !(Bint[code - 1] < y)) --code;
    while (code < (uint32_t)(o.N_r - 1) && Bint[code] < y) ++code;
    const int t = oc / o.K, j = oc % o.K;
    o.codes[((int64_t)t * o.n + rr) * CODE_STRIDE + j] = (uint8_t)code;
    // the column minimum (maximum) lies in the lowest (highest) region
    if (code == 0) atomicMin(&o.minmax[oc * 2 + 0], fkey(y));
    if (code == (uint32_t)(o.N_r - 1)) atomicMax(&o.minmax[oc * 2 + 1], fkey(y));
  }
}

template <int MODE>
static int project_impl(const float *X, int64_t ldx, const uint32_t *rows, int64_t nrows, int d,
                        const float *A, int LK, ProjArgs o, cudaStream_t st) {
  if (nrows <= 0) return DETLSH_OK;
  DL_CUDA(cudaMemsetAsync(o.fb_count, 0, sizeof(uint32_t), st));
  const int W = (MODE == 2) ? (EN_COLS / o.K) * o.K : PJ_COLS;
  int tc = 0;
  if constexpr (MODE == 2) {
    if (!rows && ldx == d) DL_TRY(launch_encode_tc(X, nrows, d, A, LK, W, o, st, &tc));
  }
  if (tc) {
    // the tensor-core encoder ran
  } else if constexpr (MODE == 2) {
    // gamma >= u / (1 - EN_CH u), u = 2^-24, rounded up
    o.gamma = std::nextafter((float)(0x1p-24 * (1.0 + 2.0 * EN_CH * 0x1p-24) * (1.0 + 1e-9)), INFINITY);
    const size_t dyn = encode_smem_bytes();
    DL_CUDA(cudaFuncSetAttribute(k_encode, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    int dev = 0, sms = 0, per = 0;
    DL_CUDA(cudaGetDevice(&dev));
    DL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_encode, EN_THREADS, dyn));
    const int64_t ny = ceil_div(LK, W), tiles = ceil_div(nrows, EN_ROWS);
    // persistent: one wave of CTAs, split over the column tiles
    const int64_t gx = std::min<int64_t>(tiles, std::max<int64_t>((int64_t)sms * std::max(per, 1) / ny, 1));
    k_encode<<<dim3((unsigned)gx, (unsigned)ny), EN_THREADS, dyn, st>>>(X, ldx, nrows, d, A, LK, W, o);
    dl_count_launch();
    DL_CUDA(cudaGetLastError());
  } else {
    // batches below two waves of 64-row tiles take 16-row tiles
    int dev = 0, sms = 0;
    DL_CUDA(cudaGetDevice(&dev));
    DL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t ny = ceil_div(LK, W);
    if (ceil_div(nrows, PJ_ROWS) * ny < 2 * (int64_t)sms) {
      dim3 grid((unsigned)ceil_div(nrows, 16), (unsigned)ny);
      k_project<MODE, 1><<<grid, PJ_THREADS, 0, st>>>(X, ldx, rows, nrows, d, A, LK, W, o);
    } else {
      dim3 grid((unsigned)ceil_div(nrows, PJ_ROWS), (unsigned)ny);
      k_project<MODE, PJ_ROWS / 16><<<grid, PJ_THREADS, 0, st>>>(X, ldx, rows, nrows, d, A, LK, W, o);
    }
    dl_count_launch();
    DL_CUDA(cudaGetLastError());
  }
  k_project_exact<MODE><<<2048, 256, 0, st>>>(X, ldx, rows, nrows, d, A, LK, o);
  dl_count_launch();
  DL_CUDA(cudaGetLastError());
  return DETLSH_OK;
}

int project_rows(const float *X, int64_t ldx, const uint32_t *rows, int64_t nrows, int d,
                 const float *A, int LK, int mode, ProjArgs o, cudaStream_t st) {
  switch (mode) {
    case 0: return project_impl<0>(X, ldx, rows, nrows, d, A, LK, o, st);
    case 1: return project_impl<1>(X, ldx, rows, nrows, d, A, LK, o, st);
    case 2: return project_impl<2>(X, ldx, rows, nrows, d, A, LK, o, st);
  }
  return DETLSH_ERR_INVALID_ARG;
}

}  // namespace dl
