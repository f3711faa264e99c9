// Split-precision FP64 GEMM on the BF16 tensor cores (tcgen05 + TMEM + TMA),
// the Ozaki scheme: every FP64 operand row (of op(A)) / column (of op(B)) is
// scaled by a power of two 2^e so that its entries lie in (-1/2, 1/2), rounded
// to the fixed-point integer N = round(x 2^(6S - e)) and written in S balanced
// base-64 digits,
//     x 2^-e = sum_{s=1..S} d_s 2^{-6s} (+ rounding below 2^{-6S-1}),   |d_s| <= 32,
// each stored pre-scaled (d_s 2^{-6s}) as BF16, which holds it exactly.  A
// product is the sum over digit pairs (s, t) with s + t <= S + 2 of BF16 x BF16
// GEMMs (53 for S = 9: the pairs at level S + 2 dominate the error of the ones
// left out, so keeping them cuts it by about twenty).  Balanced digits make the dropped pairs and the rounding zero-mean
// (truncated digits bias every term of a Gram diagonal the same way) and keep
// |d_s d_t| <= 2^10, so a level (fixed s + t) of p pairs summed over k terms
// stays below p k 2^10 units of its last place: exact in FP32 while that is
// <= 2^24.  Levels 2..8 (p <= 7) therefore accumulate exactly in their own TMEM
// accumulator over K-chunks of 2048; the levels >= 9 share one FP32
// accumulator, whose rounding lies 2^-42 below the leading level.  After every
// chunk the epilogue adds the exact levels to an int64 counting units of 2^-48
// and the merged one to a float; at the end it joins them with one FMA and
// applies 2^(e_i + f_j) through the exponent field, alpha and beta in FP64.
// Accuracy: |C - AB| <~ 8 sqrt(K) 2^-6S max|A_i.| max|B_.j|, dominated by the
// rounding of N against a row maximum in [1/4, 1/2) (S = 9: FP64 grade).
//
// FP16 form: FP16 has three more significand bits than BF16 but
// cannot hold a digit pre-scaled by 2^-7s (its range ends at 2^-24), so its
// slices are the raw balanced base-128 digits, |d_s| <= 64 (exact in FP16).
// S = 8 slices (56 bits) and the pairs with s + t <= S + 1 = 9: 36 slice-pair
// products instead of 53.  Every level L = 2..9 keeps its own accumulator of
// raw integer products, |d_s d_t| <= 2^12, exact in FP32 over K-chunks of 512
// (8 pairs x 512 x 2^12 = 2^24); the epilogue adds levels 2..7 to an int64 of
// 2^-49 units (shifted by 49 - 7L) and levels 8 and 9 to one float in 2^-56
// units, joined as iacc + f 2^-7 before the scale 2^(e_i + f_j - 49).  The
// error is the BF16 form's (CPU model: 1.43e-15 against 1.40e-15 of the row and
// column maxima on the same operands).
//
// FP8 form (E4M3, tcgen05 kind::f8f6f4): E4M3 holds every integer |d| <= 16
// exactly but nothing pre-scaled below 2^-9, so its slices are raw balanced
// base-32 digits, |d_s| <= 16: S = 11 slices (55 bits) and the pairs with
// s + t <= S + 2 = 13 (76 slice pairs, 38 16-bit-product equivalents at FP8's
// doubled rate; dropping level 13 would multiply the error by five).
// |d_s d_t| <= 2^8, so a level of p <= 11 pairs stays exact in FP32 over
// K-chunks of 4096.  Each of the 12 levels keeps its own accumulator of BN = 32
// columns (384 of TMEM's 512); the epilogue adds levels 2..9 to an int64 of
// 2^-48 units and levels 10..13 to one float in 2^-65 units, joined as
// iacc + f 2^-17.  A K block is 128 one-byte elements, the same 128-byte
// swizzled rows as the 16-bit forms, and one MMA takes K = 32 (32 bytes), so
// the shared-memory layout and descriptors are the 16-bit forms' byte for byte.
// The slice planes take 11 bytes per element against 18.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <mutex>

#include "tc_ptx.cuh"
#include "zolo_internal.h"

namespace zolo {
namespace {

constexpr int kBeta = 6;          // BF16 form: base-64 digits
constexpr int kTileM = 128;
constexpr int kRowBytes = 128;     // one 128-byte swizzle row of K per tile row
// The slice forms: digit width, element bytes (K elements per 128-byte row),
// exact-accumulation span of a level's sums, TMEM accumulators, tile width BN
// and the largest 0-based level s + t kept (1-based S + 2 for BF16 and FP8,
// S + 1 for FP16).  BF16: levels 2..8 exact, >= 9 merged in the last
// accumulator; FP16 and FP8: one accumulator per level.
template <int FORM> struct Form;
template <> struct Form<kFormBF16> {
  static constexpr int kBits = 6, kElem = 2, kChunkK = 2048, kAcc = 8, kBN = 64;
  __host__ __device__ static constexpr int top(int S) { return S; }
};
template <> struct Form<kFormFP16> {
  static constexpr int kBits = 7, kElem = 2, kChunkK = 512, kAcc = 8, kBN = 64;
  __host__ __device__ static constexpr int top(int S) { return S - 1; }
};
template <> struct Form<kFormFP8> {
  static constexpr int kBits = 5, kElem = 1, kChunkK = 4096, kAcc = 12, kBN = 32;
  __host__ __device__ static constexpr int top(int S) { return S; }
};
template <int FORM> __host__ __device__ constexpr int form_bk() { return kRowBytes / Form<FORM>::kElem; }
constexpr int kARing = 4;
constexpr int kFusedSliceK = 2048;  // slicing in one launch per product up to this padded K
constexpr int kGroupM = 8;         // tile rows per CTA group (L2 reuse of the A slices)
constexpr int kEpiWarps = 16;      // four per TMEM lane quarter, each owning a quarter of the columns
constexpr int kThreads = 64 + 32 * kEpiWarps;   // warp 0 TMA, warp 1 MMA, the rest epilogue

// ----------------------------------------------------------------- slicing
// One batch entry per blockIdx.z; operand b starts at X + b * strideX.
// Row i of op(X) (rows x K):  trans = 0: X[i + k ldx] (rows contiguous),
//                             trans = 1: X[k + i ldx] (row contiguous along k).

// e_i with max_k |op(X)_ik| < 2^(e_i - 1) (0 for a zero row).  Integer
// arithmetic on the FP64 bit patterns (|x| orders like its magnitude bits); no
// FP64 pipe work.
__device__ __forceinline__ int exp_above(unsigned long long mag) {
  if (mag == 0) return 0;
  const int ef = (int)(mag >> 52);
  return ef ? ef - 1021 : -1021;   // normal: |x| < 2^(ef-1022); subnormal: < 2^-1022
}

// With ek != nullptr, element (i, k) counts as x 2^(esign ek[k]) (the inner-index
// equilibration): e_i bounds the shifted row.
__global__ void row_exp_kernel(const double* __restrict__ X, int64_t ldx, int64_t strideX, int trans,
                               int rows, int K, int* __restrict__ e_out, int rows_pad,
                               const int* __restrict__ ek, int esign, int K_pad) {
  __shared__ long long red[8][33];
  const double* Xb = X + blockIdx.z * strideX;
  const int* ekb = ek ? ek + blockIdx.z * K_pad : nullptr;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  const unsigned long long kMag = 0x7FFFFFFFFFFFFFFFull;
  // without shifts: the largest magnitude pattern; with shifts: the largest
  // shifted exponent bound (both reduce with max)
  long long mx = ek ? LLONG_MIN : 0;
  auto take = [&](double x, int k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x) & kMag;
    if (!ekb) {
      mx = (long long)b > mx ? (long long)b : mx;
    } else if (b != 0) {
      const long long e = exp_above(b) + esign * ekb[k];
      mx = e > mx ? e : mx;
    }
  };
  auto finish = [&](long long v) -> int {
    if (!ekb) return exp_above((unsigned long long)v);
    return v == LLONG_MIN ? 0 : (int)v;
  };
  if (!trans) {   // 32 rows per block along tx, k split over ty
    const int i = blockIdx.x * 32 + tx;
    if (i < rows)
      for (int k = ty; k < K; k += 8) take(Xb[i + (int64_t)k * ldx], k);
    red[ty][tx] = mx;
    __syncthreads();
    if (ty == 0) {
      for (int y = 1; y < 8; ++y) mx = red[y][tx] > mx ? red[y][tx] : mx;
      if (i < rows_pad) e_out[blockIdx.z * rows_pad + i] = finish(mx);
    }
  } else {        // 8 rows per block, one warp per row, lanes along k
    const int i = blockIdx.x * 8 + ty;
    if (i < rows)
      for (int k = tx; k < K; k += 32) take(Xb[k + (int64_t)i * ldx], k);
    for (int o = 16; o > 0; o >>= 1) {
      const long long t = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = t > mx ? t : mx;
    }
    if (tx == 0 && i < rows_pad) e_out[blockIdx.z * rows_pad + i] = finish(mx);
  }
}

// ek[k] = the exponent bound of column k of the (rows x K) view of op(X)
// (0 for a zero column or k >= K): scaling that column by 2^-ek[k] puts its
// largest magnitude in [1/4, 1/2).
__global__ void col_exp_kernel(const double* __restrict__ X, int64_t ldx, int64_t strideX, int trans,
                               int rows, int K, int* __restrict__ ek, int K_pad) {
  __shared__ unsigned long long red[8][33];
  const double* Xb = X + blockIdx.z * strideX;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  const unsigned long long kMag = 0x7FFFFFFFFFFFFFFFull;
  const int k0 = blockIdx.x * 32;
  if (trans) {    // element (i, k) = X[k + i ldx]: threads along k, rows split over ty
    unsigned long long mx = 0;
    const int k = k0 + tx;
    if (k < K)
      for (int i = ty; i < rows; i += 8) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(Xb[k + (int64_t)i * ldx]) & kMag;
        mx = b > mx ? b : mx;
      }
    red[ty][tx] = mx;
  } else {        // element (i, k) = X[i + k ldx]: one warp per column, lanes along i
    for (int kk = ty; kk < 32; kk += 8) {
      unsigned long long mx = 0;
      const int k = k0 + kk;
      if (k < K)
        for (int i = tx; i < rows; i += 32) {
          const unsigned long long b = (unsigned long long)__double_as_longlong(Xb[i + (int64_t)k * ldx]) & kMag;
          mx = b > mx ? b : mx;
        }
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = t > mx ? t : mx;
      }
      if (tx == 0) red[0][kk] = mx;   // row 0 collects the columns
    }
    __syncthreads();
    if (ty == 0) {
      const int k = k0 + tx;
      if (k < K_pad) ek[blockIdx.z * K_pad + k] = (k < K) ? exp_above(red[0][tx]) : 0;
    }
    return;
  }
  __syncthreads();
  if (ty == 0) {
    unsigned long long mx = red[0][tx];
    for (int y = 1; y < 8; ++y) mx = red[y][tx] > mx ? red[y][tx] : mx;
    const int k = k0 + tx;
    if (k < K_pad) ek[blockIdx.z * K_pad + k] = (k < K) ? exp_above(mx) : 0;
  }
}

// N = round(x 2^(bS - e)) from the bit pattern (|x| < 2^(e-1), so |N| <= 2^(bS-1));
// ties round away from zero.  b = the digit width (6, or 7 for FP16).
template <int S, int B = kBeta>
__device__ __forceinline__ long long fixed_point(double x, int e) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned long long mag = bits & 0x7FFFFFFFFFFFFFFFull;
  if (mag == 0) return 0;
  const int ef = (int)(mag >> 52);
  const unsigned long long M = (mag & ((1ull << 52) - 1)) | (ef ? (1ull << 52) : 0ull);
  const int E = ef ? ef - 1075 : -1074;          // |x| = M 2^E
  const int k = E - e + B * S;                   // |x| < 2^(e-1) keeps k <= bS - 54
  unsigned long long F;
  if (k >= 0) F = k < 11 ? M << k : 0;
  else F = -k < 63 ? (M + (1ull << (-k - 1))) >> (-k) : 0;
  return (bits >> 63) ? -(long long)F : (long long)F;
}

// The S slice values d_s 2^-6s of x against the row bound 2^(ee - 1): balanced
// digits from the least significant one up; the leading digit takes what is
// left, |d_1| <= 32 because |N| <= 2^(6S-1).  Each is exact in FP32 and BF16
// (at most six significant bits).
template <int S, int FORM>
__device__ __forceinline__ void slice_values(double x, int ee, float* v) {
  constexpr int B = Form<FORM>::kBits;
  constexpr bool raw = FORM != kFormBF16;
  long long N = fixed_point<S, B>(x, ee);
#pragma unroll
  for (int s = S; s >= 2; --s) {
    int d = (int)(N & ((1 << B) - 1));
    d = d >= (1 << (B - 1)) ? d - (1 << B) : d;
    // BF16: the digit pre-scaled by 2^-Bs; FP16 and FP8: the raw digit (scaled
    // in the epilogue)
    v[s - 1] = raw ? (float)d : (float)d * __int_as_float((127 - B * s) << 23);
    N = (N - d) >> B;
  }
  v[0] = raw ? (float)N : (float)N * __int_as_float((127 - B) << 23);
}

// S slices of op(X), each rows_pad x K_pad elements of the form's type (BF16,
// FP16 or E4M3), K contiguous; batch entry b at out + b * S * rows_pad * K_pad,
// slice s (1-based) at + (s-1) * rows_pad * K_pad elements.  32 x 64 tiles
// through shared memory: the read runs along X's contiguous dimension, and each
// thread writes two neighbouring K entries per plane so that a warp stores whole
// 128-byte (16-bit forms) or 64-byte (FP8) lines.  Xb, ob and ekb are the batch
// entry's; er(r) gives the exponent of tile row r (rows i0 + r).
template <int S, int FORM, class ExpOf>
__device__ __forceinline__ void slice_tile(double (*tile)[65], const double* __restrict__ Xb,
                                           int64_t ldx, int trans, int rows, int K, ExpOf er,
                                           uint8_t* __restrict__ ob, int rows_pad, int K_pad,
                                           const int* __restrict__ ekb, int esign, int i0, int k0) {
  constexpr int kE = Form<FORM>::kElem;
  const size_t plane = (size_t)rows_pad * K_pad;  // elements
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  if (!trans) {     // rows contiguous: tx runs along i
    const int i = i0 + tx;
    for (int r = ty; r < 64; r += 8) {
      const int k = k0 + r;
      tile[tx][r] = (i < rows && k < K) ? Xb[i + (int64_t)k * ldx] : 0.0;
    }
  } else {          // K contiguous: tx runs along k
    for (int r = ty; r < 32; r += 8) {
      const int i = i0 + r;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = k0 + h * 32 + tx;
        tile[r][h * 32 + tx] = (i < rows && k < K) ? Xb[k + (int64_t)i * ldx] : 0.0;
      }
    }
  }
  __syncthreads();
  const int kl = 2 * tx, k = k0 + kl;             // this thread's two K entries
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r;
    if (i >= rows_pad) continue;
    float va[S], vb[S];
    if (i < rows) {
      // element x 2^(esign ek[k]) against the row bound 2^(e_i - 1)
      const int ei = er(r);
      const int ea = ekb ? ei - esign * ekb[k] : ei;
      const int eb2 = ekb ? ei - esign * ekb[k + 1] : ei;
      slice_values<S, FORM>(tile[r][kl], ea, va);
      slice_values<S, FORM>(tile[r][kl + 1], eb2, vb);
    } else {
#pragma unroll
      for (int s = 0; s < S; ++s) va[s] = vb[s] = 0.f;
    }
    uint8_t* o = ob + ((size_t)i * K_pad + k) * kE;
    if (FORM == kFormFP8) {   // two E4M3 bytes per plane (|d| <= 16: exact)
#pragma unroll
      for (int s = 0; s < S; ++s)
        *reinterpret_cast<__nv_fp8x2_storage_t*>(o + s * plane) =
            __nv_cvt_float2_to_fp8x2(make_float2(va[s], vb[s]), __NV_SATFINITE, __NV_E4M3);
    } else if (FORM == kFormFP16) {
#pragma unroll
      for (int s = 0; s < S; ++s)
        *reinterpret_cast<__half2*>(o + s * plane * 2) = __floats2half2_rn(va[s], vb[s]);
    } else {
#pragma unroll
      for (int s = 0; s < S; ++s)
        *reinterpret_cast<__nv_bfloat162*>(o + s * plane * 2) = __floats2bfloat162_rn(va[s], vb[s]);
    }
  }
}

// One 32 x 64 tile per block, with the row exponents row_exp_kernel wrote.
template <int S, int FORM>
__global__ void __launch_bounds__(256)
slice_kernel(const double* __restrict__ X, int64_t ldx, int64_t strideX, int trans,
             int rows, int K, const int* __restrict__ e_in,
             uint8_t* __restrict__ out, int rows_pad, int K_pad,
             const int* __restrict__ ek, int esign) {
  __shared__ double tile[32][65];                 // [row][k]
  const int* eb = e_in + blockIdx.z * rows_pad + blockIdx.y * 32;
  const size_t plane = (size_t)rows_pad * K_pad;
  slice_tile<S, FORM>(tile, X + blockIdx.z * strideX, ldx, trans, rows, K,
                      [&](int r) { return eb[r]; },
                      out + (size_t)blockIdx.z * S * plane * Form<FORM>::kElem, rows_pad, K_pad,
                      ek ? ek + blockIdx.z * K_pad : nullptr, esign, blockIdx.y * 32,
                      blockIdx.x * 64);
}

// One operand of a fused slicing launch.
struct SliceOp {
  const double* X;
  int64_t ldx, strideX;
  int trans, rows, rows_pad, esign;
  int* e;                   // row exponents out (batch x rows_pad)
  uint8_t* out;             // slice planes
};

// Row exponents and slices of both operands of a product in one launch: block
// x < nblk_a takes 32 rows of op(A), the rest 32 rows of op(B)^T, blockIdx.z the
// batch entry.  The block first finds its rows' exponents (the max over all K,
// as row_exp_kernel), keeps them in shared memory, then slices its rows tile by
// tile along K: one launch instead of four for the small products, whose K runs
// are short (the caller uses it for K_pad <= 2048).
template <int S, int FORM>
__global__ void __launch_bounds__(256)
slice_fused_kernel(const SliceOp a, const SliceOp b, int nblk_a, int K, int K_pad,
                   const int* __restrict__ ek) {
  __shared__ double tile[32][65];
  __shared__ long long red[8][33];
  __shared__ int es[32];
  const bool on_b = (int)blockIdx.x >= nblk_a;
  const SliceOp o = on_b ? b : a;
  const int i0 = (on_b ? (int)blockIdx.x - nblk_a : (int)blockIdx.x) * 32;
  const double* Xb = o.X + blockIdx.z * o.strideX;
  const int* ekb = ek ? ek + blockIdx.z * K_pad : nullptr;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  const unsigned long long kMag = 0x7FFFFFFFFFFFFFFFull;
  // the row bound as row_exp_kernel forms it: the largest magnitude pattern, or
  // with the inner-index shifts the largest shifted exponent bound
  auto take = [&](long long& mx, double x, int k) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x) & kMag;
    if (!ekb) {
      mx = (long long)bits > mx ? (long long)bits : mx;
    } else if (bits != 0) {
      const long long e = exp_above(bits) + o.esign * ekb[k];
      mx = e > mx ? e : mx;
    }
  };
  auto finish = [&](long long v) -> int {
    if (!ekb) return exp_above((unsigned long long)v);
    return v == LLONG_MIN ? 0 : (int)v;
  };
  if (!o.trans) {   // rows contiguous: tx runs along i, k split over ty
    const int i = i0 + tx;
    long long mx = ekb ? LLONG_MIN : 0;
    if (i < o.rows)
      for (int k = ty; k < K; k += 8) take(mx, Xb[i + (int64_t)k * o.ldx], k);
    red[ty][tx] = mx;
    __syncthreads();
    if (ty == 0) {
      for (int y = 1; y < 8; ++y) mx = red[y][tx] > mx ? red[y][tx] : mx;
      es[tx] = finish(mx);
    }
  } else {          // K contiguous: one warp per row, lanes along k
    for (int r = ty; r < 32; r += 8) {
      const int i = i0 + r;
      long long mx = ekb ? LLONG_MIN : 0;
      if (i < o.rows)
        for (int k = tx; k < K; k += 32) take(mx, Xb[k + (int64_t)i * o.ldx], k);
      for (int s = 16; s > 0; s >>= 1) {
        const long long t = __shfl_xor_sync(0xffffffffu, mx, s);
        mx = t > mx ? t : mx;
      }
      if (tx == 0) es[r] = finish(mx);
    }
  }
  __syncthreads();
  if (ty == 0 && i0 + tx < o.rows_pad) o.e[blockIdx.z * o.rows_pad + i0 + tx] = es[tx];
  const size_t plane = (size_t)o.rows_pad * K_pad;
  uint8_t* ob = o.out + (size_t)blockIdx.z * S * plane * Form<FORM>::kElem;
  for (int k0 = 0; k0 < K_pad; k0 += 64) {
    slice_tile<S, FORM>(tile, Xb, o.ldx, o.trans, o.rows, K, [&](int r) { return es[r]; }, ob,
                        o.rows_pad, K_pad, ekb, o.esign, i0, k0);
    __syncthreads();   // the tile is refilled
  }
}

// ----------------------------------------------------------------- GEMM
// The epilogue's conversions by integer operations: FP64 instructions, int64
// and float conversions to FP64 among them, go through the FP64 units, the
// scarce ones on this part, and the epilogue of a product with a short K does
// as much FP64 work per output as its MMAs do tensor work.

// x 2^k for an int64 x, rounded to nearest (ties to even) like (double)x, then
// scaled exactly: the leading one found by a count of leading zeros, 53 bits
// kept, the exponent assembled; a result outside the normal range takes the
// FP64 route.
__device__ __forceinline__ double i64_scaled(long long x, int k) {
  if (x == 0) return 0.0;
  const unsigned long long sgn = x < 0 ? 0x8000000000000000ull : 0ull;
  const unsigned long long a = x < 0 ? 0ull - (unsigned long long)x : (unsigned long long)x;
  int msb = 63 - __clzll((long long)a);
  unsigned long long m;
  if (msb <= 52) {
    m = a << (52 - msb);
  } else {
    const int sh = msb - 52;
    const unsigned long long rem = a & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    m = a >> sh;
    if (rem > half || (rem == half && (m & 1ull))) {
      ++m;
      if (m >> 53) {
        m >>= 1;
        ++msb;
      }
    }
  }
  const int be = msb + k + 1023;
  if (be <= 0 || be >= 2047) return ldexp((double)x, k);
  return __longlong_as_double((long long)(sgn | ((unsigned long long)be << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

// f 2^k for a float f, exact: the float's fields moved into an FP64 pattern
// (zero keeps its sign; subnormal floats and results outside the normal range
// take the FP64 route).
__device__ __forceinline__ double f32_scaled(float f, int k) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sgn = (unsigned long long)(u >> 31) << 63;
  if ((u & 0x7FFFFFFFu) == 0) return __longlong_as_double((long long)sgn);
  const int ef = (int)((u >> 23) & 0xFFu);
  const int be = ef - 127 + k + 1023;
  if (ef == 0 || ef == 255 || be <= 0 || be >= 2047) return ldexp((double)f, k);
  return __longlong_as_double(
      (long long)(sgn | ((unsigned long long)be << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

struct SplitEpi {
  double* C;                // output (column-major), per-batch stride
  int64_t ldc, strideC;
  const double* Cin;
  int64_t ldcin, strideCin;
  double beta;
  double alpha[kGemmMaxBatch];
  const int* ea;            // row exponents, batch-major (batch x Mpad)
  const int* eb;            // column exponents (batch x Npad)
  int M, N, K, Mpad, Npad;
  int batch, reduce, swap;  // swap: the tile computes C^T (rows of the tile are columns of C)
  int* err;
  int stall;                // test hook: the MMA issuer first waits on a barrier nothing completes
  long long stall_ns;
  int nan_rows;             // an exponent of 1026 marks a row or column with an Inf or NaN
                            // (off with the inner-index equilibration, whose shifted
                            // exponents may exceed it)
};

template <int BN, int S>
struct SmemLayout {
  static constexpr int kBTile = BN * 128;          // bytes of one B slice tile (BN rows of 128 bytes)
  static constexpr int kBStage = S * kBTile;
  static constexpr int kATile = kTileM * 128;      // 16 KB
  static constexpr int kOffB = 0;
  static constexpr int kOffA = 2 * kBStage;
  static constexpr int kOffBar = kOffA + kARing * kATile;
  static constexpr int kBars = 2 + 2 + 2 * kARing + 3 + 1;   // the last: never completed
  static constexpr int kBytes = kOffBar + kBars * 8 + 16;
  static constexpr int kAlloc = kBytes + 1024;     // slack for 1024-byte alignment
};

template <int BN, int S, int FORM>
__global__ void __launch_bounds__(kThreads, 1)
split_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const SplitEpi p) {
  using L = SmemLayout<BN, S>;
  using F = Form<FORM>;
  constexpr int kChunkK = F::kChunkK;
  constexpr int kBK = form_bk<FORM>();
  constexpr int kAcc = F::kAcc;
  static_assert(kAcc * BN <= 512, "the level accumulators must fit in TMEM");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sB = sm + L::kOffB;
  uint8_t* sA = sm + L::kOffA;
  uint64_t* bar = (uint64_t*)(sm + L::kOffBar);
  uint64_t* bfull = bar;
  uint64_t* bempty = bar + 2;
  uint64_t* afull = bar + 4;
  uint64_t* aempty = afull + kARing;
  uint64_t* tfull = aempty + kARing;
  uint64_t* tempty = tfull + 1;
  uint64_t* tdone = tfull + 2;
  uint64_t* never = tfull + 3;         // initialised, never arrived at (test hook)
  uint32_t* tslot = (uint32_t*)(bar + L::kBars);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // CTAs in groups of kGroupM tile rows: one wave covers kGroupM rows of A
  // tiles (kept in L2) while B streams, instead of all of B for two rows
  int tm, tn;
  {
    const int num_n = gridDim.x, num_m = gridDim.y;
    const int pid = blockIdx.y * num_n + blockIdx.x;
    const int first_m = pid / (kGroupM * num_n) * kGroupM;
    const int gm = num_m - first_m < kGroupM ? num_m - first_m : kGroupM;
    const int idx = pid - first_m * num_n;
    tm = first_m + idx % gm;
    tn = idx / gm;
  }
  const int m0 = tm * kTileM, n0 = tn * BN;
  const int nkb = (p.K + kBK - 1) / kBK;
  const int nchunk_k = (nkb + (kChunkK / kBK) - 1) / (kChunkK / kBK);
  const int b_first = p.reduce ? 0 : blockIdx.z;
  const int b_last = p.reduce ? p.batch : blockIdx.z + 1;
  const int nchunks = nchunk_k * (b_last - b_first);
  int* err = p.err;

  if (threadIdx.x == 0) {
    tc::prefetch_tmap(&tmA);
    tc::prefetch_tmap(&tmB);
    for (int i = 0; i < 2; ++i) { tc::mbar_init(&bfull[i], 1); tc::mbar_init(&bempty[i], 1); }
    for (int i = 0; i < kARing; ++i) { tc::mbar_init(&afull[i], 1); tc::mbar_init(&aempty[i], 1); }
    tc::mbar_init(tfull, 1);
    tc::mbar_init(tempty, kEpiWarps);
    tc::mbar_init(tdone, 1);
    tc::mbar_init(never, 1);
    tc::fence_barrier_init();
  }
  if (warp == 1) tc::tmem_alloc<512>(tslot);
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    int kbg = 0, ia = 0;
    bool ok = true;
    int kbg_armed = 0, ia_armed = 0;   // loads issued (for the error-path drain)
    for (int b = b_first; b < b_last && ok; ++b) {
      const int arow = b * S * p.Mpad + m0, brow = b * S * p.Npad + n0;
      for (int kb = 0; kb < nkb && ok; ++kb, ++kbg) {
        const int sb = kbg & 1;
        if (kbg >= 2 && !(ok = tc::mbar_wait(&bempty[sb], ((kbg >> 1) & 1) ^ 1, err))) break;
        tc::mbar_arrive_expect_tx(&bfull[sb], L::kBStage);
        kbg_armed = kbg + 1;
        for (int t = 0; t < S; ++t)
          tc::tma_load_2d(sB + sb * L::kBStage + t * L::kBTile, &tmB, &bfull[sb], kb * kBK,
                          brow + t * p.Npad);
        for (int s = 0; s < S; ++s, ++ia) {
          const int sa = ia % kARing;
          if (ia >= kARing && !(ok = tc::mbar_wait(&aempty[sa], ((ia / kARing) & 1) ^ 1, err))) break;
          tc::mbar_arrive_expect_tx(&afull[sa], L::kATile);
          ia_armed = ia + 1;
          tc::tma_load_2d(sA + sa * L::kATile, &tmA, &afull[sa], kb * kBK, arow + s * p.Mpad);
        }
      }
    }
    if (*(volatile int*)err) {
      // something failed: wait (bounded) until every load this thread issued has landed
      for (int k = kbg_armed > 2 ? kbg_armed - 2 : 0; k < kbg_armed; ++k)
        tc::mbar_wait_drain(&bfull[k & 1], (k >> 1) & 1);
      for (int k = ia_armed > kARing ? ia_armed - kARing : 0; k < ia_armed; ++k)
        tc::mbar_wait_drain(&afull[k % kARing], (k / kARing) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    // One thread issues 4 MMAs per slice pair and K block (32 bytes of K each):
    // the descriptors are formed once and advanced by adding to their
    // start-address field (address >> 4, 14 bits; shared addresses stay below
    // 256 KB so no carry leaves the field), and the slice-pair loops are unrolled.
    const uint32_t idesc = FORM == kFormFP8    ? tc::idesc_e4m3_f32(kTileM, BN)
                           : FORM == kFormFP16 ? tc::idesc_f16_f32(kTileM, BN)
                                               : tc::idesc_bf16_f32(kTileM, BN);
    const uint64_t adesc0 = tc::sdesc_k128(tc::smem_u32(sA));
    const uint64_t bdesc0 = tc::sdesc_k128(tc::smem_u32(sB));
    int kbg = 0, ia = 0;
    bool ok = true;
    if (p.stall) {
      tc::mbar_stall(never, err, p.stall_ns);
      ok = false;
    }
    for (int c = 0; c < nchunks && ok; ++c) {
      if (c > 0 && !(ok = tc::mbar_wait(tempty, (c - 1) & 1, err))) break;
      tc::tc_fence_after();
      uint32_t fresh = (1u << kAcc) - 1;   // accumulator a starts (accumulate = 0) at its first MMA
      const int kc = c % nchunk_k;
      const int kb_end = min(nkb, (kc + 1) * (kChunkK / kBK));
      for (int kb = kc * (kChunkK / kBK); kb < kb_end && ok; ++kb, ++kbg) {
        const int sb = kbg & 1;
        if (!(ok = tc::mbar_wait(&bfull[sb], (kbg >> 1) & 1, err))) break;
        tc::tc_fence_after();
        const uint64_t bd = bdesc0 + (uint64_t)((sb * L::kBStage) >> 4);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const int sa = ia % kARing;
          if (!(ok = tc::mbar_wait(&afull[sa], (ia / kARing) & 1, err))) break;
          ++ia;
          tc::tc_fence_after();
          const uint64_t ad = adesc0 + (uint64_t)((sa * L::kATile) >> 4);
          constexpr int kTop = F::top(S);   // largest s + t (0-based) kept
#pragma unroll
          for (int t = 0; t < (kTop - s + 1 < S ? kTop - s + 1 : S); ++t) {
            const int lvl = s + t;                 // 0 -> level 2
            // FP16 and FP8: one accumulator per level (raw digits of different
            // scales must not share one); BF16: levels >= 9 share the last
            const int acc = FORM != kFormBF16 ? lvl : (lvl < kAcc - 1 ? lvl : kAcc - 1);
            const uint32_t d = tmem + acc * BN;
            const uint64_t bt = bd + (uint64_t)((t * L::kBTile) >> 4);
            const uint32_t first = (fresh >> acc) & 1u;
#pragma unroll
            for (int kk = 0; kk < kRowBytes / 32; ++kk) {
              const uint32_t accum = (first && kk == 0) ? 0u : 1u;
              if (FORM == kFormFP8) tc::mma_f8(d, ad + 2 * kk, bt + 2 * kk, idesc, accum);
              else tc::mma_bf16(d, ad + 2 * kk, bt + 2 * kk, idesc, accum);
            }
            fresh &= ~(1u << acc);
          }
          tc::mma_commit(&aempty[sa]);
        }
        tc::mma_commit(&bempty[sb]);
      }
      tc::mma_commit(tfull);
    }
    tc::mma_commit(tdone);   // arrives once every MMA issued above has completed
  } else if (warp >= 2) {
    // ---------------- epilogue: drain chunks into integer accumulators
    // Level L (2..8) of a chunk is an integer multiple of 2^-6L below 2^24 of
    // those units, so it is added exactly to an int64 counting units of 2^-48
    // (per chunk below 2^57.1: exact for 56 chunks, so gemm_split cuts a longer
    // K into products of at most 56 x 2048).  The merged
    // levels >= 9 go into a float, 2^-42 below the leading level.  FP64 is used
    // only when a batch entry's result is written (two conversions, one FMA, the
    // beta term; the power-of-two scale goes into the exponent field).
    constexpr int HALF = BN / (kEpiWarps / 4);     // columns of this warp
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;              // which column slice
    const int row = m0 + q * 32 + lane;            // tile row
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    long long iacc[HALF];
    float fm[HALF];
#pragma unroll
    for (int j = 0; j < HALF; ++j) {
      iacc[j] = 0;
      fm[j] = 0.f;
    }
    bool ok = true;
    const int z = p.reduce ? 0 : blockIdx.z;
    double* C = p.C + (int64_t)z * p.strideC;
    const double* Cin = p.Cin ? p.Cin + (int64_t)z * p.strideCin : nullptr;
    for (int c = 0; c < nchunks; ++c) {
      if (!(ok = tc::mbar_wait(tfull, c & 1, err))) break;
      tc::tc_fence_after();
      // one TMEM load (and one wait for it) per 16 columns where the warp has 16
      constexpr int kLd = HALF % 16 == 0 ? 16 : 8;
#pragma unroll
      for (int a = 0; a < kAcc; ++a) {
#pragma unroll
        for (int g = 0; g < HALF / kLd; ++g) {
          float v[kLd];
          if constexpr (kLd == 16) tc::tmem_ld16(tmem + lane_off + a * BN + half * HALF + g * kLd, v);
          else tc::tmem_ld8(tmem + lane_off + a * BN + half * HALF + g * kLd, v);
          if (FORM == kFormFP8) {
            // raw integer level sums (|.| <= 2^24): levels 2..9 into 2^-48 units
            // (level 2 of a 4096-chunk is below 2^20: 2^58 per chunk, so about
            // 29 chunks fit); levels 10..13 into one float in units of 2^-65
            // (times 2^(65 - 5L), exact)
            const int L = a + 2;
#pragma unroll
            for (int i = 0; i < kLd; ++i) {
              if (L <= 9) iacc[g * kLd + i] += (long long)__float2int_rn(v[i]) << (48 - 5 * L);
              else fm[g * kLd + i] += v[i] * __int_as_float((127 + 65 - 5 * L) << 23);
            }
          } else if (FORM == kFormFP16) {
            // raw integer level sums (|.| <= 2^24): levels 2..7 into 2^-49 units;
            // levels 8 and 9 into one float in units of 2^-56 (level 9 times
            // 2^-7, exact), whose rounding lies about 2^-56 below the leading level
            const int L = a + 2;
#pragma unroll
            for (int i = 0; i < kLd; ++i) {
              if (L <= 7) iacc[g * kLd + i] += (long long)__float2int_rn(v[i]) << (49 - 7 * L);
              else if (L == 8) fm[g * kLd + i] += v[i];
              else fm[g * kLd + i] += v[i] * 0x1p-7f;
            }
          } else if (a < kAcc - 1) {
            const int L = a + 2;
            // times 2^6L: an exact integer below 2^24
            const float up = __int_as_float((127 + kBeta * L) << 23);
#pragma unroll
            for (int i = 0; i < kLd; ++i)
              iacc[g * kLd + i] += (long long)__float2int_rn(v[i] * up) << (48 - kBeta * L);
          } else {
            // merged levels >= 9 stay in a float (2^-24 of a value 2^-30 below the
            // leading level: rounding them to the int64's unit would cost 2^-49)
#pragma unroll
            for (int i = 0; i < kLd; ++i) fm[g * kLd + i] += v[i];
          }
        }
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(tempty);
      // end of a batch entry: scale, combine with beta C_in (first entry) or with
      // the running sum already in C (reduce mode), write, reset
      if ((c + 1) % nchunk_k == 0) {
        const int b = b_first + c / nchunk_k;
        const bool first = c / nchunk_k == 0;
        const int ei = p.ea[b * p.Mpad + row];
        const int* ebb = p.eb + b * p.Npad + n0 + half * HALF;
        const double al = p.alpha[b];
        // eight outputs at a time: their addends (beta C_in, or the running sum
        // in reduce mode) loaded together first, then formed and stored (a load
        // after a store to C could alias it, so a plain loop waits for each)
        const bool use_cin = Cin && p.beta != 0.0;
#pragma unroll
        for (int j0 = 0; j0 < HALF; j0 += 8) {
          double add[8];
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int col = n0 + half * HALF + j0 + jj;
            const int ci = p.swap ? col : row, cj = p.swap ? row : col;
            add[jj] = 0.0;
            if (row < (p.swap ? p.N : p.M) && col < (p.swap ? p.M : p.N)) {
              if (!first) add[jj] = C[ci + (int64_t)cj * p.ldc];
              else if (use_cin) add[jj] = Cin[ci + (int64_t)cj * p.ldcin];
            }
          }
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int j = j0 + jj;
            const int col = n0 + half * HALF + j;
            const int ci = p.swap ? col : row, cj = p.swap ? row : col;
            if (row < (p.swap ? p.N : p.M) && col < (p.swap ? p.M : p.N)) {
              // the integer part and the float part, each scaled by the power of
              // two 2^(e_i + f_j) in its exponent field, joined by one FP64 add
              // (the same single rounding as converting the int64 and adding the
              // float part at its weight)
              const int ej = __ldg(ebb + j), e = ei + ej;
              double v;
              if (FORM == kFormFP8)
                v = i64_scaled(iacc[j], e - 48) + f32_scaled(fm[j], e - 48 - 17);
              else if (FORM == kFormFP16)
                v = i64_scaled(iacc[j], e - 49) + f32_scaled(fm[j], e - 49 - 7);
              else
                v = i64_scaled(iacc[j], e - 48) + f32_scaled(fm[j], e);
              // an Inf or NaN in the row of op(A) or the column of op(B): the
              // digits carry no value, so the output is NaN (as the FP64 product
              // gives NaN or Inf there)
              if (p.nan_rows && (ei >= 1026 || ej >= 1026)) v = __longlong_as_double(0x7FF8000000000000ll);
              if (al == -1.0) v = __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ull);
              else if (al != 1.0) v *= al;
              if (first) {
                if (use_cin) v = fma(p.beta, add[jj], v);
              } else {
                v += add[jj];
              }
              C[ci + (int64_t)cj * p.ldc] = v;
            }
            iacc[j] = 0;
            fm[j] = 0.f;
          }
        }
      }
    }
    (void)ok;
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    if (lane == 0) tc::mbar_wait_drain(tdone, 0);
    __syncwarp();
    tc::tc_fence_after();
    tc::tmem_dealloc<512>(tmem);
  }
}

// ----------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &f, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)f;
  });
  return fn;
}

// 2-D map over a (rows x K_pad) matrix of the form's slice type, K contiguous,
// box of one 128-byte row (64 16-bit or 128 one-byte elements) x box_rows,
// 128-byte swizzle
template <int FORM>
bool make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t K_pad, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K_pad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)K_pad * Form<FORM>::kElem};
  cuuint32_t box[2] = {(cuuint32_t)form_bk<FORM>(), (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  const CUtensorMapDataType ty = FORM == kFormFP8    ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                 : FORM == kFormFP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                     : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  return enc(m, ty, 2,
             const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

template <int S, int FORM>
cudaError_t slice_operand(const double* X, int64_t ldx, int64_t strideX, int trans, int rows, int K,
                          int batch, int* e, uint8_t* out, int rows_pad, int K_pad,
                          const int* ek, int esign, cudaStream_t st) {
  {
    ProfScope ps(kProfSlice, st, 0.0, 8.0 * batch * rows * (double)K);
    if (!trans) {
      ps.blocks((const void*)row_exp_kernel, dim3(32, 8), 0, dim3((rows_pad + 31) / 32, 1, batch));
      row_exp_kernel<<<dim3((rows_pad + 31) / 32, 1, batch), dim3(32, 8), 0, st>>>(
          X, ldx, strideX, 0, rows, K, e, rows_pad, ek, esign, K_pad);
    } else {
      ps.blocks((const void*)row_exp_kernel, dim3(32, 8), 0, dim3((rows_pad + 7) / 8, 1, batch));
      row_exp_kernel<<<dim3((rows_pad + 7) / 8, 1, batch), dim3(32, 8), 0, st>>>(
          X, ldx, strideX, 1, rows, K, e, rows_pad, ek, esign, K_pad);
    }
  }
  ProfScope ps(kProfSlice, st, 0.0,
               (8.0 + (double)Form<FORM>::kElem * S) * batch * rows_pad * (double)K_pad);
  dim3 grid((unsigned)(K_pad / 64), (unsigned)(rows_pad / 32), batch);
  ps.blocks((const void*)slice_kernel<S, FORM>, dim3(32, 8), 0, dim3(grid));
  slice_kernel<S, FORM><<<grid, dim3(32, 8), 0, st>>>(X, ldx, strideX, trans, rows, K, e, out,
                                                      rows_pad, K_pad, ek, esign);
  return cudaGetLastError();
}

template <int BN, int S, int FORM>
cudaError_t run_split(const GemmArgs& g, SplitWork& w, cudaStream_t st) {
  constexpr int kE = Form<FORM>::kElem;
  // orientation: put the larger output dimension on the 128-row tile side
  const bool swap = g.M < kTileM && g.N > g.M;
  const int M = swap ? g.N : g.M, N = swap ? g.M : g.N, K = g.K;
  const int Mpad = (int)round_up(M, kTileM), Npad = (int)round_up(N, BN),
            Kpad = (int)round_up(K, form_bk<FORM>());
  const int nb = g.batch;
  const size_t need_a = (size_t)nb * S * Mpad * Kpad, need_b = (size_t)nb * S * Npad * Kpad;
  const bool keq = g.k_equilibrate != 0;
  // the workspace counts 16-bit units
  if ((need_a + need_b) * kE > w.slice_elems * 2 ||
      (size_t)nb * (Mpad + Npad + (keq ? Kpad : 0)) > w.exp_elems)
    return cudaErrorMemoryAllocation;
  uint8_t* sa = static_cast<uint8_t*>(w.slices);
  uint8_t* sb = sa + need_a * kE;
  int* ea = w.exps;
  int* eb = w.exps + (size_t)nb * Mpad;
  int* ek = keq ? eb + (size_t)nb * Npad : nullptr;
  cudaError_t err;
  // op(A) rows: M x K.  With swap the tile's A side is op(B)^T (rows = columns of op(B)).
  //   op(A) row i, col k:   transA = 0: A[i + k lda]   transA = 1: A[k + i lda]
  //   op(B)^T row j, col k: transB = 0: B[k + j ldb]   transB = 1: B[j + k ldb]
  const double* Xa = swap ? g.B : g.A;
  const double* Xb = swap ? g.A : g.B;
  const int64_t lda = swap ? g.ldb : g.lda, ldb = swap ? g.lda : g.ldb;
  const int64_t sta = swap ? g.strideB : g.strideA, stb = swap ? g.strideA : g.strideB;
  const int ta = swap ? (g.transB ? 0 : 1) : g.transA;
  const int tb = swap ? g.transA : (g.transB ? 0 : 1);
  // inner-index equilibration: op(B)'s rows k are the columns of the (rows x K)
  // view of the tile's B side (A side when swapped); they are scaled by 2^-ek[k]
  // and op(A)'s columns by 2^+ek[k]
  const int sign_a = swap ? -1 : 1;
  if (keq) {
    ProfScope ps(kProfSlice, st, 0.0, 8.0 * nb * (double)N * K);
    const double* Xo = swap ? Xa : Xb;
    ps.blocks((const void*)col_exp_kernel, dim3(32, 8), 0, dim3((unsigned)(Kpad / 32), 1, nb));
    col_exp_kernel<<<dim3((unsigned)(Kpad / 32), 1, nb), dim3(32, 8), 0, st>>>(
        Xo, swap ? lda : ldb, swap ? sta : stb, swap ? ta : tb, swap ? M : N, K, ek, Kpad);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  if (Kpad <= kFusedSliceK) {
    // short K runs: both operands' exponents and slices in one launch
    const SliceOp oa{Xa, lda, sta, ta, M, Mpad, sign_a, ea, sa};
    const SliceOp ob{Xb, ldb, stb, tb, N, Npad, -sign_a, eb, sb};
    ProfScope ps(kProfSlice, st, 0.0,
                 (16.0 + (double)Form<FORM>::kElem * S) * nb * (double)(Mpad + Npad) * Kpad);
    ps.blocks((const void*)slice_fused_kernel<S, FORM>, dim3(32, 8), 0,
              dim3((unsigned)((Mpad + Npad) / 32), 1, nb));
    slice_fused_kernel<S, FORM><<<dim3((unsigned)((Mpad + Npad) / 32), 1, nb), dim3(32, 8), 0, st>>>(
        oa, ob, Mpad / 32, K, Kpad, ek);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  } else {
    if ((err = slice_operand<S, FORM>(Xa, lda, sta, ta, M, K, nb, ea, sa, Mpad, Kpad, ek, sign_a,
                                      st)) != cudaSuccess)
      return err;
    if ((err = slice_operand<S, FORM>(Xb, ldb, stb, tb, N, K, nb, eb, sb, Npad, Kpad, ek, -sign_a,
                                      st)) != cudaSuccess)
      return err;
  }
  CUtensorMap mA, mB;
  if (!make_map<FORM>(&mA, sa, (int64_t)nb * S * Mpad, Kpad, kTileM) ||
      !make_map<FORM>(&mB, sb, (int64_t)nb * S * Npad, Kpad, BN))
    return cudaErrorInvalidValue;
  SplitEpi p{};
  p.C = g.Cout; p.ldc = g.ldcout; p.strideC = g.strideCout;
  p.Cin = g.Cin; p.ldcin = g.ldcin; p.strideCin = g.strideCin; p.beta = g.beta;
  for (int b = 0; b < kGemmMaxBatch; ++b) p.alpha[b] = g.alpha[b];
  p.ea = ea; p.eb = eb;
  p.M = g.M; p.N = g.N; p.K = K; p.Mpad = Mpad; p.Npad = Npad;
  p.batch = nb; p.reduce = g.reduce; p.swap = swap ? 1 : 0;
  p.err = w.err;
  p.stall = w.stall;
  p.stall_ns = w.stall_ns;
  p.nan_rows = keq ? 0 : 1;
  using L = SmemLayout<BN, S>;
  if ((err = smem_attr_once((const void*)split_gemm_kernel<BN, S, FORM>, L::kAlloc)) != cudaSuccess) {
    if (std::getenv("ZOLO_DEBUG"))
      std::fprintf(stderr, "zolo: cudaFuncSetAttribute(%d B): %s\n", L::kAlloc,
                   cudaGetErrorString(err));
    return err;
  }
  dim3 grid((unsigned)(Npad / BN), (unsigned)(Mpad / kTileM), g.reduce ? 1 : nb);
  ProfScope ps(kProfSplitGemm, st, gemm_flops(g), 0.0);
  ps.blocks((const void*)split_gemm_kernel<BN, S, FORM>, dim3(kThreads), L::kAlloc, dim3(grid));
  split_gemm_kernel<BN, S, FORM><<<grid, kThreads, L::kAlloc, st>>>(mA, mB, p);
  err = cudaGetLastError();
  if (err != cudaSuccess && std::getenv("ZOLO_DEBUG")) {
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, split_gemm_kernel<BN, S, FORM>);
    std::fprintf(stderr,
                 "zolo: split_gemm_kernel<%d,%d> launch (grid %u x %u x %u, %d threads, %d B smem): %s"
                 " [maxThreadsPerBlock %d, numRegs %d, localSizeBytes %zu, maxDynamicSmem %d]\n",
                 BN, S, grid.x, grid.y, grid.z, kThreads, L::kAlloc, cudaGetErrorString(err),
                 fa.maxThreadsPerBlock, fa.numRegs, fa.localSizeBytes,
                 fa.maxDynamicSharedSizeBytes);
  }
  return err;
}

}  // namespace

cudaError_t gemm_split(const GemmArgs& g, SplitWork& w, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.K <= 0 || g.batch > kGemmMaxBatch) return gemm_f64(g, st);
  // The int64 that holds an output's exact level sums has room for a bounded
  // number of K-chunks at the digit bounds (BF16: 2^57.1 per 2048-chunk, FP16:
  // 2^56.1 per 512-chunk, FP8: 2^58.1 per 4096-chunk); a longer K runs as
  // consecutive products whose partial results are added in FP64.
  const int64_t kmax = w.form == kFormFP16 ? 120 * 512 : w.form == kFormFP8 ? 28 * 4096 : 56 * 2048;
  if (g.K > kmax) {
    for (int64_t k0 = 0; k0 < g.K; k0 += kmax) {
      GemmArgs h = g;
      h.K = (int)std::min<int64_t>(kmax, g.K - k0);
      h.A = g.A + (g.transA ? k0 : k0 * g.lda);   // op(A) columns k0..
      h.B = g.B + (g.transB ? k0 * g.ldb : k0);   // op(B) rows k0..
      if (k0 > 0) {
        h.Cin = g.Cout;
        h.ldcin = g.ldcout;
        h.strideCin = g.reduce ? 0 : g.strideCout;
        h.beta = 1.0;
      }
      const cudaError_t e = gemm_split(h, w, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  // batch entries per launch that the slice workspace and the exponent array hold
  const size_t per = split_slice_elems(g.M, g.N, g.K, 1, w.slices_s, w.form);
  const size_t rows = split_exp_elems(g.M, g.N, g.K, 1, g.k_equilibrate, w.form);
  int gs = (int)std::min<size_t>(g.batch, w.slice_elems / std::max<size_t>(per, 1));
  gs = (int)std::min<size_t>((size_t)gs, w.exp_elems / std::max<size_t>(rows, 1));
  if (gs < 1) return cudaErrorMemoryAllocation;
  auto run = [&](const GemmArgs& h) {
    if (w.form == kFormFP8) return run_split<Form<kFormFP8>::kBN, 11, kFormFP8>(h, w, st);
    if (w.form == kFormFP16) return run_split<64, 8, kFormFP16>(h, w, st);
    return w.slices_s == 9 ? run_split<64, 9, kFormBF16>(h, w, st)
                           : run_split<64, 8, kFormBF16>(h, w, st);
  };
  if (gs >= g.batch) return run(g);
  for (int b0 = 0; b0 < g.batch; b0 += gs) {
    GemmArgs h = g;
    h.batch = std::min(gs, g.batch - b0);
    h.A = g.A + b0 * g.strideA;
    h.B = g.B + b0 * g.strideB;
    for (int b = 0; b < h.batch; ++b) h.alpha[b] = g.alpha[b0 + b];
    if (g.reduce) {
      if (b0 > 0) { h.Cin = g.Cout; h.ldcin = g.ldcout; h.strideCin = 0; h.beta = 1.0; }
    } else {
      h.Cout = g.Cout + b0 * g.strideCout;
      if (g.Cin) h.Cin = g.Cin + b0 * g.strideCin;
    }
    cudaError_t e = run(h);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void split_prepare() {
  smem_attr_once((const void*)split_gemm_kernel<64, 8, kFormBF16>, SmemLayout<64, 8>::kAlloc);
  smem_attr_once((const void*)split_gemm_kernel<64, 9, kFormBF16>, SmemLayout<64, 9>::kAlloc);
  smem_attr_once((const void*)split_gemm_kernel<64, 8, kFormFP16>, SmemLayout<64, 8>::kAlloc);
  smem_attr_once((const void*)split_gemm_kernel<Form<kFormFP8>::kBN, 11, kFormFP8>,
                 SmemLayout<Form<kFormFP8>::kBN, 11>::kAlloc);
  encode_fn();
}

thread_local SplitWork* t_split = nullptr;

void set_split_engine(SplitWork* w) { t_split = w; }
SplitWork* get_split_engine() { return t_split; }

// Estimated seconds on GB300 of one call on the FP64 pipe and on the split
// tensor-core path (slicing traffic + output traffic + slice-pair products +
// launch latency).
bool split_preferred(const GemmArgs& g, const SplitWork& w) { return split_time_ratio(g, w) < 1.0; }

namespace {
// The padded tile sides, slice bytes per element and slice-pair products (in
// 16-bit-MMA equivalents: FP8 runs at twice the rate) of one call in a form.
struct SplitShape {
  double ra, rb, kp, elem_bytes, pairs;
};
SplitShape split_shape(const GemmArgs& g, const SplitWork& w) {
  const bool swap = g.M < kTileM && g.N > g.M;
  const bool fp8 = w.form == kFormFP8;
  const double S = w.slices_s;
  SplitShape sh;
  sh.ra = (double)round_up(swap ? g.N : g.M, kTileM);
  sh.rb = (double)round_up(swap ? g.M : g.N, fp8 ? Form<kFormFP8>::kBN : 64);
  sh.kp = (double)round_up(g.K, fp8 ? form_bk<kFormFP8>() : form_bk<kFormBF16>());
  sh.elem_bytes = fp8 ? 1.0 : 2.0;
  // slice pairs: s + t <= S + 2 (BF16, FP8), s + t <= S + 1 (FP16)
  const double pairs = w.form == kFormFP16 ? S * (S + 1) / 2 : S * (S + 1) / 2 + (S - 1);
  sh.pairs = fp8 ? pairs / 2 : pairs;
  return sh;
}
}  // namespace

double split_time_ratio(const GemmArgs& g, const SplitWork& w) {
  const SplitShape sh = split_shape(g, w);
  const double S = w.slices_s;
  const double slice_bytes = g.batch * (8.0 + sh.elem_bytes * S) * (sh.ra + sh.rb) * sh.kp;
  const double out_bytes = (g.reduce ? 1 : g.batch) * 8.0 * g.M * (double)g.N * (g.beta != 0.0 ? 2 : 1);
  const double products = sh.pairs * 2.0 * sh.ra * sh.rb * sh.kp * g.batch;
  if (w.throughput) {
    // GPU-seconds of each path when other calls fill the rest of the chip: the
    // FP64 pipe at its measured 1.2 TFLOP/s, the slice-pair products at 1.7 PFLOP/s
    // of BF16 issue, the slicing and output traffic at 6 TB/s
    return ((slice_bytes + out_bytes) / 6e12 + products / 1.7e15) / (gemm_flops(g) / 1.2e12);
  }
  const double t64 = gemm_flops(g) / 0.9e12;
  const double tsplit = slice_bytes / 4e12 + out_bytes / 5e12 + products / 0.7e15 + 30e-6;
  return tsplit / t64;
}

// Exponents run_split writes: one per padded tile row and column of every batch
// entry, plus one per padded inner index with the equilibration.
size_t split_exp_elems(int64_t M, int64_t N, int64_t K, int batch, int k_equilibrate, int form) {
  const bool swap = M < kTileM && N > M;
  const bool fp8 = form == kFormFP8;
  const int64_t rows = swap ? N : M, cols = swap ? M : N;
  const int64_t bk = fp8 ? form_bk<kFormFP8>() : form_bk<kFormBF16>();
  return (size_t)batch * (size_t)(round_up(rows, kTileM) + round_up(cols, fp8 ? Form<kFormFP8>::kBN : 64) +
                                  (k_equilibrate ? round_up(K, bk) : 0));
}

// Slice planes of one call, in 16-bit units (two FP8 slices per unit).
size_t split_slice_elems(int64_t M, int64_t N, int64_t K, int batch, int S, int form) {
  const bool swap = M < kTileM && N > M;
  const bool fp8 = form == kFormFP8;
  const int64_t rows = swap ? N : M, cols = swap ? M : N;
  const int64_t bk = fp8 ? form_bk<kFormFP8>() : form_bk<kFormBF16>();
  const size_t elems = (size_t)batch * S *
                       (round_up(rows, kTileM) + round_up(cols, fp8 ? Form<kFormFP8>::kBN : 64)) *
                       round_up(K, bk);
  return fp8 ? (elems + 1) / 2 : elems;
}

}  // namespace zolo
