// Split-precision FP64 GEMM on the BF16 tensor cores (tcgen05 + TMEM + TMA),
// the Ozaki scheme: every FP64 operand row (of op(A)) / column (of op(B)) is
// scaled by a power of two 2^e so that its entries lie in (-1, 1), and cut into
// S signed 6-bit digits by truncation,
//     x 2^-e = sum_{s=1..S} d_s 2^{-6s} + O(2^{-6S}),   |d_s| <= 63,
// stored pre-scaled (d_s 2^{-6s}) as BF16, which holds them exactly.  A product
// is then sum over pairs (s, t), s + t <= S + 1, of BF16 x BF16 GEMMs whose
// FP32 accumulation is exact as long as each sum stays below 2^24 units of its
// last place: with |d| <= 63 a level (fixed s + t) of p pairs over k terms needs
// p k 2^12 <= 2^24.  Levels 2..5 (p <= 4) therefore accumulate exactly in their
// own TMEM accumulator over K-chunks of 1024; the levels >= 6 share one FP32
// accumulator whose rounding (2^-24 of a term already 2^-36 below the leading
// level) is below the slicing error.  The epilogue adds the five accumulators in
// FP64 after every chunk and applies 2^(e_i + f_j), alpha and beta.
// Accuracy: |C - AB| <~ K 2^-6S max|A_i.| max|B_.j| (normwise ~2^-48 for S = 8).
#include <cuda.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <mutex>

#include "tc_ptx.cuh"
#include "zolo_internal.h"

namespace zolo {
namespace {

constexpr int kBeta = 6;
constexpr int kTileM = 128;
constexpr int kBK = 64;            // one 128-byte swizzle row of BF16
constexpr int kChunkK = 1024;      // exact-accumulation span of the level sums
constexpr int kARing = 4;
constexpr int kThreads = 192;      // warp 0 TMA, warp 1 MMA, warps 2..5 epilogue

// ----------------------------------------------------------------- slicing
// max-exponent of each row of op(X) (rows x K): e with max|x| < 2^e (0 for a zero row)
__global__ void row_exp_kernel(const double* __restrict__ X, int64_t ldx, int trans, int rows, int K,
                               int* __restrict__ e_out) {
  // trans = 0: op(X) = X (column-major, rows contiguous): one thread per row.
  // trans = 1: op(X) = X^T: row i is column i of X: one warp per row.
  if (!trans) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    double mx = 0.0;
    for (int k = 0; k < K; ++k) mx = fmax(mx, fabs(X[i + (int64_t)k * ldx]));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);
    e_out[i] = e;
  } else {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= rows) return;
    double mx = 0.0;
    for (int k = lane; k < K; k += 32) mx = fmax(mx, fabs(X[k + (int64_t)w * ldx]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);
    if (lane == 0) e_out[w] = e;
  }
}

// S slices of op(X), each rows_pad x K_pad BF16, K contiguous, at out + s*rows_pad*K_pad.
// 32 x 32 tiles through shared memory so that both the read (along X's
// contiguous dimension) and the write (along K) are coalesced.
template <int S>
__global__ void slice_kernel(const double* __restrict__ X, int64_t ldx, int trans, int rows, int K,
                             const int* __restrict__ e_in, __nv_bfloat16* __restrict__ out,
                             int rows_pad, int K_pad) {
  __shared__ double tile[32][33];
  const int i0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    double v = 0.0;
    if (!trans) {   // X[i + k ldx]: tx runs along i
      const int i = i0 + tx, k = k0 + r;
      if (i < rows && k < K) v = X[i + (int64_t)k * ldx];
      tile[tx][r] = v;    // tile[i][k]
    } else {        // X[k + i ldx]: tx runs along k
      const int i = i0 + r, k = k0 + tx;
      if (i < rows && k < K) v = X[k + (int64_t)i * ldx];
      tile[r][tx] = v;
    }
  }
  __syncthreads();
  const size_t plane = (size_t)rows_pad * K_pad;
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, k = k0 + tx;
    if (i >= rows_pad || k >= K_pad) continue;
    double y = (i < rows) ? ldexp(tile[r][tx], -e_in[i]) : 0.0;
    __nv_bfloat16* o = out + (size_t)i * K_pad + k;
#pragma unroll
    for (int s = 1; s <= S; ++s) {
      const double t = y * 64.0;
      const double d = trunc(t);
      y = t - d;
      o[(s - 1) * plane] = __double2bfloat16(ldexp(d, -kBeta * s));
    }
  }
}

// ----------------------------------------------------------------- GEMM
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
};

template <int BN, int S>
struct SmemLayout {
  static constexpr int kBTile = BN * 128;          // bytes of one B slice tile (BN x 64 BF16)
  static constexpr int kBStage = S * kBTile;
  static constexpr int kATile = kTileM * 128;      // 16 KB
  static constexpr int kOffB = 0;
  static constexpr int kOffA = 2 * kBStage;
  static constexpr int kOffBar = kOffA + kARing * kATile;
  static constexpr int kBars = 2 + 2 + 2 * kARing + 3;
  static constexpr int kBytes = kOffBar + kBars * 8 + 16;
  static constexpr int kAlloc = kBytes + 1024;     // slack for 1024-byte alignment
};

template <int BN, int S>
__global__ void __launch_bounds__(kThreads, 1)
split_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const SplitEpi p) {
  using L = SmemLayout<BN, S>;
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
  uint32_t* tslot = (uint32_t*)(bar + L::kBars);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kTileM, n0 = blockIdx.x * BN;
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
    tc::mbar_init(tempty, 4);
    tc::mbar_init(tdone, 1);
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
    const uint32_t idesc = tc::idesc_bf16_f32(kTileM, BN);
    int kbg = 0, ia = 0;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      if (c > 0 && !(ok = tc::mbar_wait(tempty, (c - 1) & 1, err))) break;
      tc::tc_fence_after();
      uint32_t fresh = 0x1F;   // accumulator a starts (accumulate = 0) at its first MMA
      const int kc = c % nchunk_k;
      const int kb_end = min(nkb, (kc + 1) * (kChunkK / kBK));
      for (int kb = kc * (kChunkK / kBK); kb < kb_end && ok; ++kb, ++kbg) {
        const int sb = kbg & 1;
        if (!(ok = tc::mbar_wait(&bfull[sb], (kbg >> 1) & 1, err))) break;
        tc::tc_fence_after();
        const uint32_t b0 = tc::smem_u32(sB + sb * L::kBStage);
        for (int s = 0; s < S; ++s, ++ia) {
          const int sa = ia % kARing;
          if (!(ok = tc::mbar_wait(&afull[sa], (ia / kARing) & 1, err))) break;
          tc::tc_fence_after();
          const uint32_t a0 = tc::smem_u32(sA + sa * L::kATile);
          for (int t = 0; s + t <= S - 1; ++t) {   // level (s+1)+(t+1) <= S+1
            const int lvl = s + t;                 // 0 -> level 2
            const int acc = lvl < 4 ? lvl : 4;
            const uint32_t d = tmem + acc * BN;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint32_t accumulate = ((fresh >> acc) & 1) && kk == 0 ? 0u : 1u;
              tc::mma_bf16(d, tc::sdesc_k128(a0 + kk * 32), tc::sdesc_k128(b0 + t * L::kBTile + kk * 32),
                           idesc, accumulate);
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
    // ---------------- epilogue: drain chunks into FP64 registers
    const int q = warp & 3;
    const int row = m0 + q * 32 + lane;            // tile row
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    double acc[BN];
#pragma unroll
    for (int j = 0; j < BN; ++j) acc[j] = 0.0;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const int b = b_first + c / nchunk_k;
      const int* ebb = p.eb + b * p.Npad + n0;
      if (!(ok = tc::mbar_wait(tfull, c & 1, err))) break;
      tc::tc_fence_after();
      const int ei = p.ea[b * p.Mpad + row];
      const double al = p.alpha[b];
#pragma unroll
      for (int g = 0; g < BN / 16; ++g) {
        double part[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) part[i] = 0.0;
#pragma unroll
        for (int a = 0; a < 5; ++a) {
          float v[16];
          tc::tmem_ld16(tmem + lane_off + a * BN + g * 16, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) part[i] += (double)v[i];
        }
#pragma unroll
        for (int i = 0; i < 16; ++i)
          acc[g * 16 + i] = fma(al, ldexp(part[i], ei + __ldg(ebb + g * 16 + i)), acc[g * 16 + i]);
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(tempty);
    }
    if (ok) {
      const int z = p.reduce ? 0 : blockIdx.z;
      double* C = p.C + (int64_t)z * p.strideC;
      const double* Cin = p.Cin ? p.Cin + (int64_t)z * p.strideCin : nullptr;
#pragma unroll
      for (int j = 0; j < BN; ++j) {
        const int col = n0 + j;
        // tile (row, col) is C(row, col), or C(col, row) when the tile computes C^T
        const int ci = p.swap ? col : row, cj = p.swap ? row : col;
        if (row < (p.swap ? p.N : p.M) && col < (p.swap ? p.M : p.N)) {
          double v = acc[j];
          if (Cin && p.beta != 0.0) v = fma(p.beta, Cin[ci + (int64_t)cj * p.ldcin], v);
          C[ci + (int64_t)cj * p.ldc] = v;
        }
      }
    }
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

// 2-D map over a (rows x K_pad) BF16 matrix, K contiguous, box 64 x box_rows, 128-byte swizzle
bool make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t K_pad, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K_pad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)K_pad * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

template <int S>
cudaError_t slice_operand(const double* X, int64_t ldx, int trans, int rows, int K, int* e,
                          __nv_bfloat16* out, int rows_pad, int K_pad, cudaStream_t st) {
  {
    ProfScope ps(kProfSlice, st, 0.0, 8.0 * rows * (double)K);
    if (!trans) row_exp_kernel<<<(rows + 255) / 256, 256, 0, st>>>(X, ldx, 0, rows, K, e);
    else row_exp_kernel<<<(rows * 32 + 255) / 256, 256, 0, st>>>(X, ldx, 1, rows, K, e);
  }
  ProfScope ps(kProfSlice, st, 0.0, (8.0 + 2.0 * S) * rows_pad * (double)K_pad);
  dim3 grid((unsigned)(K_pad / 32), (unsigned)(rows_pad / 32));
  slice_kernel<S><<<grid, dim3(32, 8), 0, st>>>(X, ldx, trans, rows, K, e, out, rows_pad, K_pad);
  return cudaGetLastError();
}

template <int BN, int S>
cudaError_t run_split(const GemmArgs& g, SplitWork& w, cudaStream_t st) {
  // orientation: put the larger output dimension on the 128-row tile side
  const bool swap = g.M < kTileM && g.N > g.M;
  const int M = swap ? g.N : g.M, N = swap ? g.M : g.N, K = g.K;
  const int Mpad = (int)round_up(M, kTileM), Npad = (int)round_up(N, BN), Kpad = (int)round_up(K, kBK);
  const int nb = g.batch;
  const size_t need_a = (size_t)nb * S * Mpad * Kpad, need_b = (size_t)nb * S * Npad * Kpad;
  if (need_a + need_b > w.slice_elems || (size_t)nb * (Mpad + Npad) > w.exp_elems)
    return cudaErrorMemoryAllocation;
  __nv_bfloat16* sa = static_cast<__nv_bfloat16*>(w.slices);
  __nv_bfloat16* sb = sa + need_a;
  int* ea = w.exps;
  int* eb = w.exps + (size_t)nb * Mpad;
  cudaError_t err;
  for (int b = 0; b < nb; ++b) {
    // op(A) rows: M x K.  With swap the tile's A side is op(B)^T, rows = columns of op(B).
    const double* Xa = swap ? g.B + b * g.strideB : g.A + b * g.strideA;
    const double* Xb = swap ? g.A + b * g.strideA : g.B + b * g.strideB;
    const int64_t lda = swap ? g.ldb : g.lda, ldb = swap ? g.lda : g.ldb;
    // tile-A operand = op(A) (or op(B)^T): rows along M.  op(A) row i, col k:
    //   transA = 0: A[i + k lda]  (rows contiguous)   transA = 1: A[k + i lda]
    // op(B)^T row j, col k = op(B)[k][j]: transB = 0: B[k + j ldb]  -> "trans" layout
    const int ta = swap ? (g.transB ? 0 : 1) : g.transA;
    const int tb = swap ? g.transA : (g.transB ? 0 : 1);
    if ((err = slice_operand<S>(Xa, lda, ta, M, K, ea + (size_t)b * Mpad,
                                sa + (size_t)b * S * Mpad * Kpad, Mpad, Kpad, st)) != cudaSuccess)
      return err;
    if ((err = slice_operand<S>(Xb, ldb, tb, N, K, eb + (size_t)b * Npad,
                                sb + (size_t)b * S * Npad * Kpad, Npad, Kpad, st)) != cudaSuccess)
      return err;
  }
  CUtensorMap mA, mB;
  if (!make_map(&mA, sa, (int64_t)nb * S * Mpad, Kpad, kTileM) ||
      !make_map(&mB, sb, (int64_t)nb * S * Npad, Kpad, BN))
    return cudaErrorInvalidValue;
  SplitEpi p{};
  p.C = g.Cout; p.ldc = g.ldcout; p.strideC = g.strideCout;
  p.Cin = g.Cin; p.ldcin = g.ldcin; p.strideCin = g.strideCin; p.beta = g.beta;
  for (int b = 0; b < kGemmMaxBatch; ++b) p.alpha[b] = g.alpha[b];
  p.ea = ea; p.eb = eb;
  p.M = g.M; p.N = g.N; p.K = K; p.Mpad = Mpad; p.Npad = Npad;
  p.batch = nb; p.reduce = g.reduce; p.swap = swap ? 1 : 0;
  p.err = w.err;
  using L = SmemLayout<BN, S>;
  static bool attr_set = false;
  if (!attr_set) {
    if ((err = cudaFuncSetAttribute(split_gemm_kernel<BN, S>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, L::kAlloc)) !=
        cudaSuccess)
      return err;
    attr_set = true;
  }
  dim3 grid((unsigned)(Npad / BN), (unsigned)(Mpad / kTileM), g.reduce ? 1 : nb);
  ProfScope ps(kProfSplitGemm, st, gemm_flops(g), 0.0);
  split_gemm_kernel<BN, S><<<grid, kThreads, L::kAlloc, st>>>(mA, mB, p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_split(const GemmArgs& g, SplitWork& w, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.K <= 0 || g.batch > kGemmMaxBatch) return gemm_f64(g, st);
  // batch entries per launch that the slice workspace holds
  const size_t per = split_slice_elems(g.M, g.N, g.K, 1, w.slices_s);
  const int64_t rows = std::max<int64_t>(round_up(std::max(g.M, g.N), kTileM), 64) * 2;
  int gs = (int)std::min<size_t>(g.batch, w.slice_elems / std::max<size_t>(per, 1));
  gs = (int)std::min<int64_t>(gs, (int64_t)(w.exp_elems / rows));
  if (gs < 1) return cudaErrorMemoryAllocation;
  auto run = [&](const GemmArgs& h) {
    return w.slices_s == 9 ? run_split<64, 9>(h, w, st) : run_split<64, 8>(h, w, st);
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

thread_local SplitWork* t_split = nullptr;

void set_split_engine(SplitWork* w) { t_split = w; }

cudaError_t gemm_any(const GemmArgs& g, cudaStream_t st) {
  // the tensor-core path pays a slicing pass per operand: small products stay on DFMA
  if (t_split && (double)g.M * g.N * g.K >= 4.0e6) return gemm_split(g, *t_split, st);
  return gemm_f64(g, st);
}

size_t split_slice_elems(int64_t M, int64_t N, int64_t K, int batch, int S) {
  const bool swap = M < kTileM && N > M;
  const int64_t rows = swap ? N : M, cols = swap ? M : N;
  return (size_t)batch * S * (round_up(rows, kTileM) + round_up(cols, 64)) * round_up(K, kBK);
}

}  // namespace zolo
