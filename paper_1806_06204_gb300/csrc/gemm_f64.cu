// FP64 GEMM on the FP64 FMA pipe (DFMA), batched or batch-reduced.
//
// On GB300 the FP64 rate is ~1.2 TFLOP/s (about 2 DFMA per clock per SM) while
// HBM delivers ~6.7 TB/s, so every FP64 contraction here is bound by the FMA
// pipe, not by memory: a 64x64 output tile per CTA with 4x4 outputs per thread
// reaches the pipe's rate with plain shared-memory staging.  tcgen05 has no
// FP64 kind, and the FP64 mma.sync path measured slower than DFMA on this part.
#include <algorithm>

#include "zolo_internal.h"

namespace zolo {
namespace {

template <int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
gemm_f64_kernel(const GemmArgs g) {
  constexpr int RT = BM / TM;           // threads along rows
  constexpr int CT = BN / TN;           // threads along columns
  constexpr int NT = RT * CT;
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];

  const int m0 = blockIdx.y * BM;
  const int n0 = blockIdx.x * BN;
  if (g.c_upper && m0 > n0 + BN - 1) return;   // tile strictly below the diagonal
  const int tid = threadIdx.x;
  const int tr = tid % RT;
  const int tc = tid / RT;

  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

  const int bbeg = g.reduce ? 0 : blockIdx.z;
  const int bend = g.reduce ? g.batch : blockIdx.z + 1;
  const int kbeg = g.b_lower ? (n0 / BK) * BK : 0;

  for (int b = bbeg; b < bend; ++b) {
    const double* A = g.A + (int64_t)b * g.strideA;
    const double* B = g.B + (int64_t)b * g.strideB;
    const double alpha = g.alpha[b];
    for (int k0 = kbeg; k0 < g.K; k0 += BK) {
      for (int e = tid; e < BM * BK; e += NT) {
        int i, kk;
        if (!g.transA) { i = e % BM; kk = e / BM; } else { kk = e % BK; i = e / BK; }
        const int gi = m0 + i, gk = k0 + kk;
        double v = 0.0;
        if (gi < g.M && gk < g.K)
          v = g.transA ? A[gk + (int64_t)gi * g.lda] : A[gi + (int64_t)gk * g.lda];
        As[kk][i] = alpha * v;
      }
      for (int e = tid; e < BK * BN; e += NT) {
        int kk, j;
        if (!g.transB) { kk = e % BK; j = e / BK; } else { j = e % BN; kk = e / BN; }
        const int gk = k0 + kk, gj = n0 + j;
        double v = 0.0;
        if (gk < g.K && gj < g.N)
          v = g.transB ? B[gj + (int64_t)gk * g.ldb] : B[gk + (int64_t)gj * g.ldb];
        Bs[kk][j] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double a[TM], bv[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[kk][tr + i * RT];
#pragma unroll
        for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tc + j * CT];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
      }
      __syncthreads();
    }
  }

  const int z = g.reduce ? 0 : blockIdx.z;
  double* C = g.Cout + (int64_t)z * g.strideCout;
  const double* Cin = g.Cin ? g.Cin + (int64_t)z * g.strideCin : nullptr;
  const bool use_in = Cin != nullptr && g.beta != 0.0;
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int gj = n0 + tc + j * CT;
    if (gj >= g.N) continue;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int gi = m0 + tr + i * RT;
      if (gi >= g.M) continue;
      double v = acc[i][j];
      if (use_in) v = fma(g.beta, Cin[gi + (int64_t)gj * g.ldcin], v);
      C[gi + (int64_t)gj * g.ldcout] = v;
    }
  }
}

__global__ void gemm_beta_only(const GemmArgs g) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)g.M * g.N) return;
  const int64_t i = e % g.M, j = e / g.M;
  const int z = blockIdx.z;
  double* C = g.Cout + (int64_t)z * g.strideCout;
  const double* Cin = g.Cin ? g.Cin + (int64_t)z * g.strideCin : nullptr;
  C[i + j * g.ldcout] = (Cin && g.beta != 0.0) ? g.beta * Cin[i + j * g.ldcin] : 0.0;
}

template <int BM, int BN>
cudaError_t launch(const GemmArgs& g, cudaStream_t st) {
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.reduce ? 1 : g.batch);
  const double bytes = 8.0 * g.batch * ((double)g.M * g.K + (double)g.K * g.N) +
                       8.0 * (g.reduce ? 1 : g.batch) * (double)g.M * g.N * (g.beta != 0.0 ? 2 : 1);
  ProfScope ps(kProfGemm, st, gemm_flops(g), bytes);
  gemm_f64_kernel<BM, BN, 16, 4, 4><<<grid, (BM / 4) * (BN / 4), 0, st>>>(g);
  return cudaGetLastError();
}

}  // namespace

// Algorithmic flops of one call: the products the structure leaves non-zero.
double gemm_flops(const GemmArgs& g) {
  double per = 2.0 * g.M * (double)g.N * g.K;
  if (g.c_upper) per = (double)g.K * g.N * (g.N + 1.0);
  else if (g.b_lower) per = 2.0 * g.M * ((double)g.N * g.K - 0.5 * (double)g.N * (g.N - 1.0));
  return per * g.batch;
}

cudaError_t gemm_f64(const GemmArgs& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.batch > kGemmMaxBatch) return cudaErrorInvalidValue;
  if (g.K <= 0) {
    // empty contraction: C_out = beta * C_in (or 0)
    const int nz = g.reduce ? 1 : g.batch;
    dim3 grid((unsigned)((g.M * (int64_t)g.N + 255) / 256), 1, nz);
    ProfScope ps(kProfOther, st);
    gemm_beta_only<<<grid, 256, 0, st>>>(g);
    return cudaGetLastError();
  }
  return g.M <= 32 ? launch<32, 128>(g, st) : launch<64, 64>(g, st);
}

}  // namespace zolo
