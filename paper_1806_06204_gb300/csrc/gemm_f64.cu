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

// ksplit > 1: blockIdx.z = batch entry * ksplit + K slice; the slice's raw sum
// goes to P (ld M, one M x N plane per (slice, entry)) for splitk_reduce_kernel.
template <int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
gemm_f64_kernel(const GemmArgs g, int ksplit, double* __restrict__ P) {
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

  const int zs = blockIdx.z % ksplit;          // K slice
  const int zb = blockIdx.z / ksplit;          // batch entry (output plane)
  const int bbeg = g.reduce ? 0 : zb;
  const int bend = g.reduce ? g.batch : zb + 1;
  int kbeg = g.b_lower ? (n0 / BK) * BK : 0;
  int kend = g.K;
  if (ksplit > 1) {
    // slices of whole BK steps, so every step lies in exactly one slice
    const int kc = ((g.K + ksplit - 1) / ksplit + BK - 1) / BK * BK;
    kbeg = max(kbeg, zs * kc);
    kend = min(g.K, (zs + 1) * kc);
  }

  for (int b = bbeg; b < bend; ++b) {
    const double* A = g.A + (int64_t)b * g.strideA;
    const double* B = g.B + (int64_t)b * g.strideB;
    const double alpha = g.alpha[b];
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
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

  const int z = g.reduce ? 0 : zb;
  if (ksplit > 1) {
    const int nz = g.reduce ? 1 : g.batch;
    double* Pz = P + ((int64_t)zs * nz + z) * (int64_t)g.M * g.N;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gj = n0 + tc + j * CT;
      if (gj >= g.N) continue;
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const int gi = m0 + tr + i * RT;
        if (gi < g.M) Pz[gi + (int64_t)gj * g.M] = acc[i][j];
      }
    }
    return;
  }
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

// C_z = sum_s P[s][z] (+ beta Cin_z), written only where the one-pass kernel with
// BM x BN tiles writes (c_upper: tiles on or above the diagonal).
template <int BM, int BN>
__global__ void splitk_reduce_kernel(const GemmArgs g, int ksplit, const double* __restrict__ P) {
  const int nz = g.reduce ? 1 : g.batch;
  const int64_t mn = (int64_t)g.M * g.N;
  const int z = blockIdx.y;
  double* C = g.Cout + (int64_t)(g.reduce ? 0 : z) * g.strideCout;
  const double* Cin = g.Cin ? g.Cin + (int64_t)(g.reduce ? 0 : z) * g.strideCin : nullptr;
  const bool use_in = Cin != nullptr && g.beta != 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < mn;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % g.M, j = e / g.M;
    if (g.c_upper && (i / BM) * BM > (j / BN) * BN + BN - 1) continue;
    double v = 0.0;
    for (int s = 0; s < ksplit; ++s) v += P[((int64_t)s * nz + z) * mn + e];
    if (use_in) v = fma(g.beta, Cin[i + j * g.ldcin], v);
    C[i + j * g.ldcout] = v;
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
cudaError_t launch(const GemmArgs& g, int ksplit, double* P, cudaStream_t st) {
  const int nz = g.reduce ? 1 : g.batch;
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, nz * ksplit);
  const double bytes = 8.0 * g.batch * ((double)g.M * g.K + (double)g.K * g.N) +
                       8.0 * nz * (double)g.M * g.N * (g.beta != 0.0 ? 2 : 1);
  {
    ProfScope ps(kProfGemm, st, gemm_flops(g), bytes);
    ps.blocks((const void*)gemm_f64_kernel<BM, BN, 16, 4, 4>, dim3((BM / 4) * (BN / 4)), 0,
              dim3(grid));
    gemm_f64_kernel<BM, BN, 16, 4, 4><<<grid, (BM / 4) * (BN / 4), 0, st>>>(g, ksplit, P);
  }
  if (ksplit > 1) {
    if (cudaError_t e = cudaGetLastError()) return e;
    const int64_t mn = (int64_t)g.M * g.N;
    const unsigned bx = (unsigned)std::min<int64_t>((mn + 255) / 256, 2048);
    ProfScope ps(kProfOther, st, 0.0, 8.0 * nz * mn * (ksplit + 1));
    ps.blocks((const void*)splitk_reduce_kernel<BM, BN>, dim3(256), 0, dim3(bx, nz));
    splitk_reduce_kernel<BM, BN><<<dim3(bx, nz), 256, 0, st>>>(g, ksplit, P);
  }
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

int gemm_f64_default_variant(const GemmArgs& g) {
  return g.M <= 32 ? kGemmV32x128 : kGemmV64x64;
}

size_t gemm_f64_scratch_elems(const GemmArgs& g, int variant) {
  const int ks = variant == kGemmVSplitK2 ? 2 : variant == kGemmVSplitK4 ? 4 :
                 variant == kGemmVSplitK8 ? 8 : 1;
  if (ks == 1) return 0;
  return (size_t)ks * (g.reduce ? 1 : g.batch) * (size_t)g.M * (size_t)g.N;
}

cudaError_t gemm_f64_variant(const GemmArgs& g, int variant, double* scratch,
                             size_t scratch_elems, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.batch > kGemmMaxBatch) return cudaErrorInvalidValue;
  if (g.K <= 0) {
    // empty contraction: C_out = beta * C_in (or 0)
    const int nz = g.reduce ? 1 : g.batch;
    dim3 grid((unsigned)((g.M * (int64_t)g.N + 255) / 256), 1, nz);
    ProfScope ps(kProfOther, st);
    ps.blocks((const void*)gemm_beta_only, dim3(256), 0, dim3(grid));
    gemm_beta_only<<<grid, 256, 0, st>>>(g);
    return cudaGetLastError();
  }
  const size_t need = gemm_f64_scratch_elems(g, variant);
  if (need > 0 && (scratch == nullptr || need > scratch_elems)) variant = kGemmV64x64;
  switch (variant) {
    case kGemmV32x128: return launch<32, 128>(g, 1, nullptr, st);
    case kGemmV32x64: return launch<32, 64>(g, 1, nullptr, st);
    case kGemmVSplitK2: return launch<64, 64>(g, 2, scratch, st);
    case kGemmVSplitK4: return launch<64, 64>(g, 4, scratch, st);
    case kGemmVSplitK8: return launch<64, 64>(g, 8, scratch, st);
    default: return launch<64, 64>(g, 1, nullptr, st);
  }
}

}  // namespace zolo
