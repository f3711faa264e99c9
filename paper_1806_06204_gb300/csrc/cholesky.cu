// Cholesky form of one Zolo-PD iteration (Algorithm 1 step (d)):
//   Z_j = X^T X + c_{2j-1} I = R_j^T R_j   (upper R_j; the paper's "L = Chol(Z)"
//   with X L^{-1} L^{-*} is consistent only for this upper factor),
//   T_j = a_j (X R_j^{-1}) R_j^{-T}.
// Blocked right-looking Cholesky: the NB x NB diagonal block is factored in
// shared memory by one CTA per shift, which also inverts it; the row panel is
// R_kk^{-T} Z_k,rest and the trailing update a SYRK, both on the FP64 GEMM.
// The triangular solves go block column by block column, each step a GEMM
// update followed by a product with the inverted diagonal block.
#include <cmath>

#include "zolo_internal.h"

namespace zolo {
namespace {

constexpr int kDiagThreads = 256;

template <int NB>
__global__ void __launch_bounds__(kDiagThreads)
chol_diag_kernel(double* Z, int64_t strideZ, int64_t n, int64_t k0, int nbk, double* Rinv,
                 int64_t strideRinv, int* status) {
  // S holds R on and above the diagonal; the inverse R^{-1} (also upper) is
  // kept transposed in the strictly lower part, its diagonal in Dinv.
  __shared__ double S[NB][NB + 1];
  __shared__ double Dinv[NB];
  __shared__ int s_fail;
  double* Zj = Z + blockIdx.x * strideZ;
  double* Ij = Rinv + blockIdx.x * strideRinv + (k0 / NB) * (int64_t)(NB * NB);
  const int tid = threadIdx.x;
  if (tid == 0) s_fail = 0;
  for (int e = tid; e < NB * NB; e += kDiagThreads) {
    const int i = e % NB, k = e / NB;
    S[i][k] = (i <= k && k < nbk) ? Zj[(k0 + i) + (k0 + k) * n] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < nbk; ++j) {
    if (tid == 0) {
      const double d = S[j][j];
      if (!(d > 0.0) || !isfinite(d)) {
        s_fail = 1;
        S[j][j] = 1.0;
      } else {
        S[j][j] = sqrt(d);
      }
    }
    __syncthreads();
    const double djj = S[j][j];
    for (int k = j + 1 + tid; k < nbk; k += kDiagThreads) S[j][k] /= djj;
    __syncthreads();
    for (int e = tid; e < nbk * nbk; e += kDiagThreads) {
      const int i = e % nbk, k = e / nbk;
      if (i > j && i <= k) S[i][k] = fma(-S[j][i], S[j][k], S[i][k]);
    }
    __syncthreads();
  }
  // inverse of the upper-triangular block, column k by thread k:
  // Inv(k,k) = 1/R(k,k);  Inv(i,k) = -sum_{l=i+1..k} R(i,l) Inv(l,k) / R(i,i)
  if (tid < nbk) {
    const int k = tid;
    const double dk = 1.0 / S[k][k];
    Dinv[k] = dk;
    for (int i = k - 1; i >= 0; --i) {
      double s = S[i][k] * dk;
      for (int l = i + 1; l < k; ++l) s = fma(S[i][l], S[k][l], s);
      S[k][i] = -s / S[i][i];
    }
  }
  __syncthreads();
  for (int e = tid; e < NB * NB; e += kDiagThreads) {
    const int i = e % NB, k = e / NB;
    if (i < nbk && k < nbk && i <= k) Zj[(k0 + i) + (k0 + k) * n] = S[i][k];
    double inv = 0.0;
    if (i < nbk && k < nbk) inv = i == k ? Dinv[k] : (i < k ? S[k][i] : 0.0);
    Ij[e] = inv;
  }
  if (tid == 0 && s_fail) atomicOr(status + kStatCholFail, 1);
}

}  // namespace

cudaError_t cholesky_upper_batched(const CholBuffers& b, int64_t n, int r, int* status,
                                   cudaStream_t st) {
  constexpr int NB = kCholNB;
  cudaError_t err;
  for (int64_t k0 = 0; k0 < n; k0 += NB) {
    const int nbk = (int)(n - k0 < NB ? n - k0 : NB);
    {
      ProfScope ps(kProfCholDiag, st, r * 2.0 / 3.0 * (double)nbk * nbk * nbk);
      chol_diag_kernel<NB><<<r, kDiagThreads, 0, st>>>(b.Z, b.strideZ, n, k0, nbk, b.Rinv,
                                                       b.strideRinv, status);
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const int64_t rest = n - k0 - nbk;
    if (rest <= 0) break;
    double* panel = b.Z + k0 + (k0 + nbk) * n;
    GemmArgs g;   // panel <- Rinv_kk^T panel (in place: each tile reads only its own columns)
    g.M = nbk; g.N = (int)rest; g.K = nbk; g.transA = 1; g.transB = 0;
    g.A = b.Rinv + (k0 / NB) * (int64_t)(NB * NB); g.lda = NB; g.strideA = b.strideRinv;
    g.B = panel; g.ldb = n; g.strideB = b.strideZ;
    g.Cout = panel; g.ldcout = n; g.strideCout = b.strideZ;
    g.batch = r;
    for (int j = 0; j < r; ++j) g.alpha[j] = 1.0;
    if ((err = gemm_any(g, st)) != cudaSuccess) return err;
    GemmArgs u;   // trailing SYRK, upper tiles only
    double* trail = b.Z + (k0 + nbk) + (k0 + nbk) * n;
    u.M = u.N = (int)rest; u.K = nbk; u.transA = 1; u.transB = 0;
    u.A = panel; u.lda = n; u.strideA = b.strideZ;
    u.B = panel; u.ldb = n; u.strideB = b.strideZ;
    u.Cin = trail; u.ldcin = n; u.strideCin = b.strideZ; u.beta = 1.0;
    u.Cout = trail; u.ldcout = n; u.strideCout = b.strideZ;
    u.batch = r; u.c_upper = 1;
    for (int j = 0; j < r; ++j) u.alpha[j] = -1.0;
    if ((err = gemm_any(u, st)) != cudaSuccess) return err;
  }
  return cudaSuccess;
}

cudaError_t trsm_right_upper_batched(const double* X, int64_t ldx, const CholBuffers& b, double* Y,
                                     int64_t strideY, double* tmp, int64_t strideTmp, int64_t m,
                                     int64_t n, int r, cudaStream_t st) {
  constexpr int NB = kCholNB;
  cudaError_t err;
  const int nblk = (int)((n + NB - 1) / NB);
  // Y R = X, block column by block column
  for (int jb = 0; jb < nblk; ++jb) {
    const int64_t j0 = (int64_t)jb * NB;
    const int nbj = (int)(n - j0 < NB ? n - j0 : NB);
    GemmArgs g;   // tmp = X_j - Y_{<j} R_{<j, j}
    g.M = (int)m; g.N = nbj; g.K = (int)j0; g.transA = 0; g.transB = 0;
    g.A = Y; g.lda = m; g.strideA = strideY;
    g.B = b.Z + j0 * n; g.ldb = n; g.strideB = b.strideZ;
    g.Cin = X + j0 * ldx; g.ldcin = ldx; g.strideCin = 0; g.beta = 1.0;
    g.Cout = tmp; g.ldcout = m; g.strideCout = strideTmp;
    g.batch = r;
    for (int j = 0; j < r; ++j) g.alpha[j] = -1.0;
    if ((err = gemm_any(g, st)) != cudaSuccess) return err;
    GemmArgs h;   // Y_j = tmp Rinv_jj
    h.M = (int)m; h.N = nbj; h.K = nbj; h.transA = 0; h.transB = 0;
    h.A = tmp; h.lda = m; h.strideA = strideTmp;
    h.B = b.Rinv + jb * (int64_t)(NB * NB); h.ldb = NB; h.strideB = b.strideRinv;
    h.Cout = Y + j0 * m; h.ldcout = m; h.strideCout = strideY;
    h.batch = r;
    for (int j = 0; j < r; ++j) h.alpha[j] = 1.0;
    if ((err = gemm_any(h, st)) != cudaSuccess) return err;
  }
  return cudaSuccess;
}

cudaError_t trsm_pair_batched(const double* X, int64_t ldx, const CholBuffers& b, double* Y,
                              int64_t strideY, double* tmp, int64_t strideTmp, int64_t m,
                              int64_t n, int r, cudaStream_t st) {
  constexpr int NB = kCholNB;
  cudaError_t err;
  const int nblk = (int)((n + NB - 1) / NB);
  if ((err = trsm_right_upper_batched(X, ldx, b, Y, strideY, tmp, strideTmp, m, n, r, st)) !=
      cudaSuccess)
    return err;
  // backward: W R^T = Y, last block column first, W overwriting Y
  for (int jb = nblk - 1; jb >= 0; --jb) {
    const int64_t j0 = (int64_t)jb * NB;
    const int nbj = (int)(n - j0 < NB ? n - j0 : NB);
    const int64_t rest = n - j0 - nbj;
    GemmArgs g;   // tmp = Y_j - W_{>j} (R_{j, >j})^T
    g.M = (int)m; g.N = nbj; g.K = (int)rest; g.transA = 0; g.transB = 1;
    g.A = Y + (j0 + nbj) * m; g.lda = m; g.strideA = strideY;
    g.B = b.Z + j0 + (j0 + nbj) * n; g.ldb = n; g.strideB = b.strideZ;
    g.Cin = Y + j0 * m; g.ldcin = m; g.strideCin = strideY; g.beta = 1.0;
    g.Cout = tmp; g.ldcout = m; g.strideCout = strideTmp;
    g.batch = r;
    for (int j = 0; j < r; ++j) g.alpha[j] = -1.0;
    if ((err = gemm_any(g, st)) != cudaSuccess) return err;
    GemmArgs h;   // W_j = tmp Rinv_jj^T
    h.M = (int)m; h.N = nbj; h.K = nbj; h.transA = 0; h.transB = 1;
    h.A = tmp; h.lda = m; h.strideA = strideTmp;
    h.B = b.Rinv + jb * (int64_t)(NB * NB); h.ldb = NB; h.strideB = b.strideRinv;
    h.Cout = Y + j0 * m; h.ldcout = m; h.strideCout = strideY;
    h.batch = r;
    for (int j = 0; j < r; ++j) h.alpha[j] = 1.0;
    if ((err = gemm_any(h, st)) != cudaSuccess) return err;
  }
  return cudaSuccess;
}

}  // namespace zolo
