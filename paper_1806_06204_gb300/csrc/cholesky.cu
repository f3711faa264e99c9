// Cholesky form of one Zolo-PD iteration (Algorithm 1 step (d)):
//   Z_j = X^T X + c_{2j-1} I = R_j^T R_j   (upper R_j; the paper's "L = Chol(Z)"
//   with X L^{-1} L^{-*} is consistent only for this upper factor),
//   T_j = a_j (X R_j^{-1}) R_j^{-T}.
// Blocked right-looking Cholesky: the NB x NB diagonal block is factored in
// shared memory by one CTA per shift, which also inverts it; the row panel is
// R_kk^{-T} Z_k,rest and the trailing update a SYRK, both on the FP64 GEMM.
// The triangular solves are recursive: halve the columns, solve one half,
// update the other with one GEMM whose inner dimension is the half's width,
// solve it; 64-column leaves are products with the inverted diagonal block.
// Every column of the right-hand side is read by O(log n) GEMMs (the
// block-column-by-block-column form reads the solved part once per block, which
// on the split path re-slices it n/64 times).
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
  __shared__ double s_rd;
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
  // FP64 division is a long dependent sequence on this part: each pivot's
  // reciprocal is formed once, by the thread that takes the square root, and the
  // row is scaled by multiplication (and the inverse below reuses it)
  for (int j = 0; j < nbk; ++j) {
    if (tid == 0) {
      const double d = S[j][j];
      double sd = 1.0;
      if (!(d > 0.0) || !isfinite(d)) {
        s_fail = 1;
      } else {
        sd = sqrt(d);
      }
      S[j][j] = sd;
      s_rd = 1.0 / sd;
      Dinv[j] = s_rd;
    }
    __syncthreads();
    const double rjj = s_rd;
    for (int k = j + 1 + tid; k < nbk; k += kDiagThreads) S[j][k] *= rjj;
    __syncthreads();
    // trailing update of rows j+1.. : thread (row i, column group g) takes the
    // columns k = g, g + 4, ... of row i at and right of the diagonal
    {
      static_assert(kDiagThreads == 4 * NB, "four threads per row of the block");
      const int i = tid >> 2, g = tid & 3;
      if (i > j && i < nbk) {
        const double sji = S[j][i];
        for (int k = i + ((g - i) & 3); k < nbk; k += 4) S[i][k] = fma(-sji, S[j][k], S[i][k]);
      }
    }
    __syncthreads();
  }
  // inverse of the upper-triangular block, column k by the four threads
  // 4k..4k+3 (each sums every fourth term, a shuffle joins them):
  // Inv(k,k) = 1/R(k,k);  Inv(i,k) = -sum_{l=i+1..k} R(i,l) Inv(l,k) / R(i,i)
  static_assert(kDiagThreads >= 4 * NB, "four threads per column of the inverse");
  {
    const int k = tid >> 2, sub = tid & 3;
    const unsigned grp = 0xFu << (tid & 28);   // the four lanes of this column
    if (k < nbk) {
      const double dk = Dinv[k];
      for (int i = k - 1; i >= 0; --i) {
        double s = 0.0;
        for (int l = i + 1 + sub; l < k; l += 4) s = fma(S[i][l], S[k][l], s);
        s += __shfl_xor_sync(grp, s, 1);
        s += __shfl_xor_sync(grp, s, 2);
        s = fma(S[i][k], dk, s);
        if (sub == 0) S[k][i] = -s * Dinv[i];
        __syncwarp(grp);   // the next row's terms read this entry
      }
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

namespace {

// Upper-triangular inverse of one NB x NB diagonal block of R (one CTA per
// block): column k of the inverse by back substitution, one thread per column.
template <int NB>
__global__ void __launch_bounds__(NB)
tri_inv_kernel(const double* __restrict__ R, int64_t n, double* __restrict__ Rinv, int* status) {
  __shared__ double S[NB][NB + 1];
  __shared__ double Y[NB][NB + 1];
  const int64_t k0 = (int64_t)blockIdx.x * NB;
  const int nbk = n - k0 < NB ? (int)(n - k0) : NB;
  const int k = threadIdx.x;
  for (int i = 0; i < NB; ++i) S[i][k] = (i < nbk && k < nbk) ? R[(k0 + i) + (k0 + k) * n] : 0.0;
  __syncthreads();
  if (k < nbk) {
    // Y(:, k) = R^{-1} e_k, rows k down to 0
    bool bad = !(S[k][k] != 0.0);
    Y[k][k] = bad ? 0.0 : 1.0 / S[k][k];
    for (int i = k - 1; i >= 0; --i) {
      double s = 0.0;
      for (int l = i + 1; l <= k; ++l) s = fma(S[i][l], Y[l][k], s);
      bad |= !(S[i][i] != 0.0);
      Y[i][k] = bad ? 0.0 : -s / S[i][i];
    }
    if (bad) atomicOr(status + kStatNonFinite, 1);
  }
  __syncthreads();
  double* Ij = Rinv + (k0 / NB) * (int64_t)(NB * NB);
  for (int i = 0; i < NB; ++i)
    Ij[i + k * NB] = (i < nbk && k < nbk && i <= k) ? Y[i][k] : 0.0;
}

}  // namespace

cudaError_t tri_inv_diag_blocks(const double* R, int64_t n, double* Rinv, int* status,
                                cudaStream_t st) {
  ProfScope ps(kProfCholDiag, st);
  ps.blocks((const void*)tri_inv_kernel<kCholNB>, dim3(kCholNB), 0,
            dim3((unsigned)((n + kCholNB - 1) / kCholNB)));
  tri_inv_kernel<kCholNB><<<(unsigned)((n + kCholNB - 1) / kCholNB), kCholNB, 0, st>>>(R, n, Rinv,
                                                                                     status);
  return cudaGetLastError();
}

cudaError_t cholesky_upper_batched(const CholBuffers& b, int64_t n, int r, int* status,
                                   cudaStream_t st) {
  constexpr int NB = kCholNB;
  cudaError_t err;
  for (int64_t k0 = 0; k0 < n; k0 += NB) {
    const int nbk = (int)(n - k0 < NB ? n - k0 : NB);
    {
      ProfScope ps(kProfCholDiag, st, r * 2.0 / 3.0 * (double)nbk * nbk * nbk);
      ps.blocks((const void*)chol_diag_kernel<NB>, dim3(kDiagThreads), 0, dim3(r));
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

namespace {

// dst_j[:, 0:w] = src_j[:, 0:w] for r matrices of m rows (column-major).
__global__ void copy_cols_kernel(const double* __restrict__ src, int64_t lds, int64_t strideS,
                                 double* __restrict__ dst, int64_t ldd, int64_t strideD, int64_t m,
                                 int w) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * w) return;
  const int64_t i = e % m, c = e / m;
  dst[blockIdx.y * strideD + i + c * ldd] = src[blockIdx.y * strideS + i + c * lds];
}

cudaError_t copy_cols(const double* src, int64_t lds, int64_t strideS, double* dst, int64_t ldd,
                      int64_t strideD, int64_t m, int w, int r, cudaStream_t st) {
  ProfScope ps(kProfOther, st, 0.0, 16.0 * m * w * r);
  ps.blocks((const void*)copy_cols_kernel, dim3(256), 0, dim3((unsigned)((m * w + 255) / 256), r));
  copy_cols_kernel<<<dim3((unsigned)((m * w + 255) / 256), r), 256, 0, st>>>(src, lds, strideS, dst,
                                                                             ldd, strideD, m, w);
  return cudaGetLastError();
}

struct TrsmCtx {
  const CholBuffers* b;
  double* Y; int64_t strideY;
  double* tmp; int64_t strideTmp;
  int64_t m, n;
  int r;
  cudaStream_t st;
};

// split point of [j0, j0 + w): a multiple of NB near the middle
int64_t half_of(int w) {
  const int nb = kCholNB;
  const int blocks = (w + nb - 1) / nb;
  return (int64_t)((blocks + 1) / 2) * nb;
}

// Y[:, j0:j0+w] R[j0:j0+w, j0:j0+w] = rhs[:, j0:j0+w]; rhs is X (shared by the
// shifts, stride strideR = 0) at the top and Y itself once updated.
cudaError_t fwd(const TrsmCtx& c, const double* rhs, int64_t ldr, int64_t strideR, int64_t j0, int w) {
  cudaError_t err;
  const CholBuffers& b = *c.b;
  if (w <= kCholNB) {
    const double* A = rhs + j0 * ldr;
    int64_t lda = ldr, strideA = strideR;
    if (rhs == c.Y) {   // in place: the product reads its own output, so copy first
      if ((err = copy_cols(rhs + j0 * ldr, ldr, strideR, c.tmp, c.m, c.strideTmp, c.m, w, c.r, c.st)) !=
          cudaSuccess)
        return err;
      A = c.tmp; lda = c.m; strideA = c.strideTmp;
    }
    GemmArgs h;   // Y_j = rhs_j Rinv_jj
    h.M = (int)c.m; h.N = w; h.K = w; h.transA = 0; h.transB = 0;
    h.A = A; h.lda = lda; h.strideA = strideA;
    h.B = b.Rinv + (j0 / kCholNB) * (int64_t)(kCholNB * kCholNB); h.ldb = kCholNB;
    h.strideB = b.strideRinv;
    h.Cout = c.Y + j0 * c.m; h.ldcout = c.m; h.strideCout = c.strideY;
    h.batch = c.r;
    for (int j = 0; j < c.r; ++j) h.alpha[j] = 1.0;
    return gemm_any(h, c.st);
  }
  const int64_t h1 = half_of(w);
  const int w2 = (int)(w - h1);
  if ((err = fwd(c, rhs, ldr, strideR, j0, (int)h1)) != cudaSuccess) return err;
  GemmArgs g;   // Y_2 = rhs_2 - Y_1 R_12
  g.M = (int)c.m; g.N = w2; g.K = (int)h1; g.transA = 0; g.transB = 0;
  g.A = c.Y + j0 * c.m; g.lda = c.m; g.strideA = c.strideY;
  g.B = b.Z + j0 + (j0 + h1) * c.n; g.ldb = c.n; g.strideB = b.strideZ;
  g.Cin = rhs + (j0 + h1) * ldr; g.ldcin = ldr; g.strideCin = strideR; g.beta = 1.0;
  g.Cout = c.Y + (j0 + h1) * c.m; g.ldcout = c.m; g.strideCout = c.strideY;
  g.batch = c.r;
  for (int j = 0; j < c.r; ++j) g.alpha[j] = -1.0;
  if ((err = gemm_any(g, c.st)) != cudaSuccess) return err;
  return fwd(c, c.Y, c.m, c.strideY, j0 + h1, w2);
}

// W[:, j0:j0+w] R[j0:j0+w, j0:j0+w]^T = Y[:, j0:j0+w], W overwriting Y.
cudaError_t bwd(const TrsmCtx& c, int64_t j0, int w) {
  cudaError_t err;
  const CholBuffers& b = *c.b;
  if (w <= kCholNB) {
    if ((err = copy_cols(c.Y + j0 * c.m, c.m, c.strideY, c.tmp, c.m, c.strideTmp, c.m, w, c.r, c.st)) !=
        cudaSuccess)
      return err;
    GemmArgs h;   // W_j = Y_j Rinv_jj^T
    h.M = (int)c.m; h.N = w; h.K = w; h.transA = 0; h.transB = 1;
    h.A = c.tmp; h.lda = c.m; h.strideA = c.strideTmp;
    h.B = b.Rinv + (j0 / kCholNB) * (int64_t)(kCholNB * kCholNB); h.ldb = kCholNB;
    h.strideB = b.strideRinv;
    h.Cout = c.Y + j0 * c.m; h.ldcout = c.m; h.strideCout = c.strideY;
    h.batch = c.r;
    for (int j = 0; j < c.r; ++j) h.alpha[j] = 1.0;
    return gemm_any(h, c.st);
  }
  const int64_t h1 = half_of(w);
  const int w2 = (int)(w - h1);
  if ((err = bwd(c, j0 + h1, w2)) != cudaSuccess) return err;
  GemmArgs g;   // Y_1 -= W_2 R_12^T
  g.M = (int)c.m; g.N = (int)h1; g.K = w2; g.transA = 0; g.transB = 1;
  g.A = c.Y + (j0 + h1) * c.m; g.lda = c.m; g.strideA = c.strideY;
  g.B = b.Z + j0 + (j0 + h1) * c.n; g.ldb = c.n; g.strideB = b.strideZ;
  g.Cin = c.Y + j0 * c.m; g.ldcin = c.m; g.strideCin = c.strideY; g.beta = 1.0;
  g.Cout = c.Y + j0 * c.m; g.ldcout = c.m; g.strideCout = c.strideY;
  g.batch = c.r;
  for (int j = 0; j < c.r; ++j) g.alpha[j] = -1.0;
  if ((err = gemm_any(g, c.st)) != cudaSuccess) return err;
  return bwd(c, j0, (int)h1);
}

}  // namespace

cudaError_t trsm_right_upper_batched(const double* X, int64_t ldx, const CholBuffers& b, double* Y,
                                     int64_t strideY, double* tmp, int64_t strideTmp, int64_t m,
                                     int64_t n, int r, cudaStream_t st) {
  if (n <= 0 || m <= 0) return cudaSuccess;
  TrsmCtx c{&b, Y, strideY, tmp, strideTmp, m, n, r, st};
  return fwd(c, X, ldx, 0, 0, (int)n);
}

cudaError_t trsm_pair_batched(const double* X, int64_t ldx, const CholBuffers& b, double* Y,
                              int64_t strideY, double* tmp, int64_t strideTmp, int64_t m,
                              int64_t n, int r, cudaStream_t st) {
  if (n <= 0 || m <= 0) return cudaSuccess;
  cudaError_t err;
  if ((err = trsm_right_upper_batched(X, ldx, b, Y, strideY, tmp, strideTmp, m, n, r, st)) !=
      cudaSuccess)
    return err;
  TrsmCtx c{&b, Y, strideY, tmp, strideTmp, m, n, r, st};
  return bwd(c, 0, (int)n);
}

}  // namespace zolo
