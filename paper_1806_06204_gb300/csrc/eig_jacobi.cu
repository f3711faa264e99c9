// Eigendecomposition of H for Zolo-SVD (Algorithm 2, step 2; ELPA in the paper).
//
// H = R^T R (Cholesky, upper R).  One-sided Jacobi rotations from the right on
// X = R^T make its columns mutually orthogonal: X Z = W diag(s) with W
// orthonormal, so H = X X^T = W diag(s^2) W^T.  The eigenvectors are the
// normalised columns of the converged X and the eigenvalues are taken as the
// Rayleigh quotients w_i^T H w_i (the squared column norms carry the rounding
// of every rotation applied to the column).  On the geometric spectra of this
// workload two-sided Jacobi on H converges only linearly in the absolute
// off-diagonal norm; the Cholesky factor restores quadratic convergence.
//
// Mixed precision.  FP32 runs 58x faster than FP64 on this part, so the sweeps
// that only need to bring the columns close to orthogonal run in FP32 on a copy
// X32 = R^T with the rotations accumulated in Z32 (one cooperative launch per
// sweep: the n-1 rounds of the round-robin ordering are separated by a bounded
// grid barrier).  Z is then made orthonormal in FP64 (Cholesky QR), X = R^T Z is
// formed in FP64, and FP64 sweeps (one launch per round, one CTA per column
// pair) finish from cosines ~1e-5 in a few quadratically convergent sweeps.
// FP32 sweeps stop when no cosine exceeds 8e-6 (25 sweeps at most).  FP64 sweeps
// stop when no pair has |x_p . x_q| > 8 eps ||x_p|| ||x_q||, or once two sweeps
// have started with every cosine below sqrt(n) eps (the rounding level of an
// n-term dot product).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "zolo_internal.h"

namespace zolo {
namespace {

constexpr int kJacThreads = 256;
constexpr double kEps = 2.220446049250313e-16;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kJacThreads)
jacobi_round_kernel(double* X, int64_t ldx, int64_t m, int n_even, int n_real, int round, double tol,
                    int* status) {
  __shared__ double red[3][kJacThreads / 32];
  __shared__ double s_c, s_s;
  __shared__ int s_rot;
  const int i = blockIdx.x;
  auto elem = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + round) % (n_even - 1); };
  int p = elem(i), q = elem(n_even - 1 - i);
  if (p > q) { const int t = p; p = q; q = t; }
  if (q >= n_real) return;
  double* xp = X + p * ldx;
  double* xq = X + q * ldx;
  double a = 0.0, b = 0.0, g = 0.0;
  for (int64_t r = threadIdx.x; r < m; r += kJacThreads) {
    const double u = xp[r], v = xq[r];
    a = fma(u, u, a);
    b = fma(v, v, b);
    g = fma(u, v, g);
  }
  a = warp_sum(a); b = warp_sum(b); g = warp_sum(g);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { red[0][w] = a; red[1][w] = b; red[2][w] = g; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0, sg = 0.0;
    for (int k = 0; k < kJacThreads / 32; ++k) { sa += red[0][k]; sb += red[1][k]; sg += red[2][k]; }
    const double cosv = (sa > 0.0 && sb > 0.0) ? fabs(sg) / (sqrt(sa) * sqrt(sb)) : 0.0;
    atomicMax(status + kStatJacobiMaxCos, __float_as_int((float)cosv));
    int rot = (sg != 0.0) && (fabs(sg) > tol * sqrt(sa) * sqrt(sb));
    double c = 1.0, s = 0.0;
    if (rot) {
      const double zeta = (sb - sa) / (2.0 * sg);
      const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
      c = 1.0 / sqrt(fma(t, t, 1.0));
      s = c * t;
      atomicAdd(status + kStatJacobiRot, 1);
    }
    s_c = c; s_s = s; s_rot = rot;
  }
  __syncthreads();
  if (!s_rot) return;
  const double c = s_c, s = s_s;
  for (int64_t r = threadIdx.x; r < m; r += kJacThreads) {
    const double u = xp[r], v = xq[r];
    xp[r] = c * u - s * v;
    xq[r] = fma(s, u, c * v);
  }
}

// Bounded grid-wide barrier for a cooperative launch (all blocks co-resident).
__device__ bool grid_barrier(unsigned* count, unsigned* gen, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vg = gen;
    const unsigned g = *vg;
    __threadfence();
    if (atomicAdd(count, 1u) == gridDim.x - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      long long i = 0;
      while (*vg == g) {
        if (++i > (1ll << 22) || *(volatile int*)err) {
          atomicExch(err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)err == 0;
}

// One FP32 sweep: every round of the round-robin ordering, pairs distributed over
// the blocks; rotations applied to X32 and accumulated into Z32.
__global__ void __launch_bounds__(kJacThreads)
jacobi32_sweep_kernel(float* X, float* Z, int64_t ld, int64_t m, int n_even, int n_real, float tol,
                      int* status, unsigned* bar, int* err) {
  __shared__ float red[3][kJacThreads / 32];
  __shared__ float s_c, s_s;
  __shared__ int s_rot;
  const int npairs = n_even / 2;
  for (int round = 0; round < n_even - 1; ++round) {
    for (int i = blockIdx.x; i < npairs; i += gridDim.x) {
      auto elem = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + round) % (n_even - 1); };
      int p = elem(i), q = elem(n_even - 1 - i);
      if (p > q) { const int t = p; p = q; q = t; }
      if (q >= n_real) continue;
      float* xp = X + p * ld;
      float* xq = X + q * ld;
      float a = 0.f, b = 0.f, g = 0.f;
      for (int64_t r = threadIdx.x; r < m; r += kJacThreads) {
        const float u = xp[r], v = xq[r];
        a = fmaf(u, u, a);
        b = fmaf(v, v, b);
        g = fmaf(u, v, g);
      }
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        g += __shfl_xor_sync(0xffffffffu, g, o);
      }
      const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
      if (l == 0) { red[0][w] = a; red[1][w] = b; red[2][w] = g; }
      __syncthreads();
      if (threadIdx.x == 0) {
        float sa = 0.f, sb = 0.f, sg = 0.f;
        for (int k = 0; k < kJacThreads / 32; ++k) { sa += red[0][k]; sb += red[1][k]; sg += red[2][k]; }
        int rot = (sg != 0.f) && (fabsf(sg) > tol * sqrtf(sa) * sqrtf(sb));
        float c = 1.f, sn = 0.f;
        if (rot) {
          const float zeta = (sb - sa) / (2.f * sg);
          const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
          c = 1.f / sqrtf(fmaf(t, t, 1.f));
          sn = c * t;
          atomicAdd(status + kStatJacobiRot, 1);
        }
        s_c = c; s_s = sn; s_rot = rot;
      }
      __syncthreads();
      if (s_rot) {
        const float c = s_c, sn = s_s;
        float* zp = Z + p * ld;
        float* zq = Z + q * ld;
        for (int64_t r = threadIdx.x; r < m; r += kJacThreads) {
          const float u = xp[r], v = xq[r];
          xp[r] = c * u - sn * v;
          xq[r] = fmaf(sn, u, c * v);
          const float y = zp[r], z = zq[r];
          zp[r] = c * y - sn * z;
          zq[r] = fmaf(sn, y, c * z);
        }
      }
      __syncthreads();
    }
    if (!grid_barrier(bar, bar + 1, err)) return;
  }
}

__global__ void to_f32_kernel(const double* __restrict__ X, float* __restrict__ Y, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    Y[e] = (float)X[e];
}

__global__ void to_f64_kernel(const float* __restrict__ X, double* __restrict__ Y, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    Y[e] = (double)X[e];
}

__global__ void identity_f32_kernel(float* Z, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n;
       e += (int64_t)gridDim.x * blockDim.x)
    Z[e] = (e % n) == (e / n) ? 1.f : 0.f;
}

__global__ void column_norms_kernel(const double* __restrict__ X, int64_t ldx, int64_t m,
                                    double* __restrict__ out) {
  __shared__ double red[kJacThreads / 32];
  const double* x = X + blockIdx.x * ldx;
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < m; r += kJacThreads) s = fma(x[r], x[r], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kJacThreads / 32; ++k) t += red[k];
    out[blockIdx.x] = sqrt(t);
  }
}

__global__ void column_dots_kernel(const double* __restrict__ A, int64_t lda,
                                   const double* __restrict__ B, int64_t ldb, int64_t m,
                                   double* __restrict__ out) {
  __shared__ double red[kJacThreads / 32];
  const double* a = A + blockIdx.x * lda;
  const double* b = B + blockIdx.x * ldb;
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < m; r += kJacThreads) s = fma(a[r], b[r], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kJacThreads / 32; ++k) t += red[k];
    out[blockIdx.x] = t;
  }
}

__global__ void scale_columns_kernel(double* X, int64_t ldx, int64_t m, const double* s, int invert) {
  const double f = invert ? (s[blockIdx.y] > 0.0 ? 1.0 / s[blockIdx.y] : 1.0) : s[blockIdx.y];
  double* x = X + blockIdx.y * ldx;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x)
    x[r] *= f;
}

__global__ void gather_columns_kernel(const double* __restrict__ X, int64_t ldx, double* __restrict__ Y,
                                      int64_t ldy, int64_t m, const int* __restrict__ perm,
                                      const double* __restrict__ sign) {
  const int j = blockIdx.y;
  const double f = sign ? sign[j] : 1.0;
  const double* x = X + perm[j] * ldx;
  double* y = Y + j * ldy;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x)
    y[r] = f * x[r];
}

__global__ void transpose_lower_kernel(const double* __restrict__ R, int64_t ldr, double* __restrict__ X,
                                       int64_t ldx, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, j = e / n;
    X[i + j * ldx] = i >= j ? R[j + i * ldr] : 0.0;
  }
}

unsigned rows_grid(int64_t m) {
  const int64_t b = (m + 255) / 256;
  return (unsigned)std::min<int64_t>(std::max<int64_t>(b, 1), 64);
}

}  // namespace

cudaError_t column_norms(const double* X, int64_t ldx, int64_t m, int64_t n, double* out,
                         cudaStream_t st) {
  ProfScope ps(kProfOther, st);
  column_norms_kernel<<<(unsigned)n, kJacThreads, 0, st>>>(X, ldx, m, out);
  return cudaGetLastError();
}

cudaError_t column_dots(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t m,
                        int64_t n, double* out, cudaStream_t st) {
  ProfScope ps(kProfOther, st);
  column_dots_kernel<<<(unsigned)n, kJacThreads, 0, st>>>(A, lda, B, ldb, m, out);
  return cudaGetLastError();
}

cudaError_t scale_columns(double* X, int64_t ldx, int64_t m, int64_t n, const double* s, int invert,
                          cudaStream_t st) {
  ProfScope ps(kProfOther, st);
  scale_columns_kernel<<<dim3(rows_grid(m), (unsigned)n), 256, 0, st>>>(X, ldx, m, s, invert);
  return cudaGetLastError();
}

cudaError_t gather_columns(const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t m,
                           int64_t n, const int* perm, const double* sign, cudaStream_t st) {
  ProfScope ps(kProfOther, st);
  gather_columns_kernel<<<dim3(rows_grid(m), (unsigned)n), 256, 0, st>>>(X, ldx, Y, ldy, m, perm,
                                                                         sign);
  return cudaGetLastError();
}

cudaError_t transpose_lower(const double* R, int64_t ldr, double* X, int64_t ldx, int64_t n,
                            cudaStream_t st) {
  const int64_t b = std::min<int64_t>((n * n + 255) / 256, 4096);
  ProfScope ps(kProfOther, st);
  transpose_lower_kernel<<<(unsigned)std::max<int64_t>(b, 1), 256, 0, st>>>(R, ldr, X, ldx, n);
  return cudaGetLastError();
}

cudaError_t jacobi_round(double* X, int64_t ldx, int64_t m, int64_t n_even, int64_t n_real,
                         int round, double tol, int* status, cudaStream_t st) {
  ProfScope ps(kProfJacobi, st, 12.0 * (double)m * (double)(n_even / 2),
               32.0 * (double)m * (double)(n_even / 2));
  jacobi_round_kernel<<<(unsigned)(n_even / 2), kJacThreads, 0, st>>>(X, ldx, m, (int)n_even,
                                                                      (int)n_real, round, tol,
                                                                      status);
  return cudaGetLastError();
}

// Full driver.  Returns 0; 1 = CUDA error, 2 = no convergence, 3 = a bounded
// wait expired.  lam_out (host, n) receives the eigenvalues in the order of V's
// columns (descending |lambda|).
int eig_sym_jacobi(const double* H, int64_t ldh, int64_t n, double* V, int64_t ldv, double* lam_out,
                   const EigWork& w, int* sweeps, cudaStream_t st) {
  // ---- Cholesky H = R^T R (shifted by 10 n eps ||H||_F if it breaks down)
  CholBuffers cb{w.R, 0, w.Rinv, 0};
  int hstat[kStatSlots] = {0, 0, 0, 0};
  double shift = 0.0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (cudaMemsetAsync(w.status, 0, sizeof(int) * kStatSlots, st) != cudaSuccess) return 1;
    if (copy_matrix(H, ldh, w.R, n, n, n, st) != cudaSuccess) return 1;
    if (shift != 0.0 && init_shifted(w.R, w.R, 0, n, &shift, 1, st) != cudaSuccess) return 1;
    if (cholesky_upper_batched(cb, n, 1, w.status, st) != cudaSuccess) return 1;
    if (cudaMemcpyAsync(hstat, w.status, sizeof(hstat), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return 1;
    if (cudaStreamSynchronize(st) != cudaSuccess) return 1;
    if (!hstat[kStatCholFail]) break;
    if (attempt == 1) return 2;
    if (frob_norm2(H, ldh, n, n, w.HV, w.lam, st) != cudaSuccess) return 1;
    double nrm2 = 0.0;
    if (cudaMemcpyAsync(&nrm2, w.lam, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return 1;
    if (cudaStreamSynchronize(st) != cudaSuccess) return 1;
    shift = 10.0 * (double)n * kEps * sqrt(nrm2);
  }
  const int64_t nn = n * n;
  const unsigned eg = (unsigned)std::min<int64_t>((nn + 255) / 256, 4096);
  const int64_t n_even = n + (n & 1);
  int total_sweeps = 0;
  // ---- FP32 phase on X32 = R^T, rotations accumulated in Z32
  if (cudaMemsetAsync(w.err, 0, sizeof(int), st) != cudaSuccess) return 1;
  if (transpose_lower(w.R, n, w.X, n, n, st) != cudaSuccess) return 1;
  {
    ProfScope ps(kProfOther, st);
    to_f32_kernel<<<eg, 256, 0, st>>>(w.X, w.X32, nn);
  }
  {
    ProfScope ps(kProfOther, st);
    identity_f32_kernel<<<eg, 256, 0, st>>>(w.Z32, n);
  }
  if (n > 1) {
    int occ = 0, dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jacobi32_sweep_kernel, kJacThreads, 0) !=
            cudaSuccess)
      return 1;
    const int grid = (int)std::min<int64_t>(n_even / 2, (int64_t)std::max(1, occ) * sms);
    const float tol32 = 8e-6f;
    for (int sw = 0; sw < 25; ++sw) {
      if (cudaMemsetAsync(w.status + kStatJacobiRot, 0, sizeof(int), st) != cudaSuccess) return 1;
      if (cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), st) != cudaSuccess) return 1;
      float* X32 = w.X32;
      float* Z32 = w.Z32;
      int64_t ld = n, mm = n;
      int ne = (int)n_even, nr = (int)n;
      float tol = tol32;
      int* status = w.status;
      unsigned* bar = w.bar;
      int* err = w.err;
      void* args[] = {&X32, &Z32, &ld, &mm, &ne, &nr, &tol, &status, &bar, &err};
      {
        ProfScope ps(kProfJacobi32, st, 18.0 * (double)n * (double)n * (double)(n_even - 1) / 2.0);
        if (cudaLaunchCooperativeKernel((const void*)jacobi32_sweep_kernel, grid, kJacThreads, args,
                                        0, st) != cudaSuccess)
          return 1;
      }
      int rot = 0, herr = 0;
      if (cudaMemcpyAsync(&rot, w.status + kStatJacobiRot, sizeof(int), cudaMemcpyDeviceToHost, st) !=
              cudaSuccess ||
          cudaMemcpyAsync(&herr, w.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return 1;
      if (herr) return 3;
      ++total_sweeps;
      if (rot == 0) break;
    }
  }
  // ---- Z orthonormal in FP64 (Cholesky QR: Z^T Z = R_z^T R_z, Z <- Z R_z^{-1})
  {
    ProfScope ps(kProfOther, st);
    to_f64_kernel<<<eg, 256, 0, st>>>(w.Z32, w.Z, nn);
  }
  {
    GemmArgs g;
    g.M = g.N = (int)n; g.K = (int)n; g.transA = 1;
    g.A = w.Z; g.lda = n; g.B = w.Z; g.ldb = n; g.Cout = w.HV; g.ldcout = n; g.c_upper = 1;
    g.alpha[0] = 1.0;
    if (gemm_f64(g, st) != cudaSuccess) return 1;
    CholBuffers cz{w.HV, 0, w.Rinv, 0};
    if (cudaMemsetAsync(w.status, 0, sizeof(int) * kStatSlots, st) != cudaSuccess) return 1;
    if (cholesky_upper_batched(cz, n, 1, w.status, st) != cudaSuccess) return 1;
    if (trsm_right_upper_batched(w.Z, n, cz, w.X, 0, w.tmp, 0, n, n, 1, st) != cudaSuccess) return 1;
  }
  // ---- X = R^T Z in FP64 (w.Z <- R^T, w.HV <- R^T Z)
  if (transpose_lower(w.R, n, w.Z, n, n, st) != cudaSuccess) return 1;
  {
    GemmArgs g;
    g.M = g.N = g.K = (int)n;
    g.A = w.Z; g.lda = n; g.B = w.X; g.ldb = n; g.Cout = w.HV; g.ldcout = n;
    g.alpha[0] = 1.0;
    if (gemm_f64(g, st) != cudaSuccess) return 1;
  }
  double* X = w.HV;
  // ---- FP64 sweeps
  const double tol_strict = 8.0 * kEps, tol_loose = sqrt((double)n) * kEps;
  bool converged = n == 1;
  int quiet = 0;
  for (int sw = 0; sw < 40 && !converged; ++sw) {
    if (cudaMemsetAsync(w.status + kStatJacobiRot, 0, 2 * sizeof(int), st) != cudaSuccess) return 1;
    for (int round = 0; round < n_even - 1; ++round)
      if (jacobi_round(X, n, n, n_even, n, round, tol_strict, w.status, st) != cudaSuccess) return 1;
    int rs[2] = {0, 0};
    if (cudaMemcpyAsync(rs, w.status + kStatJacobiRot, sizeof(rs), cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
      return 1;
    if (cudaStreamSynchronize(st) != cudaSuccess) return 1;
    ++total_sweeps;
    float maxcos;
    memcpy(&maxcos, &rs[1], sizeof(float));
    if (rs[0] == 0) converged = true;
    else if (maxcos <= tol_loose && ++quiet >= 2) converged = true;
  }
  *sweeps = total_sweeps;
  if (!converged) return 2;
  // ---- eigenvectors (normalised columns) and Rayleigh quotients
  if (column_norms(X, n, n, n, w.lam, st) != cudaSuccess) return 1;
  if (scale_columns(X, n, n, n, w.lam, 1, st) != cudaSuccess) return 1;
  GemmArgs g;
  g.M = g.N = g.K = (int)n;
  g.A = H; g.lda = ldh; g.B = X; g.ldb = n; g.Cout = w.Z; g.ldcout = n;
  g.alpha[0] = 1.0;
  if (gemm_f64(g, st) != cudaSuccess) return 1;
  if (column_dots(X, n, w.Z, n, n, n, w.lam, st) != cudaSuccess) return 1;
  std::vector<double> lam(n);
  if (cudaMemcpyAsync(lam.data(), w.lam, sizeof(double) * n, cudaMemcpyDeviceToHost, st) !=
      cudaSuccess)
    return 1;
  if (cudaStreamSynchronize(st) != cudaSuccess) return 1;
  std::vector<int> perm(n);
  for (int64_t i = 0; i < n; ++i) perm[i] = (int)i;
  std::stable_sort(perm.begin(), perm.end(),
                   [&](int a, int b) { return std::fabs(lam[a]) > std::fabs(lam[b]); });
  for (int64_t i = 0; i < n; ++i) lam_out[i] = lam[perm[i]];
  if (cudaMemcpyAsync(w.perm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return 1;
  if (gather_columns(X, n, V, ldv, n, n, w.perm, nullptr, st) != cudaSuccess) return 1;
  // the host vectors must outlive the async copy
  if (cudaStreamSynchronize(st) != cudaSuccess) return 1;
  return 0;
}

}  // namespace zolo
