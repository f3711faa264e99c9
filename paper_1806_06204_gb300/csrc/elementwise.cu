// Memory-bound kernels of the iteration: scaling, stacked-matrix set-up, the
// r-way combination X_{k+1} = M_hat (X_k + sum_j T_j) with its two norms, and
// the symmetrisation of H.  All are single passes over column-major data with
// consecutive threads on consecutive rows (coalesced), grid-stride loops and a
// fixed grid so that per-block partial sums reduce deterministically.
#include <cmath>

#include "zolo_internal.h"

namespace zolo {
namespace {

constexpr int kThreads = 256;
constexpr int kReduceBlocks = 1024;   // fixed: partial-sum buffers hold 2 * 1024 doubles

struct Vec8 {
  double v[kGemmMaxBatch];
};

__global__ void scale_copy_kernel(const double* __restrict__ A, int64_t lda, double* __restrict__ X,
                                  int64_t ldx, int64_t m, int64_t n, double s) {
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % m, j = e / m;
    X[i + j * ldx] = s * A[i + j * lda];
  }
}

__global__ void init_stacked_kernel(const double* __restrict__ X, int64_t ldx, double* W,
                                    int64_t strideW, int64_t m, int64_t n, Vec8 sc) {
  const int64_t ldw = m + n, total = ldw * n;
  double* Wj = W + blockIdx.y * strideW;
  const double s = sc.v[blockIdx.y];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % ldw, j = e / ldw;
    Wj[e] = i < m ? X[i + j * ldx] : ((i - m) == j ? s : 0.0);
  }
}

__global__ void init_q_identity_kernel(double* Q, int64_t strideQ, int64_t m, int64_t n) {
  const int64_t ldq = m + n, total = ldq * n;
  double* Qj = Q + blockIdx.y * strideQ;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % ldq, j = e / ldq;
    Qj[e] = (i == j) ? 1.0 : 0.0;
  }
}

__global__ void init_shifted_kernel(const double* G, double* Z, int64_t strideZ,
                                    int64_t n, Vec8 sh) {
  const int64_t total = n * n;
  double* Zj = Z + blockIdx.y * strideZ;
  const double s = sh.v[blockIdx.y];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, j = e / n;
    Zj[e] = G[e] + (i == j ? s : 0.0);
  }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;   // valid in thread 0
}

__global__ void combine_kernel(const double* __restrict__ X, int64_t ldx, double* __restrict__ Xn,
                               int64_t ldxn, int64_t m, int64_t n, double mhat,
                               const double* __restrict__ T, int64_t ldt, int64_t strideT, Vec8 coef,
                               int nt, double* __restrict__ partials, int* status) {
  __shared__ double red[32];
  const int64_t total = m * n;
  double d2 = 0.0, x2 = 0.0;
  bool bad = false;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % m, j = e / m;
    const double x = X[i + j * ldx];
    double s = x;
    for (int t = 0; t < nt; ++t) s = fma(coef.v[t], T[i + j * ldt + t * strideT], s);
    const double y = mhat * s;
    Xn[i + j * ldxn] = y;
    const double d = y - x;
    d2 = fma(d, d, d2);
    x2 = fma(y, y, x2);
    bad |= !isfinite(y);
  }
  if (bad) atomicOr(status + kStatNonFinite, 1);
  const double sd = block_sum(d2, red);
  const double sx = block_sum(x2, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sd;
    partials[2 * blockIdx.x + 1] = sx;
  }
}

// S = sum_t coef_t T_t (T_t at T + t strideT): the shifted terms of one rank's
// shifts, before the sum over ranks.
__global__ void weighted_sum_kernel(const double* __restrict__ T, int64_t ldt, int64_t strideT,
                                    Vec8 coef, int nt, double* __restrict__ S, int64_t lds,
                                    int64_t m, int64_t n) {
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % m, j = e / m;
    double s = 0.0;
    for (int t = 0; t < nt; ++t) s = fma(coef.v[t], T[i + j * ldt + t * strideT], s);
    S[i + j * lds] = s;
  }
}

__global__ void guard_check_kernel(const unsigned char* __restrict__ p, size_t bytes,
                                   int* __restrict__ flag) {
  bool bad = false;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < bytes;
       e += (size_t)gridDim.x * blockDim.x)
    bad |= p[e] != 0xFF;
  if (bad) atomicOr(flag, 1);
}

__global__ void flag_to_double_kernel(const int* __restrict__ flag, double* __restrict__ out) {
  *out = *flag ? 1.0 : 0.0;
}

__global__ void finish_pairs_kernel(const double* __restrict__ partials, int nblocks,
                                    double* __restrict__ out) {
  __shared__ double red[32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    a += partials[2 * i];
    b += partials[2 * i + 1];
  }
  const double sa = block_sum(a, red);
  const double sb = block_sum(b, red);
  if (threadIdx.x == 0) {
    out[0] = sa;
    out[1] = sb;
  }
}

__global__ void frob_kernel(const double* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                            double* __restrict__ partials) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double v = A[(e % m) + (e / m) * lda];
    s = fma(v, v, s);
  }
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = t;
    partials[2 * blockIdx.x + 1] = 0.0;
  }
}

// Partial sums of ||G - I||_F^2 from the upper triangle of a symmetric G (each
// off-diagonal entry counted twice).
__global__ void gram_dev_kernel(const double* __restrict__ G, int64_t ldg, int64_t n,
                                double* __restrict__ partials) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, j = e / n;
    if (i > j) continue;
    const double d = G[i + j * ldg] - (i == j ? 1.0 : 0.0);
    s = fma(i == j ? 1.0 : 2.0, d * d, s);
  }
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = t;
    partials[2 * blockIdx.x + 1] = 0.0;
  }
}

// Row sums of |A| over a chunk of kAbsChunk columns: part[i + c m] for chunk c.
constexpr int kAbsChunk = 256;

__global__ void row_abs_partial_kernel(const double* __restrict__ A, int64_t lda, int64_t m,
                                       int64_t n, double* __restrict__ part) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t j0 = (int64_t)blockIdx.y * kAbsChunk;
  const int64_t j1 = j0 + kAbsChunk < n ? j0 + kAbsChunk : n;
  double s = 0.0;
  for (int64_t j = j0; j < j1; ++j) s += fabs(A[i + j * lda]);
  part[i + (int64_t)blockIdx.y * m] = s;
}

// One warp per column: colsum[j] = sum_i |A(i, j)|.
__global__ void col_abs_kernel(const double* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                               double* __restrict__ colsum) {
  const int64_t j = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= n) return;
  const int l = threadIdx.x & 31;
  double s = 0.0;
  for (int64_t i = l; i < m; i += 32) s += fabs(A[i + j * lda]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (l == 0) colsum[j] = s;
}

__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  }
  return s;   // valid in thread 0
}

// out[1] = max_j colsum[j] = ||A||_1, out[2] = max_i sum_c part[i + c m] = ||A||_inf.
__global__ void abs_norms_finish_kernel(const double* __restrict__ part, int64_t m, int nchunk,
                                        const double* __restrict__ colsum, int64_t n,
                                        double* __restrict__ out) {
  __shared__ double red[32];
  double rmax = 0.0, cmax = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    double r = 0.0;
    for (int c = 0; c < nchunk; ++c) r += part[i + c * m];
    rmax = fmax(rmax, r);
  }
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) cmax = fmax(cmax, colsum[j]);
  const double a = block_max(cmax, red);
  const double b = block_max(rmax, red);
  if (threadIdx.x == 0) {
    out[1] = a;
    out[2] = b;
  }
}

// W(i, j) = W(j, i) for i > j: the lower triangle from the upper one.
__global__ void mirror_upper_kernel(double* __restrict__ W, int64_t ldw, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, j = e / n;
    if (i > j) W[i + j * ldw] = W[j + i * ldw];
  }
}

__global__ void symmetrize_kernel(const double* __restrict__ M, int64_t ldm, double* __restrict__ H,
                                  int64_t ldh, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, j = e / n;
    H[i + j * ldh] = 0.5 * (M[i + j * ldm] + M[j + i * ldm]);
  }
}

__global__ void check_finite_kernel(const double* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                                    int* status) {
  bool bad = false;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * n;
       e += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(A[(e % m) + (e / m) * lda]);
  if (bad) atomicOr(status + kStatNonFinite, 1);
}

unsigned grid_for(int64_t total) {
  const int64_t b = (total + kThreads - 1) / kThreads;
  return (unsigned)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

Vec8 pack(const double* v, int r) {
  Vec8 p{};
  for (int i = 0; i < r && i < kGemmMaxBatch; ++i) p.v[i] = v[i];
  return p;
}

}  // namespace

cudaError_t scale_copy(const double* A, int64_t lda, double* X, int64_t ldx, int64_t m, int64_t n,
                       double s, cudaStream_t st) {
  ProfScope ps(kProfOther, st);
  ps.blocks((const void*)scale_copy_kernel, dim3(kThreads), 0, dim3(grid_for(m * n)));
  scale_copy_kernel<<<grid_for(m * n), kThreads, 0, st>>>(A, lda, X, ldx, m, n, s);
  return cudaGetLastError();
}

cudaError_t copy_matrix(const double* A, int64_t lda, double* B, int64_t ldb, int64_t m, int64_t n,
                        cudaStream_t st) {
  return cudaMemcpy2DAsync(B, ldb * sizeof(double), A, lda * sizeof(double), m * sizeof(double), n,
                           cudaMemcpyDeviceToDevice, st);
}

cudaError_t init_stacked(const double* X, int64_t ldx, double* W, int64_t strideW, int64_t m,
                         int64_t n, const double* sqrt_c, int r, cudaStream_t st) {
  dim3 grid(grid_for((m + n) * n), r);
  ProfScope ps(kProfOther, st);
  ps.blocks((const void*)init_stacked_kernel, dim3(kThreads), 0, dim3(grid));
  init_stacked_kernel<<<grid, kThreads, 0, st>>>(X, ldx, W, strideW, m, n, pack(sqrt_c, r));
  return cudaGetLastError();
}

cudaError_t init_q_identity(double* Q, int64_t strideQ, int64_t m, int64_t n, int r,
                            cudaStream_t st) {
  dim3 grid(grid_for((m + n) * n), r);
  ProfScope ps(kProfOther, st);
  ps.blocks((const void*)init_q_identity_kernel, dim3(kThreads), 0, dim3(grid));
  init_q_identity_kernel<<<grid, kThreads, 0, st>>>(Q, strideQ, m, n);
  return cudaGetLastError();
}

cudaError_t init_shifted(const double* G, double* Z, int64_t strideZ, int64_t n, const double* shift,
                         int r, cudaStream_t st) {
  dim3 grid(grid_for(n * n), r);
  ProfScope ps(kProfOther, st);
  ps.blocks((const void*)init_shifted_kernel, dim3(kThreads), 0, dim3(grid));
  init_shifted_kernel<<<grid, kThreads, 0, st>>>(G, Z, strideZ, n, pack(shift, r));
  return cudaGetLastError();
}

cudaError_t combine(const double* X, int64_t ldx, double* Xn, int64_t ldxn, int64_t m, int64_t n,
                    double mhat, const double* T, int64_t ldt, int64_t strideT, const double* coef,
                    int nt, double* partials, double* norms, int* status, cudaStream_t st) {
  {
    ProfScope ps(kProfCombine, st, 2.0 * (double)m * n * (nt + 2), 8.0 * (double)m * n * (nt + 2));
    ps.blocks((const void*)combine_kernel, dim3(kThreads), 0, dim3(kReduceBlocks));
    combine_kernel<<<kReduceBlocks, kThreads, 0, st>>>(X, ldx, Xn, ldxn, m, n, mhat, T, ldt,
                                                       strideT, pack(coef, nt), nt, partials,
                                                       status);
  }
  ProfScope ps(kProfOther, st);
  ps.blocks((const void*)finish_pairs_kernel, dim3(1024), 0, dim3(1));
  finish_pairs_kernel<<<1, 1024, 0, st>>>(partials, kReduceBlocks, norms);
  return cudaGetLastError();
}

cudaError_t weighted_sum(const double* T, int64_t ldt, int64_t strideT, const double* coef, int nt,
                         double* S, int64_t lds, int64_t m, int64_t n, cudaStream_t st) {
  ProfScope ps(kProfCombine, st, 2.0 * (double)m * n * nt, 8.0 * (double)m * n * (nt + 1));
  ps.blocks((const void*)weighted_sum_kernel, dim3(kThreads), 0, dim3(grid_for(m * n)));
  weighted_sum_kernel<<<grid_for(m * n), kThreads, 0, st>>>(T, ldt, strideT, pack(coef, nt), nt, S,
                                                             lds, m, n);
  return cudaGetLastError();
}

cudaError_t guard_fill(void* p, size_t bytes, cudaStream_t st) {
  return cudaMemsetAsync(p, 0xFF, bytes, st);
}

cudaError_t guard_check(const void* p, size_t bytes, int* flag, cudaStream_t st) {
  ProfScope ps(kProfOther, st);
  ps.blocks((const void*)guard_check_kernel, dim3(256), 0,
            dim3((unsigned)((bytes + 255) / 256 < 64 ? (bytes + 255) / 256 : 64)));
  guard_check_kernel<<<(unsigned)((bytes + 255) / 256 < 64 ? (bytes + 255) / 256 : 64), 256, 0, st>>>(
      static_cast<const unsigned char*>(p), bytes, flag);
  return cudaGetLastError();
}

cudaError_t flag_to_double(const int* flag, double* out, cudaStream_t st) {
  ProfScope ps(kProfOther, st);
  ps.blocks((const void*)flag_to_double_kernel, dim3(1), 0, dim3(1));
  flag_to_double_kernel<<<1, 1, 0, st>>>(flag, out);
  return cudaGetLastError();
}

cudaError_t mirror_upper(double* W, int64_t ldw, int64_t n, cudaStream_t st) {
  ProfScope ps(kProfOther, st);
  ps.blocks((const void*)mirror_upper_kernel, dim3(kThreads), 0, dim3(grid_for(n * n)));
  mirror_upper_kernel<<<grid_for(n * n), kThreads, 0, st>>>(W, ldw, n);
  return cudaGetLastError();
}

cudaError_t symmetrize(const double* M, int64_t ldm, double* H, int64_t ldh, int64_t n,
                       cudaStream_t st) {
  ProfScope ps(kProfOther, st);
  ps.blocks((const void*)symmetrize_kernel, dim3(kThreads), 0, dim3(grid_for(n * n)));
  symmetrize_kernel<<<grid_for(n * n), kThreads, 0, st>>>(M, ldm, H, ldh, n);
  return cudaGetLastError();
}

cudaError_t check_finite(const double* A, int64_t lda, int64_t m, int64_t n, int* status,
                         cudaStream_t st) {
  ProfScope ps(kProfOther, st);
  ps.blocks((const void*)check_finite_kernel, dim3(kThreads), 0, dim3(grid_for(m * n)));
  check_finite_kernel<<<grid_for(m * n), kThreads, 0, st>>>(A, lda, m, n, status);
  return cudaGetLastError();
}

int64_t alpha_bound_part_elems(int64_t m, int64_t n) {
  return m * ((n + kAbsChunk - 1) / kAbsChunk);
}

cudaError_t alpha_bound_sums(const double* A, int64_t lda, int64_t m, int64_t n, double* part,
                             double* colsum, double* partials, double* out, cudaStream_t st) {
  if (cudaError_t e = frob_norm2(A, lda, m, n, partials, out, st)) return e;
  const int nchunk = (int)((n + kAbsChunk - 1) / kAbsChunk);
  {
    ProfScope ps(kProfOther, st);
    ps.blocks((const void*)row_abs_partial_kernel, dim3(256), 0,
              dim3((unsigned)((m + 255) / 256), nchunk));
    row_abs_partial_kernel<<<dim3((unsigned)((m + 255) / 256), nchunk), 256, 0, st>>>(A, lda, m, n,
                                                                                      part);
  }
  {
    ProfScope ps(kProfOther, st);
    ps.blocks((const void*)col_abs_kernel, dim3(256), 0, dim3((unsigned)((n + 7) / 8)));
    col_abs_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(A, lda, m, n, colsum);
  }
  ProfScope ps(kProfOther, st);
  ps.blocks((const void*)abs_norms_finish_kernel, dim3(1024), 0, dim3(1));
  abs_norms_finish_kernel<<<1, 1024, 0, st>>>(part, m, nchunk, colsum, n, out);
  return cudaGetLastError();
}

double alpha_from_sums(const double* sums) {
  // ||A||_2 <= ||A||_F and ||A||_2^2 <= ||A||_1 ||A||_inf: the smaller of the two
  const double fro = std::sqrt(sums[0]);
  const double holder = std::sqrt(sums[1]) * std::sqrt(sums[2]);
  if (!std::isfinite(fro)) return fro;
  return holder < fro ? holder : fro;
}

cudaError_t gram_identity_dev2(const double* G, int64_t ldg, int64_t n, double* partials,
                               double* out, cudaStream_t st) {
  {
    ProfScope ps(kProfOther, st);
    ps.blocks((const void*)gram_dev_kernel, dim3(kThreads), 0, dim3(kReduceBlocks));
    gram_dev_kernel<<<kReduceBlocks, kThreads, 0, st>>>(G, ldg, n, partials);
  }
  ProfScope ps(kProfOther, st);
  ps.blocks((const void*)finish_pairs_kernel, dim3(1024), 0, dim3(1));
  finish_pairs_kernel<<<1, 1024, 0, st>>>(partials, kReduceBlocks, out);
  return cudaGetLastError();
}

cudaError_t frob_norm2(const double* A, int64_t lda, int64_t m, int64_t n, double* partials,
                       double* out, cudaStream_t st) {
  {
    ProfScope ps(kProfOther, st);
    ps.blocks((const void*)frob_kernel, dim3(kThreads), 0, dim3(kReduceBlocks));
    frob_kernel<<<kReduceBlocks, kThreads, 0, st>>>(A, lda, m, n, partials);
  }
  ProfScope ps(kProfOther, st);
  ps.blocks((const void*)finish_pairs_kernel, dim3(1024), 0, dim3(1));
  finish_pairs_kernel<<<1, 1024, 0, st>>>(partials, kReduceBlocks, out);
  return cudaGetLastError();
}

}  // namespace zolo
