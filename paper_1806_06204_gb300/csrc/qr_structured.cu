// Structured Householder QR of the stacked matrix [X; sqrt(c) I] (Section 3.1,
// Eq. 12) and the explicit thin Q = [Q1; Q2] (the structured ORGQR).
//
// Layout: the stacked (m+n) x n matrix is stored densely, column-major with
// ld = m + n (top block rows 0..m-1, bottom block rows m..m+n-1).  The bottom
// block starts diagonal; Householder vector c (column c) is non-zero only on
// top rows c..m-1 and bottom rows 0..c, i.e. on the CONTIGUOUS stored rows
// c..m+c: m+1 entries instead of m+n-c (the paper's "at most m+1 nonzero
// elements").  A set of columns [c0, c0 + w) therefore lives in the row window
// [c0, c0 + m + w), and its compact-WY update (I - V T V^T) touches only that
// window: every step costs O((m + w) w n) whatever n is.
//
// Two levels of blocking.  Panels of NB = 32 columns are factored by one kernel
// (one CTA, or one 8-CTA cluster, per shift) and applied at once only to the
// rest of their block of NBb = 128 columns.  The block's reflectors are then
// merged into one compact-WY factor T_b (from the Gram matrix V_b^T V_b, below)
// and applied to all later columns with three GEMMs whose inner dimension is the
// block width: the wide products see the trailing matrix once per 128 columns,
// not once per 32, and no GEMM dimension is padded up from 32.  The explicit Q
// applies the same block reflectors in reverse order.
//
// Q2 (the bottom block of Q) stays exactly upper triangular: the explicit V
// holds exact zeros outside each reflector's support, so every product that the
// structure makes zero is an exact zero in floating point too.
#include <cooperative_groups.h>

#include <cmath>

#include "zolo_internal.h"

namespace zolo {
namespace {

constexpr int kPanelCluster = 8;            // CTAs per shift in the cluster panel
constexpr int64_t kClusterPanelMinRows = 512;

// Reduce-scatter of 32 per-lane partial sums across a warp: on return lane q
// holds the warp's total of value q.  Each step keeps the half of the values
// selected by one lane bit and adds the partner's copy of that half: 16 + 8 +
// 4 + 2 + 1 = 31 adds per lane, where one butterfly per value costs 5 x 32 (the
// FP64 adds, not the shuffles, bound the panel on this part).
__device__ __forceinline__ double warp_reduce_scatter32(double (&a)[32], int lane) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const double send = up ? a[j] : a[j + h];
      const double keep = up ? a[j + h] : a[j];
      a[j] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  return a[0];
}

// Cluster form of the panel factorisation: CG CTAs per shift (one thread-block
// cluster), each owning a contiguous slice of the panel's row window.  Per
// column, every CTA reduces its rows' part of the norm (and the owner of the
// diagonal row contributes alpha), the partials are exchanged through
// distributed shared memory, every CTA forms the same beta/tau from the same
// ordered sum, scales its rows of v, and the same exchange gives the dot
// products for the update and for T.  Two hardware cluster barriers per
// column; the partial buffers alternate between columns so that no third
// barrier is needed before they are rewritten.  All rows a CTA reads or writes
// in W and V are its own, so the only cross-CTA traffic is the partials.
template <int NB, int CG, int KT>
__global__ void __cluster_dims__(CG, 1, 1) __launch_bounds__(KT)
qr_panel_cluster_kernel(double* W, int64_t strideW, int64_t ldw, int64_t m, int64_t c0, int nbp,
                        double* V, int64_t strideV, int64_t ldv, double* T, int64_t strideT,
                        int* status) {
  namespace cgrp = cooperative_groups;
  cgrp::cluster_group cluster = cgrp::this_cluster();
  constexpr int kT = KT, kWarps = kT / 32;
  __shared__ double part[2][NB + 2];        // [0, NB): dots, NB: norm^2, NB+1: alpha
  __shared__ double red[kWarps][NB + 2];
  __shared__ double dots[NB];
  __shared__ double cf[NB];                // -tau dots[q]: the update's coefficients
  __shared__ double Ts[NB][NB + 1];
  __shared__ double s_tau, s_scal, s_beta;

  const int rank = (int)cluster.block_rank();
  const int shift = blockIdx.x / CG;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* Wj = W + shift * strideW;
  double* Vp = V + shift * strideV + c0 * ldv;
  double* Tp = T + shift * strideT + (c0 / NB) * (int64_t)(NB * NB);
  const int64_t height = m + NB;
  const int64_t chunk = (height + CG - 1) / CG;
  const int64_t lo = c0 + rank * chunk;                   // my window rows [lo, hi)
  const int64_t hi = lo + chunk < c0 + height ? lo + chunk : c0 + height;

  for (int e = tid; e < NB * (NB + 1); e += kT) (&Ts[0][0])[e] = 0.0;

  for (int i = 0; i < nbp; ++i) {
    const int64_t c = c0 + i;
    const int buf = i & 1;
    double* col = Wj + c * ldw;
    const int64_t r0 = lo > c ? lo : c;                  // my part of the support [c, m + c]
    const int64_t r1 = hi < m + c + 1 ? hi : m + c + 1;
    // ---- 1. partial norm of the tail (rows > c) and alpha from the owner of row c
    double ss = 0.0;
    for (int64_t r = (r0 > c + 1 ? r0 : c + 1) + tid; r < r1; r += kT) {
      const double v = col[r];
      ss = fma(v, v, ss);
    }
    // the block's partials are summed by warp 0 (kWarps - 1 + 5 FP64 warp
    // instructions; a butterfly in every warp would take 5 per warp, and an FP64
    // instruction costs its unit a whole warp slot however few lanes it uses)
    double* flat = &red[0][0];
    flat[tid] = ss;
    __syncthreads();
    if (warp == 0) {
      double t = flat[lane];
#pragma unroll
      for (int w = 1; w < kWarps; ++w) t += flat[lane + 32 * w];
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) {
        part[buf][NB] = t;
        part[buf][NB + 1] = (c >= lo && c < hi) ? col[c] : 0.0;
      }
    }
    cluster.sync();
    if (tid == 0) {
      double s = 0.0, alpha = 0.0;
      for (int rk = 0; rk < CG; ++rk) {
        const double* rp = cluster.map_shared_rank(&part[buf][0], rk);
        s += rp[NB];
        alpha += rp[NB + 1];
      }
      double beta, tau, scal;
      if (s == 0.0) {
        beta = alpha; tau = 0.0; scal = 0.0;
      } else {
        beta = -copysign(sqrt(fma(alpha, alpha, s)), alpha);
        tau = (beta - alpha) / beta;
        scal = 1.0 / (alpha - beta);
      }
      if (rank == 0 && (!isfinite(beta) || !isfinite(tau))) atomicOr(status + kStatNonFinite, 1);
      s_beta = beta; s_tau = tau; s_scal = scal;
    }
    __syncthreads();
    const double tau = s_tau, scal = s_scal;
    // ---- 2. my rows of v, and of the explicit reflector (zeros outside the support)
    double* Vcol = Vp + (int64_t)i * ldv;
    for (int64_t r = lo + tid; r < hi; r += kT) {
      double v;
      if (r < c || r > m + c) {
        v = 0.0;
      } else if (r == c) {
        v = 1.0;
      } else {
        v = col[r] * scal;
        col[r] = v;
      }
      Vcol[r - c0] = v;
    }
    __syncthreads();
    if (tid == 0 && c >= lo && c < hi) col[c] = s_beta;
    // ---- 3. partial dots of v with the later panel columns and the earlier reflectors
    double acc[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) acc[q] = 0.0;
    for (int64_t r = r0 + tid; r < r1; r += kT) {
      const double v = Vcol[r - c0];
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        if (q < nbp && q != i) {
          const double o = q > i ? Wj[r + (c0 + q) * ldw] : Vp[(r - c0) + (int64_t)q * ldv];
          acc[q] = fma(v, o, acc[q]);
        }
      }
    }
    static_assert(NB == 32, "one dot product per lane");
    red[warp][lane] = warp_reduce_scatter32(acc, lane);
    __syncthreads();
    if (tid < NB) {
      double t = 0.0;
      for (int w = 0; w < kWarps; ++w) t += red[w][tid];
      part[buf][tid] = t;
    }
    cluster.sync();
    if (tid < NB) {
      double t = 0.0;
      for (int rk = 0; rk < CG; ++rk) t += cluster.map_shared_rank(&part[buf][0], rk)[tid];
      dots[tid] = t;
      cf[tid] = -tau * t;
    }
    __syncthreads();
    // ---- 4. my rows of the later panel columns: W[:, q] -= tau * dots[q] * v
    //         (the coefficients formed once above: the stores through pq may
    //         alias shared memory for the compiler, so a product written here
    //         would be redone for every row)
    for (int64_t r = r0 + tid; r < r1; r += kT) {
      const double v = Vcol[r - c0];
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        if (q > i && q < nbp) {
          double* pq = Wj + r + (c0 + q) * ldw;
          *pq = fma(cf[q], v, *pq);
        }
      }
    }
    // ---- 5. T(0:i, i) = -tau T(0:i, 0:i) V^T v_i (same in every CTA)
    if (tid < i) {
      double t = 0.0;
      for (int pc = tid; pc < i; ++pc) t = fma(Ts[tid][pc], dots[pc], t);
      Ts[tid][i] = -tau * t;
    }
    if (tid == 0) Ts[i][i] = tau;
    __syncthreads();
  }
  if (rank == 0)
    for (int e = tid; e < NB * NB; e += kT) Tp[e] = Ts[e % NB][e / NB];
  cluster.sync();   // no CTA leaves while another may still read its partials
}

// T_b of one block: its panel factors on the 32 x 32 diagonal blocks, zero
// elsewhere (ld NBb).  Grid (ceil(nbb^2 / 256), r).
__global__ void tb_init_kernel(const double* __restrict__ T, int64_t strideT, double* __restrict__ Tb,
                               int64_t strideTb, int panel0, int nbb) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nbb * nbb) return;
  const int i = e % nbb, j = e / nbb;
  double v = 0.0;
  if (i / kQrNB == j / kQrNB)
    v = T[blockIdx.y * strideT + (int64_t)(panel0 + i / kQrNB) * kQrNB * kQrNB + (i % kQrNB) +
          (j % kQrNB) * kQrNB];
  Tb[blockIdx.y * strideTb + i + (int64_t)j * kQrBlock] = v;
}

// One merge level of the block factor: for each pair of neighbouring diagonal
// blocks [a, a+h) and [a+h, a+h+w) of T_b (already merged up to width h),
//     T_b[a:a+h, a+h:a+h+w] = -T_11 (V_1^T V_2) T_22,
// which makes (I - V_1 T_11 V_1^T)(I - V_2 T_22 V_2^T) = I - V T V^T.  One CTA
// per column j of the right block, per pair and per shift; thread i owns row i.
__global__ void __launch_bounds__(kQrBlock / 2)
tb_merge_kernel(const double* __restrict__ G, int64_t strideG, double* __restrict__ Tb,
                int64_t strideTb, int nbb, int h) {
  __shared__ double x[kQrBlock / 2];
  const int j = blockIdx.x, i = threadIdx.x;
  const int a = blockIdx.y * 2 * h, b0 = a + h;
  const int w = nbb - b0 < h ? nbb - b0 : h;
  if (w <= 0 || j >= w) return;
  const double* Gs = G + blockIdx.z * strideG;
  double* T = Tb + blockIdx.z * strideTb;
  constexpr int ld = kQrBlock;
  if (i < h) {
    double t = 0.0;
    for (int k = 0; k <= j; ++k) t = fma(Gs[(a + i) + (int64_t)(b0 + k) * ld], T[(b0 + k) + (int64_t)(b0 + j) * ld], t);
    x[i] = t;
  }
  __syncthreads();
  if (i < h) {
    double t = 0.0;
    for (int k = i; k < h; ++k) t = fma(T[(a + i) + (int64_t)(a + k) * ld], x[k], t);
    T[(a + i) + (int64_t)(b0 + j) * ld] = -t;
  }
}

// Shared-memory form of the panel factorisation: each of the CG CTAs of a
// shift (one cluster; CG = 1 is a single CTA) loads its rows of the panel's 32
// columns into shared memory once, factors them there, and writes W, V and T
// back at the end.  The per-column steps are those of the cluster kernel above
// (norm and dot-product partials exchanged through distributed shared memory in
// rank order, so every CTA forms the same beta, tau and dots); only the panel's
// storage moves from L2 to shared memory, which removes the L2 round trips of
// the ~80 accesses per row and column.  The reflector's unit diagonal is kept
// implicit (the diagonal slot holds beta once it is formed), so no second copy
// of V is needed.  Rows per CTA: ceil((m + NB) / CG) <= kSmemPanelRows.
constexpr int kSmemPanelRows = 768;

// A one-CTA "cluster" needs no cluster barrier and no distributed shared memory:
// the panel kernels of one CTA per shift (the batched call's common case) use a
// CTA barrier and their own partial sums.
template <int CG>
__device__ __forceinline__ void panel_sync(cooperative_groups::cluster_group& cluster) {
  if constexpr (CG == 1) __syncthreads();
  else cluster.sync();
}
template <int CG>
__device__ __forceinline__ const double* panel_part(cooperative_groups::cluster_group& cluster,
                                                    double* p, int rank) {
  if constexpr (CG == 1) return p;
  else return cluster.map_shared_rank(p, rank);
}

template <int NB, int CG>
__global__ void __cluster_dims__(CG, 1, 1) __launch_bounds__(256)
qr_panel_smem_kernel(double* W, int64_t strideW, int64_t ldw, int64_t m, int64_t c0, int nbp,
                     double* V, int64_t strideV, int64_t ldv, double* T, int64_t strideT,
                     int* status) {
  namespace cgrp = cooperative_groups;
  cgrp::cluster_group cluster = cgrp::this_cluster();
  constexpr int kT = 256, kWarps = kT / 32;
  extern __shared__ double Ws[];              // NB columns x Rs rows, column-major
  __shared__ double part[2][NB + 2];          // [0, NB): dots, NB: norm^2, NB+1: alpha
  __shared__ double red[kWarps][NB + 2];
  __shared__ double dots[NB];
  __shared__ double cf[NB];                // -tau dots[q]: the update's coefficients
  __shared__ double Ts[NB][NB + 1];
  __shared__ double s_tau, s_scal, s_beta;

  const int rank = (int)cluster.block_rank();
  const int shift = blockIdx.x / CG;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* Wj = W + shift * strideW;
  double* Vp = V + shift * strideV + c0 * ldv;
  double* Tp = T + shift * strideT + (c0 / NB) * (int64_t)(NB * NB);
  const int64_t height = m + NB;
  const int Rs = (int)((height + CG - 1) / CG);
  const int64_t lo = c0 + (int64_t)rank * Rs;             // my window rows [lo, hi)
  const int64_t hi = lo + Rs < c0 + height ? lo + Rs : c0 + height;
  const int64_t rows_w = ldw;                             // rows that exist in W (m + n)
  const int nr = hi > lo ? (int)(hi - lo) : 0;

  for (int q = 0; q < NB; ++q)
    for (int rr = tid; rr < Rs; rr += kT) {
      const int64_t r = lo + rr;
      Ws[q * Rs + rr] = (q < nbp && rr < nr && r < rows_w) ? Wj[r + (c0 + q) * ldw] : 0.0;
    }
  for (int e = tid; e < NB * (NB + 1); e += kT) (&Ts[0][0])[e] = 0.0;
  __syncthreads();

  for (int i = 0; i < nbp; ++i) {
    const int64_t c = c0 + i;
    const int buf = i & 1;
    double* col = Ws + i * Rs;
    const int64_t r0 = lo > c ? lo : c;                  // my part of the support [c, m + c]
    const int64_t r1 = hi < m + c + 1 ? hi : m + c + 1;
    // ---- 1. partial norm of the tail (rows > c) and alpha from the owner of row c
    double ss = 0.0;
    for (int64_t r = (r0 > c + 1 ? r0 : c + 1) + tid; r < r1; r += kT) {
      const double v = col[r - lo];
      ss = fma(v, v, ss);
    }
    // the block's partials are summed by warp 0 (kWarps - 1 + 5 FP64 warp
    // instructions; a butterfly in every warp would take 5 per warp, and an FP64
    // instruction costs its unit a whole warp slot however few lanes it uses)
    double* flat = &red[0][0];
    flat[tid] = ss;
    __syncthreads();
    if (warp == 0) {
      double t = flat[lane];
#pragma unroll
      for (int w = 1; w < kWarps; ++w) t += flat[lane + 32 * w];
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) {
        part[buf][NB] = t;
        part[buf][NB + 1] = (c >= lo && c < hi) ? col[c - lo] : 0.0;
      }
    }
    panel_sync<CG>(cluster);
    if (tid == 0) {
      double sum = 0.0, alpha = 0.0;
      for (int rk = 0; rk < CG; ++rk) {
        const double* rp = panel_part<CG>(cluster, &part[buf][0], rk);
        sum += rp[NB];
        alpha += rp[NB + 1];
      }
      double beta, tau, scal;
      if (sum == 0.0) {
        beta = alpha; tau = 0.0; scal = 0.0;
      } else {
        beta = -copysign(sqrt(fma(alpha, alpha, sum)), alpha);
        tau = (beta - alpha) / beta;
        scal = 1.0 / (alpha - beta);
      }
      if (rank == 0 && (!isfinite(beta) || !isfinite(tau))) atomicOr(status + kStatNonFinite, 1);
      s_beta = beta; s_tau = tau; s_scal = scal;
    }
    __syncthreads();
    const double tau = s_tau, scal = s_scal;
    // ---- 2. my rows of v below the diagonal; the diagonal slot takes beta
    //         (v's unit diagonal is implicit from here on)
    for (int64_t r = (r0 > c + 1 ? r0 : c + 1) + tid; r < r1; r += kT) col[r - lo] *= scal;
    if (tid == 0 && c >= lo && c < hi) col[c - lo] = s_beta;
    __syncthreads();
    // ---- 3. dots of v with the other panel columns (the later ones for the
    //         update, the earlier reflectors for T): warp w takes the four columns
    //         4w..4w+3 over all my rows, lanes striding the rows, so each dot is
    //         reduced over 32 lanes (a four-value reduce-scatter, six adds a
    //         lane) instead of over every thread of the CTA
    static_assert(NB == 4 * kWarps, "four dot products per warp");
    {
      double a4[4] = {0.0, 0.0, 0.0, 0.0};
      const int q0 = 4 * warp;
      for (int64_t r = r0 + lane; r < r1; r += 32) {
        const double v = (r == c) ? 1.0 : col[r - lo];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int q = q0 + k;
          if (q < nbp && q != i) {
            // earlier reflector q: support rows [c0+q, m+c0+q]; r >= c > c0+q
            const double o = (q > i || r <= m + c0 + q) ? Ws[q * Rs + (r - lo)] : 0.0;
            a4[k] = fma(v, o, a4[k]);
          }
        }
      }
      // lanes with bit 16 keep values 2, 3 and send 0, 1 (and the reverse), then
      // bit 8 halves again; three butterflies finish the remaining value
      const bool up16 = (lane & 16) != 0, up8 = (lane & 8) != 0;
      const double k0 = up16 ? a4[2] : a4[0], k1 = up16 ? a4[3] : a4[1];
      const double s0 = up16 ? a4[0] : a4[2], s1 = up16 ? a4[1] : a4[3];
      const double b0 = k0 + __shfl_xor_sync(0xffffffffu, s0, 16);
      const double b1 = k1 + __shfl_xor_sync(0xffffffffu, s1, 16);
      double t = (up8 ? b1 : b0) + __shfl_xor_sync(0xffffffffu, up8 ? b0 : b1, 8);
      t += __shfl_xor_sync(0xffffffffu, t, 4);
      t += __shfl_xor_sync(0xffffffffu, t, 2);
      t += __shfl_xor_sync(0xffffffffu, t, 1);
      // lane 8 (2 * up16 + up8) holds column q0 + that index's dot
      if ((lane & 7) == 0) {
        const int q = q0 + 2 * (up16 ? 1 : 0) + (up8 ? 1 : 0);
        part[buf][q] = (q < nbp && q != i) ? t : 0.0;
      }
    }
    panel_sync<CG>(cluster);
    if (tid < NB) {
      double t = 0.0;
      for (int rk = 0; rk < CG; ++rk) t += panel_part<CG>(cluster, &part[buf][0], rk)[tid];
      dots[tid] = t;
      cf[tid] = -tau * t;
    }
    __syncthreads();
    // ---- 4. my rows of the later panel columns: W[:, q] -= tau * dots[q] * v
    //         (the coefficients formed once above: the stores to Ws may alias
    //         dots for the compiler, so a product written here would be redone
    //         for every row)
    for (int64_t r = r0 + tid; r < r1; r += kT) {
      const double v = (r == c) ? 1.0 : col[r - lo];
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        if (q > i && q < nbp) {
          double* pq = Ws + q * Rs + (r - lo);
          *pq = fma(cf[q], v, *pq);
        }
      }
    }
    // ---- 5. T(0:i, i) = -tau T(0:i, 0:i) V^T v_i (same in every CTA)
    if (tid < i) {
      double t = 0.0;
      for (int pc = tid; pc < i; ++pc) t = fma(Ts[tid][pc], dots[pc], t);
      Ts[tid][i] = -tau * t;
    }
    if (tid == 0) Ts[i][i] = tau;
    __syncthreads();
  }
  // ---- write back: W (R above the diagonal, beta on it, v below), the explicit
  //      reflectors (unit diagonal, exact zeros outside each support) and T
  for (int q = 0; q < nbp; ++q) {
    const int64_t cq = c0 + q;
    for (int rr = tid; rr < nr; rr += kT) {
      const int64_t r = lo + rr;
      const double w = Ws[q * Rs + rr];
      if (r < rows_w) Wj[r + cq * ldw] = w;
      Vp[(r - c0) + (int64_t)q * ldv] = (r < cq || r > m + cq) ? 0.0 : (r == cq ? 1.0 : w);
    }
  }
  if (rank == 0)
    for (int e = tid; e < NB * NB; e += kT) Tp[e] = Ts[e % NB][e / NB];
  panel_sync<CG>(cluster);   // no CTA leaves while another may still read its partials
}

// ------------------------------------------------------- skinny products
// C_t = A[:, i0:i0+mt]^T B[:, j0:j0+nt] over K rows, for up to three tiles t
// with mt <= 64, nt <= 96: the products whose output is a few thousand entries
// and whose inner dimension is the whole row window (m + w).  One GEMM tile per
// shift would leave most SMs idle for the length of K, so K is cut into chunks
// of kTsRows rows: each CTA stages one chunk of the columns it needs in shared
// memory and writes its partial tile; a second kernel sums the partials chunk
// by chunk in order (deterministic, FP64).
constexpr int kTsRows = 64;
constexpr int kTsThreads = 256;
constexpr int kTsMaxTile = 64 * 96;   // entries of one tile
struct TsTiles {
  int n;
  int i0[3], j0[3], mt[3], nt[3];
};

__global__ void __launch_bounds__(kTsThreads)
ts_partial_kernel(const double* __restrict__ A, int64_t lda, int64_t strideA,
                  const double* __restrict__ B, int64_t ldb, int64_t strideB, int64_t K,
                  TsTiles tl, double* __restrict__ P) {
  __shared__ double sA[kTsRows][65];
  __shared__ double sB[kTsRows][97];
  const int chunk = blockIdx.x, t = blockIdx.y, z = blockIdx.z;
  const int mt = tl.mt[t], nt = tl.nt[t];
  const double* Az = A + z * strideA + (int64_t)tl.i0[t] * lda;
  const double* Bz = B + z * strideB + (int64_t)tl.j0[t] * ldb;
  const int64_t k0 = (int64_t)chunk * kTsRows;
  const int kc = K - k0 < kTsRows ? (int)(K - k0) : kTsRows;
  for (int e = threadIdx.x; e < kTsRows * mt; e += kTsThreads) {
    const int k = e % kTsRows, i = e / kTsRows;
    sA[k][i] = k < kc ? Az[k0 + k + (int64_t)i * lda] : 0.0;
  }
  for (int e = threadIdx.x; e < kTsRows * nt; e += kTsThreads) {
    const int k = e % kTsRows, j = e / kTsRows;
    sB[k][j] = k < kc ? Bz[k0 + k + (int64_t)j * ldb] : 0.0;
  }
  __syncthreads();
  double* Pz = P + (((int64_t)chunk * gridDim.z + z) * gridDim.y + t) * kTsMaxTile;
  for (int e = threadIdx.x; e < mt * nt; e += kTsThreads) {
    const int i = e % mt, j = e / mt;
    double acc = 0.0;
#pragma unroll 8
    for (int k = 0; k < kTsRows; ++k) acc = fma(sA[k][i], sB[k][j], acc);
    Pz[e] = acc;
  }
}

__global__ void ts_reduce_kernel(const double* __restrict__ P, int nchunks, TsTiles tl,
                                 double* __restrict__ C, int64_t ldc, int64_t strideC) {
  const int t = blockIdx.y, z = blockIdx.z;
  const int mt = tl.mt[t], nt = tl.nt[t];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= mt * nt) return;
  double s = 0.0;
  for (int c = 0; c < nchunks; ++c)
    s += P[(((int64_t)c * gridDim.z + z) * gridDim.y + t) * kTsMaxTile + e];
  C[z * strideC + (tl.i0[t] + e % mt) + (int64_t)(tl.j0[t] + e / mt) * ldc] = s;
}

// C[i0.., j0..] = A[:, i0..]^T B[:, j0..] for the tiles of tl, r shifts (strides
// per shift), K rows; P holds the partials.
cudaError_t ts_product(const double* A, int64_t lda, int64_t strideA, const double* B, int64_t ldb,
                       int64_t strideB, int64_t K, const TsTiles& tl, double* C, int64_t ldc,
                       int64_t strideC, int r, double* P, int64_t elemsP, cudaStream_t st) {
  const int nchunks = (int)((K + kTsRows - 1) / kTsRows);
  if ((int64_t)nchunks * r * tl.n * kTsMaxTile > elemsP) return cudaErrorInvalidValue;
  for (int t = 0; t < tl.n; ++t)
    if (tl.mt[t] > 64 || tl.nt[t] > 96 || tl.mt[t] < 1 || tl.nt[t] < 1) return cudaErrorInvalidValue;
  double fl = 0.0;
  for (int t = 0; t < tl.n; ++t) fl += 2.0 * tl.mt[t] * tl.nt[t] * (double)K * r;
  {
    ProfScope ps(kProfGemm, st, fl, 0.0);
    ps.blocks((const void*)ts_partial_kernel, dim3(kTsThreads), 0, dim3(nchunks, tl.n, r));
    ts_partial_kernel<<<dim3(nchunks, tl.n, r), kTsThreads, 0, st>>>(A, lda, strideA, B, ldb,
                                                                     strideB, K, tl, P);
  }
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  ProfScope ps(kProfOther, st);
  ps.blocks((const void*)ts_reduce_kernel, dim3(256), 0, dim3(kTsMaxTile / 256, tl.n, r));
  ts_reduce_kernel<<<dim3(kTsMaxTile / 256, tl.n, r), 256, 0, st>>>(P, nchunks, tl, C, ldc, strideC);
  return cudaGetLastError();
}

// C <- (I - V op(T) V^T) C for r shifts, on the row window of C, as
// W1 = V^T C, W2 = op(T) W1, C -= V W2 (transT = 1 applies Q^T, the
// factorisation's update; transT = 0 applies Q, the explicit-Q build).
cudaError_t apply_block(const QrBuffers& b, const double* Vw, int64_t ldv, const double* Tw,
                        int ldt, int64_t strideT, double* C, int64_t ldw, int64_t rows, int w,
                        int64_t ncols, int r, int transT, cudaStream_t st) {
  cudaError_t err;
  GemmArgs g;
  g.M = w; g.N = (int)ncols; g.K = (int)rows; g.transA = 1; g.transB = 0;
  g.A = Vw; g.lda = ldv; g.strideA = b.strideV;
  g.B = C; g.ldb = ldw; g.strideB = b.strideW;
  g.Cout = b.W1; g.ldcout = kQrBlock; g.strideCout = b.strideW1;
  g.batch = r;
  for (int j = 0; j < r; ++j) g.alpha[j] = 1.0;
  if (w <= 32 && ncols <= 96) {
    // a panel's own block: a skinny output over the whole window, split over K
    TsTiles tl{1, {0}, {0}, {w}, {(int)ncols}};
    err = ts_product(Vw, ldv, b.strideV, C, ldw, b.strideW, rows, tl, b.W1, kQrBlock, b.strideW1,
                     r, b.P, b.elemsP, st);
  } else {
    err = gemm_any(g, st);
  }
  if (err != cudaSuccess) return err;
  GemmArgs h = g;
  h.K = w; h.transA = transT;
  h.A = Tw; h.lda = ldt; h.strideA = strideT;
  h.B = b.W1; h.ldb = kQrBlock; h.strideB = b.strideW1;
  h.Cout = b.W2; h.strideCout = b.strideW2;
  if ((err = gemm_any(h, st)) != cudaSuccess) return err;
  GemmArgs u = g;
  u.M = (int)rows; u.N = (int)ncols; u.K = w; u.transA = 0; u.transB = 0;
  u.A = Vw; u.lda = ldv; u.strideA = b.strideV;
  u.B = b.W2; u.ldb = kQrBlock; u.strideB = b.strideW2;
  u.Cin = C; u.ldcin = ldw; u.strideCin = b.strideW; u.beta = 1.0;
  u.Cout = C; u.ldcout = ldw; u.strideCout = b.strideW;
  for (int j = 0; j < r; ++j) u.alpha[j] = -1.0;
  // the rows of W2 follow the trailing matrix, whose size decays across the
  // block's reflectors like the singular values: equilibrate them
  u.k_equilibrate = 1;
  return gemm_any(u, st);
}

}  // namespace

int64_t qr_partial_elems(int64_t m, int r) {
  const int64_t nchunks = (m + kQrBlock + kTsRows - 1) / kTsRows;
  return nchunks * r * 3 * kTsMaxTile;
}

cudaError_t structured_qr_q(const QrBuffers& b, int64_t m, int64_t n, int r, int* status,
                            cudaStream_t st, bool explicit_q, bool narrow_panels) {
  constexpr int NB = kQrNB, NBb = kQrBlock;
  {
    const int bytes = (int)(sizeof(double) * NB * kSmemPanelRows);
    if (smem_attr_once((const void*)qr_panel_smem_kernel<NB, 2>, bytes) != cudaSuccess ||
        smem_attr_once((const void*)qr_panel_smem_kernel<NB, 4>, bytes) != cudaSuccess ||
        smem_attr_once((const void*)qr_panel_smem_kernel<NB, 1>, bytes) != cudaSuccess ||
        smem_attr_once((const void*)qr_panel_smem_kernel<NB, kPanelCluster>, bytes) != cudaSuccess)
      return cudaErrorInvalidConfiguration;
  }
  const int64_t ldw = m + n;
  const int64_t ldv = m + NBb;
  cudaError_t err;
  const int nblocks = (int)((n + NBb - 1) / NBb);
  // CTAs per shift of the panel kernel.  The panel is a chain of dependent
  // column steps on a few SMs.  Alone (one matrix, r shifts in flight) it goes
  // fastest on an 8-CTA cluster, which splits each column's rows eight ways;
  // when many problems are in flight (narrow_panels) the same SMs serve more
  // panels at once with the fewest CTAs whose rows fit in shared memory (one
  // CTA up to m = 736, two up to 1504).  0: the global-memory cluster kernel.
  int cg = 0;
  if (narrow_panels) {
    for (int c = 1; c <= kPanelCluster; c *= 2)
      if ((m + NB + c - 1) / c <= kSmemPanelRows) { cg = c; break; }
  } else if (m + NB <= kSmemPanelRows && m < kClusterPanelMinRows) {
    cg = 1;
  } else if ((m + NB + kPanelCluster - 1) / kPanelCluster <= kSmemPanelRows) {
    cg = kPanelCluster;
  }
  const int64_t rows_cta = cg ? (m + NB + cg - 1) / cg : 0;
  // every V entry outside the rows a panel writes must be an exact zero
  if ((err = cudaMemsetAsync(b.V, 0, sizeof(double) * r * b.strideV, st)) != cudaSuccess) return err;
  // ---------------- factorisation (structured GEQRF)
  for (int blk = 0; blk < nblocks; ++blk) {
    const int64_t c0b = (int64_t)blk * NBb;
    const int nbb = (int)(n - c0b < NBb ? n - c0b : NBb);
    for (int p = 0; p * NB < nbb; ++p) {
      const int64_t c0 = c0b + (int64_t)p * NB;
      const int nbp = nbb - p * NB < NB ? nbb - p * NB : NB;
      // V rows are relative to the block start: this panel's window starts p*NB down
      double* Vpan = b.V + (int64_t)p * NB;
      {
        ProfScope ps(kProfPanel, st, 3.0 * r * (double)(m + 1) * nbp * nbp,
                     8.0 * r * (double)(m + NB) * nbp * 2.0);
        const size_t smem = sizeof(double) * NB * rows_cta;
        if (cg == 0)
          ps.blocks((const void*)qr_panel_cluster_kernel<NB, kPanelCluster, 512>, dim3(512), 0,
                    dim3(r * kPanelCluster));
        else
          ps.blocks((const void*)qr_panel_smem_kernel<NB, 1>, dim3(256), smem, dim3(r * cg));
        if (cg == 1)
          qr_panel_smem_kernel<NB, 1><<<r, 256, smem, st>>>(
              b.W, b.strideW, ldw, m, c0, nbp, Vpan, b.strideV, ldv, b.T, b.strideT, status);
        else if (cg == 2)
          qr_panel_smem_kernel<NB, 2><<<r * 2, 256, smem, st>>>(
              b.W, b.strideW, ldw, m, c0, nbp, Vpan, b.strideV, ldv, b.T, b.strideT, status);
        else if (cg == 4)
          qr_panel_smem_kernel<NB, 4><<<r * 4, 256, smem, st>>>(
              b.W, b.strideW, ldw, m, c0, nbp, Vpan, b.strideV, ldv, b.T, b.strideT, status);
        else if (cg == kPanelCluster)
          qr_panel_smem_kernel<NB, kPanelCluster><<<r * kPanelCluster, 256, smem, st>>>(
              b.W, b.strideW, ldw, m, c0, nbp, Vpan, b.strideV, ldv, b.T, b.strideT, status);
        else
          // tall panels (m > 8 x 768 rows): 512 threads per CTA halve each thread's
          // share of the rows on the serial chain of every column
          qr_panel_cluster_kernel<NB, kPanelCluster, 512><<<r * kPanelCluster, 512, 0, st>>>(
              b.W, b.strideW, ldw, m, c0, nbp, Vpan, b.strideV, ldv, b.T, b.strideT, status);
      }
      if ((err = cudaGetLastError()) != cudaSuccess) return err;
      // the rest of this block's columns
      const int64_t nin = c0b + nbb - (c0 + nbp);
      if (nin > 0) {
        const double* Vp = Vpan + c0 * ldv;
        const double* Tp = b.T + (c0 / NB) * (int64_t)(NB * NB);
        if ((err = apply_block(b, Vp, ldv, Tp, NB, b.strideT, b.W + c0 + (c0 + nbp) * ldw, ldw,
                               m + nbp, nbp, nin, r, 1, st)) != cudaSuccess)
          return err;
      }
    }
    // ---- the block factor T_b: panel factors on the diagonal, merged pairwise
    const double* Vb = b.V + c0b * ldv;
    double* Tb = b.Tb + (int64_t)blk * NBb * NBb;
    {
      ProfScope ps(kProfOther, st);
      ps.blocks((const void*)tb_init_kernel, dim3(256), 0, dim3((nbb * nbb + 255) / 256, r));
      tb_init_kernel<<<dim3((nbb * nbb + 255) / 256, r), 256, 0, st>>>(b.T, b.strideT, Tb,
                                                                      b.strideTb, (int)(c0b / NB), nbb);
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (nbb > NB) {
      // the blocks of G = V_b^T V_b that the merges read: [0,32)x[32,64),
      // [64,96)x[96,128) and [0,64)x[64,128) (clipped to the block), in FP64 on
      // every path: they are small next to the columns' norms, and T_b carries
      // their error into every update
      static_assert(kQrBlock == 4 * kQrNB, "the merge levels assume four panels per block");
      TsTiles tl{};
      auto add = [&](int i0, int j0, int mt, int nt) {
        nt = nbb - j0 < nt ? nbb - j0 : nt;
        if (nt > 0) { tl.i0[tl.n] = i0; tl.j0[tl.n] = j0; tl.mt[tl.n] = mt; tl.nt[tl.n] = nt; ++tl.n; }
      };
      add(0, 32, 32, 32);
      add(64, 96, 32, 32);
      add(0, 64, 64, 64);
      if ((err = ts_product(Vb, ldv, b.strideV, Vb, ldv, b.strideV, m + nbb, tl, b.G, NBb, b.strideG,
                            r, b.P, b.elemsP, st)) != cudaSuccess)
        return err;
      for (int h = NB; h < nbb; h *= 2) {
        const int pairs = (nbb + 2 * h - 1) / (2 * h);
        {
          ProfScope ps(kProfOther, st);
          ps.blocks((const void*)tb_merge_kernel, dim3(NBb / 2), 0, dim3(h, pairs, r));
          tb_merge_kernel<<<dim3(h, pairs, r), NBb / 2, 0, st>>>(b.G, b.strideG, Tb, b.strideTb,
                                                                 nbb, h);
        }
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
      }
    }
    // ---- all later columns, once per block
    const int64_t ntr = n - c0b - nbb;
    if (ntr > 0 &&
        (err = apply_block(b, Vb, ldv, Tb, NBb, b.strideTb, b.W + c0b + (c0b + nbb) * ldw, ldw,
                           m + nbb, nbb, ntr, r, 1, st)) != cudaSuccess)
      return err;
  }
  if (!explicit_q) return cudaSuccess;
  // ---------------- explicit Q (structured ORGQR), overwriting W
  if ((err = init_q_identity(b.W, b.strideW, m, n, r, st)) != cudaSuccess) return err;
  for (int blk = nblocks - 1; blk >= 0; --blk) {
    const int64_t c0b = (int64_t)blk * NBb;
    const int nbb = (int)(n - c0b < NBb ? n - c0b : NBb);
    if ((err = apply_block(b, b.V + c0b * ldv, ldv, b.Tb + (int64_t)blk * NBb * NBb, NBb,
                           b.strideTb, b.W + c0b + c0b * ldw, ldw, m + nbb, nbb, n - c0b, r, 0,
                           st)) != cudaSuccess)
      return err;
  }
  return cudaSuccess;
}

}  // namespace zolo
