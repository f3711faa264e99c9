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
// X32 = R^T with the rotations accumulated in Z32, as block Jacobi on 16-column
// blocks (one cooperative launch per sweep, rounds separated by a bounded grid
// barrier).  Z is then made orthonormal in FP64 (Cholesky QR), X = R^T Z is
// formed in FP64, and FP64 sweeps (one cooperative dataflow launch per sweep,
// one CTA per column pair at a time) finish from cosines ~1e-4 in a few
// quadratically convergent sweeps.
// FP32 sweeps stop when fewer than n rotations (cosines above 8e-6) were needed
// in a sweep (25 sweeps at most): the FP64 sweeps start from cosines of about
// 1e-4 whatever the last FP32 sweeps do, since Z's FP32 rounding, times R^T,
// sets them.  FP64 sweeps stop when no pair has |x_p . x_q| > 8 eps ||x_p||
// ||x_q||, or after a sweep in which every cosine was below sqrt(n) eps (the
// rounding level of an n-term dot product): its rotations were of that size,
// so the next sweep would find the same rounding-level cosines again.
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

// Per-column round counters of the FP64 sweep: acquire/release at GPU scope.
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits until *ver >= want, two seconds at most (by the global timer), giving up
// at once when another block has set the error flag; false (and *err set) on
// time-out.
__device__ bool wait_round(const int* ver, int want, int* err) {
  if (ld_acquire(ver) >= want) return true;
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (unsigned k = 0;; ++k) {
    if (ld_acquire(ver) >= want) return true;
    if ((k & 63u) == 63u) {
      if (*(volatile int*)err) return false;
      uint64_t t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > 2000000000ull) break;
    }
    __nanosleep(32);
  }
  atomicExch(err, 1);
  return false;
}

// One FP64 sweep (the n_even - 1 rounds of the round-robin ordering, n_even / 2
// column pairs each) in one cooperative launch, as a dataflow: pair (round k, i)
// is work item k * n_even / 2 + i, block b takes the items b, b + gridDim.x, ...
// in order, and an item starts as soon as the two items of round k - 1 that
// held its columns are done (per-column round counters, acquire / release),
// instead of after a launch boundary that waits for the whole round.  Every
// block is resident (cooperative launch) and takes its items in increasing
// order, and an item waits only for lower-numbered items, so the lowest
// unfinished item can always run.  Columns are read through L2 (__ldcg): this
// SM's L1 may hold a column from an earlier round.
//
// Per pair: the squared column norms are tracked in nrm2 (formed afresh at the
// start of every sweep): a rotation with t = tan(theta) changes them exactly to
// a - t g and b + t g, so only the cross product of the pair is formed.  The
// rotations are the scaled ("fast") form: column j is held as dsc[j] * x~_j, the
// cosine goes into the scales (dsc_p <- c dsc_p, dsc_q <- c dsc_q) and each
// stored column takes one FMA, x~_p -= t (dsc_q / dsc_p) x~_q and
// x~_q += t (dsc_p / dsc_q) x~_p: three FP64 operations per row and pair instead
// of five (the FP64 pipe is the bound).  Near convergence c = 1 - O(t^2), so the
// scales stay within rounding of 1 over a sweep; the caller folds them into the
// columns between sweeps.
// An FP64 instruction occupies its sub-partition's FP64 unit for a whole warp
// slot however few lanes are active, so the block's 256 partial dot products
// are summed by one warp (7 + 5 warp instructions instead of 5 per warp plus 8
// on one lane), and the warp that sums them and forms the rotation changes with
// the item: the scalar work spreads over the SM's four sub-partitions.
__global__ void __launch_bounds__(kJacThreads)
jacobi_sweep_kernel(double* X, int64_t ldx, int64_t m, int n_even, int n_real, double tol,
                    int* status, double* nrm2, double* dsc, int* ver, int* err, int stall,
                    long long stall_ns) {
  __shared__ double part[kJacThreads];
  __shared__ double s_al, s_be;
  __shared__ int s_rot, s_ok, never;
  const int npairs = n_even / 2;
  const int64_t items = (int64_t)(n_even - 1) * npairs;
  if (stall && blockIdx.x == 0) {
    // test hook of the error exit: item 0 first waits, bounded, on a flag that
    // nothing sets; the blocks whose items need its columns leave on the flag
    if (threadIdx.x == 0) {
      never = 0;
      long long t0;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      for (;;) {
        if (*(volatile int*)&never) break;
        long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > stall_ns) break;
        __nanosleep(256);
      }
      atomicExch(err, 1);
    }
    __syncthreads();
    return;
  }
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int round = (int)(it / npairs), i = (int)(it - (int64_t)round * npairs);
    auto elem = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + round) % (n_even - 1); };
    int p = elem(i), q = elem(n_even - 1 - i);
    if (p > q) { const int t = p; p = q; q = t; }
    const bool real = q < n_real;      // the pair with the padding column is no work
    if (threadIdx.x == 0)
      s_ok = !*(volatile int*)err && wait_round(ver + p, round, err) &&
             (!real || wait_round(ver + q, round, err));
    __syncthreads();
    if (!s_ok) return;
    if (real) {
      double* xp = X + p * ldx;
      double* xq = X + q * ldx;
      double g = 0.0;
      for (int64_t r = threadIdx.x; r < m; r += kJacThreads) g = fma(__ldcg(xp + r), __ldcg(xq + r), g);
      part[threadIdx.x] = g;
      __syncthreads();
      const int lead = (int)(it & (kJacThreads / 32 - 1));   // the warp that forms the rotation
      if ((int)(threadIdx.x >> 5) == lead) {
        const int l = threadIdx.x & 31;
        double sg = part[l];
#pragma unroll
        for (int k = 1; k < kJacThreads / 32; ++k) sg += part[l + 32 * k];
        sg = warp_sum(sg);
        if (l == 0) {
          // One lane's scalar work costs whole FP64 warp instructions on this
          // part, so only what fixes the rotation exactly is FP64: the cosine
          // test and the angle are formed in FP32 (an angle off by 1e-7 only
          // slows convergence by that factor), while c = (1 + t^2)^(-1/2) for
          // the t actually applied, the norm and scale updates are FP64 (Newton
          // steps from FP32 seeds).
          const double dp = __ldcg(dsc + p), dq = __ldcg(dsc + q);
          sg *= dp * dq;                                  // cross product of the true columns
          const double sa = __ldcg(nrm2 + p), sb = __ldcg(nrm2 + q);
          const float fa = (float)sa, fb = (float)sb;     // below float range: left as converged
          const float cosv = (fa > 0.f && fb > 0.f) ? fabsf((float)sg) * rsqrtf(fa) * rsqrtf(fb) : 0.f;
          atomicMax(status + kStatJacobiMaxCos, __float_as_int(cosv));
          const int rot = (sg != 0.0) && (cosv > (float)tol);
          if (rot) {
            const float zeta = (float)((sb - sa) / (2.0 * sg));
            const float az = fabsf(zeta);
            const float tf = (az > 1e18f ? 0.5f / az : 1.f / (az + sqrtf(fmaf(az, az, 1.f))));
            const double t = zeta >= 0.f ? (double)tf : -(double)tf;
            const double x = fma(t, t, 1.0);
            double c = (double)rsqrtf((float)x);
            c = c * fma(-0.5 * x * c, c, 1.5);
            c = c * fma(-0.5 * x * c, c, 1.5);
            double rp = (double)(1.f / (float)dp), rq = (double)(1.f / (float)dq);
            rp = rp * fma(-dp, rp, 2.0); rp = rp * fma(-dp, rp, 2.0);
            rq = rq * fma(-dq, rq, 2.0); rq = rq * fma(-dq, rq, 2.0);
            nrm2[p] = fma(-t, sg, sa);
            nrm2[q] = fma(t, sg, sb);
            dsc[p] = c * dp;
            dsc[q] = c * dq;
            s_al = t * (dq * rp);
            s_be = t * (dp * rq);
            atomicAdd(status + kStatJacobiRot, 1);
          }
          s_rot = rot;
        }
      }
      __syncthreads();
      if (s_rot) {
        const double al = s_al, be = s_be;
        for (int64_t r = threadIdx.x; r < m; r += kJacThreads) {
          const double u = __ldcg(xp + r), v = __ldcg(xq + r);
          xp[r] = fma(-al, v, u);
          xq[r] = fma(be, u, v);
        }
      }
    }
    // publish: the block barrier orders every thread's stores before thread 0's
    // release of the columns' round counters (a release at GPU scope covers what
    // happens before it in the block), which the next pair's acquire pairs with
    __syncthreads();
    if (threadIdx.x == 0) {
      st_release(ver + p, round + 1);
      if (real) st_release(ver + q, round + 1);
    }
  }
}

__global__ void fill_kernel(double* d, int64_t n, double v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = v;
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

// One FP32 sweep of block Jacobi: the columns are grouped in blocks of kJB,
// the blocks paired by the round-robin ordering, and each CTA takes one block
// pair per round: it forms the Gram matrix G = C^T C of the pair's 2 kJB
// columns (one pass over the rows, staged through shared memory), runs
// kJInner cyclic Jacobi sweeps on G in shared memory (the rotation from the
// 2x2 Gram entries of a column pair is the one-sided rotation of those two
// columns; J^T G J keeps G current), and applies the accumulated rotation Q to
// the pair's columns of X32 and Z32 in one more pass.  Each column is read a
// few times per visit instead of once per rotation.  Rounds are separated by a
// bounded grid barrier.  A rotation is counted when |g_pq| > tol sqrt(g_pp g_qq).
constexpr int kJB = 16;                // columns per block
constexpr int kJW = 2 * kJB;           // columns of a block pair
constexpr int kJRows = 256;            // rows per staged chunk (one per thread when loading)
constexpr int kJLd = kJRows + 1;       // chunk leading dimension: conflict-free column and row walks
constexpr int kJInner = 1;             // Jacobi sweeps on G per visit

__global__ void __launch_bounds__(kJacThreads, 2)
jacobi32_block_sweep_kernel(float* X, float* Z, int64_t ld, int64_t m, int nb_even, int n_real,
                            float tol, int* status, unsigned* bar, int* err, int stall,
                            long long stall_ns, int split, float* Gp) {
  static_assert(kJacThreads == 256 && kJW == 32 && kJRows == kJacThreads, "thread mapping below");
  __shared__ float Ct[kJW * kJLd];             // chunk, column-major: Ct[j * kJLd + r]
  __shared__ float G[kJW][kJW + 1];
  __shared__ float Qm[kJW][kJW + 1];
  __shared__ __align__(16) float Q4[kJW][kJW]; // Q for the vectorised product
  __shared__ float s_c[kJB], s_s[kJB];
  __shared__ int s_a[kJB], s_b[kJB];
  if (stall && blockIdx.x == 0) {
    // test hook of the error exit: wait, bounded, on a flag that nothing sets
    __shared__ int never;
    if (threadIdx.x == 0) {
      never = 0;
      long long t0;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      for (;;) {
        if (*(volatile int*)&never) break;
        long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > stall_ns) break;
        __nanosleep(256);
      }
      atomicExch(err, 1);
    }
    __syncthreads();
    return;
  }
  __shared__ int s_rot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int npairs = nb_even / 2;
  // split = 2: two blocks per block pair, each on half of the rows, so that an
  // SM holds two blocks (16 warps) where one left it latency-bound; their Gram
  // partials meet through Gp after a grid barrier (the host launches exactly
  // 2 x npairs blocks then, so every block reaches that barrier once per round)
  const int half = split == 2 ? (int)(blockIdx.x & 1) : 0;
  const int64_t mh = split == 2 ? ((m + 1) / 2 + kJRows - 1) / kJRows * kJRows : m;
  const int64_t row_lo = half * mh;
  const int64_t row_hi = row_lo + mh < m ? row_lo + mh : m;
  for (int round = 0; round < nb_even - 1; ++round) {
    for (int pi = blockIdx.x / split; pi < npairs; pi += gridDim.x / split) {
      auto elem = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + round) % (nb_even - 1); };
      int P = elem(pi), Qb = elem(nb_even - 1 - pi);
      if (P > Qb) { const int t = P; P = Qb; Qb = t; }
      auto col = [&](int j) { return j < kJB ? P * kJB + j : Qb * kJB + (j - kJB); };
      // chunk loader: thread = row, all 32 columns (coalesced along each column).
      // The next chunk is fetched into registers while the current one is used.
      float pf[kJW];
      auto fetch = [&](const float* M, int64_t r0) {
        const int64_t r = r0 + tid;
#pragma unroll
        for (int j = 0; j < kJW; ++j) {
          const int c = col(j);
          pf[j] = (c < n_real && r < row_hi) ? M[(int64_t)c * ld + r] : 0.f;
        }
      };
      auto stage = [&]() {
#pragma unroll
        for (int j = 0; j < kJW; ++j) Ct[j * kJLd + tid] = pf[j];
      };
      // ---- 1. Gram G = C^T C: 16 row groups; thread owns the 8x8 block (bi, bj)
      //         of G over the rows r = g (mod 16) of each chunk
      {
        const int g = tid >> 4, t = tid & 15, bi = t >> 2, bj = t & 3;
        float acc[8][8];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
        fetch(X, row_lo);
        for (int64_t r0 = row_lo; r0 < row_hi; r0 += kJRows) {
          stage();
          __syncthreads();
          if (r0 + kJRows < row_hi) fetch(X, r0 + kJRows);
          for (int r = g; r < kJRows; r += 16) {
            float va[8], vb[8];
#pragma unroll
            for (int a = 0; a < 8; ++a) va[a] = Ct[(8 * bi + a) * kJLd + r];
#pragma unroll
            for (int b = 0; b < 8; ++b) vb[b] = Ct[(8 * bj + b) * kJLd + r];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
              for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(va[a], vb[b], acc[a][b]);
          }
          __syncthreads();
        }
        // groups 2w and 2w+1 share warp w (lanes l and l ^ 16): fold them, then
        // sum the 8 warps' partials through the chunk buffer
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) acc[a][b] += __shfl_xor_sync(0xffffffffu, acc[a][b], 16);
        if (lane < 16)
#pragma unroll
          for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) Ct[warp * kJW * kJW + (8 * bi + a) * kJW + (8 * bj + b)] = acc[a][b];
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = tid + kJacThreads * u, i = e >> 5, jj = e & 31;
          float sum = 0.f;
#pragma unroll
          for (int w = 0; w < kJacThreads / 32; ++w) sum += Ct[w * kJW * kJW + e];
          G[i][jj] = sum;
          Qm[i][jj] = i == jj ? 1.f : 0.f;
          if (split == 2) Gp[((int64_t)pi * 2 + half) * kJW * kJW + e] = sum;
        }
      }
      if (split == 2) {
        // both halves' partials, summed in the same order by both blocks (read
        // through L2: the partner wrote them on another SM)
        if (!grid_barrier(bar, bar + 1, err)) return;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = tid + kJacThreads * u, i = e >> 5, jj = e & 31;
          G[i][jj] = __ldcg(Gp + (int64_t)pi * 2 * kJW * kJW + e) +
                     __ldcg(Gp + ((int64_t)pi * 2 + 1) * kJW * kJW + e);
        }
      }
      if (tid == 0) s_rot = 0;
      __syncthreads();
      // ---- 2. cyclic Jacobi on G (round-robin over the 32 indices, 16 disjoint
      //         rotations per step); Q accumulates the rotations
      for (int sw = 0; sw < kJInner; ++sw) {
        for (int step = 0; step < kJW - 1; ++step) {
          if (tid < kJB) {
            auto e2 = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + step) % (kJW - 1); };
            int a = e2(tid), b = e2(kJW - 1 - tid);
            if (a > b) { const int t = a; a = b; b = t; }
            const float ga = G[a][a], gb = G[b][b], gab = G[a][b];
            float c = 1.f, sn = 0.f;
            if (col(b) < n_real && gab != 0.f && fabsf(gab) > tol * sqrtf(ga) * sqrtf(gb)) {
              const float zeta = (gb - ga) / (2.f * gab);
              const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
              c = 1.f / sqrtf(fmaf(t, t, 1.f));
              sn = c * t;
              atomicAdd(&s_rot, 1);
            }
            s_a[tid] = a; s_b[tid] = b; s_c[tid] = c; s_s[tid] = sn;
          }
          __syncthreads();
          // rows a, b of G (J^T G): 16 rotations x 32 entries, two per thread
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int e = tid + kJacThreads * u, t = e >> 5, k = e & 31;
            const int a = s_a[t], b = s_b[t];
            const float c = s_c[t], sn = s_s[t];
            const float x = G[a][k], y = G[b][k];
            G[a][k] = c * x - sn * y;
            G[b][k] = fmaf(sn, x, c * y);
          }
          __syncthreads();
          // columns a, b of G and of Q (G J, Q J)
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int e = tid + kJacThreads * u, t = e >> 5, k = e & 31;
            const int a = s_a[t], b = s_b[t];
            const float c = s_c[t], sn = s_s[t];
            const float x = G[k][a], y = G[k][b];
            G[k][a] = c * x - sn * y;
            G[k][b] = fmaf(sn, x, c * y);
            const float qx = Qm[k][a], qy = Qm[k][b];
            Qm[k][a] = c * qx - sn * qy;
            Qm[k][b] = fmaf(sn, qx, c * qy);
          }
          __syncthreads();
        }
      }
      const int nrot = s_rot;
      if (tid == 0 && nrot && half == 0) atomicAdd(status + kStatJacobiRot, nrot);
      // ---- 3. X and Z columns of the pair times Q (skipped when nothing rotated):
      //         thread computes rows 8 rt .. 8 rt + 7, columns 4 ct .. 4 ct + 3
      if (nrot) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = tid + kJacThreads * u;
          Q4[e >> 5][e & 31] = Qm[e >> 5][e & 31];
        }
        const int rt = tid >> 3, ct = tid & 7;
        for (int which = 0; which < 2; ++which) {
          float* M = which ? Z : X;
          fetch(M, row_lo);
          for (int64_t r0 = row_lo; r0 < row_hi; r0 += kJRows) {
            stage();
            __syncthreads();
            if (r0 + kJRows < row_hi) fetch(M, r0 + kJRows);
            float o[8][4];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
              for (int b = 0; b < 4; ++b) o[a][b] = 0.f;
#pragma unroll 4
            for (int k = 0; k < kJW; ++k) {
              const float4 q = *reinterpret_cast<const float4*>(&Q4[k][4 * ct]);
#pragma unroll
              for (int a = 0; a < 8; ++a) {
                const float cv = Ct[k * kJLd + 8 * rt + a];
                o[a][0] = fmaf(cv, q.x, o[a][0]);
                o[a][1] = fmaf(cv, q.y, o[a][1]);
                o[a][2] = fmaf(cv, q.z, o[a][2]);
                o[a][3] = fmaf(cv, q.w, o[a][3]);
              }
            }
            __syncthreads();
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
              for (int b = 0; b < 4; ++b) Ct[(4 * ct + b) * kJLd + 8 * rt + a] = o[a][b];
            __syncthreads();
            const int64_t r = r0 + tid;
#pragma unroll 8
            for (int j = 0; j < kJW; ++j) {
              const int c = col(j);
              if (c < n_real && r < row_hi) M[(int64_t)c * ld + r] = Ct[j * kJLd + tid];
            }
            __syncthreads();
          }
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
  ps.blocks((const void*)column_norms_kernel, dim3(kJacThreads), 0, dim3((unsigned)n));
  column_norms_kernel<<<(unsigned)n, kJacThreads, 0, st>>>(X, ldx, m, out);
  return cudaGetLastError();
}

cudaError_t column_dots(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t m,
                        int64_t n, double* out, cudaStream_t st) {
  ProfScope ps(kProfOther, st);
  ps.blocks((const void*)column_dots_kernel, dim3(kJacThreads), 0, dim3((unsigned)n));
  column_dots_kernel<<<(unsigned)n, kJacThreads, 0, st>>>(A, lda, B, ldb, m, out);
  return cudaGetLastError();
}

cudaError_t scale_columns(double* X, int64_t ldx, int64_t m, int64_t n, const double* s, int invert,
                          cudaStream_t st) {
  ProfScope ps(kProfOther, st);
  ps.blocks((const void*)scale_columns_kernel, dim3(256), 0, dim3(rows_grid(m), (unsigned)n));
  scale_columns_kernel<<<dim3(rows_grid(m), (unsigned)n), 256, 0, st>>>(X, ldx, m, s, invert);
  return cudaGetLastError();
}

cudaError_t gather_columns(const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t m,
                           int64_t n, const int* perm, const double* sign, cudaStream_t st) {
  ProfScope ps(kProfOther, st);
  ps.blocks((const void*)gather_columns_kernel, dim3(256), 0, dim3(rows_grid(m), (unsigned)n));
  gather_columns_kernel<<<dim3(rows_grid(m), (unsigned)n), 256, 0, st>>>(X, ldx, Y, ldy, m, perm,
                                                                         sign);
  return cudaGetLastError();
}

cudaError_t transpose_lower(const double* R, int64_t ldr, double* X, int64_t ldx, int64_t n,
                            cudaStream_t st) {
  const int64_t b = std::min<int64_t>((n * n + 255) / 256, 4096);
  ProfScope ps(kProfOther, st);
  ps.blocks((const void*)transpose_lower_kernel, dim3(256), 0,
            dim3((unsigned)std::max<int64_t>(b, 1)));
  transpose_lower_kernel<<<(unsigned)std::max<int64_t>(b, 1), 256, 0, st>>>(R, ldr, X, ldx, n);
  return cudaGetLastError();
}

// One FP64 sweep: n_even - 1 rounds of n_even / 2 pairs (ProfScope: 6 flops and
// 32 bytes per row and pair).
cudaError_t jacobi_sweep(double* X, int64_t ldx, int64_t m, int64_t n_even, int64_t n_real,
                         double tol, int* status, double* nrm2, double* dsc, int* ver, int* err,
                         int stall, long long stall_ns, cudaStream_t st) {
  int occ = 0, dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jacobi_sweep_kernel, kJacThreads, 0) !=
          cudaSuccess)
    return cudaErrorUnknown;
  const int64_t items = (n_even - 1) * (n_even / 2);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)std::max(1, occ) * sms));
  if (cudaMemsetAsync(ver, 0, sizeof(int) * n_even, st) != cudaSuccess) return cudaErrorUnknown;
  ProfScope ps(kProfJacobi, st, 6.0 * (double)m * (double)items, 32.0 * (double)m * (double)items);
  ps.blocks((const void*)jacobi_sweep_kernel, dim3(kJacThreads), 0, dim3(grid));
  int ne = (int)n_even, nr = (int)n_real;
  void* args[] = {&X, &ldx, &m, &ne, &nr, &tol, &status, &nrm2, &dsc, &ver, &err, &stall, &stall_ns};
  return cudaLaunchCooperativeKernel((const void*)jacobi_sweep_kernel, grid, kJacThreads, args, 0, st);
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
    ps.blocks((const void*)to_f32_kernel, dim3(256), 0, dim3(eg));
    to_f32_kernel<<<eg, 256, 0, st>>>(w.X, w.X32, nn);
  }
  {
    ProfScope ps(kProfOther, st);
    ps.blocks((const void*)identity_f32_kernel, dim3(256), 0, dim3(eg));
    identity_f32_kernel<<<eg, 256, 0, st>>>(w.Z32, n);
  }
  if (n > 1) {
    int occ = 0, dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jacobi32_block_sweep_kernel, kJacThreads,
                                                      0) != cudaSuccess)
      return 1;
    const int nb = (int)((n + kJB - 1) / kJB);
    const int nb_even = nb + (nb & 1);
    // two blocks per block pair when they all fit at once and a half has rows
    // to spare (n >= 512); the partial Gram matrices go to Z, unused until the
    // FP32 phase ends
    const int split = (int64_t)nb_even <= (int64_t)std::max(1, occ) * sms && n >= 2 * kJRows ? 2 : 1;
    const int grid =
        split == 2 ? nb_even : (int)std::min<int64_t>(nb_even / 2, (int64_t)std::max(1, occ) * sms);
    float* Gp = reinterpret_cast<float*>(w.Z);
    const float tol32 = 8e-6f;
    for (int sw = 0; sw < 25; ++sw) {
      if (cudaMemsetAsync(w.status + kStatJacobiRot, 0, sizeof(int), st) != cudaSuccess) return 1;
      if (cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), st) != cudaSuccess) return 1;
      float* X32 = w.X32;
      float* Z32 = w.Z32;
      int64_t ld = n, mm = n;
      int ne = nb_even, nr = (int)n;
      float tol = tol32;
      int* status = w.status;
      unsigned* bar = w.bar;
      int* err = w.err;
      int stall = sw == 0 ? w.stall : 0;
      long long stall_ns = w.stall_ns;
      int sp = split;
      void* args[] = {&X32, &Z32, &ld, &mm, &ne, &nr, &tol, &status, &bar, &err, &stall, &stall_ns,
                      &sp, &Gp};
      {
        // Gram and two products with Q per block pair: 6 (2 kJB)^2 m flops
        ProfScope ps(kProfJacobi32, st,
                     6.0 * kJW * kJW * (double)n * (double)(nb_even / 2) * (double)(nb_even - 1));
        ps.blocks((const void*)jacobi32_block_sweep_kernel, dim3(kJacThreads), 0, dim3(grid));
        if (cudaLaunchCooperativeKernel((const void*)jacobi32_block_sweep_kernel, grid, kJacThreads,
                                        args, 0, st) != cudaSuccess)
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
      if (rot < n) break;
    }
  }
  // ---- Z orthonormal in FP64 (Cholesky QR: Z^T Z = R_z^T R_z, Z <- Z R_z^{-1})
  {
    ProfScope ps(kProfOther, st);
    ps.blocks((const void*)to_f64_kernel, dim3(256), 0, dim3(eg));
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
  for (int sw = 0; sw < 40 && !converged; ++sw) {
    if (cudaMemsetAsync(w.status + kStatJacobiRot, 0, 2 * sizeof(int), st) != cudaSuccess) return 1;
    // fold the previous sweep's column scales in, then the squared column norms
    // afresh (w.lam and w.tmp are free until the Rayleigh quotients)
    if (sw > 0 && scale_columns(X, n, n, n, w.tmp, 0, st) != cudaSuccess) return 1;
    {
      ProfScope ps(kProfOther, st);
      ps.blocks((const void*)fill_kernel, dim3(256), 0, dim3((unsigned)((n + 255) / 256)));
      fill_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w.tmp, n, 1.0);
    }
    if (column_dots(X, n, X, n, n, n, w.lam, st) != cudaSuccess) return 1;
    if (jacobi_sweep(X, n, n, n_even, n, tol_strict, w.status, w.lam, w.tmp, w.ver, w.err,
                     sw == 0 ? w.stall64 : 0, w.stall_ns, st) != cudaSuccess)
      return 1;
    int rs[2] = {0, 0}, herr = 0;
    if (cudaMemcpyAsync(rs, w.status + kStatJacobiRot, sizeof(rs), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(&herr, w.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return 1;
    if (cudaStreamSynchronize(st) != cudaSuccess) return 1;
    if (herr) return 3;
    ++total_sweeps;
    float maxcos;
    memcpy(&maxcos, &rs[1], sizeof(float));
    if (rs[0] == 0) converged = true;
    else if (maxcos <= tol_loose) converged = true;
  }
  *sweeps = total_sweeps;
  if (!converged) return 2;
  if (n > 1 && scale_columns(X, n, n, n, w.tmp, 0, st) != cudaSuccess) return 1;
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
