// C ABI of libzolo and the host orchestration of Zolo-PD / Zolo-SVD.
//
// zolo_pd follows Algorithm 1: X_0 = A / alpha, l_0 = beta / alpha, r from
// Table 1's guidance, then the a-priori l-schedule (Algorithm 1 step (c),
// stopping when 1 - l <= 1e-15 as Table 1 does) fixes every iteration's
// coefficients before any GPU work, so the whole decomposition is queued
// without a device round trip.  Each iteration forms the r shifted problems at
// once (the paper's r process groups, Algorithm 3 step 4(c), become r batch
// entries of one launch), in the QR form of Eq. (12) while the bound
// (1 + c_1)/(l^2 + c_1) on kappa(Z_1) exceeds 100 and in the Cholesky form of
// Algorithm 1 step (d) afterwards, and sums them on the device (the paper's
// DGSUM2D, Algorithm 3 step 4(d)) fused into X_{k+1} = M_hat (X_k + sum T_j)
// together with ||X_{k+1} - X_k||_F and ||X_{k+1}||_F.  H = (Qp^T A + A^T Qp)/2
// uses the original A (Algorithm 1 step 5).
#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/zolo.h"
#include "zolo_internal.h"

using namespace zolo;

// Per-matrix device norms: ||X_{k+1} - X_k||^2, ||X_{k+1}||^2 per iteration,
// then the estimates ||A - Qp H||^2, ||A||^2, ||Qp^T Qp - I||^2 (opts.estimate).
constexpr int kEstSlot = 2 * (kMaxIters + 2);
constexpr int kNormSlots = kEstSlot + 4;
constexpr int kPhaseEvents = 32;
constexpr int kAsyncSlots = 64;

// Host record of one zolo_pd_async call (pinned): the device status words and
// norms are copied here at the end of the call's work, and a host function
// turns them into the caller's zolo_info_t.
struct AsyncSlot {
  int stat[kStatSlots];
  int err;
  double norms[kNormSlots];
  zolo_info_t base;        // the schedule's part, known at enqueue time
  zolo_info_t* out;
  int64_t n;
  int estimate;
  volatile int busy;       // set at enqueue, cleared by the host function
};

// One concurrent lane of zolo_pd_batched: a stream with its own workspace.
struct BatchSlot {
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* slices = nullptr;
  size_t slice_elems = 0;
  int* exps = nullptr;
  size_t exp_elems = 0;
  int* err = nullptr;
  // the handle's kernel choices as this lane replays them, with the lane's own
  // scratch for split-K partial sums (lanes run concurrently)
  std::unique_ptr<GemmTuner> tuner;
  uint64_t tuner_gen = ~0ull;
};

struct BatchGraph {
  std::vector<uint64_t> key;
  cudaGraphExec_t exec = nullptr;
  uint64_t launches = 0;         // kernels recorded in the graph
};

struct zolo_handle_s {
  int device = 0;
  std::vector<BatchSlot> slots;
  cudaEvent_t fork = nullptr;
  cudaEvent_t joined = nullptr;
  cudaStream_t cap = nullptr;    // the stream the batch graph is captured on and launched from
  double* brec = nullptr;        // per-matrix device records (status + norms)
  size_t brec_count = 0;
  double* hrec = nullptr;        // pinned host mirror of brec
  size_t hrec_count = 0;
  std::vector<BatchGraph> graphs;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* io = nullptr;
  size_t io_bytes = 0;
  void* slices = nullptr;     // split-precision slice planes (16-bit units)
  size_t slice_elems = 0;
  int* exps = nullptr;        // slice exponents
  size_t exp_elems = 0;
  int* err = nullptr;         // device error flag of the tensor-core kernels
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  // r measured fastest per (m, n, prec, round(-log10 l_0))
  std::map<std::array<int64_t, 4>, int> tuned_r;
  // contraction kernel measured fastest per shape (zolo_autotune)
  GemmTuner tuner;
  // zolo_debug_stall: which kernel waits on a barrier nothing completes (0: none,
  // ZOLO_STALL_SPLIT_GEMM, ZOLO_STALL_JACOBI32, ZOLO_STALL_JACOBI64) and for how long
  int dbg_stall = 0;
  long long dbg_ns = 0;
  cudaEvent_t ph_ev[kPhaseEvents] = {};   // phase boundaries of one call
  AsyncSlot* async = nullptr;              // pinned ring of zolo_pd_async records
  int async_next = 0;
  bool batch_graphs = true;                // zolo_pd_batched records and replays a graph
  bool guards = false;                     // zolo_debug_guards
  int* guard_flag = nullptr;               // set by the guard check
};

namespace {

constexpr double kEps = 2.220446049250313e-16;

bool is_split(int prec) {
  return prec == ZOLO_SPLIT_BF16 || prec == ZOLO_SPLIT_FP16 || prec == ZOLO_SPLIT_FP8;
}
// The slice form and count of a split precision.
int split_form(int prec) {
  return prec == ZOLO_SPLIT_FP8 ? kFormFP8 : prec == ZOLO_SPLIT_FP16 ? kFormFP16 : kFormBF16;
}
int split_slices(int prec) {
  return prec == ZOLO_SPLIT_FP8 ? 11 : prec == ZOLO_SPLIT_FP16 ? 8 : 9;
}

// Guard zones (zolo_debug_guards): in a call made with them on, every buffer
// carved from the workspace is followed by kGuardBytes of 0xFF (an FP64 NaN
// pattern) and the QR, Cholesky and eigensolver regions stop sharing memory;
// the zones of the last layout placed in the workspace are listed here.
constexpr size_t kGuardBytes = 4096;
thread_local bool t_guard_on = false;
thread_local std::vector<std::pair<size_t, size_t>> t_guards;   // (offset, bytes)

// Bump allocator over one device block; with base == nullptr it only sizes.
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    if (t_guard_on) {
      off = (off + 255) & ~size_t(255);
      if (base) t_guards.emplace_back(off, kGuardBytes);
      off += kGuardBytes;
    }
    return p;
  }
};

struct PdBufs {
  double *X, *Xn, *S, *M, *partials, *norms;
  int* status;
  double *Qp_int, *H_int;   // zolo_svd only
  QrBuffers qr;
  CholBuffers ch;
  double *Y, *tmp;
  int64_t strideY, strideTmp;
  EigWork eig;
};

// Workspace layout for (m, n, r).  The QR, Cholesky and eigensolver regions
// are never live at the same time and share one union region.
size_t layout(void* base, int64_t m, int64_t n, int r, bool svd, PdBufs* b) {
  if (base && t_guard_on) t_guards.clear();
  Carve c(base);
  PdBufs t{};
  t.X = c.take<double>(m * n);
  t.Xn = c.take<double>(m * n);
  t.S = c.take<double>(m * n + 8);   // + the sharded path's breakdown count
  t.M = c.take<double>(n * n);
  t.partials = c.take<double>(2 * 1024);
  t.norms = c.take<double>(kNormSlots);
  t.status = c.take<int>(kStatSlots);
  if (svd) {
    t.Qp_int = c.take<double>(m * n);
    t.H_int = c.take<double>(n * n);
  }
  const size_t union_start = (c.off + 255) & ~size_t(255);
  // QR region
  {
    Carve q(base);
    q.off = t_guard_on ? c.off : union_start;   // guard mode: no sharing
    const int64_t npan = (n + kQrNB - 1) / kQrNB;
    t.qr.strideW = (m + n) * n;
    t.qr.W = q.take<double>(r * t.qr.strideW);
    const int64_t nblk = (n + kQrBlock - 1) / kQrBlock;
    t.qr.strideV = (m + kQrBlock) * n;
    t.qr.V = q.take<double>(r * t.qr.strideV);
    t.qr.strideT = npan * kQrNB * kQrNB;
    t.qr.T = q.take<double>(r * t.qr.strideT);
    t.qr.strideTb = nblk * kQrBlock * kQrBlock;
    t.qr.Tb = q.take<double>(r * t.qr.strideTb);
    t.qr.strideG = kQrBlock * kQrBlock;
    t.qr.G = q.take<double>(r * t.qr.strideG);
    t.qr.elemsP = qr_partial_elems(m, r);
    t.qr.P = q.take<double>(t.qr.elemsP);
    t.qr.strideW1 = kQrBlock * n;
    t.qr.W1 = q.take<double>(r * t.qr.strideW1);
    t.qr.strideW2 = kQrBlock * n;
    t.qr.W2 = q.take<double>(r * t.qr.strideW2);
    c.off = std::max(c.off, q.off);
  }
  // Cholesky region
  {
    Carve q(base);
    q.off = t_guard_on ? c.off : union_start;   // guard mode: no sharing
    const int64_t nblk = (n + kCholNB - 1) / kCholNB;
    t.ch.strideZ = n * n;
    t.ch.Z = q.take<double>(r * t.ch.strideZ);
    t.ch.strideRinv = nblk * kCholNB * kCholNB;
    t.ch.Rinv = q.take<double>(r * t.ch.strideRinv);
    t.strideY = m * n;
    t.Y = q.take<double>(r * t.strideY);
    t.strideTmp = m * kCholNB;
    t.tmp = q.take<double>(r * t.strideTmp);
    c.off = std::max(c.off, q.off);
  }
  // eigensolver region
  if (svd) {
    Carve q(base);
    q.off = t_guard_on ? c.off : union_start;   // guard mode: no sharing
    const int64_t nblk = (n + kCholNB - 1) / kCholNB;
    t.eig.R = q.take<double>(n * n);
    t.eig.X = q.take<double>(n * n);
    t.eig.HV = q.take<double>(std::max<int64_t>(n * n, 2 * 1024));
    t.eig.Rinv = q.take<double>(nblk * kCholNB * kCholNB);
    t.eig.lam = q.take<double>(std::max<int64_t>(n, 2));
    t.eig.perm = q.take<int>(n);
    t.eig.status = t.status;
    t.eig.X32 = q.take<float>(n * n);
    t.eig.Z32 = q.take<float>(n * n);
    t.eig.Z = q.take<double>(n * n);
    t.eig.tmp = q.take<double>(n * kCholNB);
    t.eig.bar = q.take<unsigned>(2);
    t.eig.ver = q.take<int>(n + 1);
    t.eig.err = q.take<int>(1);
    c.off = std::max(c.off, q.off);
  }
  if (b) *b = t;
  return c.off + 256;
}

int ensure_ws(zolo_handle_t h, size_t bytes) {
  if (h->ws_bytes >= bytes) return 0;
  if (h->ws) cudaFree(h->ws);
  h->ws = nullptr;
  h->ws_bytes = 0;
  if (cudaMalloc(&h->ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    return ZOLO_ENOMEM;
  }
  h->ws_bytes = bytes;
  return 0;
}

// Fill the listed guard zones of the workspace and clear the flag (guard mode).
int guards_arm(zolo_handle_t h, cudaStream_t st) {
  if (!t_guard_on) return 0;
  if (!h->guard_flag && cudaMalloc(&h->guard_flag, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    h->guard_flag = nullptr;
    return ZOLO_ENOMEM;
  }
  if (cudaMemsetAsync(h->guard_flag, 0, sizeof(int), st) != cudaSuccess) return ZOLO_ECUDA;
  for (const auto& g : t_guards)
    if (guard_fill(static_cast<char*>(h->ws) + g.first, g.second, st) != cudaSuccess)
      return ZOLO_ECUDA;
  return 0;
}

// Check every listed zone still holds 0xFF; ZOLO_EGUARD if not (synchronises).
int guards_check(zolo_handle_t h, cudaStream_t st) {
  if (!t_guard_on || !h->guard_flag) return 0;
  for (const auto& g : t_guards)
    if (guard_check(static_cast<const char*>(h->ws) + g.first, g.second, h->guard_flag, st) !=
        cudaSuccess)
      return ZOLO_ECUDA;
  int f = 0;
  if (cudaMemcpyAsync(&f, h->guard_flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ZOLO_ECUDA;
  return f ? ZOLO_EGUARD : 0;
}

// Guard mode for the calls of one entry point on this thread.
struct GuardScope {
  explicit GuardScope(bool on) {
    t_guard_on = on;
    t_guards.clear();
  }
  ~GuardScope() {
    t_guard_on = false;
    t_guards.clear();
  }
};

// Slice-plane units for the largest contraction of a decomposition of an
// m x n matrix (one batch entry, the larger of the BF16 form's nine slices and
// the FP8 form's eleven, whose K runs are padded to 128).
size_t split_elems_per_entry(int64_t m, int64_t n) {
  const int64_t shapes[][3] = {{kQrNB, n, m + kQrNB}, {m + kQrNB, n, kQrNB}, {m, n, n},
                               {n, n, m}, {m, kCholNB, n}, {m, n, n}};
  size_t mx = 0;
  for (auto& sh : shapes)
    mx = std::max({mx, split_slice_elems(sh[0], sh[1], sh[2], 1, 9, kFormBF16),
                   split_slice_elems(sh[0], sh[1], sh[2], 1, 11, kFormFP8)});
  return mx;
}

// Grow the handle's slice workspace to hold `want` elements (at least `need`).
int ensure_split(zolo_handle_t h, size_t need, size_t want, size_t exps) {
  if (!h->err && cudaMalloc(&h->err, sizeof(int)) != cudaSuccess) return ZOLO_ENOMEM;
  if (h->slice_elems < need) {
    if (h->slices) cudaFree(h->slices);
    h->slices = nullptr;
    h->slice_elems = 0;
    size_t n = std::max(want, need);
    while (cudaMalloc(&h->slices, n * 2) != cudaSuccess) {
      cudaGetLastError();
      h->slices = nullptr;
      if (n == need) return ZOLO_ENOMEM;
      n = std::max(need, n / 2);
    }
    h->slice_elems = n;
  }
  if (h->exp_elems < exps) {
    if (h->exps) cudaFree(h->exps);
    if (cudaMalloc(&h->exps, exps * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      h->exps = nullptr;
      h->exp_elems = 0;
      return ZOLO_ENOMEM;
    }
    h->exp_elems = exps;
  }
  return 0;
}

// Installs the split tensor-core engine for the contractions of one call.
struct SplitScope {
  SplitWork w{};
  bool on = false;
  ~SplitScope() { set_split_engine(nullptr); }
  int begin(zolo_handle_t h, int64_t m, int64_t n, int r, cudaStream_t st, int prec) {
    const size_t per = split_elems_per_entry(m, n);
    const size_t budget = (size_t)8 << 30;   // 16 GB of BF16 planes at most
    size_t want = std::max(per, std::min(per * (size_t)r, budget));
    const size_t exps = (size_t)2 * kGemmMaxBatch * (size_t)(std::max(m, n) + m + n + 512);
    if (int e = ensure_split(h, per, want, exps)) return e;
    if (cudaMemsetAsync(h->err, 0, sizeof(int), st) != cudaSuccess) return ZOLO_ECUDA;
    w.slices = h->slices;
    w.slice_elems = h->slice_elems;
    w.exps = h->exps;
    w.exp_elems = h->exp_elems;
    w.err = h->err;
    w.slices_s = split_slices(prec);
    w.form = split_form(prec);
    w.stall = h->dbg_stall == ZOLO_STALL_SPLIT_GEMM;
    w.stall_ns = h->dbg_ns;
    set_split_engine(&w);
    on = true;
    return 0;
  }
};

#define CK(x)                                  \
  do {                                         \
    if ((x) != cudaSuccess) return ZOLO_ECUDA; \
  } while (0)

struct Run {
  int64_t m, n;
  int r;
  PdBufs b;
  cudaStream_t st;
  bool inv_chol = false;   // Cholesky-form iterations through W = sum_j a_j Z_j^{-1}
  bool narrow_panels = false;   // many problems in flight: panels on the fewest CTAs
};

// opts.chol_form = 0: the explicit-inverse Cholesky form when its modelled flops,
// r (n^3 for R_j^{-1} by solves against I + n^3 / 2 for the triangular product)
// + 2 m n^2 for X W, are below 85% of the 2 r m n^2 of the triangular solves.
bool use_inverse_form(int chol_form, int64_t m, int64_t n, int r) {
  if (chol_form != 0) return chol_form == 2;
  const double dm = (double)m, dn = (double)n;
  const double inv = r * 1.5 * dn * dn * dn + 2.0 * dm * dn * dn;
  const double trsm = 2.0 * r * dm * dn * dn;
  return inv < 0.85 * trsm;
}

// One Zolo-PD iteration from X into Xn; norms_k receives (||Xn - X||^2, ||Xn||^2).
int iterate(const Run& R, const Coefficients& co, bool qr, const double* X, double* Xn,
            double* norms_k) {
  const int64_t m = R.m, n = R.n;
  const int r = co.r;
  const PdBufs& b = R.b;
  if (qr) {
    double sq[kMaxR];
    for (int j = 0; j < r; ++j) sq[j] = std::sqrt(co.c[2 * j]);
    CK(init_stacked(X, m, b.qr.W, b.qr.strideW, m, n, sq, r, R.st));
    CK(structured_qr_q(b.qr, m, n, r, b.status, R.st, true, R.narrow_panels));
    GemmArgs g;   // S = sum_j a_j / sqrt(c_{2j-1}) Q1_j Q2_j^T   (Q2_j upper triangular)
    g.M = (int)m; g.N = (int)n; g.K = (int)n; g.transA = 0; g.transB = 1;
    g.A = b.qr.W; g.lda = m + n; g.strideA = b.qr.strideW;
    g.B = b.qr.W + m; g.ldb = m + n; g.strideB = b.qr.strideW;
    g.Cout = b.S; g.ldcout = m;
    g.batch = r; g.reduce = 1; g.b_lower = 1;
    for (int j = 0; j < r; ++j) g.alpha[j] = co.a[j] / sq[j];
    CK(gemm_any(g, R.st));
    const double one = 1.0;
    CK(combine(X, m, Xn, m, m, n, co.mhat, b.S, m, 0, &one, 1, b.partials, norms_k, b.status,
               R.st));
  } else {
    GemmArgs g;   // G = X^T X (upper triangle), shared by every shift
    g.M = g.N = (int)n; g.K = (int)m; g.transA = 1; g.transB = 0;
    g.A = X; g.lda = m; g.B = X; g.ldb = m;
    g.Cout = b.M; g.ldcout = n; g.c_upper = 1;
    g.alpha[0] = 1.0;
    CK(gemm_any(g, R.st));
    double shifts[kMaxR];
    for (int j = 0; j < r; ++j) shifts[j] = co.c[2 * j];
    CK(init_shifted(b.M, b.ch.Z, b.ch.strideZ, n, shifts, r, R.st));
    CK(cholesky_upper_batched(b.ch, n, r, b.status, R.st));
    if (R.inv_chol) {
      // R_j^{-1} = I R_j^{-1} (n x n, ld n, in Y_j; exactly upper triangular:
      // the zero rows of I stay zero through the solves); G is consumed, so M
      // holds the identity
      CK(init_q_identity(b.M, 0, 0, n, 1, R.st));
      CK(trsm_right_upper_batched(b.M, n, b.ch, b.Y, b.strideY, b.tmp, b.strideTmp, n, n, r,
                                  R.st));
      GemmArgs w;   // W = sum_j a_j R_j^{-1} R_j^{-T}: upper tiles, op(B) lower triangular
      w.M = w.N = w.K = (int)n; w.transA = 0; w.transB = 1;
      w.A = b.Y; w.lda = n; w.strideA = b.strideY;
      w.B = b.Y; w.ldb = n; w.strideB = b.strideY;
      w.Cout = b.S; w.ldcout = n;
      w.batch = r; w.reduce = 1; w.b_lower = 1; w.c_upper = 1;
      for (int j = 0; j < r; ++j) w.alpha[j] = co.a[j];
      CK(gemm_any(w, R.st));
      CK(mirror_upper(b.S, n, n, R.st));
      GemmArgs t;   // T = X W into Y_0 (m x n)
      t.M = (int)m; t.N = (int)n; t.K = (int)n;
      t.A = X; t.lda = m; t.B = b.S; t.ldb = n;
      t.Cout = b.Y; t.ldcout = m;
      t.alpha[0] = 1.0;
      CK(gemm_any(t, R.st));
      const double one = 1.0;
      CK(combine(X, m, Xn, m, m, n, co.mhat, b.Y, m, 0, &one, 1, b.partials, norms_k, b.status,
                 R.st));
    } else {
      CK(trsm_pair_batched(X, m, b.ch, b.Y, b.strideY, b.tmp, b.strideTmp, m, n, r, R.st));
      CK(combine(X, m, Xn, m, m, n, co.mhat, b.Y, m, b.strideY, co.a, r, b.partials, norms_k,
                 b.status, R.st));
    }
  }
  return 0;
}

// The rank's share of one iteration on the sharded path (Algorithm 3 step 4(c):
// process group j forms T_j): S = sum of T_j over the shifts of `co` (a
// sub-range of the iteration's shifts, re-indexed from 0), in the form the
// iteration takes.  The kernels are iterate()'s; the terms are left unsummed
// with X and M_hat so that the other ranks' shares can be added first.
// `scratch` (m x n, not X) holds W = sum_j a_j Z_j^{-1} in the inverse form.
int shift_terms(const Run& R, const Coefficients& co, bool qr, const double* X, double* S,
                double* scratch) {
  const int64_t m = R.m, n = R.n;
  const int r = co.r;
  const PdBufs& b = R.b;
  if (qr) {
    double sq[kMaxR];
    for (int j = 0; j < r; ++j) sq[j] = std::sqrt(co.c[2 * j]);
    CK(init_stacked(X, m, b.qr.W, b.qr.strideW, m, n, sq, r, R.st));
    CK(structured_qr_q(b.qr, m, n, r, b.status, R.st, true, R.narrow_panels));
    GemmArgs g;   // sum_j a_j / sqrt(c_{2j-1}) Q1_j Q2_j^T   (Q2_j upper triangular)
    g.M = (int)m; g.N = (int)n; g.K = (int)n; g.transA = 0; g.transB = 1;
    g.A = b.qr.W; g.lda = m + n; g.strideA = b.qr.strideW;
    g.B = b.qr.W + m; g.ldb = m + n; g.strideB = b.qr.strideW;
    g.Cout = S; g.ldcout = m;
    g.batch = r; g.reduce = 1; g.b_lower = 1;
    for (int j = 0; j < r; ++j) g.alpha[j] = co.a[j] / sq[j];
    CK(gemm_any(g, R.st));
    return 0;
  }
  GemmArgs g;   // G = X^T X (upper triangle)
  g.M = g.N = (int)n; g.K = (int)m; g.transA = 1; g.transB = 0;
  g.A = X; g.lda = m; g.B = X; g.ldb = m;
  g.Cout = b.M; g.ldcout = n; g.c_upper = 1;
  g.alpha[0] = 1.0;
  CK(gemm_any(g, R.st));
  double shifts[kMaxR];
  for (int j = 0; j < r; ++j) shifts[j] = co.c[2 * j];
  CK(init_shifted(b.M, b.ch.Z, b.ch.strideZ, n, shifts, r, R.st));
  CK(cholesky_upper_batched(b.ch, n, r, b.status, R.st));
  if (R.inv_chol) {
    CK(init_q_identity(b.M, 0, 0, n, 1, R.st));
    CK(trsm_right_upper_batched(b.M, n, b.ch, b.Y, b.strideY, b.tmp, b.strideTmp, n, n, r, R.st));
    GemmArgs w;   // W = sum_j a_j R_j^{-1} R_j^{-T} (upper tiles, then mirrored)
    w.M = w.N = w.K = (int)n; w.transA = 0; w.transB = 1;
    w.A = b.Y; w.lda = n; w.strideA = b.strideY;
    w.B = b.Y; w.ldb = n; w.strideB = b.strideY;
    w.Cout = scratch; w.ldcout = n;
    w.batch = r; w.reduce = 1; w.b_lower = 1; w.c_upper = 1;
    for (int j = 0; j < r; ++j) w.alpha[j] = co.a[j];
    CK(gemm_any(w, R.st));
    CK(mirror_upper(scratch, n, n, R.st));
    GemmArgs t;   // X W
    t.M = (int)m; t.N = (int)n; t.K = (int)n;
    t.A = X; t.lda = m; t.B = scratch; t.ldb = n;
    t.Cout = S; t.ldcout = m;
    t.alpha[0] = 1.0;
    CK(gemm_any(t, R.st));
    return 0;
  }
  CK(trsm_pair_batched(X, m, b.ch, b.Y, b.strideY, b.tmp, b.strideTmp, m, n, r, R.st));
  CK(weighted_sum(b.Y, m, b.strideY, co.a, r, S, m, m, n, R.st));
  return 0;
}

// The sharded path's exchange: this rank's shifts, the sum over ranks, then
// the combination X_{k+1} = M_hat (X + S) (Algorithm 3 steps 4(c)-(d), with the
// caller's sum in place of DGSUM2D).  S carries one more double, this rank's
// Cholesky-breakdown flag, so that every rank learns of a breakdown from the
// same sum; *redo = true when any rank saw one (no combination then).
struct ShardCtx {
  int rank = 0, nranks = 1;
  zolo_sum_fn fn = nullptr;
  void* ctx = nullptr;
};

int iterate_sharded(const Run& R, const Coefficients& co, bool qr, const double* X, double* Xn,
                    double* norms_k, const ShardCtx& sh, bool* redo) {
  const int64_t m = R.m, n = R.n;
  const PdBufs& b = R.b;
  int j0 = 0, j1 = 0;
  zolo_shift_range(co.r, sh.rank, sh.nranks, &j0, &j1);
  Coefficients sub = co;
  sub.r = j1 - j0;
  for (int j = 0; j < sub.r; ++j) {
    sub.c[2 * j] = co.c[2 * (j0 + j)];
    sub.c[2 * j + 1] = co.c[2 * (j0 + j) + 1];
    sub.a[j] = co.a[j0 + j];
  }
  CK(cudaMemsetAsync(b.status + kStatCholFail, 0, sizeof(int), R.st));
  if (sub.r > 0) {
    if (int e = shift_terms(R, sub, qr, X, b.S, Xn)) return e;
  } else {
    CK(cudaMemsetAsync(b.S, 0, sizeof(double) * m * n, R.st));
  }
  CK(flag_to_double(b.status + kStatCholFail, b.S + m * n, R.st));
  if (sh.fn && sh.fn(b.S, m * n + 1, R.st, sh.ctx) != 0) return ZOLO_ECOMM;
  double fails = 0.0;
  CK(cudaMemcpyAsync(&fails, b.S + m * n, sizeof(double), cudaMemcpyDeviceToHost, R.st));
  CK(cudaStreamSynchronize(R.st));
  *redo = fails != 0.0;
  if (*redo) return 0;
  const double one = 1.0;
  CK(combine(X, m, Xn, m, m, n, co.mhat, b.S, m, 0, &one, 1, b.partials, norms_k, b.status, R.st));
  return 0;
}

int read_status(const Run& R, int* hstat) {
  CK(cudaMemcpyAsync(hstat, R.b.status, sizeof(int) * kStatSlots, cudaMemcpyDeviceToHost, R.st));
  CK(cudaStreamSynchronize(R.st));
  return 0;
}

// opts.estimate: ||A - Qp H||_F^2 and ||A||_F^2, then ||Qp^T Qp - I||_F^2 into
// b.norms[kEstSlot ..] (S and M are free once H is formed).
int enqueue_estimates(const PdBufs& b, const double* A, int64_t lda, const double* Qp, int64_t ldq,
                      const double* H, int64_t ldh, int64_t m, int64_t n, cudaStream_t st) {
  GemmArgs g;   // A - Qp H
  g.M = (int)m; g.N = (int)n; g.K = (int)n;
  g.A = Qp; g.lda = ldq; g.B = H; g.ldb = ldh;
  g.Cin = A; g.ldcin = lda; g.beta = 1.0; g.Cout = b.S; g.ldcout = m;
  g.alpha[0] = -1.0;
  CK(gemm_any(g, st));
  CK(frob_norm2(b.S, m, m, n, b.partials, b.norms + kEstSlot, st));
  CK(frob_norm2(A, lda, m, n, b.partials, b.norms + kEstSlot + 1, st));
  GemmArgs q;   // Qp^T Qp, upper tiles
  q.M = q.N = (int)n; q.K = (int)m; q.transA = 1;
  q.A = Qp; q.lda = ldq; q.B = Qp; q.ldb = ldq;
  q.Cout = b.M; q.ldcout = n; q.c_upper = 1;
  q.alpha[0] = 1.0;
  CK(gemm_any(q, st));
  CK(gram_identity_dev2(b.M, n, n, b.partials, b.norms + kEstSlot + 2, st));
  return 0;
}

void fill_estimates(zolo_info_t* info, const double* norms, int64_t n) {
  const double* e = norms + kEstSlot;
  info->bwd_est = e[1] > 0.0 ? std::sqrt(e[0] / e[1]) : 0.0;
  info->orth_est = std::sqrt(std::max(e[2], 0.0) / (double)n);
}

const char* const kPhaseNames[ZOLO_PHASES] = {
    "zolo: bounds", "zolo: QR-form iteration", "zolo: Cholesky-form iteration",
    "zolo: Newton-Schulz", "zolo: H", "zolo: estimates", "zolo: eig(H)", "zolo: U = Qp V"};

// Device time per phase of one call: an event on the call's stream at every
// phase boundary (and an NVTX range per phase on the calling thread), read once
// the stream has been synchronised.
struct PhaseClock {
  zolo_handle_t h = nullptr;
  cudaStream_t st = nullptr;
  int n = 0;
  int phase[kPhaseEvents] = {};
  bool nvtx_open = false;
  void start(zolo_handle_t hh, cudaStream_t s) {
    h = hh;
    st = s;
    n = 0;
    for (int i = 0; i < kPhaseEvents; ++i)
      if (!h->ph_ev[i] && cudaEventCreate(&h->ph_ev[i]) != cudaSuccess) {
        h->ph_ev[i] = nullptr;
        h = nullptr;   // no clock for this call
        cudaGetLastError();
        return;
      }
  }
  void record(int p) {
    if (h && n < kPhaseEvents && cudaEventRecord(h->ph_ev[n], st) == cudaSuccess) phase[n++] = p;
  }
  void mark(int p) {
    if (nvtx_open) nvtxRangePop();
    nvtxRangePushA(kPhaseNames[p]);
    nvtx_open = true;
    record(p);
  }
  void stop() {
    if (nvtx_open) nvtxRangePop();
    nvtx_open = false;
    record(-1);
  }
  void read(float* ms) {
    for (int k = 0; k + 1 < n; ++k) {
      float t = 0.f;
      if (phase[k] >= 0 && cudaEventElapsedTime(&t, h->ph_ev[k], h->ph_ev[k + 1]) == cudaSuccess)
        ms[phase[k]] += t;
    }
    cudaGetLastError();
  }
  ~PhaseClock() {
    if (nvtx_open) nvtxRangePop();
  }
};

int validate(zolo_handle_t h, const void* A, int64_t m, int64_t n, int64_t lda, const void* P,
             int64_t ldp, const void* Q, int64_t ldq, const zolo_opts_t* o) {
  if (!h) return -1;
  if (!A) return -2;
  if (n < 1) return -4;
  if (m < n) return -3;
  if (lda < m) return -5;
  if (!P) return -6;
  if (ldp < m) return -7;
  if (!Q) return -8;
  if (ldq < n) return -9;
  if (o) {
    if (o->r < ZOLO_R_TUNED || o->r > kMaxR || !std::isfinite(o->alpha) || !std::isfinite(o->beta) ||
        o->max_iter < 1 || o->max_iter > kMaxIters || o->ns_steps < 0 ||
        o->ns_steps > 4 || (o->prec != ZOLO_FP64 && !is_split(o->prec)) ||
        o->force_qr < -1 || o->force_qr > 1 || o->chol_form < 0 || o->chol_form > 2 ||
        o->estimate < 0 || o->estimate > 1 ||
        (o->alpha > 0.0 && o->beta > o->alpha))
      return -10;
  } else {
    return -10;
  }
  return 0;
}

// The PD core on device buffers; Qp/H are written (may be internal buffers).
// beta = alpha / ||R^{-1}||_F with R the triangular factor of a Householder QR
// of X0 = A / alpha (the structured QR with c = 0, no explicit Q): since
// ||R^{-1}||_F >= ||R^{-1}||_2 = 1 / sigma_min(X0), a lower bound of
// sigma_min(A), loose by at most sqrt(n).  R^{-1} comes from the recursive
// triangular solve with the identity as right-hand side.  Uses the workspace
// of an r = 1 layout; returns ZOLO_ENONFINITE for a zero pivot.
int estimate_beta(const double* A, int64_t lda, int64_t m, int64_t n, double alpha, const PdBufs& b,
                  cudaStream_t st, double* beta) {
  CK(cudaMemsetAsync(b.status, 0, sizeof(int) * kStatSlots, st));
  CK(scale_copy(A, lda, b.X, m, m, n, 1.0 / alpha, st));
  const double zero = 0.0;
  CK(init_stacked(b.X, m, b.qr.W, b.qr.strideW, m, n, &zero, 1, st));
  CK(structured_qr_q(b.qr, m, n, 1, b.status, st, false));
  // R (the upper triangle of W's top n x n block; what lies below is never read)
  // into X with ld n; the QR region is free from here on
  CK(copy_matrix(b.qr.W, m + n, b.X, n, n, n, st));
  CK(tri_inv_diag_blocks(b.X, n, b.ch.Rinv, b.status, st));
  CK(init_q_identity(b.ch.Z, 0, 0, n, 1, st));
  CholBuffers cb{b.X, 0, b.ch.Rinv, 0};
  CK(trsm_right_upper_batched(b.ch.Z, n, cb, b.Y, 0, b.tmp, 0, n, n, 1, st));
  CK(frob_norm2(b.Y, n, n, n, b.partials, b.norms, st));
  double nrm2 = 0.0;
  int hst[kStatSlots];
  CK(cudaMemcpyAsync(&nrm2, b.norms, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hst, b.status, sizeof(hst), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hst[kStatNonFinite] || !(nrm2 > 0.0) || !std::isfinite(nrm2)) return ZOLO_ENONFINITE;
  *beta = alpha / std::sqrt(nrm2);
  return 0;
}

// device name with blanks as '_' (the tuning cache file's first line)
std::string device_tag(int dev) {
  cudaDeviceProp p;
  std::string tag = "unknown";
  if (cudaGetDeviceProperties(&p, dev) == cudaSuccess) tag = p.name;
  for (char& c : tag)
    if (c == ' ' || c == '\t' || c == '\n') c = '_';
  return tag;
}

std::array<int64_t, 4> tune_key(int64_t m, int64_t n, int prec, double ell0) {
  return {m, n, prec, (int64_t)std::lround(-std::log10(ell0))};
}

int pd_core(zolo_handle_t h, const double* A, int64_t m, int64_t n, int64_t lda, double* Qp,
            int64_t ldq, double* H, int64_t ldh, const zolo_opts_t& o, zolo_info_t* info,
            cudaStream_t st, bool svd, PdBufs* out_bufs, const ShardCtx* shard = nullptr,
            PhaseClock* pc = nullptr);

// r = ZOLO_R_TUNED: the cached r for this key, else every r whose schedule
// converges within max_iter is run on A itself and timed, and the fastest kept.
// The workspace (and the slice planes) are sized for r = 8 first, so that no
// trial pays for an allocation; a trial under 50 ms is timed three times (min).
int tune_r(zolo_handle_t h, const double* A, int64_t m, int64_t n, int64_t lda, double* Qp,
           int64_t ldq, double* H, int64_t ldh, const zolo_opts_t& o, double alpha, double beta,
           double ell0, cudaStream_t st, bool svd, PdBufs* out_bufs, int* r_out) {
  const auto key = tune_key(m, n, o.prec, ell0);
  const auto hit = h->tuned_r.find(key);
  if (hit != h->tuned_r.end()) {
    *r_out = hit->second;
    return 0;
  }
  {
    PdBufs tb;
    if (int e = ensure_ws(h, layout(nullptr, m, n, kMaxR, svd, &tb))) return e;
    if (is_split(o.prec)) {
      SplitScope pre;
      if (int e = pre.begin(h, m, n, kMaxR, st, o.prec)) return e;
    }
  }
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) {
    if (t0) cudaEventDestroy(t0);
    return ZOLO_ECUDA;
  }
  float best = 0.f;
  int best_r = 0, e = 0;
  for (int r = 1; r <= kMaxR && !e; ++r) {
    Schedule s;
    if (build_schedule(ell0, r, o.max_iter, &s) != 0 || !s.converged) continue;
    zolo_opts_t oo = o;
    oo.r = r;
    oo.alpha = alpha;
    oo.beta = beta;
    float ms = 0.f;
    for (int rep = 0; rep < 3 && !e; ++rep) {
      zolo_info_t ti{};
      float t = 0.f;
      if (cudaEventRecord(t0, st) != cudaSuccess) { e = ZOLO_ECUDA; break; }
      e = pd_core(h, A, m, n, lda, Qp, ldq, H, ldh, oo, &ti, st, svd, out_bufs);
      if (e) break;
      if (cudaEventRecord(t1, st) != cudaSuccess || cudaEventSynchronize(t1) != cudaSuccess ||
          cudaEventElapsedTime(&t, t0, t1) != cudaSuccess) {
        e = ZOLO_ECUDA;
        break;
      }
      ms = rep == 0 ? t : std::min(ms, t);
      if (ms >= 50.f) break;
    }
    if (e) break;
    if (best_r == 0 || ms < best) {
      best = ms;
      best_r = r;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (e) return e;
  if (best_r == 0) best_r = kMaxR;   // no schedule converges within max_iter
  h->tuned_r[key] = best_r;
  *r_out = best_r;
  return 0;
}

int pd_core(zolo_handle_t h, const double* A, int64_t m, int64_t n, int64_t lda, double* Qp,
            int64_t ldq, double* H, int64_t ldh, const zolo_opts_t& o, zolo_info_t* info,
            cudaStream_t st, bool svd, PdBufs* out_bufs, const ShardCtx* shard,
            PhaseClock* pc) {
  if (pc) pc->mark(ZOLO_PHASE_BOUNDS);
  // alpha: caller's bound or min(||A||_F, sqrt(||A||_1 ||A||_inf))
  double alpha = o.alpha;
  int r_sched = o.r;
  if (alpha <= 0.0) {
    PdBufs tmpb;
    const size_t bytes = layout(nullptr, m, n, 1, svd, &tmpb);
    if (int e = ensure_ws(h, bytes)) return e;
    layout(h->ws, m, n, 1, svd, &tmpb);
    // row partial sums in X (m * ceil(n / 256) <= m n), column sums in Xn
    CK(alpha_bound_sums(A, lda, m, n, tmpb.X, tmpb.Xn, tmpb.partials, tmpb.norms, st));
    double sums[3];
    CK(cudaMemcpyAsync(sums, tmpb.norms, sizeof(sums), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    alpha = alpha_from_sums(sums);
    if (!(alpha > 0.0) || !std::isfinite(alpha)) return ZOLO_ENONFINITE;
  }
  double beta = o.beta;
  if (!(beta > 0.0)) {
    PdBufs eb;
    const size_t bytes1 = layout(nullptr, m, n, 1, svd, &eb);
    if (int e = ensure_ws(h, bytes1)) return e;
    layout(h->ws, m, n, 1, svd, &eb);
    if (int e = estimate_beta(A, lda, m, n, alpha, eb, st, &beta)) return e;
  }
  const double ell0 = std::min(1.0, beta / alpha);
  if (r_sched == ZOLO_R_TUNED)
    if (int e = tune_r(h, A, m, n, lda, Qp, ldq, H, ldh, o, alpha, beta, ell0, st, svd, out_bufs,
                       &r_sched))
      return e;
  Schedule sch;
  if (build_schedule(ell0, r_sched, o.max_iter, &sch) != 0) return -10;
  const int r = sch.r;
  Run R{m, n, r, {}, st};
  R.inv_chol = use_inverse_form(o.chol_form, m, n, r);
  info->chol_form = R.inv_chol ? 2 : 1;
  const size_t bytes = layout(nullptr, m, n, r, svd, &R.b);
  if (int e = ensure_ws(h, bytes)) return e;
  layout(h->ws, m, n, r, svd, &R.b);
  if (out_bufs) *out_bufs = R.b;
  const PdBufs& b = R.b;
  if (int e = guards_arm(h, st)) return e;
  SplitScope split;
  if (is_split(o.prec))
    if (int e = split.begin(h, m, n, r, st, o.prec)) return e;
  CK(cudaMemsetAsync(b.status, 0, sizeof(int) * kStatSlots, st));
  CK(cudaMemsetAsync(b.norms, 0, sizeof(double) * kNormSlots, st));

  double* X = b.X;
  double* Xn = b.Xn;
  CK(scale_copy(A, lda, X, m, m, n, 1.0 / alpha, st));
  CK(check_finite(X, m, m, n, b.status, st));

  info->r = r;
  info->ell[0] = ell0;
  info->chol_fallbacks = 0;
  int it = 0;
  int hstat[kStatSlots];
  std::vector<Coefficients> cos;
  std::vector<bool> qrs;
  for (int k = 0; k < sch.iters; ++k) {
    const Coefficients& co = sch.co[k];
    bool qr = o.force_qr == 1 ? true : (o.force_qr == 0 ? false : sch.use_qr[k]);
    if (pc) pc->mark(qr ? ZOLO_PHASE_QR : ZOLO_PHASE_CHOL);
    if (shard) {
      // each rank forms its own shifts' terms; the caller's sum joins them
      bool redo = false;
      if (int e = iterate_sharded(R, co, qr, X, Xn, b.norms + 2 * it, *shard, &redo)) return e;
      if (redo) {   // a Cholesky breakdown on some rank: every rank redoes it in the QR form
        qr = true;
        info->chol_fallbacks++;
        if (int e = iterate_sharded(R, co, qr, X, Xn, b.norms + 2 * it, *shard, &redo)) return e;
      }
    } else if (int e = iterate(R, co, qr, X, Xn, b.norms + 2 * it)) {
      return e;
    } else if (!qr) {
      // a non-positive Cholesky pivot: redo this iteration in the QR form (X is intact)
      if (int e = read_status(R, hstat)) return e;
      if (hstat[kStatCholFail]) {
        CK(cudaMemsetAsync(b.status + kStatCholFail, 0, sizeof(int), st));
        qr = true;
        info->chol_fallbacks++;
        if (int e = iterate(R, co, qr, X, Xn, b.norms + 2 * it)) return e;
      }
    }
    info->used_qr[it] = qr ? 1 : 0;
    info->ell[it + 1] = sch.ell[k + 1];
    std::swap(X, Xn);
    ++it;
  }
  // Algorithm 1 step (d), applied literally when asked for
  int status = ZOLO_OK;
  if (o.posteriori && it > 0) {
    const double thr = std::pow(kEps, 1.0 / (2 * r + 1));
    double ell = sch.ell[sch.iters];
    while (true) {
      double nk[2];
      CK(cudaMemcpyAsync(nk, b.norms + 2 * (it - 1), sizeof(nk), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      const double delta = std::sqrt(nk[0] / nk[1]);
      if (delta <= thr) break;
      if (it >= o.max_iter) {
        status = ZOLO_ENOTCONV;
        break;
      }
      Coefficients co;
      compute_coefficients(std::min(1.0, ell), r, &co);
      if (int e = iterate(R, co, false, X, Xn, b.norms + 2 * it)) return e;
      if (int e = read_status(R, hstat)) return e;
      bool qr = false;
      if (hstat[kStatCholFail]) {
        CK(cudaMemsetAsync(b.status + kStatCholFail, 0, sizeof(int), st));
        qr = true;
        info->chol_fallbacks++;
        if (int e = iterate(R, co, true, X, Xn, b.norms + 2 * it)) return e;
      }
      ell = 1.0 - co.gap;
      info->used_qr[it] = qr;
      info->ell[it + 1] = ell;
      std::swap(X, Xn);
      ++it;
    }
  }
  // Newton-Schulz refinement steps (on the split path in the iteration's slice form)
  if (pc && o.ns_steps > 0) pc->mark(ZOLO_PHASE_NS);
  for (int s = 0; s < o.ns_steps; ++s) {
    GemmArgs g;
    g.M = g.N = (int)n; g.K = (int)m; g.transA = 1;
    g.A = X; g.lda = m; g.B = X; g.ldb = m; g.Cout = b.M; g.ldcout = n;
    g.alpha[0] = 1.0;
    CK(gemm_any(g, st));
    GemmArgs u;
    u.M = (int)m; u.N = (int)n; u.K = (int)n;
    u.A = X; u.lda = m; u.B = b.M; u.ldb = n;
    u.Cin = X; u.ldcin = m; u.beta = 1.5; u.Cout = Xn; u.ldcout = m;
    u.alpha[0] = -0.5;
    CK(gemm_any(u, st));
    std::swap(X, Xn);
  }
  // H = (Qp^T A + A^T Qp) / 2 with the original A
  if (pc) pc->mark(ZOLO_PHASE_H);
  {
    GemmArgs g;
    g.M = g.N = (int)n; g.K = (int)m; g.transA = 1;
    g.A = X; g.lda = m; g.B = A; g.ldb = lda; g.Cout = b.M; g.ldcout = n;
    g.alpha[0] = 1.0;
    CK(gemm_any(g, st));
    CK(symmetrize(b.M, n, H, ldh, n, st));
    CK(copy_matrix(X, m, Qp, ldq, m, n, st));
  }
  if (o.estimate) {
    if (pc) pc->mark(ZOLO_PHASE_EST);
    if (int e = enqueue_estimates(b, A, lda, Qp, ldq, H, ldh, m, n, st)) return e;
  }
  // final status and norms
  if (int e = guards_check(h, st)) return e;
  double hn[kNormSlots];
  CK(cudaMemcpyAsync(hn, b.norms, sizeof(hn), cudaMemcpyDeviceToHost, st));
  if (int e = read_status(R, hstat)) return e;
  info->iters = it;
  for (int k = 0; k < it; ++k) info->delta[k] = hn[2 * k + 1] > 0 ? std::sqrt(hn[2 * k] / hn[2 * k + 1]) : 0.0;
  if (o.estimate) fill_estimates(info, hn, n);
  if (split.on) {
    int herr = 0;
    CK(cudaMemcpy(&herr, h->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) return ZOLO_ETIMEOUT;
  }
  if (hstat[kStatNonFinite]) return ZOLO_ENONFINITE;
  if (hstat[kStatCholFail]) return ZOLO_ECHOL;
  return status;
}

// Concurrent lanes (streams) of zolo_pd_batched.  The batch of 512 matrices with
// n in {64..1024} measured 209 / 213 / 215 matrices/s at 16 / 32 / 64 lanes:
// past 32 the GPU is full.
constexpr int kBatchLanes = 32;

// Per-matrix device record of the batched path: status words, then norms.
constexpr int kRecDoubles = 4 + kNormSlots;

// Queue one polar decomposition on `st` without any host synchronisation:
// status and norms go to R.b.status / R.b.norms (the matrix's own record).
int pd_enqueue(const Run& R, const double* A, int64_t lda, double* Qp, int64_t ldq, double* H,
               int64_t ldh, const Schedule& sch, const zolo_opts_t& o, double alpha) {
  const int64_t m = R.m, n = R.n;
  const PdBufs& b = R.b;
  cudaStream_t st = R.st;
  CK(cudaMemsetAsync(b.status, 0, sizeof(int) * kStatSlots, st));
  CK(cudaMemsetAsync(b.norms, 0, sizeof(double) * kNormSlots, st));
  double* X = b.X;
  double* Xn = b.Xn;
  CK(scale_copy(A, lda, X, m, m, n, 1.0 / alpha, st));
  CK(check_finite(X, m, m, n, b.status, st));
  for (int k = 0; k < sch.iters; ++k) {
    const bool qr = o.force_qr == 1 ? true : (o.force_qr == 0 ? false : sch.use_qr[k]);
    if (int e = iterate(R, sch.co[k], qr, X, Xn, b.norms + 2 * k)) return e;
    std::swap(X, Xn);
  }
  for (int s = 0; s < o.ns_steps; ++s) {
    GemmArgs g;
    g.M = g.N = (int)n; g.K = (int)m; g.transA = 1;
    g.A = X; g.lda = m; g.B = X; g.ldb = m; g.Cout = b.M; g.ldcout = n;
    g.alpha[0] = 1.0;
    CK(gemm_any(g, st));
    GemmArgs u;
    u.M = (int)m; u.N = (int)n; u.K = (int)n;
    u.A = X; u.lda = m; u.B = b.M; u.ldb = n;
    u.Cin = X; u.ldcin = m; u.beta = 1.5; u.Cout = Xn; u.ldcout = m;
    u.alpha[0] = -0.5;
    CK(gemm_any(u, st));
    std::swap(X, Xn);
  }
  GemmArgs g;
  g.M = g.N = (int)n; g.K = (int)m; g.transA = 1;
  g.A = X; g.lda = m; g.B = A; g.ldb = lda; g.Cout = b.M; g.ldcout = n;
  g.alpha[0] = 1.0;
  CK(gemm_any(g, st));
  CK(symmetrize(b.M, n, H, ldh, n, st));
  CK(copy_matrix(X, m, Qp, ldq, m, n, st));
  if (o.estimate)
    if (int e = enqueue_estimates(b, A, lda, Qp, ldq, H, ldh, m, n, st)) return e;
  return 0;
}

// zolo_pd_async's host function: the copied status words and norms into the
// caller's zolo_info_t (no CUDA call is made here).
void CUDART_CB async_done(void* p) {
  AsyncSlot* s = static_cast<AsyncSlot*>(p);
  zolo_info_t inf = s->base;
  for (int k = 0; k < inf.iters; ++k)
    inf.delta[k] = s->norms[2 * k + 1] > 0.0 ? std::sqrt(s->norms[2 * k] / s->norms[2 * k + 1]) : 0.0;
  if (s->estimate) fill_estimates(&inf, s->norms, s->n);
  inf.status = s->err ? ZOLO_ETIMEOUT
                      : s->stat[kStatNonFinite] ? ZOLO_ENONFINITE
                                                : s->stat[kStatCholFail] ? ZOLO_ECHOL : ZOLO_OK;
  *s->out = inf;
  s->busy = 0;
}

int grow(void** p, size_t* have, size_t bytes) {
  if (*have >= bytes) return 0;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return ZOLO_ENOMEM;
  }
  *have = bytes;
  return 0;
}

}  // namespace

extern "C" {

void zolo_opts_default(zolo_opts_t* o) {
  if (!o) return;
  o->r = 0;
  o->alpha = 1.0;
  o->beta = 0.0;
  o->max_iter = 6;
  o->posteriori = 0;
  o->ns_steps = 0;
  o->prec = ZOLO_FP64;
  o->force_qr = -1;
  o->chol_form = 0;
  o->estimate = 0;
}

int zolo_create(zolo_handle_t* handle, int device) {
  if (!handle) return -1;
  int dev = device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return ZOLO_ECUDA;
  if (cudaSetDevice(dev) != cudaSuccess) return ZOLO_ECUDA;
  auto* h = new zolo_handle_s();
  h->device = dev;
  if (cudaEventCreate(&h->e0) != cudaSuccess || cudaEventCreate(&h->e1) != cudaSuccess) {
    delete h;
    return ZOLO_ECUDA;
  }
  *handle = h;
  return 0;
}

int zolo_destroy(zolo_handle_t h) {
  if (!h) return -1;
  cudaSetDevice(h->device);
  if (h->ws) cudaFree(h->ws);
  if (h->io) cudaFree(h->io);
  if (h->slices) cudaFree(h->slices);
  if (h->exps) cudaFree(h->exps);
  if (h->err) cudaFree(h->err);
  for (BatchSlot& sl : h->slots) {
    if (sl.st) cudaStreamDestroy(sl.st);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.ws) cudaFree(sl.ws);
    if (sl.slices) cudaFree(sl.slices);
    if (sl.exps) cudaFree(sl.exps);
    if (sl.err) cudaFree(sl.err);
  }
  for (BatchGraph& g : h->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (h->fork) cudaEventDestroy(h->fork);
  if (h->joined) cudaEventDestroy(h->joined);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->brec) cudaFree(h->brec);
  if (h->hrec) cudaFreeHost(h->hrec);
  if (h->e0) cudaEventDestroy(h->e0);
  if (h->e1) cudaEventDestroy(h->e1);
  if (h->guard_flag) cudaFree(h->guard_flag);
  for (cudaEvent_t ev : h->ph_ev)
    if (ev) cudaEventDestroy(ev);
  if (h->async) {
    for (int k = 0; k < kAsyncSlots; ++k)
      if (h->async[k].busy) {   // a host function still to run reads this ring
        cudaDeviceSynchronize();
        break;
      }
    cudaFreeHost(h->async);
  }
  delete h;
  return 0;
}

int zolo_coefficients(double ell, int r, double* c, double* a, double* Mhat, double* gap) {
  Coefficients co;
  const int e = compute_coefficients(ell, r, &co);
  if (e) return e;
  if (c) for (int i = 0; i < 2 * r; ++i) c[i] = co.c[i];
  if (a) for (int j = 0; j < r; ++j) a[j] = co.a[j];
  if (Mhat) *Mhat = co.mhat;
  if (gap) *gap = co.gap;
  return 0;
}

int zolo_workspace_bytes(int64_t m, int64_t n, int r, int prec, int svd, uint64_t* bytes) {
  if (n < 1 || n > INT32_MAX) return -2;
  if (m < n || m > INT32_MAX) return -1;
  if (r < ZOLO_R_TUNED || r > kMaxR) return -3;
  if (prec != ZOLO_FP64 && !is_split(prec)) return -4;
  if (svd != 0 && svd != 1) return -5;
  if (!bytes) return -6;
  const int rr = r > 0 ? r : kMaxR;   // r chosen by the call: at most 8 shifts
  PdBufs b;
  uint64_t total = layout(nullptr, m, n, rr, svd != 0, &b);
  if (is_split(prec)) {
    // as SplitScope::begin asks for: slice planes (BF16), exponents (int), error flag
    const size_t per = split_elems_per_entry(m, n);
    const size_t want = std::max(per, std::min(per * (size_t)rr, (size_t)8 << 30));
    const size_t exps = (size_t)2 * kGemmMaxBatch * (size_t)(std::max(m, n) + m + n + 512);
    total += want * 2 + exps * sizeof(int) + sizeof(int);
  }
  *bytes = total;
  return 0;
}

int zolo_schedule(double ell0, int r, int max_iter, double* ells, int* used_qr, int* r_used) {
  Schedule s;
  const int e = build_schedule(ell0, r, max_iter, &s);
  if (e) return e;
  if (ells) for (int k = 0; k <= s.iters; ++k) ells[k] = s.ell[k];
  if (used_qr) for (int k = 0; k < s.iters; ++k) used_qr[k] = s.use_qr[k] ? 1 : 0;
  if (r_used) *r_used = s.r;
  return s.iters;
}

int zolo_pd(zolo_handle_t h, const double* A, int64_t m, int64_t n, int64_t lda, double* Qp,
            int64_t ldq, double* H, int64_t ldh, const zolo_opts_t* opts, zolo_info_t* info,
            void* stream) {
  if (int e = validate(h, A, m, n, lda, Qp, ldq, H, ldh, opts)) return e;
  if (!info) return -11;
  std::memset(info, 0, sizeof(*info));
  if (cudaSetDevice(h->device) != cudaSuccess) return info->status = ZOLO_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  TunerScope ts(&h->tuner);
  GuardScope guard(h->guards);
  PhaseClock pc;
  pc.start(h, st);
  cudaEventRecord(h->e0, st);
  int e = pd_core(h, A, m, n, lda, Qp, ldq, H, ldh, *opts, info, st, false, nullptr, nullptr, &pc);
  pc.stop();
  cudaEventRecord(h->e1, st);
  if (cudaEventSynchronize(h->e1) == cudaSuccess) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->e0, h->e1);
    info->ms = ms;
    pc.read(info->ms_phase);
  }
  info->status = e;
  return e;
}

int zolo_pd_async(zolo_handle_t h, const double* A, int64_t m, int64_t n, int64_t lda, double* Qp,
                  int64_t ldq, double* H, int64_t ldh, const zolo_opts_t* opts, zolo_info_t* info,
                  void* stream) {
  if (int e = validate(h, A, m, n, lda, Qp, ldq, H, ldh, opts)) return e;
  const zolo_opts_t& o = *opts;
  if (!(o.alpha > 0.0) || !(o.beta > 0.0) || o.r == ZOLO_R_TUNED || o.posteriori) return -10;
  if (!info) return -11;
  std::memset(info, 0, sizeof(*info));
  if (cudaSetDevice(h->device) != cudaSuccess) return info->status = ZOLO_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!h->async) {
    void* p = nullptr;
    if (cudaMallocHost(&p, sizeof(AsyncSlot) * kAsyncSlots) != cudaSuccess) {
      cudaGetLastError();
      return info->status = ZOLO_ENOMEM;
    }
    std::memset(p, 0, sizeof(AsyncSlot) * kAsyncSlots);
    h->async = static_cast<AsyncSlot*>(p);
  }
  AsyncSlot* slot = &h->async[h->async_next];
  // a slot still waiting for its host function belongs to a call 64 back on this
  // stream: wait for it (calls on one handle are ordered on one stream)
  if (slot->busy && cudaStreamSynchronize(st) != cudaSuccess) return info->status = ZOLO_ECUDA;
  // kernels measured so far are used; none is timed here (timing synchronises)
  const bool was_tuning = h->tuner.tuning;
  h->tuner.tuning = false;
  TunerScope ts(&h->tuner);
  struct Restore {
    zolo_handle_t h;
    bool v;
    ~Restore() { h->tuner.tuning = v; }
  } restore{h, was_tuning};
  const double ell0 = std::min(1.0, o.beta / o.alpha);
  Schedule sch;
  if (build_schedule(ell0, o.r, o.max_iter, &sch) != 0) return -10;
  Run R{m, n, sch.r, {}, st};
  R.inv_chol = use_inverse_form(o.chol_form, m, n, sch.r);
  if (int e = ensure_ws(h, layout(nullptr, m, n, sch.r, false, &R.b))) return info->status = e;
  layout(h->ws, m, n, sch.r, false, &R.b);
  SplitScope split;
  if (is_split(o.prec))
    if (int e = split.begin(h, m, n, sch.r, st, o.prec)) return info->status = e;
  if (int e = pd_enqueue(R, A, lda, Qp, ldq, H, ldh, sch, o, o.alpha)) return info->status = e;
  zolo_info_t& base = slot->base;
  std::memset(&base, 0, sizeof(base));
  base.r = sch.r;
  base.iters = sch.iters;
  base.chol_form = R.inv_chol ? 2 : 1;
  base.ell[0] = sch.ell[0];
  for (int k = 0; k < sch.iters; ++k) {
    base.used_qr[k] = o.force_qr == 1 ? 1 : (o.force_qr == 0 ? 0 : sch.use_qr[k]);
    base.ell[k + 1] = sch.ell[k + 1];
  }
  slot->out = info;
  slot->n = n;
  slot->estimate = o.estimate;
  slot->err = 0;
  slot->busy = 1;
  CK(cudaMemcpyAsync(slot->stat, R.b.status, sizeof(slot->stat), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(slot->norms, R.b.norms, sizeof(slot->norms), cudaMemcpyDeviceToHost, st));
  if (split.on)
    CK(cudaMemcpyAsync(&slot->err, h->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  info->status = ZOLO_EPENDING;
  if (cudaLaunchHostFunc(st, async_done, slot) != cudaSuccess) {
    slot->busy = 0;
    return info->status = ZOLO_ECUDA;
  }
  h->async_next = (h->async_next + 1) % kAsyncSlots;
  return 0;
}

int zolo_shift_range(int r, int rank, int nranks, int* j0, int* j1) {
  if (r < 1 || r > kMaxR) return -1;
  if (nranks < 1) return -3;
  if (rank < 0 || rank >= nranks) return -2;
  if (!j0 || !j1) return -4;
  const int base = r / nranks, extra = r % nranks;
  *j0 = rank * base + std::min(rank, extra);
  *j1 = *j0 + base + (rank < extra ? 1 : 0);
  return 0;
}

int zolo_pd_sharded(zolo_handle_t h, const double* A, int64_t m, int64_t n, int64_t lda,
                    double* Qp, int64_t ldq, double* H, int64_t ldh, const zolo_opts_t* opts,
                    zolo_info_t* info, void* stream, int rank, int nranks, zolo_sum_fn sum,
                    void* ctx) {
  if (int e = validate(h, A, m, n, lda, Qp, ldq, H, ldh, opts)) return e;
  if (opts->r == ZOLO_R_TUNED || opts->posteriori) return -10;
  if (!info) return -11;
  if (nranks < 1) return -14;
  if (rank < 0 || rank >= nranks) return -13;
  if (!sum && nranks > 1) return -15;
  std::memset(info, 0, sizeof(*info));
  if (cudaSetDevice(h->device) != cudaSuccess) return info->status = ZOLO_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  TunerScope ts(&h->tuner);
  GuardScope guard(h->guards);
  ShardCtx sh;
  sh.rank = rank;
  sh.nranks = nranks;
  sh.fn = sum;
  sh.ctx = ctx;
  cudaEventRecord(h->e0, st);
  PhaseClock pc;
  pc.start(h, st);
  int e = pd_core(h, A, m, n, lda, Qp, ldq, H, ldh, *opts, info, st, false, nullptr, &sh, &pc);
  pc.stop();
  cudaEventRecord(h->e1, st);
  if (cudaEventSynchronize(h->e1) == cudaSuccess) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->e0, h->e1);
    info->ms = ms;
    pc.read(info->ms_phase);
  }
  info->status = e;
  return e;
}

int zolo_svd(zolo_handle_t h, const double* A, int64_t m, int64_t n, int64_t lda, double* U,
             int64_t ldu, double* S, double* V, int64_t ldv, const zolo_opts_t* opts,
             zolo_info_t* info, void* stream) {
  if (int e = validate(h, A, m, n, lda, U, ldu, V, ldv, opts)) return e;
  if (!S) return -8;
  if (!info) return -12;
  std::memset(info, 0, sizeof(*info));
  if (cudaSetDevice(h->device) != cudaSuccess) return info->status = ZOLO_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  TunerScope ts(&h->tuner);
  GuardScope guard(h->guards);
  cudaEventRecord(h->e0, st);
  // Qp and H go to internal buffers carved ahead of the union region; their
  // offsets do not depend on r, and sizing with r = 8 when r is chosen by the
  // schedule means pd_core never has to grow (and move) the workspace.
  PdBufs b{};
  int e = 0;
  const int r_size = opts->r <= 0 ? kMaxR : opts->r;
  {
    const size_t bytes = layout(nullptr, m, n, r_size, true, &b);
    if ((e = ensure_ws(h, bytes)) != 0) return info->status = e;
    layout(h->ws, m, n, r_size, true, &b);
  }
  double* Qp = b.Qp_int;
  double* Hm = b.H_int;
  PhaseClock pc;
  pc.start(h, st);
  e = pd_core(h, A, m, n, lda, Qp, m, Hm, n, *opts, info, st, true, &b, nullptr, &pc);
  if (e == 0) {
    pc.mark(ZOLO_PHASE_EIG);
    std::vector<double> lam(n);
    int sweeps = 0;
    b.eig.stall = h->dbg_stall == ZOLO_STALL_JACOBI32;
    b.eig.stall64 = h->dbg_stall == ZOLO_STALL_JACOBI64;
    b.eig.stall_ns = h->dbg_ns;
    const int ee = eig_sym_jacobi(Hm, n, n, V, ldv, lam.data(), b.eig, &sweeps, st);
    info->eig_sweeps = sweeps;
    if (ee == 1) e = ZOLO_ECUDA;
    else if (ee == 2) e = ZOLO_EEIG;
    else if (ee == 3) e = ZOLO_ETIMEOUT;
    if (e == 0) {
      // U = Qp V, with the sign of u_i flipped where lambda_i < 0 (sigma_i = |lambda_i|)
      std::vector<double> sv(n), sg(n);
      for (int64_t i = 0; i < n; ++i) {
        sv[i] = std::fabs(lam[i]);
        sg[i] = lam[i] < 0.0 ? -1.0 : 1.0;
      }
      pc.mark(ZOLO_PHASE_U);
      GemmArgs g;
      g.M = (int)m; g.N = (int)n; g.K = (int)n;
      g.A = Qp; g.lda = m; g.B = V; g.ldb = ldv; g.Cout = U; g.ldcout = ldu;
      g.alpha[0] = 1.0;
      if (gemm_any(g, st) != cudaSuccess) e = ZOLO_ECUDA;
      if (e == 0 && cudaMemcpyAsync(b.eig.lam, sg.data(), sizeof(double) * n,
                                    cudaMemcpyHostToDevice, st) != cudaSuccess)
        e = ZOLO_ECUDA;
      if (e == 0 && scale_columns(U, ldu, m, n, b.eig.lam, 0, st) != cudaSuccess) e = ZOLO_ECUDA;
      if (e == 0 && cudaMemcpyAsync(S, sv.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st) !=
                        cudaSuccess)
        e = ZOLO_ECUDA;
      if (cudaStreamSynchronize(st) != cudaSuccess) e = ZOLO_ECUDA;
    }
    if (e == 0) e = guards_check(h, st);   // the eigensolver's buffers too
  }
  pc.stop();
  cudaEventRecord(h->e1, st);
  if (cudaEventSynchronize(h->e1) == cudaSuccess) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->e0, h->e1);
    info->ms = ms;
    pc.read(info->ms_phase);
  }
  info->status = e;
  return e;
}

static int ensure_io(zolo_handle_t h, size_t bytes) {
  if (h->io_bytes >= bytes) return 0;
  if (h->io) cudaFree(h->io);
  h->io = nullptr;
  h->io_bytes = 0;
  if (cudaMalloc(&h->io, bytes) != cudaSuccess) {
    cudaGetLastError();
    return ZOLO_ENOMEM;
  }
  h->io_bytes = bytes;
  return 0;
}

int zolo_pd_host(zolo_handle_t h, const double* A, int64_t m, int64_t n, int64_t lda, double* Qp,
                 int64_t ldq, double* H, int64_t ldh, const zolo_opts_t* opts, zolo_info_t* info,
                 void* stream) {
  if (int e = validate(h, A, m, n, lda, Qp, ldq, H, ldh, opts)) return e;
  if (!info) return -11;
  if (cudaSetDevice(h->device) != cudaSuccess) return ZOLO_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t mn = (size_t)m * n, nn = (size_t)n * n;
  if (int e = ensure_io(h, sizeof(double) * (2 * mn + nn) + 1024)) return e;
  double* dA = static_cast<double*>(h->io);
  double* dQ = dA + mn;
  double* dH = dQ + mn;
  if (cudaMemcpy2DAsync(dA, m * sizeof(double), A, lda * sizeof(double), m * sizeof(double), n,
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
    return ZOLO_ECUDA;
  int e = zolo_pd(h, dA, m, n, m, dQ, m, dH, n, opts, info, stream);
  if (e > 0 && e != ZOLO_ENOTCONV) return e;
  if (cudaMemcpy2DAsync(Qp, ldq * sizeof(double), dQ, m * sizeof(double), m * sizeof(double), n,
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpy2DAsync(H, ldh * sizeof(double), dH, n * sizeof(double), n * sizeof(double), n,
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ZOLO_ECUDA;
  return e;
}

int zolo_svd_host(zolo_handle_t h, const double* A, int64_t m, int64_t n, int64_t lda, double* U,
                  int64_t ldu, double* S, double* V, int64_t ldv, const zolo_opts_t* opts,
                  zolo_info_t* info, void* stream) {
  if (int e = validate(h, A, m, n, lda, U, ldu, V, ldv, opts)) return e;
  if (!S) return -8;
  if (!info) return -12;
  if (cudaSetDevice(h->device) != cudaSuccess) return ZOLO_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t mn = (size_t)m * n, nn = (size_t)n * n;
  if (int e = ensure_io(h, sizeof(double) * (2 * mn + nn + n) + 2048)) return e;
  double* dA = static_cast<double*>(h->io);
  double* dU = dA + mn;
  double* dV = dU + mn;
  double* dS = dV + nn;
  if (cudaMemcpy2DAsync(dA, m * sizeof(double), A, lda * sizeof(double), m * sizeof(double), n,
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
    return ZOLO_ECUDA;
  int e = zolo_svd(h, dA, m, n, m, dU, m, dS, dV, n, opts, info, stream);
  if (e > 0 && e != ZOLO_ENOTCONV) return e;
  if (cudaMemcpy2DAsync(U, ldu * sizeof(double), dU, m * sizeof(double), m * sizeof(double), n,
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpy2DAsync(V, ldv * sizeof(double), dV, n * sizeof(double), n * sizeof(double), n,
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(S, dS, n * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ZOLO_ECUDA;
  return e;
}

int zolo_dgemm(zolo_handle_t h, int transA, int transB, int64_t m, int64_t n, int64_t k,
               double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
               double beta, double* C, int64_t ldc, int prec, int slices, void* stream) {
  if (!h) return -1;
  if (transA != 0 && transA != 1) return -2;
  if (transB != 0 && transB != 1) return -3;
  if (m < 0 || m > INT32_MAX) return -4;
  if (n < 0 || n > INT32_MAX) return -5;
  if (k < 0 || k > INT32_MAX) return -6;
  if (!std::isfinite(alpha)) return -7;
  if (k > 0 && m > 0 && !A) return -8;
  if (lda < std::max<int64_t>(1, transA ? k : m)) return -9;
  if (k > 0 && n > 0 && !B) return -10;
  if (ldb < std::max<int64_t>(1, transB ? n : k)) return -11;
  if (!std::isfinite(beta)) return -12;
  if (m > 0 && n > 0 && !C) return -13;
  if (ldc < std::max<int64_t>(1, m)) return -14;
  if (prec != ZOLO_FP64 && !is_split(prec)) return -15;
  if (slices != 0 && slices != split_slices(prec) && !(prec == ZOLO_SPLIT_BF16 && slices == 8))
    return -16;
  if (cudaSetDevice(h->device) != cudaSuccess) return ZOLO_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  TunerScope ts(&h->tuner);
  GemmArgs g;
  g.M = (int)m; g.N = (int)n; g.K = (int)k; g.transA = transA; g.transB = transB;
  g.A = A; g.lda = lda; g.B = B; g.ldb = ldb;
  g.Cin = beta != 0.0 ? C : nullptr; g.ldcin = ldc; g.beta = beta;
  g.Cout = C; g.ldcout = ldc;
  g.alpha[0] = alpha;
  if (prec == ZOLO_FP64) {
    if (gemm_f64(g, st) != cudaSuccess) return ZOLO_ECUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? 0 : ZOLO_ECUDA;
  }
  const int S = slices ? slices : prec == ZOLO_SPLIT_BF16 ? 8 : split_slices(prec);
  const size_t per = split_slice_elems(m, n, k, 1, S, split_form(prec));
  const size_t exps = (size_t)2 * (size_t)(std::max(m, n) + m + n + 512);
  if (int e = ensure_split(h, per, per, exps)) return e;
  if (cudaMemsetAsync(h->err, 0, sizeof(int), st) != cudaSuccess) return ZOLO_ECUDA;
  SplitWork w{h->slices, h->slice_elems, h->exps, h->exp_elems, h->err, S};
  w.form = split_form(prec);
  w.stall = h->dbg_stall == ZOLO_STALL_SPLIT_GEMM;
  w.stall_ns = h->dbg_ns;
  if (gemm_split(g, w, st) != cudaSuccess) return ZOLO_ECUDA;
  int herr = 0;
  if (cudaMemcpyAsync(&herr, h->err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ZOLO_ECUDA;
  return herr ? ZOLO_ETIMEOUT : 0;
}

int zolo_pd_batched(zolo_handle_t h, int count, const double* const* A, const int64_t* m,
                    const int64_t* n, const int64_t* lda, double* const* Qp, const int64_t* ldq,
                    double* const* H, const int64_t* ldh, const zolo_opts_t* opts,
                    zolo_info_t* info, void* stream) {
  if (!h) return -1;
  if (count < 0) return -2;
  if (count == 0) return 0;
  if (!A || !m || !n || !lda || !Qp || !ldq || !H || !ldh || !opts || !info) return -3;
  // kernel choices come from the handle's tuner (per lane below); none is timed
  // while the lanes are queued
  TunerScope no_tuner(nullptr);
  for (int i = 0; i < count; ++i) {
    std::memset(&info[i], 0, sizeof(zolo_info_t));
    int e = validate(h, A[i], m[i], n[i], lda[i], Qp[i], ldq[i], H[i], ldh[i], &opts[i]);
    if (e == 0 && opts[i].posteriori) e = -10;
    if (e) {
      info[i].status = e;
      return e;
    }
  }
  if (cudaSetDevice(h->device) != cudaSuccess) return ZOLO_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEventRecord(h->e0, st);
  // ---- bounds and schedules (alpha <= 0: min(||A_i||_F, sqrt(||A_i||_1 ||A_i||_inf)),
  // all sums in one pass; the scratch is reused matrix after matrix on one stream)
  std::vector<double> alpha(count), beta(count);
  std::vector<Schedule> sch(count);
  {
    std::vector<int> need;
    int64_t part_max = 0, n_max = 0;
    for (int i = 0; i < count; ++i) {
      alpha[i] = opts[i].alpha;
      if (alpha[i] <= 0.0) {
        need.push_back(i);
        part_max = std::max(part_max, alpha_bound_part_elems(m[i], n[i]));
        n_max = std::max(n_max, n[i]);
      }
    }
    if (!need.empty()) {
      double* tmp = nullptr;
      const size_t nsum = 3 * need.size();
      if (cudaMalloc(&tmp, sizeof(double) * (nsum + 2 * 1024 + part_max + n_max)) != cudaSuccess) {
        cudaGetLastError();
        return ZOLO_ENOMEM;
      }
      double* partials = tmp + nsum;
      double* part = partials + 2 * 1024;
      double* colsum = part + part_max;
      std::vector<double> nr(nsum);
      int e = 0;
      for (size_t q = 0; q < need.size() && !e; ++q) {
        const int i = need[q];
        if (alpha_bound_sums(A[i], lda[i], m[i], n[i], part, colsum, partials, tmp + 3 * q, st) !=
            cudaSuccess)
          e = ZOLO_ECUDA;
      }
      if (!e && (cudaMemcpyAsync(nr.data(), tmp, sizeof(double) * nr.size(), cudaMemcpyDeviceToHost,
                                 st) != cudaSuccess ||
                 cudaStreamSynchronize(st) != cudaSuccess))
        e = ZOLO_ECUDA;
      cudaFree(tmp);
      if (e) return e;
      for (size_t q = 0; q < need.size(); ++q) alpha[need[q]] = alpha_from_sums(&nr[3 * q]);
    }
    for (int i = 0; i < count; ++i) {
      if (!(alpha[i] > 0.0) || !std::isfinite(alpha[i])) {
        info[i].status = ZOLO_ENONFINITE;
        return ZOLO_ENONFINITE;
      }
      // beta <= 0: estimated on the handle's own workspace, before any lane starts
      beta[i] = opts[i].beta;
      if (!(beta[i] > 0.0)) {
        PdBufs eb;
        if (int e = ensure_ws(h, layout(nullptr, m[i], n[i], 1, false, &eb))) {
          info[i].status = e;
          return e;
        }
        layout(h->ws, m[i], n[i], 1, false, &eb);
        if (int e = estimate_beta(A[i], lda[i], m[i], n[i], alpha[i], eb, st, &beta[i])) {
          info[i].status = e;
          return e;
        }
      }
      const double ell0 = std::min(1.0, beta[i] / alpha[i]);
      int ri = opts[i].r;
      if (ri == ZOLO_R_TUNED) {
        const auto hit = h->tuned_r.find(tune_key(m[i], n[i], opts[i].prec, ell0));
        ri = hit != h->tuned_r.end() ? hit->second : 0;
      }
      if (build_schedule(ell0, ri, opts[i].max_iter, &sch[i]) != 0) {
        info[i].status = -10;
        return -10;
      }
    }
  }
  // ---- lanes: streams with workspace for the largest matrix of the batch.  With
  // per-kernel profiling on, one lane: every launch's event pair then times that
  // kernel alone, not its share of a GPU other lanes' kernels run on too
  const int nslots = profiling_enabled() ? 1 : std::min(count, kBatchLanes);
  int64_t mmax = 0, nmax = 0;
  int rmax = 1;
  bool any_split = false;
  for (int i = 0; i < count; ++i) {
    mmax = std::max(mmax, m[i]);
    nmax = std::max(nmax, n[i]);
    rmax = std::max(rmax, sch[i].r);
    any_split |= is_split(opts[i].prec);
  }
  if ((int)h->slots.size() < nslots) h->slots.resize(nslots);
  if (!h->fork && cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess)
    return ZOLO_ECUDA;
  const size_t ws_bytes = layout(nullptr, mmax, nmax, rmax, false, nullptr);
  for (int k = 0; k < nslots; ++k) {
    BatchSlot& sl = h->slots[k];
    if (!sl.st && cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess)
      return ZOLO_ECUDA;
    if (!sl.done && cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess)
      return ZOLO_ECUDA;
    if (int e = grow(&sl.ws, &sl.ws_bytes, ws_bytes)) return e;
    if (any_split) {
      const size_t per = split_elems_per_entry(mmax, nmax) * (size_t)rmax;
      size_t have = sl.slice_elems * 2;
      if (int e = grow(&sl.slices, &have, per * 2)) return e;
      sl.slice_elems = have / 2;
      const size_t ex = (size_t)2 * kGemmMaxBatch * (size_t)(2 * mmax + nmax + 512);
      size_t hx = sl.exp_elems * sizeof(int);
      if (int e = grow((void**)&sl.exps, &hx, ex * sizeof(int))) return e;
      sl.exp_elems = hx / sizeof(int);
      size_t he = sl.err ? sizeof(int) : 0;
      if (int e = grow((void**)&sl.err, &he, sizeof(int))) return e;
    }
  }
  // ---- per-matrix records
  {
    size_t have = h->brec_count * sizeof(double);
    if (int e = grow((void**)&h->brec, &have, sizeof(double) * kRecDoubles * (size_t)count)) return e;
    h->brec_count = have / sizeof(double);
    if (h->hrec_count < (size_t)count * kRecDoubles) {
      if (h->hrec) cudaFreeHost(h->hrec);
      h->hrec = nullptr;
      h->hrec_count = 0;
      if (cudaMallocHost(&h->hrec, sizeof(double) * kRecDoubles * (size_t)count) != cudaSuccess) {
        cudaGetLastError();
        return ZOLO_ENOMEM;
      }
      h->hrec_count = (size_t)count * kRecDoubles;
    }
  }
  // ---- kernel choices (zolo_autotune).  With tuning on, one matrix of every
  // distinct configuration (sizes, r, iteration forms, options) is decomposed
  // first on the caller's stream, outside any capture, in lane 0's workspace,
  // while the handle's tuner times the contraction shapes it meets; the lanes
  // then replay the handle's choices, each with its own split-K scratch.
  if (h->tuner.tuning) {
    TunerScope ts(&h->tuner);
    std::map<std::vector<int64_t>, int> seen;
    BatchSlot& sl = h->slots[0];
    for (int i = 0; i < count; ++i) {
      const bool inv = use_inverse_form(opts[i].chol_form, m[i], n[i], sch[i].r);
      std::vector<int64_t> cfg = {m[i], n[i], sch[i].r, sch[i].iters, opts[i].prec,
                                  opts[i].ns_steps, opts[i].force_qr, inv ? 1 : 0, opts[i].estimate};
      for (int k = 0; k < sch[i].iters; ++k) cfg.push_back(sch[i].use_qr[k] ? 1 : 0);
      if (!seen.emplace(cfg, i).second) continue;
      Run R{m[i], n[i], sch[i].r, {}, st};
      R.inv_chol = inv;
      R.narrow_panels = true;
      layout(sl.ws, m[i], n[i], sch[i].r, false, &R.b);
      SplitWork w{sl.slices, sl.slice_elems, sl.exps, sl.exp_elems, sl.err, 9};
      w.slices_s = split_slices(opts[i].prec);
      w.form = split_form(opts[i].prec);
      w.throughput = true;
      set_split_engine(is_split(opts[i].prec) ? &w : nullptr);
      const int e = pd_enqueue(R, A[i], lda[i], Qp[i], ldq[i], H[i], ldh[i], sch[i], opts[i],
                               alpha[i]);
      set_split_engine(nullptr);
      if (e) return e;
    }
    CK(cudaStreamSynchronize(st));
  }
  for (int k = 0; k < nslots; ++k) {
    BatchSlot& sl = h->slots[k];
    if (!sl.tuner) sl.tuner.reset(new GemmTuner());
    if (sl.tuner_gen != h->tuner.gen) {
      sl.tuner->choice = h->tuner.choice;
      sl.tuner_gen = h->tuner.gen;
    }
    sl.tuner->tuning = false;
    if (sl.tuner->scratch_elems < h->tuner.scratch_elems) {
      if (sl.tuner->scratch) cudaFree(sl.tuner->scratch);
      sl.tuner->scratch = nullptr;
      sl.tuner->scratch_elems = 0;
      if (cudaMalloc(&sl.tuner->scratch, h->tuner.scratch_elems * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return ZOLO_ENOMEM;
      }
      sl.tuner->scratch_elems = h->tuner.scratch_elems;
    }
  }
  if (!h->cap && cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess)
    return ZOLO_ECUDA;
  if (!h->joined && cudaEventCreateWithFlags(&h->joined, cudaEventDisableTiming) != cudaSuccess)
    return ZOLO_ECUDA;
  if (any_split) split_prepare();
  // ---- the batch as one graph: key = every pointer, size and option of the call
  std::vector<uint64_t> key;
  key.reserve(8 + 12 * (size_t)count);
  key.push_back((uint64_t)count);
  key.push_back((uint64_t)(uintptr_t)h->brec);
  key.push_back(h->tuner.gen);   // graphs recorded with older kernel choices are not replayed
  for (int k = 0; k < nslots; ++k) key.push_back((uint64_t)(uintptr_t)h->slots[k].ws);
  for (int i = 0; i < count; ++i) {
    const uint64_t f[] = {(uint64_t)(uintptr_t)A[i], (uint64_t)m[i], (uint64_t)n[i],
                          (uint64_t)lda[i], (uint64_t)(uintptr_t)Qp[i], (uint64_t)ldq[i],
                          (uint64_t)(uintptr_t)H[i], (uint64_t)ldh[i]};
    key.insert(key.end(), f, f + 8);
    uint64_t ob[sizeof(zolo_opts_t) / 8 + 1] = {};
    std::memcpy(ob, &opts[i], sizeof(zolo_opts_t));
    key.insert(key.end(), ob, ob + sizeof(zolo_opts_t) / 8 + 1);
    uint64_t ab;
    std::memcpy(&ab, &alpha[i], 8);
    key.push_back(ab);
    std::memcpy(&ab, &beta[i], 8);   // an estimated beta follows A's contents
    key.push_back(ab);
    key.push_back((uint64_t)sch[i].r);   // a tuned r may change between calls
  }
  cudaGraphExec_t exec = nullptr;
  for (BatchGraph& g : h->graphs)
    if (g.key == key) exec = g.exec;
  // largest matrices first, dealt round-robin over the lanes
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return m[a] * n[a] * n[a] * sch[a].r > m[b] * n[b] * n[b] * sch[b].r;
  });
  cudaStream_t cap = h->cap;
  auto enqueue_all = [&]() -> int {
    CK(cudaEventRecord(h->fork, cap));
    for (int k = 0; k < nslots; ++k) CK(cudaStreamWaitEvent(h->slots[k].st, h->fork, 0));
    for (int q = 0; q < count; ++q) {
      const int i = order[q];
      BatchSlot& sl = h->slots[q % nslots];
      Run R{m[i], n[i], sch[i].r, {}, sl.st};
      R.inv_chol = use_inverse_form(opts[i].chol_form, m[i], n[i], sch[i].r);
      R.narrow_panels = true;
      layout(sl.ws, m[i], n[i], sch[i].r, false, &R.b);
      double* rec = h->brec + (size_t)i * kRecDoubles;
      R.b.status = reinterpret_cast<int*>(rec);
      R.b.norms = rec + 4;
      SplitWork w{sl.slices, sl.slice_elems, sl.exps, sl.exp_elems, sl.err, 9};
      w.slices_s = split_slices(opts[i].prec);
      w.form = split_form(opts[i].prec);
      w.throughput = true;   // many lanes in flight: latency is hidden
      w.stall = h->dbg_stall == ZOLO_STALL_SPLIT_GEMM;
      w.stall_ns = h->dbg_ns;
      set_split_engine(is_split(opts[i].prec) ? &w : nullptr);
      TunerScope lane_tuner(sl.tuner.get());
      const int e = pd_enqueue(R, A[i], lda[i], Qp[i], ldq[i], H[i], ldh[i], sch[i], opts[i], alpha[i]);
      set_split_engine(nullptr);
      if (e) return e;
    }
    for (int k = 0; k < nslots; ++k) {
      CK(cudaEventRecord(h->slots[k].done, h->slots[k].st));
      CK(cudaStreamWaitEvent(cap, h->slots[k].done, 0));
    }
    return 0;
  };
  if (any_split)
    for (int k = 0; k < nslots; ++k)
      if (h->slots[k].err) CK(cudaMemsetAsync(h->slots[k].err, 0, sizeof(int), st));
  // the capture stream starts after everything queued on the caller's stream
  CK(cudaEventRecord(h->joined, st));
  CK(cudaStreamWaitEvent(cap, h->joined, 0));
  // with per-kernel profiling on, the work is queued directly (events cannot
  // bracket the nodes of a graph)
  const bool use_graph = !profiling_enabled() && h->batch_graphs;
  if (!use_graph) exec = nullptr;
  uint64_t graph_launches = 0;
  for (BatchGraph& g : h->graphs)
    if (g.exec == exec) graph_launches = g.launches;
  if (!exec && use_graph) {
    cudaGraph_t graph = nullptr;
    const uint64_t l0 = zolo_kernel_launches();
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int e = enqueue_all();
      const cudaError_t ce = cudaStreamEndCapture(cap, &graph);
      if (e == 0 && ce == cudaSuccess && graph &&
          cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
        graph_launches = zolo_kernel_launches() - l0;
        // the capture itself ran no kernel: take the recorded ones back off the counter
        add_launches(-(int64_t)graph_launches);
        h->graphs.push_back({key, exec, graph_launches});
        if (h->graphs.size() > 8) {
          cudaGraphExecDestroy(h->graphs.front().exec);
          h->graphs.erase(h->graphs.begin());
        }
      } else {
        exec = nullptr;
      }
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
    }
  }
  if (exec) {
    CK(cudaGraphLaunch(exec, cap));
    add_launches((int64_t)graph_launches);
  } else if (int e = enqueue_all()) {
    return e;
  }
  CK(cudaEventRecord(h->joined, cap));
  CK(cudaStreamWaitEvent(st, h->joined, 0));
  // ---- statuses and norms, once
  CK(cudaMemcpyAsync(h->hrec, h->brec, sizeof(double) * kRecDoubles * (size_t)count,
                     cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  int worst = 0;
  bool timeout = false;
  if (any_split)
    for (int k = 0; k < nslots; ++k) {
      int he = 0;
      if (h->slots[k].err) CK(cudaMemcpy(&he, h->slots[k].err, sizeof(int), cudaMemcpyDeviceToHost));
      timeout |= he != 0;
    }
  for (int i = 0; i < count; ++i) {
    const double* rec = h->hrec + (size_t)i * kRecDoubles;
    int stv[kStatSlots];
    std::memcpy(stv, rec, sizeof(stv));
    zolo_info_t& inf = info[i];
    inf.r = sch[i].r;
    inf.chol_form = use_inverse_form(opts[i].chol_form, m[i], n[i], sch[i].r) ? 2 : 1;
    inf.iters = sch[i].iters;
    inf.ell[0] = sch[i].ell[0];
    for (int k = 0; k < sch[i].iters; ++k) {
      inf.used_qr[k] = opts[i].force_qr == 1 ? 1 : (opts[i].force_qr == 0 ? 0 : sch[i].use_qr[k]);
      inf.ell[k + 1] = sch[i].ell[k + 1];
      const double* nk = rec + 4 + 2 * k;
      inf.delta[k] = nk[1] > 0.0 ? std::sqrt(nk[0] / nk[1]) : 0.0;
    }
    if (opts[i].estimate) fill_estimates(&inf, rec + 4, n[i]);
    int e = 0;
    if (stv[kStatCholFail]) {
      // redo this matrix on the single-matrix path, which falls back to the QR form
      zolo_info_t again;
      e = zolo_pd(h, A[i], m[i], n[i], lda[i], Qp[i], ldq[i], H[i], ldh[i], &opts[i], &again, stream);
      const double ms = inf.ms;
      inf = again;
      inf.ms = ms;
    } else if (stv[kStatNonFinite]) {
      e = ZOLO_ENONFINITE;
    } else if (timeout && is_split(opts[i].prec)) {
      e = ZOLO_ETIMEOUT;
    }
    inf.status = e;
    if (e && !worst) worst = e;
  }
  cudaEventRecord(h->e1, st);
  if (cudaEventSynchronize(h->e1) == cudaSuccess) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->e0, h->e1);
    for (int i = 0; i < count; ++i) info[i].ms = ms;
  }
  return worst;
}

int zolo_debug_guards(zolo_handle_t h, int enable) {
  if (!h) return -1;
  if (enable != 0 && enable != 1) return -2;
  h->guards = enable != 0;
  return 0;
}

int zolo_batch_graphs(zolo_handle_t h, int enable) {
  if (!h) return -1;
  if (enable != 0 && enable != 1) return -2;
  h->batch_graphs = enable != 0;
  return 0;
}

int zolo_debug_stall(zolo_handle_t h, int where, int64_t ns) {
  if (!h) return -1;
  if (where != 0 && where != ZOLO_STALL_SPLIT_GEMM && where != ZOLO_STALL_JACOBI32 &&
      where != ZOLO_STALL_JACOBI64)
    return -2;
  if (ns < 0 || ns > 1000000000) return -3;
  h->dbg_stall = where;
  h->dbg_ns = ns;
  return 0;
}

int zolo_tuned_r(zolo_handle_t h, int64_t m, int64_t n, int prec, double ell0) {
  if (!h || !(ell0 > 0.0 && ell0 <= 1.0)) return 0;
  const auto hit = h->tuned_r.find(tune_key(m, n, prec, ell0));
  return hit != h->tuned_r.end() ? hit->second : 0;
}

int zolo_autotune(zolo_handle_t h, int enable) {
  if (!h) return -1;
  if (enable != 0 && enable != 1) return -2;
  h->tuner.tuning = enable != 0;
  return 0;
}

int zolo_tune_save(zolo_handle_t h, const char* path) {
  if (!h) return -1;
  if (!path) return -2;
  FILE* f = std::fopen(path, "w");
  if (!f) return ZOLO_EIO;
  bool ok = std::fprintf(f, "zolo-tune 2 %s\n", device_tag(h->device).c_str()) > 0;
  for (const auto& kv : h->tuned_r)
    ok = ok && std::fprintf(f, "r %lld %lld %lld %lld %d\n", (long long)kv.first[0],
                            (long long)kv.first[1], (long long)kv.first[2], (long long)kv.first[3],
                            kv.second) > 0;
  for (const auto& kv : h->tuner.choice)
    ok = ok && std::fprintf(f, "g %d %d %d %d %d %d %d\n", kv.first[0], kv.first[1], kv.first[2],
                            kv.first[3], kv.first[4], kv.first[5], kv.second) > 0;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? 0 : ZOLO_EIO;
}

int zolo_tune_load(zolo_handle_t h, const char* path) {
  if (!h) return -1;
  if (!path) return -2;
  FILE* f = std::fopen(path, "r");
  if (!f) return ZOLO_EIO;
  char magic[32] = {0}, dev[256] = {0};
  int version = 0;
  int rc = 0;
  if (std::fscanf(f, "%31s %d %255s", magic, &version, dev) != 3 ||
      std::strcmp(magic, "zolo-tune") != 0 || version != 2 || device_tag(h->device) != dev) {
    rc = ZOLO_EINVAL;
  }
  std::map<std::array<int64_t, 4>, int> got_r;
  std::map<std::array<int, 7>, int> got_g;
  while (rc == 0) {
    char tag[4] = {0};
    const int t = std::fscanf(f, "%3s", tag);
    if (t == EOF) break;
    if (t != 1) {
      rc = ZOLO_EINVAL;
    } else if (std::strcmp(tag, "r") == 0) {
      long long a, b, c, d;
      int r;
      if (std::fscanf(f, "%lld %lld %lld %lld %d", &a, &b, &c, &d, &r) != 5 || r < 1 ||
          r > kMaxR || a < 1 || b < 1 || a < b || (c != ZOLO_FP64 && !is_split((int)c)) ||
          d < 0 || d > 400)
        rc = ZOLO_EINVAL;
      else
        got_r[{a, b, c, d}] = r;
    } else if (std::strcmp(tag, "g") == 0) {
      int k[6], v;
      if (std::fscanf(f, "%d %d %d %d %d %d %d", &k[0], &k[1], &k[2], &k[3], &k[4], &k[5], &v) !=
              7 ||
          k[0] < 1 || k[1] < 1 || k[2] < 1 || k[3] < 1 || k[3] > kGemmMaxBatch || k[4] < 0 ||
          k[4] > 255 || (k[5] != 0 && k[5] != 8 && k[5] != 9 && k[5] != 108 && k[5] != 211) ||
          !gemm_variant_allowed({k[0], k[1], k[2], k[3], k[4], k[5], 0}, v))
        rc = ZOLO_EINVAL;
      else
        got_g[{k[0], k[1], k[2], k[3], k[4], k[5], 0}] = v;
    } else {
      rc = ZOLO_EINVAL;
    }
  }
  std::fclose(f);
  if (rc) return rc;
  for (const auto& kv : got_r) h->tuned_r[kv.first] = kv.second;
  for (const auto& kv : got_g) h->tuner.choice[kv.first] = kv.second;
  if (!got_g.empty()) ++h->tuner.gen;
  return 0;
}

const char* zolo_strerror(int code) {
  switch (code) {
    case ZOLO_OK: return "success";
    case ZOLO_ENONFINITE: return "NaN or Inf in the input or an iterate";
    case ZOLO_ECHOL: return "Cholesky breakdown";
    case ZOLO_ENOTCONV: return "a-posteriori test failed at max_iter";
    case ZOLO_ECUDA: return "CUDA runtime error";
    case ZOLO_ENOMEM: return "device memory allocation failed";
    case ZOLO_EEIG: return "Jacobi eigensolver did not converge";
    case ZOLO_ETIMEOUT: return "a bounded device wait expired (tensor-core pipeline)";
    case ZOLO_EIO: return "tuning-cache file could not be written or read";
    case ZOLO_EINVAL: return "tuning-cache file malformed or written on another GPU";
    case ZOLO_ECOMM: return "the caller's sum over ranks reported a failure";
    case ZOLO_EPENDING: return "the asynchronous call has not completed";
    case ZOLO_EGUARD: return "a kernel wrote outside its workspace buffer (guard zone changed)";
    default: return code < 0 ? "illegal argument" : "unknown error";
  }
}

}  // extern "C"
