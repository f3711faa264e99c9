// Internal declarations shared by the libzolo translation units.
#pragma once

#include <array>
#include <cstddef>
#include <cstdint>
#include <map>

#ifdef __CUDACC__
#include <cuda_runtime.h>
#else
typedef struct CUstream_st* cudaStream_t;
#endif

namespace zolo {

constexpr int kMaxR = 8;
constexpr int kMaxIters = 8;
constexpr double kTable1Tol = 1e-15;

// ---------------------------------------------------------------- coefficients
struct Coefficients {
  double ell = 0.0;
  int r = 0;
  double c[2 * kMaxR] = {};   // c_1 .. c_{2r}
  double a[kMaxR] = {};       // a_1 .. a_r
  double mhat = 0.0;          // M_hat
  double gap = 0.0;           // 1 - Zhat(l; l)
};

struct Schedule {
  int r = 0;
  int iters = 0;
  bool converged = false;
  double ell[kMaxIters + 1] = {};
  bool use_qr[kMaxIters] = {};
  Coefficients co[kMaxIters];
};

int compute_coefficients(double ell, int r, Coefficients* out);
bool qr_form_needed(const Coefficients& co);
int build_schedule(double ell0, int r, int max_iter, Schedule* out);

#ifdef __CUDACC__

// ------------------------------------------------------------- launch scopes
enum ProfClass { kProfGemm = 0, kProfPanel, kProfCholDiag, kProfJacobi, kProfCombine, kProfOther,
                 kProfSplitGemm, kProfSlice, kProfJacobi32, kProfClasses };
// Counts the launch made inside its scope and, while profiling is on, brackets
// it with CUDA events on `st`.  flops/bytes: the launch's algorithmic work.
class ProfScope {
 public:
  ProfScope(int cls, cudaStream_t st, double flops = 0.0, double bytes = 0.0);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;
  // The launch's blocks, for its SM-time: blocks / (SMs x blocks per SM of
  // `kernel` at this block size and dynamic shared memory), at most 1.  Only
  // queried while profiling is on.
  void blocks(const void* kernel, dim3 block, size_t smem, dim3 grid);

 private:
  int cls_;
  cudaStream_t st_;
  double flops_, bytes_;
  double share_ = 1.0;
  void* a_ = nullptr;
};

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) applies to the current device
// only: set it once per (kernel, device), thread-safely.
cudaError_t smem_attr_once(const void* func, int bytes);

// Launch bookkeeping for graphs: kernels recorded at capture time are counted
// when the graph is launched.
void add_launches(int64_t n);
bool profiling_enabled();

// ----------------------------------------------------------------- device flags
// A small device array of int counters written by kernels and read once at the
// end of a call.
enum StatusSlot {
  kStatNonFinite = 0,   // a NaN/Inf was produced
  kStatCholFail = 1,    // non-positive pivot in a Cholesky diagonal block
  kStatJacobiRot = 2,   // rotations applied in the current Jacobi sweep
  kStatJacobiMaxCos = 3,  // largest |cos| between two columns seen in the sweep (float bits)
  kStatSlots = 4
};

// ------------------------------------------------------------------- FP64 GEMM
// C_out[b] = beta * C_in[b] + alpha[b] * op(A[b]) op(B[b])          (reduce = 0)
// C_out    = beta * C_in    + sum_b alpha[b] * op(A[b]) op(B[b])    (reduce = 1)
// Column-major, op = N or T.  Structural flags let the kernel skip known zeros:
//   b_lower  : op(B)[k][j] == 0 for k < j (e.g. op(B) = Q2^T with Q2 upper)
//   c_upper  : only tiles touching the upper triangle (i <= j) are computed
constexpr int kGemmMaxBatch = 16;
struct GemmArgs {
  int M = 0, N = 0, K = 0;
  int transA = 0, transB = 0;
  const double* A = nullptr; int64_t lda = 0; int64_t strideA = 0;
  const double* B = nullptr; int64_t ldb = 0; int64_t strideB = 0;
  const double* Cin = nullptr; int64_t ldcin = 0; int64_t strideCin = 0;
  double* Cout = nullptr; int64_t ldcout = 0; int64_t strideCout = 0;
  double beta = 0.0;
  double alpha[kGemmMaxBatch] = {};
  int batch = 1;
  int reduce = 0;
  int b_lower = 0;
  int c_upper = 0;
  // split path only: rescale the inner index by exact powers of two so that every
  // row of op(B) has its largest magnitude in [1/4, 1/2), moving the factors into
  // op(A)'s columns (the product is unchanged).  For products whose op(B) rows
  // differ by orders of magnitude, where one scale per output column would cost
  // the small rows their precision.
  int k_equilibrate = 0;
};
// Kernel variants of the FP64 contraction: output tile shape, and split-K
// (K cut into 2 / 4 / 8 slices of whole BK steps whose raw sums go to a scratch
// of ksplit * (reduce ? 1 : batch) * M * N doubles, then one deterministic
// reduction kernel).  kGemmVSplit names the split tensor-core path.
enum GemmVariant {
  kGemmV64x64 = 0, kGemmV32x128 = 1, kGemmV32x64 = 2,
  kGemmVSplitK2 = 3, kGemmVSplitK4 = 4, kGemmVSplitK8 = 5,
  kGemmVSplit = 8
};
// one FP64 launch of the given variant (a split-K variant without enough
// scratch runs as kGemmV64x64)
cudaError_t gemm_f64_variant(const GemmArgs& g, int variant, double* scratch,
                             size_t scratch_elems, cudaStream_t st);
size_t gemm_f64_scratch_elems(const GemmArgs& g, int variant);
int gemm_f64_default_variant(const GemmArgs& g);
// FP64 contraction: the variant the current thread's tuner chose for this
// shape, else the default one.
cudaError_t gemm_f64(const GemmArgs& g, cudaStream_t st);

// Measured kernel choice per contraction shape (sizes, batch, transposes,
// structure flags, slice count): the cache of a handle, made current for the
// calls of one API entry point by TunerScope.  With `tuning` set, a shape met
// for the first time is run with every candidate variant into a scratch output
// (the real output untouched) and timed with CUDA events; the fastest is kept.
// No tuning while the stream is being captured.
struct GemmTuner {
  std::map<std::array<int, 7>, int> choice;
  uint64_t gen = 0;      // bumped whenever `choice` changes (graph replay keys)
  bool tuning = false;
  bool busy = false;
  double* scratch = nullptr;
  size_t scratch_elems = 0;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  ~GemmTuner();
};
std::array<int, 7> gemm_key(const GemmArgs& g, int split_slices);
// C's elements overlap those of A or B (flag 128 of the key)
bool gemm_output_aliases_input(const GemmArgs& g);
// whether kernel v may serve a key (tile variants other than the built-in one
// are barred for in-place products: their CTAs would overwrite rows of B that
// other CTAs still read)
bool gemm_variant_allowed(const std::array<int, 7>& key, int v);
void set_gemm_tuner(GemmTuner* t);
GemmTuner* get_gemm_tuner();
struct TunerScope {
  GemmTuner* prev;
  explicit TunerScope(GemmTuner* t) : prev(get_gemm_tuner()) { set_gemm_tuner(t); }
  ~TunerScope() { set_gemm_tuner(prev); }
};
// algorithmic flops of one call (structural zeros excluded)
double gemm_flops(const GemmArgs& g);

// --------------------------------------------------- split-precision GEMM
// Same contract as gemm_f64 (c_upper / b_lower are computed in full), on the
// tensor cores with the operands cut into S slices of one of three forms.
enum : int {
  kFormBF16 = 0,   // S = 8 or 9 pre-scaled base-64 digits in BF16
  kFormFP16 = 1,   // S = 8 raw base-128 digits in FP16
  kFormFP8 = 2     // S = 11 raw base-32 digits in E4M3
};
struct SplitWork {
  void* slices;          // slice planes
  size_t slice_elems;    // their size in 16-bit units
  int* exps;             // per-row / per-column power-of-two exponents
  size_t exp_elems;
  int* err;              // device error flag (bounded waits)
  int slices_s;          // S
  int form = kFormBF16;
  // test hook of the failure path: with stall = 1 the MMA issuer first waits,
  // for stall_ns, on an mbarrier that nothing arrives at, then takes the
  // bounded-wait error exit
  int stall = 0;
  long long stall_ns = 0;
  // the router's cost model: false = one call alone on the GPU (its launch and
  // pipeline latency counts); true = many calls in flight at once (zolo_pd_batched's
  // lanes), where latency is hidden and each path costs the share of the GPU's
  // FP64 pipe, tensor pipe and memory bandwidth it takes
  bool throughput = false;
};
cudaError_t gemm_split(const GemmArgs& g, SplitWork& w, cudaStream_t st);
// slice planes (16-bit units) one call of the given shape needs in a form
size_t split_slice_elems(int64_t M, int64_t N, int64_t K, int batch, int S, int form = kFormBF16);
// exponent entries (ints) one call of the given shape needs
size_t split_exp_elems(int64_t M, int64_t N, int64_t K, int batch, int k_equilibrate,
                       int form = kFormBF16);
// The engine every contraction of the current call goes through: FP64 (DFMA)
// when no split workspace is installed, the split tensor-core path otherwise.
void set_split_engine(SplitWork* w);
SplitWork* get_split_engine();
// the built-in router: true when the split path's estimated time (slicing and
// output traffic, slice-pair products, launch latency) beats the FP64 pipe's
bool split_preferred(const GemmArgs& g, const SplitWork& w);
// the same estimate as a ratio: split-path time / FP64 time
double split_time_ratio(const GemmArgs& g, const SplitWork& w);
// Sets the kernels' launch attributes ahead of a stream capture.
void split_prepare();
cudaError_t gemm_any(const GemmArgs& g, cudaStream_t st);

// --------------------------------------------------------------- elementwise
cudaError_t scale_copy(const double* A, int64_t lda, double* X, int64_t ldx, int64_t m, int64_t n,
                       double s, cudaStream_t st);
cudaError_t copy_matrix(const double* A, int64_t lda, double* B, int64_t ldb, int64_t m, int64_t n,
                        cudaStream_t st);
// W_j = [X; sqrt(c_j) I] for j < r, W_j at W + j*strideW with ld = m + n
cudaError_t init_stacked(const double* X, int64_t ldx, double* W, int64_t strideW, int64_t m,
                         int64_t n, const double* sqrt_c, int r, cudaStream_t st);
// Q_j = [I_n; 0] ((m+n) x n, ld m+n) for j < r
cudaError_t init_q_identity(double* Q, int64_t strideQ, int64_t m, int64_t n, int r,
                            cudaStream_t st);
// Z_j = G + shift_j I for j < r (full copy of G, n x n, ld n)
cudaError_t init_shifted(const double* G, double* Z, int64_t strideZ, int64_t n, const double* shift,
                         int r, cudaStream_t st);
// Xn = mhat * (X + sum_j coef_j * T_j) (T_j at T + j*strideT, ld ldt; nt may be 0),
// partial sums of ||Xn - X||^2 and ||Xn||^2 to norms[0..1] (after norms_finish).
cudaError_t combine(const double* X, int64_t ldx, double* Xn, int64_t ldxn, int64_t m, int64_t n,
                    double mhat, const double* T, int64_t ldt, int64_t strideT, const double* coef,
                    int nt, double* partials, double* norms, int* status, cudaStream_t st);
// S = sum_t coef_t T_t, T_t at T + t * strideT (ld ldt), t < nt <= 8
cudaError_t weighted_sum(const double* T, int64_t ldt, int64_t strideT, const double* coef, int nt,
                         double* S, int64_t lds, int64_t m, int64_t n, cudaStream_t st);
// guard zones: fill with 0xFF bytes; set *flag if any byte differs
cudaError_t guard_fill(void* p, size_t bytes, cudaStream_t st);
cudaError_t guard_check(const void* p, size_t bytes, int* flag, cudaStream_t st);
// *out = (*flag != 0) as a double
cudaError_t flag_to_double(const int* flag, double* out, cudaStream_t st);
// H = (M + M^T) / 2
// W(i, j) = W(j, i) for i > j (n x n, ld ldw): a symmetric W from its upper triangle
cudaError_t mirror_upper(double* W, int64_t ldw, int64_t n, cudaStream_t st);
cudaError_t symmetrize(const double* M, int64_t ldm, double* H, int64_t ldh, int64_t n,
                       cudaStream_t st);
cudaError_t check_finite(const double* A, int64_t lda, int64_t m, int64_t n, int* status,
                         cudaStream_t st);
// ||G - I||_F^2 into out[0] from the upper triangle of a symmetric n x n G
// (out[1] = 0)
cudaError_t gram_identity_dev2(const double* G, int64_t ldg, int64_t n, double* partials,
                               double* out, cudaStream_t st);
// ||A||_F^2 into out[0] (via partials)
cudaError_t frob_norm2(const double* A, int64_t lda, int64_t m, int64_t n, double* partials,
                       double* out, cudaStream_t st);
// alpha >= sigma_max(A) when the caller gives none: sums[0] = ||A||_F^2, sums[1] =
// ||A||_1, sums[2] = ||A||_inf (sums: 3 device doubles, written by
// alpha_bound_sums; part: alpha_bound_part_elems(m, n) doubles, colsum: n,
// partials: 2 * 1024), then alpha_from_sums = min(||A||_F, sqrt(||A||_1 ||A||_inf))
// on the host.
int64_t alpha_bound_part_elems(int64_t m, int64_t n);
cudaError_t alpha_bound_sums(const double* A, int64_t lda, int64_t m, int64_t n, double* part,
                             double* colsum, double* partials, double* sums, cudaStream_t st);
double alpha_from_sums(const double* sums);

// ------------------------------------------------------------ structured QR
constexpr int kQrNB = 32;      // panel width (columns factored by one panel kernel)
constexpr int kQrBlock = 128;  // block width (columns per trailing update / block reflector)
struct QrBuffers {
  double* W;   int64_t strideW;   // stacked (m+n) x n per shift, ld m+n
  double* V;   int64_t strideV;   // explicit reflectors (m+NBb) x n per shift, ld m+NBb, rows
                                  // relative to the start of each column's block
  double* T;   int64_t strideT;   // nb x nb triangular factor per panel
  double* Tb;  int64_t strideTb;  // NBb x NBb triangular factor per block
  double* G;   int64_t strideG;   // NBb x NBb Gram V_b^T V_b scratch
  double* P;   int64_t elemsP;    // split-K partial products of the skinny products
  double* W1;  int64_t strideW1;  // NBb x n scratch
  double* W2;  int64_t strideW2;  // NBb x n scratch
};
// Doubles of QrBuffers::P for an m-row problem with r shifts.
int64_t qr_partial_elems(int64_t m, int r);
// Factor [X; sqrt(c_j) I] for j < r and overwrite W_j with the thin Q_j
// (explicit_q = false: leave R on and above the diagonal of W_j's top block).
// narrow_panels: many problems are in flight on other streams; the panel kernel
// then takes the fewest CTAs per shift whose rows fit in shared memory.
cudaError_t structured_qr_q(const QrBuffers& b, int64_t m, int64_t n, int r, int* status,
                            cudaStream_t st, bool explicit_q = true, bool narrow_panels = false);
// Inverses of the NB x NB diagonal blocks of an upper-triangular R (ld n) in the
// layout cholesky_upper_batched leaves in Rinv; a zero pivot sets status.
cudaError_t tri_inv_diag_blocks(const double* R, int64_t n, double* Rinv, int* status,
                                cudaStream_t st);

// ----------------------------------------------------------------- Cholesky
constexpr int kCholNB = 64;
struct CholBuffers {
  double* Z;    int64_t strideZ;     // n x n, ld n: in = Z_j (upper), out = R_j (upper)
  double* Rinv; int64_t strideRinv;  // inverses of the nb x nb diagonal blocks, nb x nb each
};
cudaError_t cholesky_upper_batched(const CholBuffers& b, int64_t n, int r, int* status,
                                   cudaStream_t st);
// Y_j = X R_j^{-1} then Y_j <- Y_j R_j^{-T} (in place), j < r.
cudaError_t trsm_pair_batched(const double* X, int64_t ldx, const CholBuffers& b, double* Y,
                              int64_t strideY, double* tmp, int64_t strideTmp, int64_t m,
                              int64_t n, int r, cudaStream_t st);

// ------------------------------------------------------------ eigensolver
struct EigWork {
  double* R;        // n x n
  double* X;        // n x n, one-sided Jacobi iterate
  double* HV;       // n x n
  double* Rinv;     // (n/nb+1) * nb * nb
  double* lam;      // n
  int* perm;        // n (device)
  int* status;
  float* X32;       // n x n, FP32 sweeps
  float* Z32;       // n x n, accumulated FP32 rotations
  double* Z;        // n x n, Z orthonormalised in FP64
  double* tmp;      // n x 64 scratch of the triangular solve
  unsigned* bar;    // grid-barrier words (2)
  int* ver;         // n + 1 per-column round counters of the FP64 sweeps
  int* err;         // bounded-wait error flag
  // test hook of the failure path: with stall = 1, block 0 of the first FP32
  // sweep waits, for stall_ns, on a flag nothing sets, then takes the
  // bounded-wait error exit (the other blocks leave the grid barrier on the flag)
  int stall = 0;
  // the same for the first FP64 sweep: block 0 waits on a flag nothing sets, the
  // blocks whose work items need its columns leave on the error flag
  int stall64 = 0;
  long long stall_ns = 0;
};
// Y <- X R^{-1} for upper R with inverted diagonal blocks (cholesky_upper_batched output)
cudaError_t trsm_right_upper_batched(const double* X, int64_t ldx, const CholBuffers& b, double* Y,
                                     int64_t strideY, double* tmp, int64_t strideTmp, int64_t m,
                                     int64_t n, int r, cudaStream_t st);
int eig_sym_jacobi(const double* H, int64_t ldh, int64_t n, double* V, int64_t ldv, double* lam_out,
                   const EigWork& w, int* sweeps, cudaStream_t st);
cudaError_t column_norms(const double* X, int64_t ldx, int64_t m, int64_t n, double* out,
                         cudaStream_t st);
cudaError_t scale_columns(double* X, int64_t ldx, int64_t m, int64_t n, const double* s, int invert,
                          cudaStream_t st);
cudaError_t column_dots(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t m,
                        int64_t n, double* out, cudaStream_t st);
cudaError_t gather_columns(const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t m,
                           int64_t n, const int* perm, const double* sign, cudaStream_t st);
cudaError_t transpose_lower(const double* R, int64_t ldr, double* X, int64_t ldx, int64_t n,
                            cudaStream_t st);
// One FP64 sweep of the one-sided Jacobi rounds (a cooperative launch; ver holds
// n_even round counters, err the bounded waits' flag).
cudaError_t jacobi_sweep(double* X, int64_t ldx, int64_t m, int64_t n_even, int64_t n_real,
                         double tol, int* status, double* nrm2, double* dsc, int* ver, int* err,
                         int stall, long long stall_ns, cudaStream_t st);

#endif  // __CUDACC__

}  // namespace zolo
