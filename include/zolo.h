/*
 * libzolo: Zolo-PD polar decomposition and Zolo-SVD on one NVIDIA GB300 (sm_103a).
 *
 * Method: Li, Liu, Du, "A new high performance and scalable SVD algorithm on
 * distributed memory systems" (arxiv 1806.06204), after Nakatsukasa & Freund.
 *
 *   A = Qp H         polar decomposition (Eq. 1), Qp m x n with orthonormal
 *                    columns, H n x n symmetric positive semidefinite;
 *   A = U diag(S) V^T  SVD from H = V diag(S) V^T and U = Qp V (Algorithm 2).
 *
 * Every matrix is real FP64, column-major with a leading dimension (LAPACK
 * convention), m >= n >= 1.  Unless an entry point says "host", every matrix
 * pointer is a DEVICE pointer on the handle's device, owned by the caller.
 * Calls are ordered on the given CUDA stream (a cudaStream_t passed as void*,
 * NULL = the legacy default stream) and return after one final stream
 * synchronisation that reads the status into `info`.
 *
 * Return codes: 0 on success; -i if argument i (1-based) is illegal, LAPACK
 * style, before any work is queued; a positive ZOLO_E* code otherwise.
 */
#ifndef ZOLO_H_
#define ZOLO_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ZOLO_MAX_R 8
#define ZOLO_MAX_ITERS 8
#define ZOLO_R_TUNED (-1)

enum {
  ZOLO_OK = 0,
  ZOLO_ENONFINITE = 1, /* NaN or Inf in the input or an iterate                */
  ZOLO_ECHOL = 2,      /* Cholesky breakdown (non-positive pivot)               */
  ZOLO_ENOTCONV = 3,   /* a-posteriori test still failing after max_iter        */
  ZOLO_ECUDA = 4,      /* a CUDA runtime call failed                            */
  ZOLO_ENOMEM = 5,     /* workspace too small / device allocation failed        */
  ZOLO_EEIG = 6,       /* the Jacobi eigensolver did not converge               */
  ZOLO_ETIMEOUT = 7,   /* a bounded device wait expired (split GEMM pipeline,
                          Jacobi grid barrier or column-pair wait)              */
  ZOLO_EIO = 8,        /* a tuning-cache file could not be written or read      */
  ZOLO_EINVAL = 9,     /* a tuning-cache file is malformed or from another GPU  */
  ZOLO_ECOMM = 10,     /* the caller's sum over ranks (zolo_pd_sharded) failed  */
  ZOLO_EPENDING = 11,  /* zolo_pd_async: the stream has not reached the end yet */
  ZOLO_EGUARD = 12     /* zolo_debug_guards: a kernel wrote outside its buffer  */
};

/* Arithmetic of the contractions.  ZOLO_FP64: plain FP64 on the FP64 FMA pipe.
   ZOLO_SPLIT_BF16: the iterations' products on the BF16 tensor cores, each FP64
   operand cut into 9 power-of-two-scaled 6-bit slices (Ozaki scheme, product
   error a few times sqrt(k) 2^-54 of max|row| max|column|); panel
   factorisations, diagonal blocks and coefficients stay FP64.
   ZOLO_SPLIT_FP16: the same on the FP16 tensor cores with 8 slices of 7-bit
   integer digits and 36 slice-pair products instead of 53 (the same error
   grade).
   ZOLO_SPLIT_FP8: the same on the FP8 (E4M3) tensor cores with 11 slices of
   5-bit integer digits and 76 slice-pair products at twice the BF16 rate
   (the same error grade).  A product whose inner dimension is longer than
   the int64 of its exact level sums can hold at the digit bounds (114688 for
   BF16 and FP8, 61440 for FP16) runs as consecutive products added in FP64. */
enum { ZOLO_FP64 = 0, ZOLO_SPLIT_BF16 = 1, ZOLO_SPLIT_FP16 = 2, ZOLO_SPLIT_FP8 = 3 };

typedef struct {
  int r;           /* order parameter, 1..8 (Eq. 6: type (2r+1, 2r)); 0 = the
                      smallest r needing at most two iterations (Table 1);
                      ZOLO_R_TUNED = the r measured fastest on this GPU for
                      (m, n, prec, l_0 to the nearest decade), see
                      zolo_tuned_r                                             */
  double alpha;    /* alpha >= sigma_max(A) (Algorithm 1 step 1); <= 0: use
                      min(||A||_F, sqrt(||A||_1 ||A||_inf)), an upper bound
                      (one pass over A)                                        */
  double beta;     /* 0 < beta <= sigma_min(A) (step 2); l_0 = beta / alpha.
                      <= 0: estimated on the device (not in the paper, which
                      assumes it known): beta = alpha / ||R^{-1}||_F with R from
                      a Householder QR of A / alpha, a lower bound of
                      sigma_min(A) (||R^{-1}||_F >= ||R^{-1}||_2) within a
                      factor sqrt(n); about 2mn^2 + n^3 more flops (in
                      zolo_pd_batched: matrix after matrix, before the
                      batch starts)                                           */
  int max_iter;    /* cap on iterations, 1..8 (default 6)                    */
  int posteriori;  /* 1: after the a-priori iterations, apply the test of
                      Algorithm 1 step (d) literally and iterate while
                      ||X_{k+1}-X_k||_F/||X_{k+1}||_F > eps^(1/(2r+1))        */
  int ns_steps;    /* Newton-Schulz steps X <- 1.5X - 0.5X(X^T X) after the
                      iteration (not in the paper), 0..4                      */
  int prec;        /* ZOLO_FP64, ZOLO_SPLIT_BF16, _FP16 or _FP8                */
  int force_qr;    /* -1: QR form while (1+c_1)/(l^2+c_1) > 100, then the
                      Cholesky form; 0: Cholesky form always; 1: QR always     */
  int chol_form;   /* how a Cholesky-form iteration applies the r factors
                      Z_j = R_j^T R_j: 1 = the triangular solves of Algorithm 1
                      (d), T_j = a_j (X R_j^{-1}) R_j^{-T}, 2r solves with m
                      rows; 2 = the explicit inverse (not in the paper):
                      W = sum_j a_j R_j^{-1} R_j^{-T} (n-row solves against I
                      and one batch-reduced product), then X W, one product
                      with m rows; the same rational function of X^T X, with
                      kappa(Z_j) <= 100 on this path.  0 = whichever has fewer
                      modelled flops: the inverse when
                      r (3/2) n^3 + 2 m n^2 < 0.85 * 2 r m n^2 (tall X, large r) */
  int estimate;    /* 1: after H, compute info.bwd_est = ||A - Qp H||_F / ||A||_F
                      and info.orth_est = ||Qp^T Qp - I||_F / sqrt(n) on the
                      device (about 3 m n^2 more flops, in opts.prec's
                      arithmetic); 0 (default): both left 0                   */
} zolo_opts_t;

/* Phases of a call timed into zolo_info_t.ms_phase (CUDA events on the call's
   stream; NVTX ranges of the same names are pushed on the calling thread):
   the bounds alpha, beta and a tuned r; the QR-form iterations (Eq. 12); the
   Cholesky-form iterations (Algorithm 1 (d)); the Newton-Schulz steps; H
   (Algorithm 1 step 5); the error estimates; and for zolo_svd the
   eigendecomposition of H and U = Qp V (Algorithm 2). */
enum {
  ZOLO_PHASE_BOUNDS = 0, ZOLO_PHASE_QR = 1, ZOLO_PHASE_CHOL = 2, ZOLO_PHASE_NS = 3,
  ZOLO_PHASE_H = 4, ZOLO_PHASE_EST = 5, ZOLO_PHASE_EIG = 6, ZOLO_PHASE_U = 7, ZOLO_PHASES = 8
};

typedef struct {
  int status;                  /* the return code of the call                */
  int iters;                   /* iterations run                             */
  int r;                       /* order parameter used                       */
  int used_qr[ZOLO_MAX_ITERS]; /* 1 if iteration k used the QR form (Eq. 12) */
  double ell[ZOLO_MAX_ITERS + 1];   /* l_0, l_1, ... (Algorithm 1 step (c))  */
  double delta[ZOLO_MAX_ITERS];     /* ||X_{k+1}-X_k||_F / ||X_{k+1}||_F      */
  int chol_fallbacks;          /* Cholesky-form iterations redone in the QR
                                  form after a non-positive pivot             */
  int eig_sweeps;              /* Jacobi sweeps (zolo_svd only)              */
  double ms;                   /* device time of the call (CUDA events)      */
  int chol_form;               /* the Cholesky form the call would take (1 =
                                  triangular solves, 2 = explicit inverse; see
                                  zolo_opts_t.chol_form)                     */
  double bwd_est;              /* ||A - Qp H||_F / ||A||_F   (opts.estimate)  */
  double orth_est;             /* ||Qp^T Qp - I||_F / sqrt(n) (opts.estimate) */
  float ms_phase[ZOLO_PHASES]; /* device time per phase (zolo_pd, zolo_svd,
                                  zolo_pd_sharded; 0 in zolo_pd_batched and
                                  zolo_pd_async)                              */
} zolo_info_t;

typedef struct zolo_handle_s* zolo_handle_t;

/* Defaults: r = 0, alpha = 1, beta = 0 (estimated), max_iter = 6,
   posteriori = 0, ns_steps = 0, prec = ZOLO_FP64, force_qr = -1,
   chol_form = 0, estimate = 0. */
void zolo_opts_default(zolo_opts_t* opts);

/* A handle binds a device and owns the library's workspace cache.
   zolo_create makes `device` current; -1 = the current device. */
int zolo_create(zolo_handle_t* handle, int device);
int zolo_destroy(zolo_handle_t handle);

/* Zolotarev coefficients for l in (0, 1], r in 1..8 (host, no GPU work):
   c[0..2r-1] = c_1..c_2r of Eq. (7), a[0..r-1] = a_1..a_r of Eq. (10) read as
   the partial-fraction residue (quotient of the two products), *Mhat = M_hat
   of Eq. (8), *gap = 1 - Zhat(l; l) (the next l is 1 - gap, Algorithm 1
   step (c)).  Any output pointer may be NULL.  Returns 0 or -1/-2. */
int zolo_coefficients(double ell, int r, double* c, double* a, double* Mhat, double* gap);

/* A-priori schedule (Table 1): l_0 = ell0 and l_{k+1} = Zhat(l_k; l_k) until
   1 - l_K <= 1e-15 or K = max_iter.  Writes ells[0..K] and used_qr[0..K-1]
   (QR form while (1+c_1)/(l_k^2+c_1) > 100) and returns K >= 0, or < 0 on
   illegal arguments.  r = 0 selects r as zolo_opts_t does (ZOLO_R_TUNED is
   illegal here: a measured r belongs to a handle, see zolo_tuned_r); *r_used
   receives the r taken (may be NULL). */
int zolo_schedule(double ell0, int r, int max_iter, double* ells, int* used_qr, int* r_used);

/* Device memory a zolo_pd (svd = 0) or zolo_svd (svd = 1) call on an m x n
   matrix keeps in its handle (host computation, no GPU work): the workspace
   for r shifts (r <= 0: for up to 8) plus, for a split precision, the slice
   planes and exponents, as the call allocates them (the planes are capped at
   16 GB; a smaller allocation is tried when that fails).  Not counted: the
   host entry points' staging copies of A and the results, and the tuner's
   scratch (zolo_autotune).  Returns 0 and writes *bytes, or -i for an illegal
   argument i (m < n, n < 1, r outside -1..8, prec, svd not 0/1, NULL). */
int zolo_workspace_bytes(int64_t m, int64_t n, int r, int prec, int svd, uint64_t* bytes);

/* Polar decomposition A = Qp H (Algorithm 1).
   A (m x n, lda >= m) is read only; Qp (m x n, ldq >= m) and H (n x n,
   ldh >= n) are written.  H is exactly symmetric. */
int zolo_pd(zolo_handle_t handle, const double* A, int64_t m, int64_t n, int64_t lda,
            double* Qp, int64_t ldq, double* H, int64_t ldh,
            const zolo_opts_t* opts, zolo_info_t* info, void* stream);

/* zolo_pd without any host synchronisation: the whole decomposition is queued
   on `stream` and the call returns at once with info->status = ZOLO_EPENDING;
   when the stream reaches the end of the queued work a host function
   (cudaLaunchHostFunc) fills *info (status, iterations, l's, deltas, the
   estimates), so *info must stay valid until then (synchronise the stream or
   an event recorded after the call before reading it; pinned or pageable host
   memory).  Needs opts.alpha > 0 and opts.beta > 0 (bounds computed on the
   device need a round trip), opts.r != ZOLO_R_TUNED and opts.posteriori = 0
   (-10 otherwise).  No Cholesky fallback can be taken without a round trip: a
   breakdown is reported as ZOLO_ECHOL in info->status (force_qr = 1 avoids
   it).  Workspace growth may allocate (cudaMalloc) on the first call of a
   shape.  Consecutive calls on one handle must use one stream (they share the
   handle's workspace); up to 64 calls may be in flight. */
int zolo_pd_async(zolo_handle_t handle, const double* A, int64_t m, int64_t n, int64_t lda,
                  double* Qp, int64_t ldq, double* H, int64_t ldh,
                  const zolo_opts_t* opts, zolo_info_t* info, void* stream);

/* SVD A = U diag(S) V^T (Algorithm 2): Zolo-PD, the eigendecomposition of H
   (one-sided block Jacobi on its Cholesky factor), U = Qp V.
   U is m x n (ldu >= m), S has n entries (descending, >= 0), V is n x n
   (ldv >= n).  All three are device pointers. */
int zolo_svd(zolo_handle_t handle, const double* A, int64_t m, int64_t n, int64_t lda,
             double* U, int64_t ldu, double* S, double* V, int64_t ldv,
             const zolo_opts_t* opts, zolo_info_t* info, void* stream);

/* ---- Shifts sharded over ranks (Section 3.2, Algorithm 3): the paper splits
   the processes into r groups, group j factors the j-th shifted problem and
   DGSUM2D sums the r terms T_j.  Here each of `nranks` ranks (one per GPU,
   each holding all of A) takes the contiguous block of the r shifts that
   zolo_shift_range gives it, forms the sum S_rank of its own T_j for every
   iteration, and hands S_rank to the caller's `sum` function, which must
   replace it by the elementwise sum over all ranks (an all-reduce, e.g. NCCL
   or torch.distributed); X_{k+1} = M_hat (X_k + S) then follows on every rank
   alike, as do the Newton-Schulz steps and H.

   zolo_shift_range: shifts [*j0, *j1) (0-based, j1 - j0 of them, possibly
   none when nranks > r) of rank `rank`: consecutive blocks, the first r mod
   nranks ranks one larger.  Host only.  Returns 0 or -i for argument i.

   zolo_sum_fn: called once per iteration (more after a Cholesky breakdown)
   with buf = a device array of `count` = m n + 1 doubles on the handle's
   device (S, column-major, ld m, then this rank's Cholesky-breakdown flag as
   0.0 / 1.0) and the call's stream; it must leave in buf, for work queued on
   that stream after it returns, the elementwise sum of every rank's buf (the
   same order of summation on every rank, so that all ranks continue with
   identical bits), and return 0; anything else makes the call return
   ZOLO_ECOMM.  A non-zero summed flag makes every rank redo that iteration in
   the QR form.

   zolo_pd_sharded: as zolo_pd, with every rank passing the same A (bitwise),
   opts and nranks; opts.r must not be ZOLO_R_TUNED and opts.posteriori must be
   0 (-10 otherwise).  rank (argument 13) in [0, nranks), nranks (14) >= 1,
   sum (15) may be NULL only when nranks = 1, ctx is passed to sum untouched.
   Every rank writes the same Qp and H. */
typedef int (*zolo_sum_fn)(double* buf, int64_t count, void* stream, void* ctx);
int zolo_shift_range(int r, int rank, int nranks, int* j0, int* j1);
int zolo_pd_sharded(zolo_handle_t handle, const double* A, int64_t m, int64_t n, int64_t lda,
                    double* Qp, int64_t ldq, double* H, int64_t ldh, const zolo_opts_t* opts,
                    zolo_info_t* info, void* stream, int rank, int nranks, zolo_sum_fn sum,
                    void* ctx);

/* Many polar decompositions in one call.  Matrix i is A[i] (m[i] x n[i],
   leading dimension lda[i]) with its own options opts[i] (its own r, bounds,
   precision); results go to Qp[i] (ldq[i]) and H[i] (ldh[i]), and info[i].
   The pointer and size arrays are HOST arrays of `count` entries; the matrix
   pointers are device pointers.  Every matrix's iterations are queued without
   host round trips on the handle's internal streams (forked from and joined
   back to `stream`), so small matrices of different sizes run concurrently;
   the whole batch is recorded as one CUDA graph and the graph is replayed when
   the same batch (pointers, sizes, options) is decomposed again.  A Cholesky
   breakdown found at the end is redone for that matrix on the single-matrix
   path.  Each matrix's result equals zolo_pd's to rounding (bit for bit below
   512 rows: with many problems in flight the batched call factors a taller
   QR panel on fewer CTAs, which sums its column norms in another order).
   opts[i].posteriori must be 0.  Returns the first non-zero status
   (info[i].status per matrix); -i codes refer to the arguments as in zolo_pd
   with the offending matrix's info[].status set. */
int zolo_pd_batched(zolo_handle_t handle, int count, const double* const* A, const int64_t* m,
                    const int64_t* n, const int64_t* lda, double* const* Qp, const int64_t* ldq,
                    double* const* H, const int64_t* ldh, const zolo_opts_t* opts,
                    zolo_info_t* info, void* stream);

/* zolo_batch_graphs(h, 0): zolo_pd_batched on this handle queues its lanes'
   work directly on every call instead of recording it as a CUDA graph and
   replaying it (for tools that cannot follow a stream capture, such as kernel
   profilers; the same kernels run, one launch each).  1 (the default) records
   and replays.  Returns 0, -1 (NULL handle) or -2 (enable not 0/1). */
int zolo_batch_graphs(zolo_handle_t handle, int enable);

/* As zolo_pd / zolo_svd, but every matrix pointer is a HOST pointer: the call
   copies A to the device, computes, and copies the results back (pageable or
   pinned host memory; pinned is faster).  Device buffers come from the
   handle's cache. */
int zolo_pd_host(zolo_handle_t handle, const double* A, int64_t m, int64_t n, int64_t lda,
                 double* Qp, int64_t ldq, double* H, int64_t ldh,
                 const zolo_opts_t* opts, zolo_info_t* info, void* stream);
int zolo_svd_host(zolo_handle_t handle, const double* A, int64_t m, int64_t n, int64_t lda,
                  double* U, int64_t ldu, double* S, double* V, int64_t ldv,
                  const zolo_opts_t* opts, zolo_info_t* info, void* stream);

/* C = alpha op(A) op(B) + beta C for device FP64 matrices (column-major,
   op = identity or transpose: trans = 0 / 1), the contraction the iterations
   run on.  prec = ZOLO_FP64 (DFMA), ZOLO_SPLIT_BF16 with `slices` = 8 or 9
   (0 = 8) six-bit slices per operand on the tensor cores, ZOLO_SPLIT_FP16
   (`slices` 0 or 8: eight seven-bit slices) or ZOLO_SPLIT_FP8 (`slices` 0 or
   11: eleven five-bit slices).  On the split path an Inf or NaN in a row of
   op(A) or a column of op(B) makes that row or column of the product NaN.
   Not in the paper as
   an interface; it exposes the building block for testing and reuse.
   Synchronises the stream before returning. */
int zolo_dgemm(zolo_handle_t handle, int transA, int transB, int64_t m, int64_t n, int64_t k,
               double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
               double beta, double* C, int64_t ldc, int prec, int slices, void* stream);

/* Allocation-free variant of zolo_dgemm with prec = ZOLO_SPLIT_BF16, for callers
   that cannot allocate device memory where they call it (their memory belongs
   to an external allocator or is reserved up front, or they must not call
   cudaMalloc/cudaFree while they run).  No counterpart in the paper.  It needs
   no handle and allocates nothing: the slice planes, exponents and error flag
   live in a 16 MiB file-scope device array that every GPU loading the library
   holds until the process exits.  Sizes whose slices do not fit are refused
   with ZOLO_ENOMEM before any device work: slices * (ceil128(rows) +
   ceil64(cols)) * ceil64(k) * 2 bytes must stay within 16 MiB - 64.25 KiB
   and ceil128(rows) + ceil64(cols) within 16384 exponents, with
   (rows, cols) = (n, m) when m < 128 and n > m, else (m, n) (so
   m = n = k = 512 fits with 8 slices, 1024 x 1024 x 512 does not, and a tall
   9000 x 8 x 8 product fits).  Every size accepted here runs.  The
   first call on a device looks up the array's device address.  All calls
   share the array: calls that overlap on the GPU race and must be serialised
   by the caller.  Matrices are device
   pointers as in zolo_dgemm; `slices` = 8 or 9 (0 = 8).  Synchronises the
   stream before returning. */
int zolo_dgemm_noalloc(int transA, int transB, int64_t m, int64_t n, int64_t k, double alpha,
                       const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                       double* C, int64_t ldc, int slices, void* stream);

/* ---- r tuned by measurement (not in the paper, whose r follows Table 1:
   there the r shifted problems run on r process groups at once; on one GPU
   they share the chip, so fewer shifts and more iterations can be faster).
   A zolo_pd / zolo_svd call with opts.r = ZOLO_R_TUNED looks up the handle's
   cache under the key (m, n, prec, round(-log10 l_0)); on a miss it runs the
   polar decomposition of its own A once for every r in 1..8 whose a-priori
   schedule converges within max_iter, times each run with CUDA events, stores
   the fastest r and then computes the result with it (so a first call costs
   up to nine decompositions).  zolo_pd_batched uses a cached r for such a
   matrix and the Table 1 rule (r = 0) when there is none.
   zolo_tuned_r returns the cached r for a key, or 0.

   ---- Contraction kernels tuned by measurement.  zolo_autotune(h, 1): from
   then on, every zolo_pd / zolo_svd / zolo_dgemm call on h that meets a
   contraction shape (M, N, K, batch, transposes, triangular-structure flags,
   slice count) for the first time runs it once with each candidate kernel
   (FP64 tiles 64x64, 32x128, 32x64; split-K in 2, 4 or 8 slices with a
   deterministic reduction; the split tensor-core path when opts.prec asks for
   it) into a scratch output, timed with CUDA events, and keeps the fastest
   for that shape; the call's own outputs are written once, by the kept
   kernel.  To bound the cost of measuring, a shape whose built-in kernel takes
   over 50 ms keeps it, and the split path (or FP64) is not timed where the
   cost model puts it 4x behind the other.  zolo_autotune(h, 0) stops measuring; choices already made stay in
   use.  Without choices the built-in rules apply (the split path where its
   cost model predicts a gain, else the 64x64 FP64 tile, 32x128 for M <= 32).
   zolo_pd_batched uses the handle's choices too: with tuning on, it first
   decomposes one matrix of every distinct configuration of the batch (sizes,
   r, iteration forms, options) on the caller's stream, outside any capture,
   while the shapes met are timed; its concurrent lanes then replay the
   choices, each with its own split-K scratch.  There the split-or-FP64 choice
   stays with the batch's throughput cost model (many calls in flight hide
   each call's latency), and only the FP64 kernels of the products it leaves
   on the FP64 pipe are measured.  A tuned kernel may sum in
   another order than the built-in one: results agree to rounding, not bit for
   bit.  Returns 0, -1 (NULL handle) or -2 (enable not 0/1).

   zolo_tune_save / zolo_tune_load write and read both caches as text: a first
   line "zolo-tune 2 <device name>", then "r m n prec decade r" lines and
   "g M N K batch flags slices kernel" lines; loading a file written on a
   device of another name, or any malformed line, returns ZOLO_EINVAL and
   keeps the caches as they were.  Both return 0, -1/-2 for a NULL argument,
   or ZOLO_EIO when the file cannot be written or read. */
int zolo_autotune(zolo_handle_t handle, int enable);
int zolo_tuned_r(zolo_handle_t handle, int64_t m, int64_t n, int prec, double ell0);
int zolo_tune_save(zolo_handle_t handle, const char* path);
int zolo_tune_load(zolo_handle_t handle, const char* path);

/* ---- Test hook of the bounded waits (no counterpart in the paper). --------
   Every wait inside a kernel of this library is bounded: when it gives up it
   sets an error flag, the kernel lets the copies and tensor-core operations it
   has in flight finish (with bounded waits), releases its tensor memory and
   returns, and the call returns ZOLO_ETIMEOUT; the context stays usable.
   zolo_debug_stall makes that path run on purpose, for tests: from then on,
   calls on this handle make the named kernel first wait, for `ns` nanoseconds
   (0 .. 1e9), on a barrier or flag that nothing completes:
     ZOLO_STALL_SPLIT_GEMM: the MMA-issuing thread of every split-precision
       product (opts.prec = ZOLO_SPLIT_BF16, FP16 or FP8, zolo_dgemm's split path),
       on an mbarrier no thread or copy arrives at;
     ZOLO_STALL_JACOBI32: block 0 of the first FP32 sweep of zolo_svd's
       eigensolver, on a flag no thread sets (the other blocks leave the grid
       barrier when they see the error flag);
     ZOLO_STALL_JACOBI64: block 0 of the first FP64 sweep, on a flag no thread
       sets, before its first column pair (the blocks whose pairs wait for that
       pair's columns leave when they see the error flag).
   where = 0 switches it off.  Returns 0, -1 (NULL handle), -2 (where) or -3
   (ns). */
/* zolo_debug_guards(h, 1): a checking mode for the workspace (no counterpart in
   the paper; a substitute for a memory checker).  In zolo_pd, zolo_svd and
   zolo_pd_sharded calls on h, every buffer carved from the handle's workspace
   is followed by a 4 KB guard zone filled with 0xFF bytes (an FP64 NaN
   pattern), and the regions that normally share memory (the QR, Cholesky and
   eigensolver buffers) are laid out one after another; after the iterations,
   H and (zolo_svd) the eigendecomposition, a kernel checks every zone, and a
   changed byte makes the call return ZOLO_EGUARD.  More workspace, slower;
   results are unchanged.  The slice planes of the split path and the batched,
   asynchronous and host entry points' own buffers are not guarded.  Returns
   0, -1 (NULL handle) or -2 (enable not 0/1). */
int zolo_debug_guards(zolo_handle_t handle, int enable);

#define ZOLO_STALL_SPLIT_GEMM 1
#define ZOLO_STALL_JACOBI32 2
#define ZOLO_STALL_JACOBI64 3
int zolo_debug_stall(zolo_handle_t handle, int where, int64_t ns);

/* Short text for a return code. */
const char* zolo_strerror(int code);

/* ---- Diagnostics (no counterpart in the paper). ---------------------------
   zolo_kernel_launches: kernels this process has launched through libzolo.
   zolo_profile(1) resets the statistics and brackets every later launch with
   a CUDA event pair on its stream (a few microseconds each); while it is on,
   zolo_pd_batched queues its matrices one after another on a single lane
   without a graph, so that every pair times its kernel alone.  zolo_profile(0)
   stops.  zolo_profile_read synchronises on the pending events, fills up to
   max_entries records (one per kernel class: launches, summed device time,
   summed algorithmic flops and bytes as stated by each launch site, and the
   SM-time: each launch's device time times the share of the GPU's resident-
   block slots its blocks take, blocks / (SMs x blocks per SM at the launch's
   occupancy), at most 1; a launch site that does not state its blocks counts
   as taking them all) and returns the number of classes.  With many calls in
   flight at once (the batched call's lanes) the SM-time shows which classes
   hold the GPU; the plain device time of a kernel on a few SMs does not. */
typedef struct {
  char name[32];
  int64_t launches;
  double ms;
  double flops;
  double bytes;
  double sm_ms;
} zolo_kstat_t;
uint64_t zolo_kernel_launches(void);
int zolo_profile(int enable);
int zolo_profile_read(zolo_kstat_t* out, int max_entries);

#ifdef __cplusplus
}
#endif

#endif /* ZOLO_H_ */
