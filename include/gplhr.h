/*
 * gplhr.h -- C ABI of libgplhr, a GB300 (sm_103a) implementation of the GPLHR
 * eigensolver: Generalized Preconditioned Locally Harmonic Residual method,
 * Vecharynski, Yang & Xue, arXiv 1506.06829.
 *
 * Problem (Sec. 1, Eq. gevp):  A x = lambda B x,  A, B sparse n x n, B = I allowed.
 * Wanted: the k eigenvalues nearest a shift sigma in C, a partial generalized
 * Schur form A V = Q R_A, B V = Q R_B (Eq. gschur; B = I: A V = V R, Eq. schur),
 * and eigenvectors x_j = V z_j.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Complex numbers are interleaved (re, im) pairs of double, as C99
 *   double _Complex / std::complex<double> / torch.complex128.
 * - Dense blocks are ROW-MAJOR n x w with a leading dimension ld >= w counted in
 *   elements: element (i, j) sits at p[i * ld + j].  (Rows of a k-wide block are
 *   contiguous so one sparse row gathers whole 16*k-byte block rows.)
 * - Small k x k / s x s matrices are row-major with ld = number of columns.
 * - "where" arguments: GPLHR_HOST (0) = pointer to host memory (pageable or
 *   pinned), GPLHR_DEVICE (1) = pointer to device memory of the context's GPU.
 * - Ownership: the library never keeps a caller pointer after a call returns;
 *   inputs are copied, outputs are written into caller-allocated memory.
 * - Errors: every call returns a gplhr_status; no exception, abort or exit
 *   crosses the ABI.  gplhr_last_error() gives a one-line message for the
 *   context (or the last failed create when called with NULL).
 * - Streams: all device work of a context runs on the stream given in
 *   gplhr_opts.stream (NULL = a stream the context creates).  Calls are
 *   synchronous with respect to the host unless stated otherwise.
 * - A context is not thread-safe; distinct contexts may be used concurrently.
 */
#ifndef GPLHR_H
#define GPLHR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GPLHR_OK = 0,
  GPLHR_EINVAL = 1,     /* invalid argument (sizes, pointers, CSR pattern, sigma)      */
  GPLHR_ENOMEM = 2,     /* device or host allocation failed                            */
  GPLHR_ECUDA = 3,      /* a CUDA runtime call failed (message has the CUDA error)     */
  GPLHR_ENOTCONV = 4,   /* maxit reached before all k pairs met tol (results readable) */
  GPLHR_ESINGULAR = 5,  /* singular (block-)Jacobi block, or orth() broke down twice   */
  GPLHR_ENUMERIC = 6,   /* NaN/Inf met in the iteration                                */
  GPLHR_ETIMEOUT = 7    /* a bounded device wait gave up                               */
} gplhr_status;

enum { GPLHR_HOST = 0, GPLHR_DEVICE = 1 };
enum { GPLHR_R64 = 0, GPLHR_C128 = 1 };                 /* CSR value types            */
enum {
  GPLHR_PREC_NONE = 0,          /* T = I                                               */
  GPLHR_PREC_JACOBI = 1,        /* T = diag(A - sigma B)^{-1}                          */
  GPLHR_PREC_BLOCK_JACOBI = 2,  /* T = blockdiag of bs x bs diagonal blocks, inverted  */
  GPLHR_PREC_CSR = 3            /* T given explicitly as a sparse matrix (C128)        */
};
/* Arithmetic of the iteration.  MIXED: a bulk phase in which the sparse products, the
 * preconditioner, the projections and block combinations compute in FP32 (complex64
 * arithmetic with FP32 accumulation, on FP64 storage), while the Cholesky-QR Gram
 * matrices, the projected pencil, its QZ and the small factors stay FP64; then FP64
 * refinement iterations once the largest residual is below switch_tol or has not
 * dropped by 10 % over stall_iters iterations.  Convergence is declared only in FP64. */
enum { GPLHR_FP64 = 0, GPLHR_MIXED = 1 };

/* Sparse matrix in CSR form (0-based, column indices sorted per row, no duplicates).
 * rowptr has n+1 entries, colind and vals nnz entries; vals are double (GPLHR_R64) or
 * interleaved complex double (GPLHR_C128).  on_device = 1 if the three arrays are
 * device pointers.  The library copies what it needs during gplhr_create. */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int32_t* rowptr;
  const int32_t* colind;
  const void* vals;
  int32_t dtype;
  int32_t on_device;
} gplhr_csr;

/* Preconditioner T ~ (A - sigma B)^{-1} (Sec. 4).  JACOBI and BLOCK_JACOBI are built
 * from A - sigma B inside gplhr_create; block_size bs >= 1 groups consecutive rows
 * [b bs, (b+1) bs) (the last block is n mod bs wide when bs does not divide n).
 * JACOBI with a constant diagonal (relative spread <= 1e-12) is T = I: every output
 * of T goes through a projector and orth(), so a constant scaling of T leaves the
 * iteration unchanged.  CSR: T is applied as a sparse product with matrix T_csr.
 * inner_steps s > 0 (Sec. 4, an inner solve as T): T R = T0 Y*, s steps of block GMRES
 * on (A - sigma B) W = R with zero start, right-preconditioned by the preconditioner T0
 * that kind / block_size / T_csr describe: Y* minimises ||R - (A - sigma B) T0 Y||_F
 * over the block Krylov space span{R, ((A - sigma B) T0) R, ...} of s blocks (block
 * Arnoldi on the device, the small least-squares problem on the host).  Needs
 * s <= 32 and s k <= 384 (EINVAL otherwise); each application of T costs s sparse
 * products with A and B and s applications of T0. */
typedef struct {
  int32_t kind;
  int32_t block_size;
  const gplhr_csr* T_csr;
  int32_t inner_steps;
} gplhr_precond;

/* Solver options.  Zero-initialised fields take the defaults in brackets. */
typedef struct {
  double tol;          /* [1e-8] backward error per pair, see gplhr_info.resid          */
  int32_t maxit;       /* [500]  iteration cap (the paper's DNC limit, Sec. 5.1)        */
  int32_t precision;   /* [GPLHR_FP64]                                                   */
  int32_t no_lock;     /* [0]    1 disables soft locking (Sec. 3.6)                      */
  int32_t products;    /* [0]    how AV, BV, AP, BP are formed: 1 = linear combinations of
                          AZ, BZ (the paper's (m+1) sparse products per iteration), 2 =
                          fresh sparse products of V and P ((m+3) per iteration), 0 = the
                          one with fewer flops for this pencil                          */
  void* stream;        /* [NULL] cudaStream_t for all device work of the context        */
  double switch_tol;   /* [1e-5] MIXED: refine in FP64 once max residual < switch_tol   */
  int32_t stall_iters; /* [5]    MIXED: ... or after this many iterations without a 10 %
                          decrease of the max residual; < 0: never on a stall            */
  int32_t pencil;      /* [0]    projected pencil: 0 = U^*BZ by a Gram product and
                          U^*(A - sigma B)Z from the factors of U's construction (Prop. 3.2
                          and the orthonormalisation of (A - sigma B)[W S P]); 1 = both
                          U^*AZ and U^*BZ by Gram products (Alg. 2 step 24 as printed)   */
  int32_t fp64_gemm;   /* [0]    FP64 block combinations and Gram products: 0 = on the
                          tensor cores (tcgen05, each double split into 7 balanced 8-bit
                          integer digits, exact accumulation of digit-pair products; a
                          combination's error is at most (K'/4 + 2) 2^-53 max|x| sum|c|
                          over K' real terms, a bound of its own: not ordered against the
                          DFMA bound K' 2^-53 sum |x| |c|, which is smaller when a row's
                          entries span decades) where the shape allows
                          (combinations: <= 32 input and output columns, n >= 512; Gram
                          products: see gplhr_gram), DFMA otherwise; 1 = DFMA only       */
  int32_t graphs;      /* [0]    1 = capture the device work of each iteration between its
                          host round trips (three segments) in CUDA graphs on first use
                          and replay them afterwards: one graph launch instead of tens of
                          kernel launches per segment, for small pencils where launch
                          overhead dominates.  A graph is kept per state that fixes the
                          launch sequence (locked pairs, m, P present, precision phase).
                          Not used while gplhr_profile timing is on or with inner GMRES
                          steps (their least squares runs on the host inside T).          */
  int32_t autotune;    /* [0]    1 = time the SpMM launch shapes (threads per CTA 64/128/256,
                          grid cap 2..64 CTAs per SM) on this pencil's A and B at create,
                          for each lane-group width the block widths 1..k select (and in
                          the FP32 bulk phase), and use the fastest; gplhr_spmm_shape
                          reports the choice.  Results do not depend on it.                */
  int32_t p_mode;      /* [0]    search directions P (Sec. 3.5, the paper's Table 2): 0 = thick
                          restart P = Z Ybar_R(:, k+1:2k) (Eq. P1); 1 = LOBPCG style
                          P = V - V_prev (Eq. P_lobpcg with C = I: every invertible C gives
                          the same trial subspace); 2 = no P, (m + 2) k trial columns.
                          EINVAL otherwise.                                                */
  int32_t no_right_proj; /* [0]  1 = omit the projector applied before T (T_L = (I - VV^*) T
                          instead of (I - VV^*) T (I - QQ^*), or (I - VV^*) T (I - VV^*) when
                          B = I): the variant the paper compares in its Table 3.            */
  int32_t variant;     /* [0]    0 = GPLHR on Schur vectors (Alg. 2); 1 = GPLHR-EIG (Alg. 3,
                          Appendix A): eigenvector iterate X with unit columns, eigenvalues
                          the Rayleigh quotients x^* A x / x^* B x, projected pair solved by
                          its eigenvectors; P of step 27 (p_mode 0) or of step 25 (p_mode 1);
                          all k pairs converge together (no locking).  FP64 only, with the
                          projector before T, no deflation, no gplhr_grad.  gplhr_vectors
                          then fills alpha, beta, lambda, X and resid and zero-fills V, Q,
                          RA, RB.  EINVAL for other values or combinations.               */
  int32_t wait_limit;  /* [0]    test hook of the failure path: the number of tests (each
                          sleeping at most 20 us) after which a wait of one role of a
                          tensor-core kernel on another role gives up; the kernel then
                          ends all its roles, waits (with the full limit) for its own
                          products in flight, frees its tensor memory, and the call returns
                          GPLHR_ETIMEOUT with the context still usable.  0 = 65536 tests
                          (~1.3 s); values above that are clamped to it; EINVAL if < 0.
                          The paper has no counterpart.                                    */
  int32_t wait_probe;  /* [0]    test hook: 1 = the epilogue of every tensor-core combination
                          also waits on an mbarrier whose phase nothing completes, so the
                          time-out path above runs deterministically (after wait_limit
                          tests).  Never set outside tests.                                */
} gplhr_opts;

/* Per-solve report.  resid[j] (j < k) is the backward error of pair j,
 *   ||A x_j - lambda_j B x_j|| / ((||A||_1 + |lambda_j| ||B||_1) ||x_j||),
 * with x_j = V z_j from the triangular factors (Sec. 5.1 measures eigen-residuals
 * of vectors made from the Schur basis).  Counters follow the paper's #mv / #prec
 * (Sec. 5): n_spmm counts products of A (and of B when B != I) with one n x w block. */
typedef struct {
  int32_t iters;
  int32_t nconv;        /* leading pairs meeting tol (locked in order)                 */
  int32_t m;            /* current m after adaptation                                  */
  int32_t n_orth_fallback; /* orth() calls that needed the shifted-Cholesky pass       */
  int32_t fp32_iters;   /* iterations run in the FP32 bulk phase (GPLHR_MIXED)         */
  int32_t bulk;         /* 1 while the iteration is still in the FP32 bulk phase        */
  int64_t n_spmm;
  int64_t n_prec;
  int64_t n_qz;
  int64_t n_launch;     /* CUDA kernels launched (since create or gplhr_profile)       */
  int64_t h2d_bytes;    /* host->device bytes moved by the iteration since start        */
  int64_t d2h_bytes;    /* device->host bytes (projected pencil for the host QZ, norms) */
  double resid[64];     /* first min(k, 64) residuals                                  */
  int64_t n_inner;      /* inner block GMRES steps (T.inner_steps per application of T;
                           their sparse products are counted in n_spmm)                 */
} gplhr_info;

typedef struct gplhr_ctx gplhr_ctx;

/* gplhr_create -- set up a GPLHR solve for the pencil (A, B) and shift sigma.
 * Paper: Algorithm 2 inputs (Sec. 3.6): a regular pair (A, B), sigma not an
 * eigenvalue, preconditioner T, block size k and expansion parameter m; the
 * trial subspace has s = (m+3)k columns (Eq. trial_partial1) and the context
 * allocates Z, U, AZ, BZ of n x s each (Sec. 3.6 storage remark).
 * A: required; B: NULL means B = I.  1 <= k <= 32, 0 <= m <= 20, (m+2) k <= 80 (the
 * widest orthonormalised block, held in one CTA's shared memory), (m+3) k <= n.
 * Errors: EINVAL (sizes, pattern, sigma not finite), ESINGULAR (a Jacobi /
 * block-Jacobi block of A - sigma B is singular), ENOMEM, ECUDA.
 * On success *out owns all device memory of the solve; free with gplhr_destroy. */
gplhr_status gplhr_create(const gplhr_csr* A, const gplhr_csr* B, double sigma_re,
                          double sigma_im, int32_t k, int32_t m, const gplhr_precond* T,
                          const gplhr_opts* opts, gplhr_ctx** out);

/* gplhr_solve -- run Algorithm 2 from the start block V0 until every pair's
 * residual is <= tol, or maxit iterations (then ENOTCONV; results readable).
 * V0: n x k row-major (ld = k), complex (is_complex = 1) or real (0), on host or
 * device per V0_where; NULL draws a Gaussian block from `seed` on the device.
 * info may be NULL.  Steps 1-4 (initial orth + ordered QZ) are part of this call. */
gplhr_status gplhr_solve(gplhr_ctx* ctx, const void* V0, int32_t V0_where, int32_t is_complex,
                         uint64_t seed, gplhr_info* info);

/* gplhr_start -- steps 1-4 of Algorithm 2 only (initial basis and factors), then
 * gplhr_iterate -- exactly `niter` passes of the while loop of Algorithm 2 (steps
 * 6-30) with the convergence/locking bookkeeping, stopping early only if all k pairs
 * meet tol.  Together they equal gplhr_solve; they exist for timing and checks. */
gplhr_status gplhr_start(gplhr_ctx* ctx, const void* V0, int32_t V0_where, int32_t is_complex,
                         uint64_t seed);
gplhr_status gplhr_iterate(gplhr_ctx* ctx, int32_t niter, gplhr_info* info);

/* gplhr_vectors -- read the current (converged) results.  Any pointer may be NULL.
 * alpha, beta, lambda: k complex each (diagonals of R_A, R_B and their ratio,
 *   Sec. 2, Eq. gevp_mod; lambda = alpha/beta, +inf when beta = 0), in ascending
 *   |lambda - sigma| order (footnote to Alg. 2 step 2).
 * X: n x k eigenvectors x_j = V z_j, unit 2-norm (Sec. 2.1: eigenvectors from the
 *   Schur basis), V, Q: n x k Schur bases (ld = k), RA, RB: k x k upper triangular
 *   (B = I: RA is R with A V = V R, Eq. schur, and RB = I).
 * resid: k backward errors recomputed with fresh products A X, B X (FP64).
 * where selects host or device for X, V, Q, RA, RB (alpha/beta/lambda/resid are
 * always host).  Errors: EINVAL if called before gplhr_start/solve. */
gplhr_status gplhr_vectors(gplhr_ctx* ctx, double* alpha, double* beta, double* lambda,
                           void* X, void* V, void* Q, void* RA, void* RB, double* resid,
                           int32_t where);

/* gplhr_grad -- gradient of a real loss of the k eigenvalues with respect to the stored
 * values of A and B, on their CSR patterns (in the input order).  Uses the first-order
 * perturbation of a simple eigenvalue (Sec. 2.1 gives the right and left Schur bases;
 * the eigenvectors come from them):
 *     d lambda_i = y_i^* (dA - lambda_i dB) x_i / (y_i^* B x_i),
 * x_i the right eigenvector from `right` (solved on (A, B) at sigma) and y_i the left one
 * from `left` (solved on (A^*, B^*) at conj(sigma), whose eigenvalues are conj(lambda));
 * pairs are matched by nearest eigenvalue (EINVAL if a match is not unique within
 * 1e-6 |lambda|).  G: 2k doubles on the host, G[2i] + i G[2i+1] = dL/dRe(lambda_i) +
 * i dL/dIm(lambda_i), in the order gplhr_vectors reports for `right`.  Outputs
 * dL/da for every stored entry of A (dA_vals, nnz(A) values) and of B (dB_vals, NULL if
 * not wanted or B = I): doubles for a real matrix (the real part, i.e. the gradient
 * with respect to real entries), interleaved complex (dL/dRe + i dL/dIm) for a complex
 * one; host or device memory per `where`.  Both contexts must be on the current GPU,
 * with equal n and k.  Errors: EINVAL, ENUMERIC (y^* B x = 0), ECUDA. */
gplhr_status gplhr_grad(gplhr_ctx* right, gplhr_ctx* left, const double* G, void* dA_vals,
                        void* dB_vals, int32_t where);

/* gplhr_create_batched -- create nctx contexts at once: many pencils of uneven size, or
 * many shifts over one pencil (spectrum slicing: pass the same A, B descriptors with
 * different shifts), each with the arguments of gplhr_create (Algorithm 2 inputs,
 * Sec. 3.6).  Arrays of nctx entries: A (required, entries non-NULL), B (NULL, or
 * entries NULL for B = I), sigma (2 nctx doubles: re, im), k, m, T (NULL, or NULL
 * entries for T = I), opts (NULL, or NULL entries for the defaults).  Every context
 * copies its matrices (as gplhr_create does; slices over one pencil do not share device
 * copies) and owns its own stream unless opts gives one.  The contexts are created
 * concurrently by nthreads host threads (<= 0: the host's hardware threads), all on the
 * current device.  out (nctx handles) receives them.  All or nothing: if any creation
 * fails, the contexts already created are destroyed, every out[i] is NULL, statuses (may
 * be NULL) holds each entry's status, the first failing status in entry order is
 * returned and gplhr_last_error(NULL) names that entry and its message.  The handles
 * then go to gplhr_solve_batched / gplhr_iterate_batched and are freed one by one with
 * gplhr_destroy. */
gplhr_status gplhr_create_batched(int32_t nctx, const gplhr_csr* const* A, const gplhr_csr* const* B,
                                  const double* sigma, const int32_t* k, const int32_t* m,
                                  const gplhr_precond* const* T, const gplhr_opts* const* opts, gplhr_ctx** out,
                                  gplhr_status* statuses, int32_t nthreads);

/* Batched solves (many pencils of uneven size, or many shifts over one pencil, each in
 * its own context).  The contexts are independent: each has its own stream and
 * buffers; a pool of nthreads host threads (<= 0: the host's hardware threads) runs
 * them concurrently, so the host QZ and synchronisations of one pencil overlap the
 * device work of the others.  Arguments are arrays of nctx entries (V0, V0_where,
 * is_complex, seeds, infos may be NULL: then gplhr_solve's defaults); statuses
 * (may be NULL) receives each context's status.  Returns GPLHR_OK if every context
 * succeeded, else the first failing status in context order.  A context must not
 * appear twice.  gplhr_iterate_batched runs niter iterations of each started context. */
gplhr_status gplhr_solve_batched(int32_t nctx, gplhr_ctx* const* ctxs, const void* const* V0,
                                 const int32_t* V0_where, const int32_t* is_complex,
                                 const uint64_t* seeds, gplhr_info* infos,
                                 gplhr_status* statuses, int32_t nthreads);
gplhr_status gplhr_iterate_batched(int32_t nctx, gplhr_ctx* const* ctxs, int32_t niter,
                                   gplhr_info* infos, gplhr_status* statuses, int32_t nthreads);

/* Persistent batched iteration: the same batches (many pencils of uneven size, many
 * shifts over one pencil), with every device segment of an iteration of Algorithm 2
 * (steps 7-24, steps 25-28, the residual with its column norms) run for ALL contexts in
 * one launch of a persistent kernel.  The host records each context's launches (the
 * kernels, grids and arguments gplhr_iterate would issue, on the FP64 / FP32 DFMA and
 * FFMA kernels, not the tensor-core ones) and merges them into one queue; the kernel,
 * launched cooperatively (every CTA resident), takes the queue's items (the launches'
 * CTAs) in order, and each item waits only for the previous launch of its own context,
 * so the contexts advance independently.  Per iteration of the whole batch: three
 * launches and two host round trips (the projected pencils for the host QZ, which runs on
 * nthreads host threads, and the residual norms for soft locking).  Each wait is bounded
 * (the contexts' opts.wait_limit, in tests of 20 us); when it runs out the call returns
 * GPLHR_ETIMEOUT (opts.wait_probe makes it run out: a test hook).  Contexts iterate in
 * lockstep and leave the batch when they converge, fail or reach their budget.  Results
 * match gplhr_iterate's to rounding (the Gram products' partial sums are split by the
 * context's share of the SMs, not by all of them).
 * Not supported (EINVAL): GPLHR-EIG contexts, inner GMRES preconditioning (its least
 * squares runs on the host inside T), profiling.  A context must not appear twice; all
 * contexts belong to the current device.
 * gplhr_iterate_persistent runs up to niter iterations of each started context;
 * gplhr_solve_persistent starts every context (steps 1-4, on host threads, as
 * gplhr_solve_batched does) and iterates until each converges or reaches its maxit
 * (ENOTCONV then, results readable).  Arguments as gplhr_solve_batched; stats (may be
 * NULL) receives the launch counts.  Returns GPLHR_OK if every context succeeded, else
 * the first failing status in context order; a message is in gplhr_last_error(NULL). */
typedef struct gplhr_persist_stats {
  int64_t launches;  /* persistent-kernel launches */
  int64_t steps;     /* queue steps (the longest context's launches) over all launches */
  int64_t ops;       /* recorded kernel launches they replaced */
  int32_t grid;      /* CTAs of the last launch */
  int32_t pad;
  double record_ms;  /* host: recording the contexts' segments (on the host threads) */
  double build_ms;   /* host: merging the programs, issuing copies and launches */
  double qz_ms;      /* host: the sorted QZ of every pencil (on the host threads) */
  double wait_ms;    /* host: waiting for the device at the two round trips */
} gplhr_persist_stats;
gplhr_status gplhr_iterate_persistent(int32_t nctx, gplhr_ctx* const* ctxs, int32_t niter,
                                      gplhr_info* infos, gplhr_status* statuses, int32_t nthreads,
                                      gplhr_persist_stats* stats);
gplhr_status gplhr_solve_persistent(int32_t nctx, gplhr_ctx* const* ctxs, const void* const* V0,
                                    const int32_t* V0_where, const int32_t* is_complex,
                                    const uint64_t* seeds, gplhr_info* infos,
                                    gplhr_status* statuses, int32_t nthreads,
                                    gplhr_persist_stats* stats);

/* gplhr_destroy -- free everything the context owns.  NULL is a no-op. */
void gplhr_destroy(gplhr_ctx* ctx);

/* Message for the last failing call on ctx (or, when called with NULL, of the last failed
 * context-free call -- gplhr_create, gplhr_create_batched, gplhr_gram_noalloc -- on the
 * calling host thread).  The string stays valid until the next call on the same context
 * (or the next context-free call on the same thread). */
const char* gplhr_last_error(const gplhr_ctx* ctx);

/* ---------------------------------------------------------------------------------
 * Step-level entry points: one building block of an iteration each, on device
 * pointers of the context's GPU, on the context's stream, synchronous on return.
 * They run the same kernels as gplhr_iterate and exist so that each step can be
 * checked against the CPU oracle on its own.
 * ------------------------------------------------------------------------------ */

/* Sparse times block (the "matblock" products of Sec. 3.6, (m+1) per iteration):
 * AX = A X and, if B != I and BX != NULL, BX = B X.  X, AX, BX: n x w, row-major. */
gplhr_status gplhr_spmm(gplhr_ctx* ctx, const void* X, int32_t ldx, int32_t w, void* AX,
                        int32_t ldax, void* BX, int32_t ldbx);

/* Preconditioner Y = T X (Sec. 4; inside T_L of Eq. prec_gen).  Y may equal X. */
gplhr_status gplhr_precond_apply(gplhr_ctx* ctx, const void* X, int32_t ldx, int32_t w,
                                 void* Y, int32_t ldy);

/* Gram product C = X^* Y (w_x x w_y, row-major, ld = w_y) over all n rows: the
 * projections and the projected pencil U^* A Z, U^* B Z (Alg. 2 steps 8, 15, 19-24).
 * arith: GPLHR_GRAM_FP64 (0) DFMA; GPLHR_GRAM_FP32 (1) FP32 arithmetic (the projection
 * coefficients of the mixed mode's bulk phase); GPLHR_GRAM_EXACT32 (2) inputs rounded
 * to FP32, every product formed exactly on the FP32 pipe and summed with compensation
 * into FP64 (the Cholesky-QR Grams and pencil of the bulk phase, whose blocks hold
 * FP32 values); GPLHR_GRAM_TENSOR (3) the FP64 product as the iteration forms it: on the
 * tensor cores (each double split into 7 integer digits against a per-column exponent
 * over 128-row windows, exact accumulation of digit products, one rounding per window,
 * FP64 sums of the windows) when n >= 2048, opts.fp64_gemm = 0 and the shape fits one of
 * the forms: wx <= 24, wy <= 16 and at most 32 loaded columns (wx + wy, or wx when Y is
 * X); the same with X and Y exchanged (C formed as (Y^* X)^*); wx <= 64, wy <= 32,
 * wx wy >= 128; wx <= 128, wy <= 32, wx wy >= 400.  Else DFMA.  EINVAL for
 * wx > max((m+3)k, 128) or wy > 2 (m+3)k. */
enum { GPLHR_GRAM_FP64 = 0, GPLHR_GRAM_FP32 = 1, GPLHR_GRAM_EXACT32 = 2, GPLHR_GRAM_TENSOR = 3 };
gplhr_status gplhr_gram(gplhr_ctx* ctx, const void* X, int32_t ldx, int32_t wx, const void* Y,
                        int32_t ldy, int32_t wy, void* C, int32_t arith);

/* Block combination Y = X C (beta = 0) or Y = Y + X C (beta = 1): the basis update of
 * Alg. 2 steps 25-28 (V = Z Y_R, Q = U Y_L, P = Z Ybar_R(:, k+1:2k)) and every projection
 * X - L (L^* X) of the iteration.  X: n x w (ld >= w), C: w x c row-major, Y: n x c
 * (ld >= c), all complex128 on the device; Y must not overlap X unless Y == X with
 * c == w and ldy == ldx (in place, beta = 0).  arith: GPLHR_COMBINE_AUTO (0) the
 * context's choice (tensor cores for <= 32 input and output columns unless
 * opts.fp64_gemm = 1), GPLHR_COMBINE_DFMA (1).  EINVAL for w or c outside [1, 2 s_max].
 * Synchronises the context's stream. */
enum { GPLHR_COMBINE_AUTO = 0, GPLHR_COMBINE_DFMA = 1 };
gplhr_status gplhr_combine(gplhr_ctx* ctx, const void* X, int32_t ldx, int32_t w, const void* C,
                           int32_t c, void* Y, int32_t ldy, int32_t beta, int32_t arith);

/* Launch shape the context uses for sparse products of a w-column block (fp32 = 1: the
 * FP32 bulk phase, w <= 64; else w <= 32): threads per CTA, grid cap in CTAs per SM and,
 * when opts.autotune measured them, the time of one A (and B) product in microseconds
 * with that shape and with the default shape (256 threads, 8 CTAs per SM); 0 otherwise.
 * Any output pointer may be NULL.  EINVAL for w out of range.  The paper has no
 * counterpart: a launch-configuration query of this implementation. */
gplhr_status gplhr_spmm_shape(gplhr_ctx* ctx, int32_t w, int32_t fp32, int32_t* threads, int32_t* grid_per_sm,
                              double* us, double* us_default);

/* gplhr_set_deflation -- compute further Schur vectors by deflation (Sec. 3.6, last
 * paragraph): with V1, Q1 the k1 right and left generalized Schur vectors found by an
 * earlier solve (n x k1 row-major complex128, ld k1; orthonormal columns), later starts
 * and solves of this context run GPLHR on the deflated pair
 *     ((I - Q1 Q1^*) A (I - V1 V1^*), (I - Q1 Q1^*) B (I - V1 V1^*)),
 * or (I - V1 V1^*) A (I - V1 V1^*) when B = I (Q1 is then ignored and may be NULL).  The
 * deflated pair is singular on span(V1), so T is deflated alike,
 * (I - V1 V1^*) T (I - Q1 Q1^*), and the start block is projected: the trial subspace stays
 * orthogonal to V1.  The new block (V2, Q2, R_A2, R_B2 from gplhr_vectors) extends the
 * partial Schur form: A [V1 V2] = [Q1 Q2] [[R_A1, Q1^* A V2], [0, R_A2]], likewise B.
 * Residuals are those of the deflated pair, normalised by ||A||_1, ||B||_1.  The library
 * copies V1, Q1 (where = HOST or DEVICE); k1 = 0 removes the deflation.  EINVAL for
 * k1 > 256, k1 + (m+3)k > n, k1 k > 2 ((m+3)k)^2, missing bases, or with inner GMRES
 * steps (opts: T.inner_steps > 0). */
gplhr_status gplhr_set_deflation(gplhr_ctx* ctx, const void* V1, const void* Q1, int32_t k1, int32_t where);

/* orth(X) in place (Alg. 1 footnote): X <- X R^{-1} with X = Q R the thin QR whose R
 * has a real positive diagonal, by Cholesky QR applied twice (a shifted Cholesky
 * first pass and a third pass when the Gram matrix is not numerically positive
 * definite).  Rinv (w x w, may be NULL) receives R^{-1}. */
gplhr_status gplhr_orth(gplhr_ctx* ctx, void* X, int32_t ldx, int32_t w, void* Rinv);

/* Instrumentation.  gplhr_profile(ctx, 1) clears the per-kernel-class counters and
 * brackets every later launch section with CUDA events on the context's stream;
 * gplhr_profile(ctx, 0) stops the timing (counters keep counting).
 * gplhr_profile_read returns for kernel class kclass -- 0 SpMM, 1 Gram (DFMA, FP32 or
 * exact-FP32 arithmetic), 2 block combine (tall-skinny times small; DFMA or FP32), 3
 * preconditioner, 4 small Cholesky, 5 other elementwise, 6 Gram on the tensor cores, 7
 * block combine on the tensor cores -- the summed event time (ms, while profiling), the
 * kernel launches,
 * and the ALGORITHMIC flops (complex multiply-add = 8, real x complex = 4) and bytes
 * (each operand read once, each result written once) of those launches. */
gplhr_status gplhr_profile(gplhr_ctx* ctx, int32_t enable);
gplhr_status gplhr_profile_read(gplhr_ctx* ctx, int32_t kclass, double* ms, int64_t* launches,
                                double* flops, double* bytes);

/* Gram product C = X^* Y that allocates nothing, for callers that cannot call
 * cudaMalloc: for instance code whose device memory is all owned by another
 * allocator or memory pool, or a loop that must not take the implicit device
 * synchronisation and latency of an allocation.  The paper has no counterpart: this
 * is a library convenience around the Gram kernel of gplhr_gram.
 * X: n x wx, Y: n x wy (row-major complex, device pointers, leading dimensions in
 * elements), C: wx x wy row-major (ld = wy), device pointer; all are the caller's and
 * must be memory of the CURRENT device (the kernels run on the current device, with
 * its copy of the scratch array; the library cannot check where a raw pointer lives).
 * Needs no context.  Limits: 1 <= n <= 2^30, wx * wy <= 16384 and wx + wy <= 768, else
 * EINVAL with a message in gplhr_last_error(NULL).  The kernel's scratch (partial sums over chunks
 * of rows) is a fixed 4 MiB array in the library's device memory, held by every GPU
 * that loads the library until the process exits; every call on a device shares it
 * and leaves it holding its own partial sums, so calls that overlap on the GPU (two
 * streams, or two threads) race and must be ordered by the caller.  The call is
 * asynchronous on `stream` (NULL = the default stream): C is complete when the stream
 * reaches this point.  The first call on a device (with that device current) also
 * looks up the scratch array's device address and sets the kernels' shared-memory
 * limit; make that first call before capturing `stream`.  Errors: EINVAL, ECUDA. */
gplhr_status gplhr_gram_noalloc(int64_t n, const void* X, int32_t ldx, int32_t wx,
                                const void* Y, int32_t ldy, int32_t wy, void* C, void* stream);

/* Ordered complex QZ of a small pencil on the host (footnote to Alg. 2 step 2):
 * Phi = YL RA YR^*, Psi = YL RB YR^* with |RA(j,j)/RB(j,j) - sigma| non-decreasing
 * and RB(j,j) real >= 0.  All matrices s x s row-major complex, host memory.
 * Phi/Psi are not modified.  No context or GPU needed.  Errors: EINVAL, ENOTCONV. */
gplhr_status gplhr_ordqz(int32_t s, const double* Phi, const double* Psi, double sigma_re,
                         double sigma_im, double* RA, double* RB, double* YL, double* YR);

/* The same ordered QZ on the device, in one CTA (s <= 80): the host routine's steps in its
 * order (Givens Hessenberg-triangular reduction, single-shift sweeps, adjacent swaps of the
 * leading nsort positions (< 0: all), unit phases), each plane rotation formed by one
 * thread and applied by all.  Phi, Psi (read) and RA, RB, YL, YR (written) are device
 * pointers to s x s row-major complex128 matrices; *status (a device int) is set to 0,
 * or to 1 when the sweeps did not converge.  Asynchronous on `stream` (NULL = the
 * default stream).  It exists so that the QZ can be timed on the device against the
 * host: an iteration of GPLHR uses the host QZ, which measured faster at every s of the
 * workloads.  Errors: EINVAL (s outside 1..80, NULL pointers), ECUDA (launch). */
gplhr_status gplhr_ordqz_device(int32_t s, const void* Phi, const void* Psi, double sigma_re,
                                double sigma_im, int32_t nsort, void* RA, void* RB, void* YL,
                                void* YR, int32_t* status, void* stream);

/* Q-free factors of Theorem 1 with Eqs. G1_fix, G2_fix: M_A = G2 G^{-1} R_A,
 * M_B = I - G1 G^{-1} R_A, G = R_A G1 + R_B G2 (k x k row-major complex, host). */
gplhr_status gplhr_mfactors(int32_t k, const double* RA, const double* RB, double* MA,
                            double* MB);

#ifdef __cplusplus
}
#endif
#endif /* GPLHR_H */
