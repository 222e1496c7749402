/*
 * tikhonov.h -- C ABI of the GB300 (sm_103a) library for randomized Tikhonov
 * regularization: min ||A x - b||^2 + lambda ||x||^2 for a list of
 * regularization parameters lambda_1..lambda_N (Meier & Nakatsukasa,
 * "Randomized algorithms for Tikhonov regularization in Linear Least Squares").
 *
 * The calls follow the paper's problem statement (Section 1, problems (1.2)-(1.4)):
 * A, b, the lambda_i and a tolerance in; x_{lambda_i} and iteration counts out.
 * A is sketched once (Section 2.1.1: SRHT or Gaussian embedding), a
 * preconditioner is formed per lambda_i from the partly exact sketch
 * (Algorithm 1 / 2: Cholesky of C + lambda_i I; Algorithms 3 / 4: the low-rank
 * Woodbury form of Sections 3.1 / 3.2), and preconditioned LSQR runs for every lambda_i.
 *
 * Conventions shared by every call:
 *  - Matrices are row-major.  A is m x n with row stride lda >= n (elements).
 *  - "device" pointers are CUDA device memory of the current device; "host"
 *    pointers are ordinary host memory.  The caller owns all memory passed in.
 *    Apart from the handle calls (tk_create ... tk_handle_solve_batched, which
 *    own a growing workspace), the library never allocates device memory:
 *    every call that needs scratch takes a caller-provided device workspace
 *    whose size tk_workspace_size() (or the call's own size query) returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Kernels are issued on it in order.  Calls that return host results
 *    synchronize the stream before returning.
 *  - The return value is a tk_status.  Argument errors are detected on the
 *    host before any launch (TK_EINVAL, nothing written).  TK_ECUDA reports a
 *    CUDA error; tk_last_error() returns its text.
 *  - m >= n selects the overdetermined algorithms (1 and 3); m < n selects the
 *    underdetermined ones (2 and 4).
 */
#ifndef TIKHONOV_H
#define TIKHONOV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define TK_API __attribute__((visibility("default")))
#else
#define TK_API
#endif

typedef enum {
  TK_OK = 0,
  TK_EINVAL = 1,    /* invalid argument (checked on the host, nothing launched) */
  TK_ENOMEM = 2,    /* workspace smaller than the size query returned */
  TK_ENOTSPD = 3,   /* Cholesky breakdown: C + lambda I not numerically positive definite */
  TK_ENOCONV = 4,   /* LSQR reached maxiter (or refinement reached max_refine) */
  TK_ENUMERIC = 5,  /* NaN/Inf met in the recurrences */
  TK_ETIMEOUT = 6,  /* a bounded device-side wait gave up */
  TK_ECUDA = 7      /* CUDA runtime error, see tk_last_error() */
} tk_status;

typedef enum { TK_F64 = 0, TK_F32 = 1 } tk_dtype;
/* Embeddings of Section 2.1.1: SRHT (signs, Walsh-Hadamard transform, row
 * sampling), Gaussian (N(0, 1/s) entries), and SPARSE (one nonzero element
 * in each column: sign_i in row h_i, both from Philox stream 4 at index i,
 * h_i = floor(w0 s / 2^32), sign_i = -1 when the low bit of w1 is set; applied
 * in O(nnz(A)) by adding each row of A into its bucket in ascending row order;
 * s <= 2^22), and SRDCT (the SRHT with the orthonormal DCT-II in place of the Hadamard transform,
 * the embedding of the paper's Fig. 1-2: X = sqrt(mp/s) S C D, same signs and rows as the SRHT,
 * computed through one complex FFT of length mp per column). */
typedef enum { TK_SKETCH_SRHT = 0, TK_SKETCH_GAUSS = 1, TK_SKETCH_SPARSE = 2, TK_SKETCH_SRDCT = 3 } tk_sketch;
/* Preconditioners: CHOL = Algorithm 1 / 2 (R_i = chol(C + lambda_i I)); LOWRANK = Algorithms 3 / 4
 * (Sections 3.1 / 3.2); QR = BP2 of Section 4.1 (m >= n): R_i from a Householder QR of the
 * (s + n) x n partly exact sketch [X A; sqrt(lambda_i) I], the same factor as CHOL in exact
 * arithmetic, without forming Y^T Y, at the cost of a QR per lambda. */
typedef enum { TK_PRECOND_CHOL = 0, TK_PRECOND_LOWRANK = 1, TK_PRECOND_QR = 2 } tk_precond;
typedef enum { TK_PREC_FP64 = 0, TK_PREC_MIXED = 1 } tk_precision;
typedef enum { TK_SCHED_BATCHED = 0, TK_SCHED_ONE_AT_A_TIME = 1 } tk_schedule;

/* Problem (1.2): device A (m x n, row stride lda, dtype) and device b (m, float64). */
typedef struct {
  int64_t m, n, lda;
  tk_dtype dtype;
  const void* A;
  const double* b;
} tk_problem;

/* Options.  tk_opts_default() fills the defaults given in brackets. */
typedef struct {
  tk_sketch sketch;       /* [SRHT] embedding of Section 2.1.1 */
  int64_t s;              /* sketch size; 0 = 4 * min(m, n) for Cholesky (16 * min(m, n) for SPARSE), capped at
                             max(m, n); min(m, n) for low rank [0] */
  tk_precond precond;     /* [CHOL] Algorithm 1/2, LOWRANK = Algorithm 3 (m >= n) / 4 (m < n, FP64), QR = BP2 */
  double alpha;           /* [2] oversampling of Algorithms 3/4: s_i = alpha * ceil(sd_i) */
  tk_precision precision; /* [FP64] or MIXED (FP32 LSQR + FP64 refinement) */
  double tol;             /* [1e-14] LSQR stopping tolerance (Paige-Saunders atol = btol) */
  int maxiter;            /* [500] LSQR iteration cap per lambda */
  int max_refine;         /* [8] refinement steps of the MIXED form */
  double inner_tol;       /* [1e-7] FP32 LSQR tolerance inside the MIXED refinement */
  double refine_tol;      /* [1e-11] MIXED stops when ||d|| <= refine_tol ||x|| */
  uint64_t seed;          /* [1] Philox key of every draw */
  tk_schedule schedule;   /* [BATCHED]: all lambda advance together; ONE_AT_A_TIME: one lambda per LSQR run */
  int lsqr_tc;            /* [2] MIXED: the two products with A of each LSQR step on the tensor cores:
                             1 = tcgen05 kind::tf32, 3-term split (float32 accuracy; needs 16-byte aligned
                             rows of A and keeps a float32 copy of A^T); 2 = BF16 products of the first 4
                             exact digits of the slices that emulate_fp64 makes (A rounded to 28 bits,
                             exact level sums; needs emulate_fp64 and m >= n; used when m n > 2^24 and
                             more than 16 lambda are active, SIMT float32 otherwise; the grouped batch
                             keeps its own products); 3 = as 2, with the two products of a step fused into
                             one kernel over one read of the digits when n <= 2048 and at most 32 lambda
                             are active; 0 = SIMT float32 */
  int group;              /* [1] tk_solve_batched: when every problem is MIXED, m >= n, BATCHED, n <= 4096,
                             N <= 64 and lsqr_tc != 1, the problems advance together in one grouped LSQR and
                             refinement (one launch per phase for all problems); 0 in any problem's options =
                             each problem solved on its own (host lanes) */
  int emulate_fp64;       /* [1] MIXED: the float64 products -- the Gram matrix, the Cholesky trailing
                             updates, and the refinement's r = b - A x and A^T r -- on the BF16 tensor
                             cores from exact integer digits (see tk_gram_emulated,
                             tk_cholesky_shifted_emulated, tk_residual) instead of the float64 pipe;
                             the same float64 accuracy.  Costs 32 bytes of workspace per element of A
                             (two sets of digit planes); 0 = float64 FMA.  The grouped batch uses the
                             emulated Gram and Cholesky and keeps its float64 refinement passes. */
  const double* x0;       /* [NULL] warm start, device N x n float64 (row i for lambdas[i]; m >= n only):
                             the solve starts from x = x0 instead of 0 and returns the same minimiser of
                             problem (1.2).  FP64: LSQR solves for the correction d in
                             min ||[A; sqrt(l) I] d - [b - A x0; -sqrt(l) x0]|| and returns x0 + d;
                             MIXED: the refinement's first round already corrects x0.  A lambda whose
                             preconditioner fails keeps x0 in X.  In tk_solve_batched each problem needs
                             its own tk_opts (n_opts = P) when x0 is set, and such problems are not
                             grouped.  The resumable state of a solve: pass a previous X back. */
} tk_opts;

/* Per-lambda report. */
typedef struct {
  int iters;          /* LSQR iterations (summed over refinement steps for MIXED) */
  int refine_steps;   /* MIXED: corrections applied; FP64: 0 */
  int istop;          /* Paige-Saunders stop reason of the last LSQR run: 1 test 1, 2 test 2, 7 maxiter */
  int64_t rank;       /* LOWRANK: truncation s_i of Algorithm 3 / 4 step 5; else 0 */
  double rnorm;       /* LSQR estimate of ||B x - b_hat|| (last run) */
  double arnorm;      /* LSQR estimate of ||M^T r|| (last run) */
  double ne_norm;     /* MIXED: ||A^T (A x - b) + lambda x|| in float64 at the last refinement check; else 0 */
  tk_status status;
} tk_info;

TK_API tk_status tk_opts_default(tk_opts* o);
TK_API const char* tk_status_str(tk_status s);
TK_API const char* tk_last_error(void);

/* Bytes of device workspace tk_solve needs for this problem, N and options. */
TK_API tk_status tk_workspace_size(const tk_problem* p, int N, const tk_opts* o, size_t* bytes);

/*
 * tk_solve -- x_{lambda_i} for i = 0..N-1 (problem (1.2); Algorithms 1, 2, 3).
 *   lambdas: host, N values > 0 (any order; results are returned in input order).
 *   X:       device, N x n float64 row-major: row i = x_{lambda_i}.
 *   info:    host, N entries (may be NULL).
 *   work:    device workspace of at least tk_workspace_size() bytes.
 * Synchronizes `stream` before returning.  Returns the worst per-lambda status
 * (TK_OK < TK_ENOCONV < TK_ENUMERIC < TK_ENOTSPD); results of the other lambdas
 * are still written.
 */
TK_API tk_status tk_solve(const tk_problem* p, const double* lambdas, int N, const tk_opts* o, void* work,
                          size_t work_bytes, void* stream, double* X, tk_info* info);

/*
 * tk_solve_batched -- P independent problems (uneven m, n) with N lambdas each
 * (the per-lambda loop of Algorithm 1 "can trivially be parallelized",
 * Section 2.1.1; here also across problems).  The problems are spread over
 * up to 8 concurrent lanes (host threads, each with its own stream joined to
 * `stream` by events, and its own slice of the workspace).
 *   o:       n_opts options, n_opts = 1 (shared) or P (one per problem, e.g.
 *            Cholesky for some problems and the low-rank form for others).
 *   lambdas: host P x N.   X[p]: device N x n_p float64.   info: host P x N (may be NULL).
 * Workspace: tk_workspace_size_batched().  Synchronizes `stream` before returning.
 */
TK_API tk_status tk_workspace_size_batched(const tk_problem* ps, int P, int N, const tk_opts* o, int n_opts,
                                           size_t* bytes);
TK_API tk_status tk_solve_batched(const tk_problem* ps, int P, const double* lambdas, int N, const tk_opts* o,
                                  int n_opts, void* work, size_t work_bytes, void* stream, double* const* X,
                                  tk_info* info);

/*
 * tk_lcurve -- the L-curve of Section 4.3 (Fig. 4): x_{lambda_i} for every
 * lambda_i, the points (||A x_i - b||, ||x_i||) of the log-log plot, and the
 * corner, where the regularization parameter of choice sits.  The paper does
 * not say how the corner is found; here it is the point of largest curvature
 * kappa = (P' Q'' - P'' Q') / (P'^2 + Q'^2)^(3/2) of P = ln ||A x - b||,
 * Q = ln ||x|| as functions of t = ln lambda (Hansen's criterion), with the
 * derivatives taken as three-point differences on the sampled grid (the end
 * points have kappa = 0 and are never the corner).
 *   Sweep 1: the N lambdas (any order; solved ascending).  Sweep 2 (N_refine
 *   > 0): N_refine parameters log-spaced strictly between the two neighbours
 *   of sweep 1's corner, solved with the same sketch, Gram matrix (or SVD of
 *   the sketch), copies and digit planes of A -- only the per-lambda
 *   factorizations and LSQR run again.  The corner is then taken on the
 *   merged grid.
 *   ||A x - b|| is formed from x in float64 (the digit residual of the mixed
 *   form with emulate_fp64, else the float64 pipe), not from LSQR estimates.
 *   N >= 3, N + N_refine <= 4096, o->x0 must be NULL.
 *   X:      device, (N + N_refine) x n float64, rows in the order of points.
 *   points: host, N + N_refine entries, ascending lambda.
 *   corner: host, index of the corner in points.
 *   work:   device, tk_lcurve_workspace_size() bytes.
 * Returns the worst per-lambda status (as tk_solve).  Synchronizes `stream`.
 */
typedef struct {
  double lambda;
  double rnorm;      /* ||A x_lambda - b|| */
  double xnorm;      /* ||x_lambda|| */
  double curvature;  /* kappa at this point (0 at both ends of the grid) */
  int iters;         /* LSQR iterations (summed over refinement rounds for MIXED) */
  tk_status status;
} tk_lcurve_point;
TK_API tk_status tk_lcurve_workspace_size(const tk_problem* p, int N, int N_refine, const tk_opts* o, size_t* bytes);
TK_API tk_status tk_lcurve(const tk_problem* p, const double* lambdas, int N, int N_refine, const tk_opts* o,
                           void* work, size_t work_bytes, void* stream, double* X, tk_lcurve_point* points,
                           int* corner);

/*
 * Handle calls -- the same solves for callers that prefer the library to own
 * the workspace (problem (1.2) as in tk_solve; no counterpart in the paper
 * beyond the solve itself).  A handle holds a stream (void* cudaStream_t,
 * NULL = legacy default stream) and the device that was current at
 * tk_create.  Each solve queries the workspace size and grows the handle's
 * device buffer with cudaMalloc when it is too small (after synchronizing the
 * stream); a later solve of the same or smaller shapes allocates nothing.
 * These are the only calls of the library that allocate device memory.
 * Solves on one handle are serialized (a mutex); use one handle per host
 * thread for concurrency.  tk_destroy synchronizes the stream, frees the
 * buffer and the handle (NULL is a no-op).  Errors as tk_solve; TK_ENOMEM if
 * cudaMalloc fails.
 */
typedef struct tk_handle tk_handle;
TK_API tk_status tk_create(tk_handle** h, void* stream);
TK_API tk_status tk_destroy(tk_handle* h);
TK_API size_t tk_handle_workspace_bytes(const tk_handle* h);
TK_API tk_status tk_handle_solve(tk_handle* h, const tk_problem* p, const double* lambdas, int N, const tk_opts* o,
                                 double* X, tk_info* info);
TK_API tk_status tk_handle_solve_batched(tk_handle* h, const tk_problem* ps, int P, const double* lambdas, int N,
                                         const tk_opts* o, int n_opts, double* const* X, tk_info* info);

/* ---- introspection calls for parity tests (each step of the path on its own) ---- */

/*
 * tk_sketch_draw -- the integer draws of the SRHT (Section 2.1.1): signs d
 * (mp values in {-1, +1}, Philox stream 0) and the s sampled rows of S
 * (ascending; the s smallest (64-bit key, row) pairs of Philox stream 1).
 *   signs: device int8[mp] (may be NULL); rows: device int64[s] (may be NULL).
 *   work:  device, at least tk_sketch_draw_workspace(mp) bytes.
 */
TK_API size_t tk_sketch_draw_workspace(int64_t mp);
TK_API tk_status tk_sketch_draw(uint64_t seed, int64_t mp, int64_t s, int8_t* signs, int64_t* rows, void* work,
                                size_t work_bytes, void* stream);

/*
 * tk_sketch_draw_static -- the same draws as tk_sketch_draw, for callers that
 * cannot allocate device memory.  The paper has no counterpart to this call.
 *
 * Some callers cannot call cudaMalloc or hand over a workspace: code that runs
 * after an "allocate once at start-up" phase has closed (real-time loops,
 * services whose memory pool owns every byte of the device), plugins invoked
 * by a host framework that gives them no allocator, or code between two
 * kernels of someone else's stream where an allocation would synchronize the
 * device.  This entry point allocates nothing: its scratch (the 64-bit
 * sampling keys) is a fixed array inside the library, TK_DRAW_STATIC_MAX_MP + 2
 * words = 8 MiB + 16 B, which every GPU that loads the library holds until
 * the process exits.
 *   mp:    1 <= mp <= TK_DRAW_STATIC_MAX_MP, else TK_EINVAL (nothing launched).
 *   signs, rows: as tk_sketch_draw (device, caller-owned, may be NULL).
 * The first call on a device looks up the array's device address; make that
 * first call before any stream capture.  The address is kept for the life of
 * the process: calling after cudaDeviceReset() (which reloads the library's
 * device code, possibly elsewhere) is not supported.  All calls share the one
 * array, so calls that overlap on the GPU (other streams, other host threads)
 * race; serialize them.  Every call synchronizes `stream` before returning.
 */
#define TK_DRAW_STATIC_MAX_MP ((int64_t)1 << 20)
TK_API tk_status tk_sketch_draw_static(uint64_t seed, int64_t mp, int64_t s, int8_t* signs, int64_t* rows,
                                       void* stream);

/*
 * tk_sketch_draw_sparse -- the integer draws of the SPARSE embedding
 * (Section 2.1.1, one nonzero element per column) and the bucket lists the
 * sketch uses: h (row of column i, int32[L]), sign (int8[L]), order (the
 * column indices sorted by h, ascending within a bucket: a stable sort,
 * int32[L]) and start (int32[s + 1]: bucket k is order[start[k] ..
 * start[k+1]-1]).  Any output may be NULL.  1 <= s <= 2^22, 1 <= L < 2^31.
 *   work: device, tk_sketch_draw_sparse_workspace(L, s) bytes.  Synchronizes `stream`.
 */
TK_API size_t tk_sketch_draw_sparse_workspace(int64_t L, int64_t s);
TK_API tk_status tk_sketch_draw_sparse(uint64_t seed, int64_t L, int64_t s, int32_t* h, int8_t* sign, int32_t* order,
                                       int32_t* start, void* work, size_t work_bytes, void* stream);

/*
 * tk_sketch_apply -- Y = X A (m >= n: Y is s x n, Algorithm 1 step 2) or
 * Y = A X (m < n: Y is m x s, Algorithm 2 step 2), float64 device output.
 * SRHT: X = sqrt(mp/s) S (H/sqrt(mp)) D with mp the next power of two of the
 * long dimension.  Gaussian: X has N(0, 1/s) entries from Philox stream 2.
 * SPARSE: one signed entry per column (see tk_sketch); Y's float64 sums run
 * over each bucket's rows in ascending order.
 * With precision MIXED (Gaussian, m >= n only) the sketch is the one the
 * mixed form uses: X and A rounded to BF16, products on the tensor cores
 * with FP32 accumulation.
 * work: device, at least tk_sketch_apply_workspace() bytes.
 */
TK_API tk_status tk_sketch_apply_workspace(const tk_problem* p, const tk_opts* o, size_t* bytes);
TK_API tk_status tk_sketch_apply(const tk_problem* p, const tk_opts* o, double* Y, void* work, size_t work_bytes,
                                 void* stream);

/*
 * tk_gram -- C = Y^T Y (Y r x c, C c x c; Algorithm 1 step 3) when
 * transpose_first != 0, else C = Y Y^T (C r x r; Algorithm 2 step 3).
 * All device float64, row-major.
 */
TK_API tk_status tk_gram(const double* Y, int64_t r, int64_t c, int transpose_first, double* C, void* stream);

/*
 * tk_gram_emulated -- C = Y^T Y as tk_gram with transpose_first, formed on
 * the BF16 tensor cores from exact integer slices of the columns of Y with
 * float64 accuracy (the Gram matrix of the mixed form with emulate_fp64; no
 * counterpart in the paper's algorithms beyond Algorithm 1 step 3 itself).
 * Only the upper triangle (j >= i) of C is defined on return.
 *   work: device, tk_gram_emulated_workspace(r, c) bytes.
 *   Returns TK_ETIMEOUT if a device-side pipeline wait gave up.
 */
TK_API size_t tk_gram_emulated_workspace(int64_t r, int64_t c);
TK_API tk_status tk_gram_emulated(const double* Y, int64_t r, int64_t c, double* C, void* work, size_t work_bytes,
                                  void* stream);

/*
 * tk_cholesky_shifted -- R_i = chol(C + lambda_i I) for i = 0..N-1
 * (Algorithm 1 step 4), upper triangular, float64.
 *   C: device n x n (symmetric, only the upper triangle is read).
 *   lambdas: host N.   R: device N x n x n (zeros below the diagonal).
 *   breakdown: host N (may be NULL): 0, or j+1 if the pivot of row j was not positive
 *              (TK_ENOTSPD), or -(j+1) if it was NaN (non-finite C: TK_ENUMERIC).
 *   work: device, tk_cholesky_workspace(n, N) bytes.
 */
TK_API size_t tk_cholesky_workspace(int64_t n, int N);
TK_API tk_status tk_cholesky_shifted(const double* C, int64_t n, const double* lambdas, int N, double* R,
                                     int* breakdown, void* work, size_t work_bytes, void* stream);

/*
 * tk_cholesky_shifted_emulated -- as tk_cholesky_shifted, with the trailing
 * updates of the blocked factorization (R_22 -= R_12^T R_12) formed on the
 * BF16 tensor cores from exact integer slices with float64 accuracy (the
 * Cholesky of the mixed form with emulate_fp64).  The diagonal blocks and the
 * panel solves stay float64.  work: tk_cholesky_emulated_workspace(n, N)
 * bytes; TK_ETIMEOUT if a device-side pipeline wait gave up.
 */
TK_API size_t tk_cholesky_emulated_workspace(int64_t n, int N);
TK_API tk_status tk_cholesky_shifted_emulated(const double* C, int64_t n, const double* lambdas, int N, double* R,
                                              int* breakdown, void* work, size_t work_bytes, void* stream);

/*
 * tk_bp2_factor -- the BP2 preconditioner of Section 4.1: R_i from a
 * Householder QR of [Y; sqrt(lambda_i) I_n] for i = 0..N-1 (Y device s x n
 * float64, row-major), upper triangular with a positive diagonal; in exact
 * arithmetic the factor tk_cholesky_shifted returns for C = Y^T Y.
 *   lambdas: host N.   R: device N x n x n (zeros below the diagonal).
 *   breakdown: host N (may be NULL): 0, k+1 for a zero column k, -(k+1) for NaN.
 *   work: device, tk_bp2_factor_workspace(s, n, N) bytes (N (s + n) n doubles).
 */
TK_API size_t tk_bp2_factor_workspace(int64_t s, int64_t n, int N);
TK_API tk_status tk_bp2_factor(const double* Y, int64_t s, int64_t n, const double* lambdas, int N, double* R,
                               int* breakdown, void* work, size_t work_bytes, void* stream);

/*
 * tk_sketch_svd -- [~, Sigma, V] = svd(Y, 'econ') of Algorithm 3 step 4 by
 * one-sided Jacobi on Y^T (no Gram matrix is formed).  Y: device s x n
 * float64 with s <= n.  sigma: device s (descending).  V: device n x s.
 * work: device, tk_sketch_svd_workspace(s, n) bytes.  sweeps: host (may be NULL).
 */
TK_API size_t tk_sketch_svd_workspace(int64_t s, int64_t n);
TK_API tk_status tk_sketch_svd(const double* Y, int64_t s, int64_t n, double* sigma, double* V, int* sweeps,
                               void* work, size_t work_bytes, void* stream);

/*
 * tk_lowrank_ranks -- Section 3.1.2 and Algorithm 3 step 5: sd_i =
 * sum_j 1/(1 + lambda_i/sigma_j^2) (float64, ascending j, no contraction) and
 * s_i = min(s, ceil(alpha * ceil(sd_i))).  sigma: device s.  lambdas: host N.
 * sd, ranks: host N.  work: device, tk_lowrank_ranks_workspace(N) bytes.
 */
TK_API size_t tk_lowrank_ranks_workspace(int N);
TK_API tk_status tk_lowrank_ranks(const double* sigma, int64_t s, const double* lambdas, int N, double alpha,
                                  double* sd, int64_t* ranks, void* work, size_t work_bytes, void* stream);

/* tk_residual -- R = b - X A^T for M rows of X and, when G is not NULL,
 * G = R A (the two float64 passes of the refinement of the mixed form:
 * residuals b - A x_l and A^T (b - A x_l); no counterpart in the paper's
 * algorithms).  emulate = 0: float64 FMA.  emulate = 1: on the BF16
 * tensor cores: every row of A (and of X) is scaled by a power of two and
 * split into 8 signed 7-bit integer slices (exact in BF16, 56 bits), the 36
 * slice products whose weight is at least 2^-56 of the row maxima are
 * accumulated exactly in FP32 over chunks of 256 values of K and then
 * exactly in int64, rounded once to float64 per output; the error is at
 * most that of a float64 GEMM (emulate = 1 requires n <= 2^27, else
 * TK_EINVAL: the exactness limit of the int64 accumulators; R A is split
 * along m so that no split holds more than 2^27 rows).
 *   p:   A (device, m x n, row stride lda, float64 or float32) and b (device, m).
 *   X:   device, M x n float64, row stride ldx >= n.
 *   R:   device, M x m float64 (row l = b - A x_l), written.
 *   G:   device, M x n float64 (row l = A^T (b - A x_l)), written; may be NULL.
 *        Emulated, A^T r is formed from the same slices of A, the row scale of A
 *        moved onto r.
 *   work: device, tk_residual_workspace(m, n, M) bytes.  Synchronizes `stream`. */
TK_API size_t tk_residual_workspace(int64_t m, int64_t n, int M);
TK_API tk_status tk_residual(const tk_problem* p, const double* X, int M, int64_t ldx, int emulate, double* R,
                             double* G, void* work, size_t work_bytes, void* stream);

/* tk_lsqr_step_products -- the two products with A of one LSQR step of the
 * mixed form (Algorithm 1 step 5 inside LSQR: A R^-1 v and A^T u), on their
 * own for parity tests of each form of them (no counterpart in the paper
 * beyond the products themselves): U <- W A^T + coef .* U (coef NULL: U <-
 * W A^T), then G = U A with the new U.  mode 0: both from the 4-digit slices
 * of A on the tensor cores, as the solve runs them while more than 16 lambda
 * are active; mode 1: the same two in one kernel over one read of A's digit
 * planes (clusters of CTAs sharing a band of rows; n <= 2048); mode 2: the
 * float32 products of at most 16 lambda from a float32 copy of A (made here
 * when A is float64), as the solve runs them for its last lambda.
 *   p: A (device, m x n, float64 or float32); W: device count x n float32;
 *   U: device count x m float32 (read when coef is not NULL, written);
 *   coef: device count float64 or NULL; G: device count x n float64, written.
 *   1 <= count <= 32.  work: tk_lsqr_step_products_workspace(m, n, count) bytes.
 *   Synchronizes `stream`; TK_ETIMEOUT if a pipeline wait gave up. */
TK_API size_t tk_lsqr_step_products_workspace(int64_t m, int64_t n, int count);
TK_API tk_status tk_lsqr_step_products(const tk_problem* p, const float* W, int count, float* U, const double* coef,
                                       double* G, int mode, void* work, size_t work_bytes, void* stream);

/* tk_autotune -- measured tile shapes for the products of the LSQR and
 * refinement passes (no counterpart in the paper: a tuning step of this
 * library).  For the problem's shape and options it runs, on the workspace
 * (tk_workspace_size() bytes, contents overwritten), every candidate tile
 * shape of the lambda-row products and every candidate split count of the
 * split-K products, for 1, 2, 4, ... and N active lambdas, times each with
 * CUDA events on `stream`, and keeps the fastest in a process-wide table that
 * every later solve of the same shapes uses (thread-safe).  A and b are read
 * but not modified.  Synchronizes the stream.  Shapes never tuned keep the
 * library's fixed rules.  tk_autotune_entries() = table size;
 * tk_autotune_clear() empties it. */
TK_API tk_status tk_autotune(const tk_problem* p, int N, const tk_opts* o, void* work, size_t work_bytes,
                             void* stream);
TK_API size_t tk_autotune_entries(void);
TK_API void tk_autotune_clear(void);
/* The table as text (one line per shape), NUL-terminated into buf (len bytes);
 * returns the length the whole text needs, NUL included. */
TK_API size_t tk_autotune_describe(char* buf, size_t len);

/* tk_wait_selftest -- the bounded device-side wait that every pipelined
 * tensor-core kernel of the library uses, on its own (no counterpart in the
 * paper: the failure path of TK_ETIMEOUT).  One thread waits on an mbarrier
 * that nothing arrives at, with a budget of budget_us microseconds (1 ..
 * 2,000,000; the kernels use 1 s per wait); the wait gives up, sets the
 * launch's error word and the call returns TK_ETIMEOUT, as a solve does when
 * one of its pipeline waits gives up.  Nothing else is in flight, so the
 * context stays usable.  TK_OK would mean the wait did not give up.
 *   work: device, at least 16 bytes.  Synchronizes `stream`. */
TK_API tk_status tk_wait_selftest(int64_t budget_us, void* work, size_t work_bytes, void* stream);

/* ---- phase profiler (tracing) ----
 * When enabled, each instrumented launch is bracketed by CUDA events on its
 * stream and tagged with its algorithmic flops and bytes: the counts of the
 * operation itself, not of the implementation -- one read of each operand and
 * one write of each result, A counted once per pass in the caller's dtype (8
 * or 4 bytes per element) whatever copy or digit planes the kernel reads.
 * impl_bytes is what the implementation moves (e.g. 8 bytes per element of A
 * for the 4 BF16 digit planes of an LSQR product, 16 for the 8 planes of a
 * float64-accurate pass, 4 for the float32 copy of a float64 A).  tk_profile_collect() waits
 * for the recorded events, fills out[TK_PHASE_COUNT] with per-phase totals
 * and clears the records.  Not for use inside CUDA graph capture. */
enum {
  TK_PHASE_SKETCH = 0,        /* Y = XA (draws, FWHT passes / Gaussian GEMM) */
  TK_PHASE_GRAM = 1,          /* C = Y^T Y */
  TK_PHASE_CHOLESKY = 2,      /* R_i = chol(C + lambda_i I), all lambda */
  TK_PHASE_SVD = 3,           /* one-sided Jacobi SVD of Y */
  TK_PHASE_PRECOND = 4,       /* R^-1 / R^-T (or low-rank) applies inside LSQR */
  TK_PHASE_AW = 5,            /* the product with A of every LSQR step (A R^-1 v for all lambda) */
  TK_PHASE_ATU = 6,           /* the product with A^T of every LSQR step */
  TK_PHASE_RES64 = 7,         /* MIXED: float64 residual b - A x */
  TK_PHASE_NE64 = 8,          /* MIXED: float64 A^T (b - A x) */
  TK_PHASE_TRINV = 9,         /* explicit R^-1 and R^-T from the float64 factors (MIXED: float32; FP64: n <= 512) */
  TK_PHASE_AW_DIGITS = 10,    /* MIXED, lsqr_tc = 2: TK_PHASE_AW on the tensor cores from digits of A */
  TK_PHASE_ATU_DIGITS = 11,   /* MIXED, lsqr_tc = 2: TK_PHASE_ATU on the tensor cores from digits of A */
  TK_PHASE_SLICE = 12,        /* MIXED, emulate_fp64: the digit planes of A (rows and columns), once per solve */
  TK_PHASE_CHOL_UPDATE = 13,  /* MIXED, emulate_fp64: the Cholesky trailing updates on the tensor cores
                                 (TK_PHASE_CHOLESKY then holds the diagonal blocks and panel solves) */
  TK_PHASE_LSQR_FUSED = 14,   /* MIXED, lsqr_tc = 3: TK_PHASE_AW_DIGITS and TK_PHASE_ATU_DIGITS of a step in one
                                 kernel over one read of the digits of A */
  TK_PHASE_COUNT = 15
};
typedef struct {
  double ms;      /* summed event time */
  double flops;   /* summed algorithmic flops */
  double bytes;   /* summed algorithmic bytes (one read of each operand, one write of each result) */
  int launches;
  double impl_bytes; /* summed bytes the implementation moves (digit planes, copies) */
} tk_phase_stats;
TK_API const char* tk_phase_name(int phase);
/* Number of kernel launches the library has issued in this process so far. */
TK_API unsigned long long tk_launch_count(void);
TK_API tk_status tk_profile_enable(int on);
TK_API tk_status tk_profile_collect(tk_phase_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* TIKHONOV_H */
