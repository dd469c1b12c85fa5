/*
 * ccg.h -- C ABI of the GB300 cooperative conjugate gradient (cCG) solver.
 *
 * Method: Bhaya, Bliman, Niedu, Pazos, "A cooperative conjugate gradient
 * method for linear systems permitting multithread implementation of low
 * complexity", arXiv:1204.0069.  Problem statement: solve A x = b for a dense
 * symmetric positive definite A (Sec. 2, Eq. "equa"), i.e. minimise
 * f(x) = x'Ax/2 - b'x, with p cooperating agents (Sec. 3.2, Algorithm 2),
 * the rank-deficiency deflation of Algorithm 3 and the stopping rule of
 * Algorithm 4.
 *
 * Conventions used by every entry point:
 *   - All matrices are row-major.  A is n x n with leading dimension lda
 *     (elements, lda >= n).  Blocks of agents (X0, X_out, V, W) are n x p
 *     row-major with leading dimension p: element (i, j) -- row i, agent j --
 *     is at [i*p + j].
 *   - Residues are gradients, r = A x - b (Sec. 2); only norms leave the
 *     library, so the sign is internal.
 *   - Pointers may be device memory (e.g. torch CUDA tensors) or host memory.
 *     Host buffers are copied to handle-owned device buffers inside the call
 *     and results are copied back; device buffers are used in place.  The
 *     caller keeps ownership of every buffer it passes; the library only
 *     borrows them for the duration of the call and never writes A or b.
 *   - Work is ordered on the handle's stream (ccg_config.stream, NULL = the
 *     legacy default stream).  Every solve returns after its results are
 *     available on the host (it synchronises that stream at the end).
 *   - Return values are status codes (ccg_status).  Nothing is thrown across
 *     the ABI.  After any error other than CCG_ERR_CUDA the handle stays
 *     usable.  A handle must not be used by two host threads at once.
 *   - Device pointers must be 8-byte aligned (16-byte aligned A with an even
 *     lda selects the vectorised A stream).
 */
#ifndef CCG_H
#define CCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CCG_MAX_AGENTS 32

/* Opaque solver handle. */
typedef struct ccg_handle_s ccg_handle;

typedef enum {
    CCG_OK = 0,              /* converged: true relative residual <= tol     */
    CCG_NOT_CONVERGED = 1,   /* warning: maxit reached; x_out = best agent   */
    CCG_ERR_INVALID = -1,    /* bad argument (sizes, tol, NULL, alignment)   */
    CCG_ERR_NOT_SPD = -2,    /* A found not positive definite (Gram pivot)   */
    CCG_ERR_NUMERICAL = -3,  /* NaN or Inf appeared                          */
    CCG_ERR_OOM = -4,        /* device allocation failed                     */
    CCG_ERR_TIMEOUT = -5,    /* an in-kernel grid barrier gave up waiting    */
    CCG_ERR_CUDA = -6        /* CUDA runtime error                           */
} ccg_status;

typedef enum {
    CCG_FP64 = 0,            /* every operation in FP64                      */
    CCG_FP32_IR = 1,         /* A in FP32, products from TF32 halves on the
                                tensor cores, FP64 refinement                 */
    CCG_BF16_IR = 2,         /* A in BF16 on the tensor cores, FP64 refinement */
    CCG_FP8_IR = 3,          /* A in FP8 E4M3 on the tensor cores, FP64 refinement */
    CCG_FP64_SLICED = 4      /* FP64 cCG (Algorithm 2, FP64 everywhere) whose block
                                products A D_k are formed on the FP8 tensor cores
                                from an error-free split of A and D_k into 14
                                slices of 4-bit integers each (the splitting of
                                Ozaki, Ogita, Oishi and Rump, Numer. Algorithms
                                59, 2012): every slice product is exact, the
                                slices are combined in FP64, and the slicing
                                (rounded to nearest) drops at most 2^-57 of each
                                row's and column's largest power of two.  The sliced copy of A (14 bytes per
                                entry) is made in each call; p <= 16.  Rows of A
                                and columns of D_k must have their largest
                                magnitude in [2^-125, 2^127]                   */
} ccg_precision;

typedef struct {
    int device;                 /* CUDA device ordinal                       */
    void* stream;               /* cudaStream_t; NULL = legacy default       */
    int precision;              /* ccg_precision                             */
    double rank_tol;            /* deflation threshold on the scaled Cholesky
                                   pivots of D'AD (Algorithm 3); default 1e-12 */
    double x0_spread;           /* initial-block spread for ccg_solve; 1.0   */
    uint64_t seed;              /* initial-block seed for ccg_solve; 0       */
    int residual_replacement;   /* 1: if the true residual at exit is above
                                   tol, restart from R = A X - b 1' (default)*/
    double barrier_timeout_ms;  /* in-kernel barrier wait limit; 10000 ms    */
    int max_ctas;               /* 0 = one CTA per SM; else an upper bound   */
    double inner_tol;           /* mixed precision: relative tolerance of each
                                   inner solve; 0 = 1e-3 (FP32), 1e-2 (BF16),
                                   1e-1 (FP8)                                 */
    int max_outer;              /* mixed precision: refinement steps; 0 = 60 */
    int explicit_residual;      /* 1: form R_{k+1} = A X_{k+1} - b 1' by a second
                                   product with A each iteration, as Algorithm 2
                                   prints it, instead of the recurrence
                                   R_{k+1} = R_k + A D_k alpha_k' (default 0).
                                   Doubles the A traffic.  CCG_FP64 only:
                                   CCG_ERR_INVALID with a mixed precision.   */
    int batch_autotune;         /* 1 (default): ccg_solve_batched times the
                                   A-pass variants on each size bucket the
                                   first time it meets it (see
                                   ccg_batch_tuning); 0: keep the table       */
    int mixed_method;           /* mixed precision: CCG_MIXED_AUTO (default:
                                   refinement for FP32; for BF16 and FP8,
                                   refinement as a probe that hands over to
                                   the preconditioned FP64 cCG when it gains
                                   less than tenfold per step),
                                   CCG_MIXED_REFINE or CCG_MIXED_PRECOND      */
    int cheb_degree;            /* CCG_MIXED_PRECOND: products with the
                                   quantised A per preconditioner application;
                                   0 = 32 (FP8, FP32) or 48 (BF16)            */
    double cheb_ratio;          /* CCG_MIXED_PRECOND: lower end of the
                                   Chebyshev interval as a fraction of the
                                   upper end (a bound on the largest
                                   eigenvalue); 0 = 1e-4                      */
} ccg_config;

/* Mixed-precision methods (ccg_config.mixed_method).
 *   CCG_MIXED_REFINE : FP64 iterative refinement x += d around inner cCG solves
 *                      on the quantised A (needs kappa(A) u_q < 1 to contract).
 *   CCG_MIXED_PRECOND: FP64 cCG (Algorithm 2, every product with the FP64 A,
 *                      formed exactly from FP8 slices for p <= 16) whose new
 *                      directions come from preconditioned residues:
 *                      D_{k+1} = Z_{k+1} + D_k beta_k', Z = q(A_q) R with q a
 *                      Chebyshev polynomial in the quantised A (cheb_degree
 *                      tensor-core products, no inner products), and
 *                      beta_k' = -(D_k'AD_k)^{-1} (AD_k)' Z_{k+1}, which keeps
 *                      D_{k+1} A-orthogonal to D_k however the preconditioner
 *                      varies (the flexible form).  Converges to the FP64
 *                      tolerance whatever kappa(A) u_q, since the quantised A
 *                      only shapes the directions.                            */
enum { CCG_MIXED_AUTO = 0, CCG_MIXED_REFINE = 1, CCG_MIXED_PRECOND = 2 };

typedef struct {
    int status;           /* ccg_status of the solve                          */
    int iterations;       /* cCG iterations = A*D_k products in the loop      */
    int agent;            /* original index of the agent returned in x_out   */
    int p_final;          /* agents still active at exit (Algorithm 3)        */
    int replacements;     /* residual replacements performed                  */
    int drops;            /* agents removed by the rank test                  */
    double relres_true;   /* ||b - A x_out|| / ||b|| computed in FP64         */
    double relres_recur;  /* min_j ||R e_j|| / ||b|| from the recurrence      */
    float device_ms;      /* device time of the solve kernel(s)               */
    int ctas;             /* CTAs of the persistent launch                    */
    int outer_steps;      /* mixed precision: refinement steps taken, or (with
                             CCG_MIXED_PRECOND) preconditioner applications;
                             iterations then counts the FP64 iterations      */
} ccg_result;

/* Fill *cfg with the defaults listed above. */
void ccg_config_init(ccg_config* cfg);

/* Create a solver handle bound to cfg->device and cfg->stream (NULL cfg =
 * defaults).  The handle owns a growable device workspace, freed by
 * ccg_destroy.  Returns CCG_ERR_INVALID on a bad device, CCG_ERR_CUDA if the
 * device cannot be initialised. */
int ccg_create(ccg_handle** out_handle, const ccg_config* cfg);

/* Release the handle and its workspace.  NULL-safe. */
int ccg_destroy(ccg_handle* handle);

/*
 * Solve A x = b with p agents (Algorithm 2 with the deflation of Algorithm 3).
 *
 *   n, A, lda : system matrix (SPD; symmetry is assumed, not checked).
 *   b         : right-hand side, n values.
 *   x0        : initial guess (n values) or NULL for zeros.  The agents'
 *               initial block is X_0 e_0 = x0 and, for j >= 1,
 *               X_0 e_j = x0 + x0_spread * u_j, where u_j(i) is uniform in
 *               [-1, 1) from SplitMix64 at counter j*n + i under cfg seed
 *               (top 53 bits).  The paper draws every agent's start at
 *               random (Sec. 5); identical starts would collapse to CG.
 *   p         : agents, 1 <= p <= min(n, 32).
 *   tol       : relative tolerance > 0.  The loop stops when
 *               min_j ||R_k e_j|| <= tol ||b|| (Algorithm 4, relative), and
 *               the solve reports CCG_OK only if the true residual of the
 *               returned agent, ||b - A x||/||b|| in FP64, is <= tol.
 *   maxit     : maximum cCG iterations (>= 0).
 *   x_out     : n values; receives the agent with the smallest residual.
 * With cfg.precision CCG_FP32_IR, CCG_BF16_IR or CCG_FP8_IR the call quantises
 * A into a handle-owned copy and runs ccg_solve_mixed (see there).
 *   res       : optional result record (host memory).
 * Errors: CCG_ERR_INVALID (n < 1, p out of range, tol <= 0, maxit < 0,
 * lda < n, NULL pointer), CCG_ERR_NOT_SPD, CCG_ERR_NUMERICAL, CCG_ERR_OOM,
 * CCG_ERR_TIMEOUT, CCG_ERR_CUDA.  b = 0 returns x = 0 after 0 iterations.
 */
int ccg_solve(ccg_handle* handle, int64_t n, const double* A, int64_t lda,
              const double* b, const double* x0, int p, double tol, int maxit,
              double* x_out, ccg_result* res);

/*
 * As ccg_solve, with the initial block given explicitly (Algorithm 2, "choose
 * X_0"): X0 is n x p row-major.  If X_out is not NULL it receives the final
 * block (n x p row-major): column j holds agent j's last iterate (for an
 * agent removed by the rank test, its iterate when it was removed).
 */
int ccg_solve_block(ccg_handle* handle, int64_t n, const double* A, int64_t lda,
                    const double* b, const double* X0, int p, double tol,
                    int maxit, double* x_out, double* X_out, ccg_result* res);

/*
 * One block product of Table 1, rows 1-3, with the same device code the
 * solver runs each iteration: W = A V (n x q), and, if M / G are not NULL,
 * the q x q Grams M = V' W (symmetrised, (M + M')/2) and G = U' V (U given,
 * n x q, may equal V).  V, U, W are n x q row-major; M, G are q x q
 * row-major.  1 <= q <= 32.  Errors as for ccg_solve.
 */
int ccg_block_product(ccg_handle* handle, int64_t n, const double* A, int64_t lda,
                      const double* V, const double* U, int q, double* W,
                      double* M, double* G, float* device_ms);

/*
 * Self-test of the in-kernel grid barrier's wait limit: launches the
 * persistent kernel with a barrier that expects one more CTA than the grid
 * holds, so every wait gives up after timeout_ms and the kernel returns.
 * Returns CCG_ERR_TIMEOUT when the limit works (the handle stays usable).
 */
int ccg_selftest_barrier_timeout(ccg_handle* handle, double timeout_ms);

/* ---- Mixed precision: a quantised copy of A on the tensor cores ---------- */

/* Storage formats of a quantised copy of A. */
typedef enum {
    CCG_LOWP_BF16 = 0,      /* bfloat16, round to nearest (2 bytes/entry)      */
    CCG_LOWP_FP8_E4M3 = 1,  /* FP8 E4M3, one FP32 scale per row: A_ij ~= s_i q_ij,
                               s_i = max_j |A_ij| / 448 (1 byte/entry)        */
    CCG_LOWP_FP32 = 2,      /* FP32 (4 bytes/entry); the tensor cores form
                               (A_hi + A_lo)(D_hi + D_lo) from TF32 halves
                               (A_lo = A - tf32(A)), about 2^-21 relative
                               error per product                              */
    CCG_LOWP_FP64_SLICED = 3 /* A_ij = 2^e_i sum_{s<14} q_s 16^-(s+1) with
                               integers q_s in [-15, 15] stored as FP8 E4M3
                               (14 bytes/entry, see CCG_FP64_SLICED); the
                               block product is FP64-accurate; q <= 16        */
} ccg_lowp_format;

/* Opaque quantised matrix (device memory owned by the object). */
typedef struct ccg_lowp_matrix_s ccg_lowp_matrix;

/*
 * Quantise A (n x n, lda; device or host FP64) into `format` on the handle's
 * device and stream.  Rows are padded to a multiple of 128 entries.  The
 * object keeps no reference to A.  Errors: CCG_ERR_INVALID (bad format, n < 1,
 * lda < n, NULL), CCG_ERR_OOM, CCG_ERR_CUDA.
 */
int ccg_lowp_create(ccg_handle* handle, int format, int64_t n, const double* A, int64_t lda,
                    ccg_lowp_matrix** out);

/*
 * Low-precision block product of Table 1, row 1: W = A_lp V for V n x q
 * (row-major FP64, 1 <= q <= 32), W n x q row-major FP64.  V is rounded to
 * BF16 (BF16 A) or split into two FP8 E4M3 terms with one scale per column
 * (FP8 A); products accumulate in FP32 on the tensor cores.  device_ms
 * (optional) receives the device time of the block product kernels.
 * Returns CCG_ERR_TIMEOUT if an in-kernel wait gave up.
 */
int ccg_lowp_block_product(ccg_handle* handle, const ccg_lowp_matrix* m, const double* V, int q,
                           double* W, float* device_ms);

/*
 * Mixed-precision solve of A x = b (FP64 result) with the quantised copy `lpA`
 * of A on the tensor cores, by cfg.mixed_method:
 *
 * CCG_MIXED_REFINE: iterative refinement in FP64 around inner
 * cCG solves on lpA.  Each step computes the FP64 residual r = b - A x, solves
 * A_lp d = r with p agents to the relative tolerance cfg.inner_tol (the
 * recurrence residual decides), and updates x += d.  The solve stops when
 * ||b - A x|| / ||b|| <= tol (CCG_OK), or returns the best x with
 * CCG_NOT_CONVERGED when maxit inner iterations or cfg.max_outer steps are
 * used up, two steps in a row fail to improve the residual, or an inner solve
 * breaks down (A_lp not positive definite) -- refinement contracts only when
 * A_lp approximates A well enough for the system's conditioning.
 * res->iterations counts inner iterations, res->outer_steps refinement steps.
 *
 * CCG_MIXED_AUTO: refinement for FP32.  For BF16 and FP8, refinement with
 * inner solves of at most 200 iterations, as long as each step gains at least
 * tenfold; otherwise the preconditioned solve below continues from the best x
 * (res->iterations and res->outer_steps then add both parts).
 *
 * CCG_MIXED_PRECOND: FP64 cCG on A (Algorithm 2 with
 * Algorithm 3's deflation and Algorithm 4's stop rule and residual check) in
 * which each new direction block is built from Z_{k+1} = q(A_lp) R_{k+1}, a
 * Chebyshev polynomial of cfg.cheb_degree products with A_lp on the interval
 * [cfg.cheb_ratio h, h], h a bound on the largest eigenvalue of A_lp (its
 * largest absolute row sum).  The block products of the FP64 iteration are
 * formed exactly from FP8 slices of A (as CCG_FP64_SLICED) for p <= 16, on the
 * FP64 pipe above.  res->iterations counts FP64 iterations, res->outer_steps
 * preconditioner applications.
 *
 * x0 may be NULL (zeros).  res->relres_true is the FP64 relative residual of
 * x_out.  lpA must have been made from this A.
 */
int ccg_solve_mixed(ccg_handle* handle, const ccg_lowp_matrix* lpA, int64_t n, const double* A,
                    int64_t lda, const double* b, const double* x0, int p, double tol,
                    int maxit, double* x_out, ccg_result* res);

/* Bytes of device memory held by the quantised matrix (entries + scales). */
int64_t ccg_lowp_bytes(const ccg_lowp_matrix* m);

/* Free the quantised matrix.  NULL-safe. */
int ccg_lowp_destroy(ccg_lowp_matrix* m);

/* ---- Many independent systems in one launch ------------------------------ */

/*
 * Solve `count` independent SPD systems A_i x_i = b_i, each with p agents
 * (Algorithm 2 with the deflation of Algorithm 3, FP64), in one persistent
 * launch: every CTA takes the next system from a queue ordered largest
 * first and solves it alone, so systems of uneven size keep all SMs busy.
 *
 *   n[i]      : sizes (host array), 1 <= p <= n[i].
 *   A         : device buffer, systems packed one after another: A_i is
 *               n_i x n_i row-major with leading dimension ld_i = n_i rounded
 *               up to even, starting at element sum_{j<i} n_j ld_j.
 *   b, x_out  : device buffers, b_i and x_i packed at element sum_{j<i} n_j.
 *   status, iterations, relres : optional host arrays of `count` entries
 *               (per-system ccg_status, iterations, true relative residual).
 *   summary   : optional: status = CCG_OK if every system converged, else the
 *               first non-OK status; iterations = sum over systems;
 *               device_ms = time of the launch; ctas = grid size.
 * Each system uses the handle's configuration (x0 = 0 with the initial-block
 * spread, residual replacement, rank tolerance).
 *
 * Precision (handle configuration): CCG_FP64 solves each system in FP64.
 * CCG_FP32_IR solves each system by FP64 iterative refinement (r = b - A x
 * and the update of x in FP64) around inner cCG solves on an FP32 copy of
 * A_i whose block product runs on the FP32 pipe; the copy is made inside
 * the launch.  The inner tolerance is cfg.inner_tol (0 = 1e-5), at most
 * cfg.max_outer refinement steps (0 = 30); refinement stops early when two
 * steps in a row do not reduce the true residual, and each x_i is the best
 * iterate.  relres[i] is the true relative residual of that x_i;
 * iterations[i] counts inner cCG iterations; summary->outer_steps is the
 * largest number of refinement steps of any system.  CCG_BF16_IR and
 * CCG_FP8_IR are not offered here (CCG_ERR_INVALID).
 *
 * Errors: CCG_ERR_INVALID (count < 0, bad sizes, host pointers for A, b,
 * x_out, unsupported precision), CCG_ERR_OOM, CCG_ERR_CUDA.
 */
int ccg_solve_batched(ccg_handle* handle, int64_t count, const int64_t* n, const double* A,
                      const double* b, int p, double tol, int maxit, double* x_out,
                      int* status, int* iterations, double* relres, ccg_result* summary);

/*
 * A-pass variant table of the batched solver (no counterpart in the paper:
 * an implementation tuning).  Systems fall into size buckets
 * [2^(k+5), 2^(k+6)), k = 0..7 (the last bucket open-ended); each bucket
 * uses one shape of the FP64 block product: 0 tiled (a k-chunk of the operand
 * staged in shared memory for the CTA's rows), 1 per-warp rows with eight
 * 16-byte loads per lane per step (512 columns), 2 per-warp rows with two
 * loads per step (128 columns, for short rows).  With cfg.batch_autotune the
 * first batched call that meets a bucket times the variants on up to two
 * systems per CTA of that bucket (6 iterations each) and keeps the fastest;
 * the table lives in the handle, per precision (CCG_FP64 / CCG_FP32_IR) and
 * agent bucket (p rounded up to a power of two).  Variants 1 and 2 exist for
 * p <= 8, variant 1 not for p <= 2.
 *   set = 0: variant[8] receives the table (-1 = not tuned yet).
 *   set = 1: the table is set from variant[8] (and counts as tuned).
 * Errors: CCG_ERR_INVALID (bad p or precision, a variant not offered).
 */
int ccg_batch_tuning(ccg_handle* handle, int p, int precision, int* variant, int set);

/* ---- Serving: a stream of solve requests --------------------------------- */

/* Opaque server. */
typedef struct ccg_server_s ccg_server;

typedef struct {
    int device;             /* CUDA device                                      */
    int workers;            /* concurrent solves (worker threads, streams); 8   */
    int precision;          /* ccg_precision of every solve; CCG_FP64            */
    double budget_bytes;    /* device bytes the admitted requests may hold; 150e9 */
    int ctas_per_worker;    /* SM share of one solve; 0 = SMs / workers          */
    int slots;              /* 0 (default): worker threads as above.  > 0: one
                               persistent serving kernel with `slots` slots of
                               SMs / slots CTAs each (continuous batching, see
                               ccg_server_create); CCG_FP64 only             */
    int64_t max_n;          /* slots mode: largest n accepted; the slots' X, R,
                               D and A D blocks are allocated for it at
                               creation; 0 = 16384                          */
    int max_p;              /* slots mode: largest p accepted (8 or 32); 0 = 8 */
} ccg_server_config;

typedef struct {
    int64_t id;             /* the id given to ccg_server_submit                */
    int status;             /* ccg_status of the solve                          */
    int iterations;
    int outer_steps;        /* mixed precision: refinement steps               */
    int worker;             /* worker, or slot in slots mode                    */
    int ctas;
    double relres_true;     /* ||b - A x|| / ||b|| in FP64                       */
    double submit_ms;       /* server clock (ms since ccg_server_create)        */
    double admit_ms;        /* admitted: a worker and the memory were free     */
    double done_ms;         /* solution in x_out                               */
} ccg_server_result;

typedef struct {
    int64_t queued, completed;
    int in_flight, peak_in_flight, ctas_per_worker;
    double reserved_bytes, peak_reserved_bytes, now_ms;
} ccg_server_stats_t;

/* Fill *cfg with the defaults listed above. */
void ccg_server_config_init(ccg_server_config* cfg);

/*
 * Start a server.
 *
 * Worker mode (slots = 0): `workers` threads, each with its own handle and
 * stream and a fixed share of the SMs.  Requests are admitted in arrival
 * order, first fit: a free worker takes the oldest queued request whose
 * device memory (its matrix, kept resident for the request's lifetime, plus
 * workspace and, for mixed precision, the quantised copy) fits in the budget
 * left by the running requests.  Requests admitted while others run execute
 * concurrently on the device.
 *
 * Slots mode (slots > 0, CCG_FP64): one persistent kernel serves every
 * request.  Its grid is split into `slots` slots of SMs / slots CTAs; each
 * slot keeps its cCG state and its X, R, D, A D blocks resident (allocated
 * once, for max_n and max_p) and takes the next admitted request from a ring
 * in host memory that the server appends to while the kernel runs, so a
 * request starts as soon as a slot is free and the work of all slots runs in
 * the same launch (continuous batching; no allocation and no launch per
 * request).  Admission is first fit in arrival order under the budget (the
 * request's matrix).  The kernel ends after a short idle time and is
 * launched again when requests arrive.  A must be 16-byte aligned with an
 * even lda, n <= max_n, p <= max_p.
 *
 * In both modes a request's grid depends only on its size and the share (or
 * slot), so its result does not depend on what else is running.
 */
int ccg_server_create(const ccg_server_config* cfg, ccg_server** out);

/*
 * Queue the solve of A x = b (device pointers, A n x n with lda; x_out n
 * values) with p agents to relative tolerance tol (ccg_solve semantics, x0 =
 * 0).  The buffers must stay valid until the request's result is polled.
 * Returns at once: CCG_OK, CCG_ERR_INVALID, or CCG_ERR_OOM if the request can
 * never fit the budget.
 */
int ccg_server_submit(ccg_server* server, int64_t id, int64_t n, const double* A, int64_t lda,
                      const double* b, double* x_out, int p, double tol, int maxit);

/* Move up to `max` finished results into out[], waiting up to wait_ms for the
 * first one; returns how many were written. */
int ccg_server_poll(ccg_server* server, ccg_server_result* out, int max, int wait_ms);

/* Current queue, in-flight, completed and memory figures. */
int ccg_server_stats(ccg_server* server, ccg_server_stats_t* stats);

/* Finish the queued and running requests, then stop.  NULL-safe. */
int ccg_server_destroy(ccg_server* server);

/* ---- Solve without any device allocation --------------------------------- */

/* Largest n * p accepted by ccg_solve_noalloc. */
#define CCG_NOALLOC_MAX_NP 131072

/*
 * ccg_solve without a handle and without allocating: no cudaMalloc, no
 * cudaFree, no pinned host buffer, no events.  The paper has no counterpart;
 * this entry exists for callers that cannot allocate device memory on the
 * fly -- for instance a process whose device memory is owned by its own
 * pool allocator or budget, or a latency-bound loop that cannot afford the
 * synchronisation an allocation may cause.
 *
 * All pointers (A, b, x0, x_out) must be device memory on `device`; host
 * pointers are rejected.  The solve runs on `stream` (NULL = legacy default
 * stream) with the default configuration of ccg_config_init (x0 spread 1,
 * seed 0, rank_tol 1e-12, residual replacement on, 10 s barrier limit) and
 * returns after the result is on the host.  res->device_ms is 0 (no events).
 *
 * Scratch: one file-scope device array of about 10.7 MB (5 blocks of
 * CCG_NOALLOC_MAX_NP doubles, per-CTA partial sums for up to 160 CTAs and the
 * solver state), held by every GPU that loads the library until the process
 * exits.  The first call on a device looks up the array's device address (a
 * runtime symbol lookup); make that first call before any stream capture.
 * Every call on a device shares the same array, so calls that overlap on the
 * GPU race: serialise them (one stream, or wait between calls).  The solver
 * state is cleared on every call.
 *
 * Errors: CCG_ERR_INVALID for arguments ccg_solve rejects, for host
 * pointers, and for n * p > CCG_NOALLOC_MAX_NP; otherwise as ccg_solve.
 */
int ccg_solve_noalloc(int device, void* stream, int64_t n, const double* A, int64_t lda,
                      const double* b, const double* x0, int p, double tol, int maxit,
                      double* x_out, ccg_result* res);

/* Name of a status code ("CCG_OK", ...). */
const char* ccg_status_string(int status);

/* Library version string. */
const char* ccg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CCG_H */
