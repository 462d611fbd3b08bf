/*
 * stiles.h - C ABI of the B300 arrowhead tile Cholesky library (libstiles.so).
 *
 * The library factorizes a sparse symmetric positive-definite matrix with a
 * block-arrowhead pattern (a variable-bandwidth band plus a thin dense arrow of
 * trailing rows/columns) by the sTiles method: a fill-reducing permutation of
 * the band part (Section III.A), a tile map in Compressed Tile Storage Format
 * (Section III.B), a tile-level symbolic factorization (Section II, step 2) and
 * the left-looking sparse tile Cholesky of Algorithm 1, whose long accumulation
 * chains are summed as trees (Section IV.A, Algorithm 3).  On top of the factor
 * it computes the log-determinant and forward/backward solves.
 *
 * Conventions common to every entry point
 * ---------------------------------------
 *  - Matrices enter as the LOWER triangle including the diagonal, in
 *    compressed sparse column form: colptr[n+1] (int64, colptr[0] = 0),
 *    rowidx[nnz] (int32, strictly ascending inside a column, every row >= the
 *    column, the diagonal entry present), values[nnz] (double).
 *  - Only the pattern defines a plan; one plan serves every matrix with the
 *    same pattern (Section III.A: preprocessing pays off when many
 *    factorizations share one structure).
 *  - Pointers marked "host or device" may point to either; the library looks
 *    the pointer up with the CUDA runtime and copies host data itself.
 *  - Caller arrays are borrowed for the duration of the call only.  Handles
 *    own all memory they allocate; the matching destroy call frees it.
 *  - "stream" is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls that return results on the host synchronize that stream.
 *  - Every call returns a stiles_status.  Nothing falls back to the CPU.
 *  - The library is not thread-safe per handle: one handle must not be used
 *    from two host threads at once.
 */
#ifndef STILES_H
#define STILES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stiles_plan stiles_plan;     /* opaque: pattern analysis, host + device arrays */
typedef struct stiles_factor stiles_factor; /* opaque: device tiles of one factorization      */
typedef struct stiles_batch stiles_batch;   /* opaque: many factorizations in one launch      */

typedef enum {
  STILES_OK = 0,
  STILES_ERR_INVALID = 1,        /* bad argument or malformed CSC input                        */
  STILES_ERR_NOT_SPD = 2,        /* a pivot was <= 0 or NaN; *info holds the permuted column  */
  STILES_ERR_NOMEM = 3,          /* host or device allocation failed                          */
  STILES_ERR_CUDA = 4,           /* a CUDA runtime call failed                                */
  STILES_ERR_TIMEOUT = 5,        /* a device wait exceeded opts.spin_limit; kernels returned  */
  STILES_ERR_NOT_CONVERGED = 6,  /* iterative refinement missed refine_tol                    */
  STILES_ERR_UNSUPPORTED = 7     /* option combination not built into this library           */
} stiles_status;

enum { STILES_ORDER_NONE = 0, STILES_ORDER_RCM = 1, STILES_ORDER_AUTO = 2, STILES_ORDER_ND = 3 };
/* Arithmetic of the off-diagonal tile updates (the SYRK/GEMM terms of Algorithm 1):
 *   F64     FP64 everywhere (DFMA/DMMA).
 *   BF16    16-bit operands on the tensor cores, FP32 accumulation, FP32 tiles, FP64 diagonal
 *   F16     POTRF; solves refined in FP64 (iterative refinement, conjugate-gradient fallback).
 *   SLICED  FP64-accurate updates on the tensor cores: FP64 tiles, each finished off-diagonal
 *           tile also split into four BF16 digit slices under a per-row power-of-two scale, every
 *           slice product accumulated exactly in FP32 and the products combined in 64-bit
 *           integers; the update carries a relative error of about 2^-33 of the row scales
 *           (sqrt(a_ii)).  POTRF, TRSM and partial sums stay FP64; the factor is stored (and
 *           exported, and used by the selected inverse) like an FP64 factor.  Its solves run
 *           their sweeps on an FP32 copy of the tiles (made after the factorization) and are
 *           refined in FP64 to refine_tol like the 16-bit factors'.  32-wide sub-tiles (block 0
 *           or 32, T a multiple of 32). */
enum { STILES_PREC_F64 = 0, STILES_PREC_BF16 = 1, STILES_PREC_F16 = 2, STILES_PREC_SLICED = 3 };

typedef struct {
  int32_t tile;       /* T, the CTSF tile size.  analyze accepts any T >= 1; factorize needs a
                         multiple of 16.  Default 32.                                           */
  int32_t ordering;   /* STILES_ORDER_*: NONE keeps the input order, RCM applies partial RCM to
                         the band rows, AUTO keeps RCM only if it gives strictly fewer L tiles
                         (Section III.A, closing rule).  ND is one level of the adaptable nested
                         dissection of Section III.A: a separator as wide as the bandwidth, cut
                         at the middle of the band and moved to the end (ahead of the arrow),
                         with the second part reversed; it adds a little fill and splits the
                         elimination into two independent chains.  Default AUTO.                */
  int32_t precision;  /* STILES_PREC_*: arithmetic of the off-diagonal tile updates.  Default F64. */
  int32_t block;      /* B, the device sub-tile size: 16, 32 or 64 dividing T; 0 = min(T, 32).   */
  int32_t tree_chunk; /* accumulation terms per tree leaf (Algorithm 3); 0 = 32.  Tasks with more
                         terms are split into leaves summed by a fixed-shape tree; a sweep task
                         keeps at least its 8 newest terms, a diagonal-chain task its 3 newest. */
  int32_t tree_fanin; /* partial tiles summed per tree node; 0 = 16.                             */
  int32_t max_refine; /* iterative-refinement steps for low-precision factors; default 20.      */
  int32_t ctas_per_sm; /* resident CTAs per SM of the persistent kernels; 0 = as many as fit.  Fewer
                         CTAs leave the critical-path task more of its SM's FP64 pipes.          */
  double refine_tol;  /* target ||b - A x||_2 / ||b||_2 of a refined solve; default 1e-10.       */
  int64_t spin_limit; /* bound on any device wait, in polling iterations; default 2^24 (about 16 s).         */
} stiles_opts;

typedef struct {
  int64_t n, n_arrow, nnz;
  int64_t tile;        /* T                                                            */
  int64_t nt;          /* tiles per side, ceil(n / T)                                  */
  int64_t nnzt;        /* tiles of L (lower, diagonal included) after symbolic closure */
  int64_t block;       /* B                                                            */
  int64_t nsub;        /* B x B sub-tiles stored (nnzt * (T/B)^2)                      */
  int64_t ntasks;      /* device factorization tasks                                   */
  int64_t npairs;      /* tile-pair updates (GEMM/SYRK terms) at sub-tile granularity  */
  int64_t nscratch;    /* tree-reduction partial tiles                                 */
  int64_t flops_potrf, flops_syrk, flops_gemm, flops_trsm, flops_total; /* at tile size T */
  int64_t factor_bytes;  /* device bytes of the tile buffer (SLICED: with the digit slices and the FP32 copy) */
  int32_t ordering_used; /* STILES_ORDER_NONE, _RCM or _ND                             */
  int32_t chain_split;  /* 1: a one-matrix FP64 launch runs the diagonal chain on reserved SMs (thin DAG) */
} stiles_plan_info;

/* Fill *opts with the defaults listed above. */
void stiles_default_opts(stiles_opts* opts);

/* Symbolic analysis (host only; no GPU needed).  Section II steps 1-2, Section III.A-B.
 *   n, colptr, rowidx : lower CSC pattern, host arrays (see conventions).
 *   n_arrow           : number of trailing arrow rows/columns (0 <= n_arrow <= n); the
 *                       ordering leaves them in place at the end.
 *   opts              : may be NULL for defaults.
 *   out               : receives a new plan; destroy with stiles_plan_destroy.
 * Errors: STILES_ERR_INVALID for malformed input (unsorted or duplicate rows, upper
 * entries, missing diagonal, T < 1), STILES_ERR_NOMEM. */
stiles_status stiles_analyze(int64_t n, const int64_t* colptr, const int32_t* rowidx, int64_t n_arrow,
                             const stiles_opts* opts, stiles_plan** out);

/* Sizes, flop counts and choices of a plan. */
stiles_status stiles_plan_get_info(const stiles_plan* plan, stiles_plan_info* info);

/* The permutation, perm[new] = old (host array of n int64). */
stiles_status stiles_plan_perm(const stiles_plan* plan, int64_t* perm);

/* The tile map of L in tile-CSC form (host arrays): tcolptr[nt+1], trowidx[nnzt]; inside a
 * tile column the diagonal tile comes first, then rows ascending.  Either pointer may be NULL. */
stiles_status stiles_plan_tilemap(const stiles_plan* plan, int64_t* tcolptr, int32_t* trowidx);

/* Numeric factorization P A P^T = L L^T (Algorithm 1).
 *   values : the nnz values in the plan's CSC order, host or device.
 *   stream : CUDA stream; the call waits for it and returns the device status.
 *   inout  : *inout == NULL allocates a new factor; a factor from an earlier call on the
 *            same plan is refactorized in place (no allocation).
 *   info   : may be NULL; on STILES_ERR_NOT_SPD receives the 1-based permuted column of
 *            the first pivot that was <= 0 or NaN (LAPACK convention), else 0.
 * Errors: STILES_ERR_NOT_SPD (the factor is then invalid), STILES_ERR_TIMEOUT,
 * STILES_ERR_CUDA, STILES_ERR_NOMEM, STILES_ERR_UNSUPPORTED (T not a multiple of 16). */
stiles_status stiles_factorize(const stiles_plan* plan, const double* values, void* stream,
                               stiles_factor** inout, int64_t* info);

/* As stiles_factorize but only enqueues the work; collect the status with
 * stiles_factor_wait.  *inout must already hold a factor of this plan, or be NULL (then
 * the allocation happens here, before anything is enqueued). */
stiles_status stiles_factorize_async(const stiles_plan* plan, const double* values, void* stream,
                                     stiles_factor** inout);
stiles_status stiles_factor_wait(stiles_factor* factor, int64_t* info);

/* log det A = 2 sum_i log L_ii, reduced on the device in a fixed order; *out on the host. */
stiles_status stiles_logdet(const stiles_factor* factor, double* out);

/* Factorize and solve in one pass (FP64 plans): the forward sweep L Y = P B runs inside the
 * factorization's persistent launch (Algorithm 1's task graph plus one task per B-row block of
 * the right-hand sides, which are held transposed as tiles after the factor's; each block is
 * the same update-and-TRSM step as an off-diagonal tile), so the forward chain follows the
 * factorization instead of running after it; then the backward sweep L^T P X = Y.  The factor
 * is left as stiles_factorize leaves it (stiles_logdet, stiles_solve, ... apply).
 *   values : as stiles_factorize;  b, x : n x nrhs device arrays, column-major, leading
 *            dimension ld >= n; 1 <= nrhs <= min(B, 16); x may equal b.
 *   inout, info : as stiles_factorize.
 * Errors: STILES_ERR_INVALID (null, sizes, host arrays), STILES_ERR_UNSUPPORTED (mixed-precision
 * plan), STILES_ERR_NOT_SPD, STILES_ERR_TIMEOUT, STILES_ERR_NOMEM, STILES_ERR_CUDA. */
stiles_status stiles_factorize_solve(const stiles_plan* plan, const double* values, const double* b, double* x,
                                     int32_t nrhs, int64_t ld, void* stream, stiles_factor** inout, int64_t* info);

/* Solve A X = B for nrhs right-hand sides: X = P^T L^{-T} L^{-1} P B.
 * For a BF16/FP16 or SLICED factor the solve refines in FP64: x <- x + solve(b - A x) with the residual
 * from the original FP64 values, until ||b - A x||_2 / ||b||_2 <= opts.refine_tol for every
 * column or opts.max_refine steps (then STILES_ERR_NOT_CONVERGED, x holding the last iterate).
 * A refinement step that does not halve the residual (the factor too inaccurate for refinement
 * to converge) hands the rest of the max_refine budget to conjugate gradients on A x = b
 * preconditioned by the same factor (FP64 residuals, dot products and updates).
 *   b, x  : n x nrhs, column-major with leading dimension ld >= n, host or device (both
 *           on the same side); x may equal b.
 *   final_relres : may be NULL; else receives max over columns of ||b - A x||_2 / ||b||_2,
 *           computed in FP64 on the device from the original values.
 * Errors: STILES_ERR_INVALID, STILES_ERR_TIMEOUT, STILES_ERR_CUDA. */
stiles_status stiles_solve(const stiles_factor* factor, const double* b, double* x, int64_t nrhs, int64_t ld,
                           void* stream, double* final_relres);

/* Refinement steps the last stiles_solve on this factor needed (largest over its right-hand-side
 * chunks): 0 for FP64 factors; for BF16/FP16 factors the number of x <- x + solve(b - A x)
 * corrections after the first solve.  -1 for a NULL factor. */
int32_t stiles_factor_refine_iters(const stiles_factor* factor);

/* Of those steps, how many were preconditioned conjugate-gradient iterations (0 unless the
 * refinement stalled).  -1 for a NULL factor. */
int32_t stiles_factor_cg_iters(const stiles_factor* factor);

/* Copy the factor out as T x T column-major tiles in tile-CSC order (nnzt * T * T doubles),
 * host or device.  Rows/columns past n are padding (identity on the diagonal). */
stiles_status stiles_factor_tiles(const stiles_factor* factor, double* out, void* stream);

void stiles_plan_destroy(stiles_plan* plan);
void stiles_factor_destroy(stiles_factor* factor);
const char* stiles_strerror(stiles_status status);

/* Human-readable detail of the last error raised on the calling host thread ("" if none). */
const char* stiles_last_error(void);

/* Device time of the last factorization of `factor` (CUDA events on its stream):
 * *ms_call from the start of the call (value copy, tile zeroing, scatter) to the end of the
 * persistent kernel, *ms_kernel of the persistent factorization kernel alone.  Either may be NULL. */
stiles_status stiles_factor_timing(const stiles_factor* factor, double* ms_call, double* ms_kernel);

/* Tracing (profiling aid).  When enabled, every persistent launch of `factor` (factorization,
 * forward and backward sweeps, selected inverse) stamps each ticket with the device global
 * timer: 4 int64 per task = start, all dependencies ready, done (ns), SM id.  Tracing costs a
 * few global stores per task.  stiles_factor_get_trace copies the stamps of launch `which`
 * (0 factorization, 1 forward, 2 backward, 3 selected inverse) to the host array
 * out[4 * ntasks]; out may be NULL to query ntasks. */
stiles_status stiles_factor_set_trace(stiles_factor* factor, int32_t enable);
stiles_status stiles_factor_get_trace(const stiles_factor* factor, int32_t which, int64_t* out, int64_t* ntasks);

/* The device task list of a plan (which: 0 factorization, 1 forward, 2 backward sweep) in ticket
 * order.  Factorization tasks are 16 int32: type (0 DIAG, 1 OFF, 2 tree leaf, 3 tree node,
 * 4 CHAIN), output, diagonal sub-tile, column, pair range [pb, pe), partial range [qb, qe),
 * second output, its column, its pair range, its partial range, and the block row and block
 * column of the tile its first accumulator updates (a tree task: its owner's).  Solve tasks are
 * 8 int32: type (0 block, 2 leaf, 3 node), output block, diagonal sub-tile, column, pair
 * range, partial range.  which = 3..6 give the selected inverse's graph (Sigma L = L^{-T} on
 * the filled sub-tile map, built on the host at the first call): 3 = tasks, 8 int32 each
 * (output sub-tile; the sub-column for a diagonal task, else -1; product range [pb, pe); load
 * range [lb, le); X-product range [xb, xe)); 4 = products, 2 int32 each (Sigma sub-tile, bit 30
 * set when read transposed; U sub-tile); 5 = loads of finished terms, 3 int32 each (the Sigma
 * sub-tile whose flag guards the term; the flag value it waits for (1); term sub-tile, bit 30
 * set when the term is in W (a diagonal task's terms), else in X);
 * 6 = X products, 1 int32 each (sub-tile of U and X).  which = 7: the tasks of the
 * factorization with the forward sweep folded in (stiles_factorize_solve; 16 int32 each as for
 * which = 0; a forward block k is an OFF task with output nsub + k).  which = 8 / 9: the
 * forward / backward sweep's operand pairs, 2 int32 each (L sub-tile, block index), indexed by
 * the solve tasks' pair ranges; which = 10 / 11: their partial lists, 1 int32 each (scratch
 * block), indexed by the partial ranges.  which = 12..14 / 15..17: the forward / backward
 * sweep's release lists of a batched (ready-queue) solve launch, 1 int32 each: 12 / 15 the
 * number of distinct tasks each task reads from (ntasks entries; the tasks with none start the
 * queue), 13 / 16 the offsets of each task's readers (ntasks + 1 entries), 14 / 17 the readers
 * (each once per producer).  *ntasks receives the number of entries.  out may be NULL to query
 * ntasks.  Errors: STILES_ERR_INVALID (null plan, which out of range). */
stiles_status stiles_plan_tasks(const stiles_plan* plan, int32_t which, int32_t* out, int64_t* ntasks);

/* Number of CUDA kernels this library has launched in this process (all threads). */
int64_t stiles_kernel_launches(void);

/* log det A from factor tiles the caller already holds, allocating no device memory.
 * The paper has no counterpart: this entry point exists for callers that cannot allocate
 * device memory -- a process that has handed its whole HBM budget to its own pool or arena,
 * or code running where a cudaMalloc would block the device or is not allowed.
 *   tiles   : device, the T x T column-major tiles of L in tile-CSC order, as written by
 *             stiles_factor_tiles (caller-owned).
 *   tcolptr : device int64[ceil(n/T) + 1], the plan's tile column pointers (the diagonal tile of
 *             column k is tile tcolptr[k]).
 *   n, tile : matrix order and T.
 *   out     : device double; receives 2 sum_i log L_ii once the stream reaches this work.
 *   stream  : cudaStream_t as void* (NULL = legacy default stream); the call does not wait.
 * Scratch is one static device array inside the library holding ceil(n/T) <= 65,536 partial
 * sums (512 KB per device, held until the library is unloaded); larger problems return
 * STILES_ERR_INVALID before any launch.  The first call on each device looks up that array's
 * device address with the device current, so make it before any stream capture.  That address
 * is kept for the life of the process: a cudaDeviceReset on the device after the first call is
 * not supported (the array would be reloaded elsewhere and the kept address would be stale).
 * Every call
 * shares the array: calls that overlap on the GPU (other streams, other host threads) race and
 * must be serialized by the caller; each call rewrites all the entries it reads.  Errors:
 * STILES_ERR_INVALID (null pointer, n < 1, tile < 1, too many tile columns), STILES_ERR_CUDA. */
stiles_status stiles_logdet_tiles_noalloc(const double* tiles, const int64_t* tcolptr, int64_t n, int32_t tile,
                                          double* out, void* stream);

/* Batched factorization (Appendix A: many independent factorizations run concurrently).
 * stiles_batch_create: device arrays for `count` plans (same precision and block size; any sizes
 *   and patterns), one merged ticket list interleaving their task lists in proportion to their
 *   lengths (each matrix keeps its own topological order), and a CUDA graph of the per-call work
 *   (tile zeroing, scatter, one persistent kernel).  The plans must outlive the batch.
 * stiles_batch_factorize: values[i] = the nnz values of matrix i, host or device; the call copies
 *   them in, replays the graph on a private stream ordered after `stream`, waits, and reports per
 *   matrix: statuses[i] (OK, NOT_SPD, TIMEOUT) and infos[i] (first bad permuted column, 1-based,
 *   else 0); either array may be NULL.  Returns the first failure or OK.
 * stiles_batch_factor: a borrowed factor handle of matrix `index` for stiles_logdet, stiles_solve
 *   and stiles_factor_tiles; it lives until the batch is destroyed (do not destroy it).  It is
 *   factorized only through its batch: stiles_factorize(_async), stiles_factor_wait and
 *   stiles_factor_timing on it return STILES_ERR_INVALID.
 * stiles_batch_logdet: all log-determinants in one launch, out[count] on the host. */
stiles_status stiles_batch_create(const stiles_plan* const* plans, int32_t count, stiles_batch** out);
stiles_status stiles_batch_factorize(stiles_batch* batch, const double* const* values, void* stream,
                                     stiles_status* statuses, int64_t* infos);
stiles_status stiles_batch_factor(const stiles_batch* batch, int32_t index, stiles_factor** out);
stiles_status stiles_batch_logdet(stiles_batch* batch, double* out, void* stream);

/* Batched solves A_i x_i = b_i (Section III.D's forward and backward sweeps, every matrix of the
 * batch in one forward and one backward persistent launch; the tickets interleave the matrices'
 * sweep task lists like stiles_batch_create does for the factorization).
 *   rhs[i], x[i] : matrix i's right-hand sides and solutions, n_i x nrhs[i] column-major with
 *                  leading dimension n_i, host or device (each pointer on its own; caller-owned);
 *                  may be NULL where nrhs[i] == 0.
 *   nrhs[i]      : 0 .. 16 right-hand sides of matrix i (0 = matrix i takes no part: its tasks are
 *                  left out of the sweeps, so a call costs what its participating matrices cost).
 *   relres       : NULL, or double[count] receiving max over matrix i's columns of
 *                  ||b - A x||_2 / ||b||_2 in FP64 (computed only when requested or refining).
 *   iters        : NULL, or int32[count] receiving the refinement steps matrix i took.
 * Mixed-precision batches refine every matrix in FP64 (x <- x + solve(b - A x)) until its own
 * residual meets its plan's refine_tol or max_refine steps; the refinement sweeps still cover the
 * whole batch but only unfinished matrices take the correction.  The batch must have been
 * factorized.  The first call allocates the batch's solve workspace (room for 16 right-hand sides
 * per matrix).  The call waits for its work; one thread at a time may use a batch.  Errors: STILES_ERR_INVALID (null pointers, nrhs out
 * of range), STILES_ERR_TIMEOUT, STILES_ERR_NOT_CONVERGED (a matrix missed refine_tol; its x is
 * still the best iterate), STILES_ERR_NOMEM, STILES_ERR_CUDA, STILES_ERR_UNSUPPORTED (more than
 * 65,535 matrices). */
stiles_status stiles_batch_solve(stiles_batch* batch, const double* const* rhs, double* const* x,
                                 const int32_t* nrhs, void* stream, double* relres, int32_t* iters);
/* Device time of the persistent factorization kernel of the last stiles_batch_factorize, in ms
 * (CUDA events recorded around the kernel inside the batch's graph).  Errors: STILES_ERR_INVALID,
 * STILES_ERR_CUDA (no factorization yet). */
stiles_status stiles_batch_timing(const stiles_batch* batch, double* ms_kernel);
/* The same kernel on a caller's device clock: its start and end in ms after base_event (a
 * cudaEvent_t as void*, created with timing enabled and recorded earlier on any stream of the
 * batch's device), so that the kernels of batches run on different streams can be compared
 * (Appendix A: concurrent factorizations; the serving loop reports their overlap).  Call after
 * stiles_batch_factorize has returned.  Errors: STILES_ERR_INVALID (null argument),
 * STILES_ERR_CUDA (an event not recorded or without timing). */
stiles_status stiles_batch_kernel_window(const stiles_batch* batch, void* base_event, double* start_ms,
                                         double* end_ms);
void stiles_batch_destroy(stiles_batch* batch);

/* Marginal variances diag(A^{-1}) of an FP64 factor (the inverses that Section I lists among
 * the standard tasks on arrowhead precision matrices; INLA's marginal variances).  Computes,
 * once per factorization, the selected inverse Sigma = (P A P^T)^{-1} on the filled sub-tile map
 * of L from Sigma L = L^{-T} in reverse column order (Sigma_mk = -sum_j Sigma_mj L_jk L_kk^{-1},
 * Sigma_kk = L_kk^{-T} L_kk^{-1} - sum_j Sigma_jk^T L_jk L_kk^{-1}) in one persistent launch, then
 * writes out[i] = (A^{-1})_ii for i < n in the original order.  out: n doubles, host or device.
 * stream: NULL = the factor's stream.  The factor keeps Sigma, its transpose and the products
 * L_jk L_kk^{-1} (three arrays of its tile size) until it is destroyed.  STILES_ERR_UNSUPPORTED for a
 * mixed-precision factor; STILES_ERR_TIMEOUT if a device wait gave up. */
stiles_status stiles_marginal_variances(stiles_factor* factor, double* out, void* stream);

/* The selected inverse itself: T x T column-major tiles of Sigma on L's tile map, in tile-CSC
 * order (the layout of stiles_factor_tiles), computed as above if it is not current.  out:
 * nnzt * T * T doubles, host or device. */
stiles_status stiles_selected_inverse_tiles(stiles_factor* factor, double* out, void* stream);

/* Tile-size autotuner (Section IV.B and Appendix B: the tile size trades the extra flops of
 * padded tiles against the parallelism of the task graph).  For each candidate in tiles[ntiles]
 * the pattern is analysed with opts (opts->tile ignored); candidates whose task flops exceed 4x
 * the smallest are skipped, the others are factorized from `values` (host or device) and timed
 * with CUDA events on `stream` (best of two).  *best_tile receives the fastest; ms[i] (may be
 * NULL) its time per candidate, -1 when skipped or failed. */
stiles_status stiles_autotune(int64_t n, const int64_t* colptr, const int32_t* rowidx, int64_t n_arrow,
                              const stiles_opts* opts, const int32_t* tiles, int32_t ntiles, const double* values,
                              void* stream, int32_t* best_tile, double* ms);

/* Measured FP64 DFMA throughput of the current device in TFLOP/s (a fixed-length FMA loop
 * on every SM, timed with CUDA events), used as the roofline denominator of the FP64 path. */
stiles_status stiles_probe_fp64_peak(double* tflops);


#ifdef __cplusplus
}
#endif

#endif /* STILES_H */
