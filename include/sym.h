/*
 * sym.h — C ABI of the GB300 supernodal Cholesky library (numeric phase of decoupled sparse
 * Cholesky, after Sympiler, arXiv 1705.06575).
 *
 * The library splits the work the way the paper does (Sec. 2.2, Sec. 3.2): a host-side symbolic
 * inspector runs once per sparsity pattern (sym_analyze*), and CUDA kernels re-run the numeric
 * factorization A = L L^T (sym_factor*) and the triangular solves (sym_solve*) for every new set
 * of values on that pattern.
 *
 * Conventions for every call:
 *   - A is symmetric positive definite; only its lower triangle is passed, in compressed sparse
 *     column form, 0-based: Ap (int64, n+1 entries), Ai (int32, Ap[n] entries, strictly
 *     increasing within a column, the diagonal present and first), Ax (float64, same order as Ai).
 *     This is the input form of Sec. 2.1 / Sec. 4.2 of the paper.
 *   - Return value 0 is success; negative values are the SYM_ERR_* codes below. No call aborts
 *     or traps; a failed call leaves the handle usable unless it says otherwise.
 *   - The caller keeps ownership of every pointer it passes. sym_analyze copies the pattern.
 *     The handle owns the factor L (device memory) and its plan; sym_free releases both.
 *   - Device pointers are plain CUDA device addresses of the current device (for example
 *     torch.Tensor.data_ptr()). "_host" variants take host pointers and copy inside.
 *   - Work is issued on the handle's stream (sym_set_stream; default: the legacy default
 *     stream). Calls on one handle are not thread-safe; different handles are independent.
 */
#ifndef SYM_H_
#define SYM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define SYM_OK 0
#define SYM_ERR_INVALID -1 /* bad pattern, permutation, option or argument */
#define SYM_ERR_NOT_SPD -2 /* non-positive or NaN pivot; see sym_last_error_column */
#define SYM_ERR_CUDA -3    /* a CUDA runtime call failed (message: sym_last_error_string) */
#define SYM_ERR_OOM -4     /* device or host allocation failed */
#define SYM_ERR_STATE -5   /* call out of order (solve before factor, host-only handle) */
#define SYM_ERR_TIMEOUT -6 /* a bounded device wait ran out */
#define SYM_ERR_LIMIT -7   /* a size exceeds a documented limit */
#define SYM_ERR_NO_CONVERGENCE -8 /* refinement stopped at its iteration limit above tolerance */

/* Orderings for sym_analyze_perm. */
#define SYM_ORDER_NATURAL 0 /* identity (then etree postorder) */
#define SYM_ORDER_GIVEN 1   /* the caller's perm (then etree postorder) */
#define SYM_ORDER_AUTO 2    /* computed from the pattern alone (the paper takes the ordering as
                               given; this is the library's addition): an approximate minimum-degree
                               ordering (quotient graph, supervariables, element absorption and the
                               approximate external degree of Amestoy, Davis and Duff) and a nested
                               dissection by breadth-first level structures (George and Liu; parts
                               of at most 96 nodes by minimum degree) are both computed and the one
                               whose factor has fewer flops (sum c_j^2) is kept; then etree
                               postorder. perm is ignored. */
/* How the ordering of a handle was obtained (sym_stats.ordering_method). */
#define SYM_ORDER_METHOD_MD 3 /* SYM_ORDER_AUTO chose minimum degree */
#define SYM_ORDER_METHOD_ND 4 /* SYM_ORDER_AUTO chose nested dissection */

/* Precision of the factor (sym_options.precision). */
#define SYM_PREC_FP64 0  /* FP64 factor and FP64 solves (the plain path) */
#define SYM_PREC_MIXED 1 /* FP32 factor (FP32 storage and arithmetic; the external updates of
                            64-wide tiles run on the tensor cores as TF32 splits, see
                            SYM_FLAG_NO_TENSOR_CORES); solves refined in FP64 by conjugate
                            gradients preconditioned with the FP32 factor, to a normwise backward
                            error <= the refinement tolerance (default 1e-12) */

/* Option flags. */
#define SYM_FLAG_HOST_ONLY 1u /* run the inspector only; no device memory, no factor/solve */
#define SYM_FLAG_NO_GRAPHS 2u /* launch kernel by kernel instead of replaying CUDA graphs */
#define SYM_FLAG_ONE_STREAM 4u /* run every factor launch on the handle's stream in list order
                                  (no lookahead overlap; results are identical either way) */
#define SYM_FLAG_NO_TENSOR_CORES 8u /* SYM_PREC_MIXED: external updates in FP32 on the SIMT
                                       pipes instead of tcgen05 TF32 splits (x = hi + lo, all four
                                       partial products accumulated in FP32) */
#define SYM_FLAG_NO_FUSED_LEVELS 16u /* run the launches of levels of narrow supernodes apart
                                        instead of as one fused launch per level and phase
                                        (SYM_EXPORT_BATCH_PANEL, _FWD_PANEL, _BWD_PANEL), for
                                        single matrices and batches */

typedef struct sym_handle_s *sym_handle;

/* Inspector options. nrelax/zrelax_permille set the relaxed-amalgamation rule: supernode S is
 * merged into the next supernode P when parent(last(S)) = last(S)+1 and, with m the merged column
 * count and z the fraction of explicit zeros in the merged trapezoid,
 *   m <= nrelax[0], or (m <= nrelax[1] and z <= zrelax[0]/1000),
 *   or (m <= nrelax[2] and z <= zrelax[1]/1000), or z <= zrelax[2]/1000;
 * passes repeat until nothing merges. The paper disables amalgamation (Sec. 4.1); set
 * amalgamate = 0 for fundamental supernodes only (Sec. 3.2). */
typedef struct {
  int32_t ordering;            /* SYM_ORDER_* */
  int32_t amalgamate;          /* 1 (default) or 0 */
  int32_t nrelax[3];           /* default 4, 16, 48 */
  int32_t zrelax_permille[3];  /* default 800, 100, 50 */
  uint32_t flags;              /* SYM_FLAG_* */
  int32_t precision;           /* SYM_PREC_* (default SYM_PREC_FP64) */
  int32_t reserved[7];
} sym_options;

/* Statistics of an analyzed pattern (sym_info). */
typedef struct {
  int64_t n;
  int64_t nnz_a;            /* entries of the lower triangle of A */
  int64_t nnz_l;            /* entries of L on its exact pattern (Eq. 1), diagonal included */
  int64_t storage_l;        /* doubles held for L (supernodal panels, padding included) */
  double flops;             /* sum_j c_j^2 over the exact pattern: the factor's useful flops */
  double solve_flops;       /* per right-hand side: 2 * (2 nnz_l - n) */
  int32_t nsuper_fund;      /* fundamental supernodes */
  int32_t nsuper;           /* supernodes after amalgamation */
  int32_t nlevels;          /* levels of the supernodal tree */
  int32_t max_ncols;        /* widest supernode */
  int64_t npairs;           /* (descendant, ancestor) update pairs */
  int64_t nlaunch_factor;   /* kernel launches per sym_factor (one matrix, current forms) */
  int64_t nlaunch_solve;    /* kernel launches per sym_solve (FP64 factors: also per pass of up to
                               8 right-hand sides of sym_solve_multi; FP32: passes of one or two) */
  double analyze_seconds;   /* host time of the inspector */
  int64_t device_bytes;     /* device memory held by the handle */
  int64_t upd_tasks;        /* tiles receiving descendant updates */
  int64_t upd_entries;      /* (tile, descendant) update entries */
  int64_t dense_tasks;      /* POTRF + TRSM + GEMM + inverse tile tasks */
  double exec_flops;        /* factor flops the kernels execute (explicit zeros included) */
  double update_flops;      /* the part of `flops` that descendant updates (SYM_KIND_UPDATE)
                               carry: column k updates column j in another supernode with
                               2 |{i in L_k : i >= j}| flops, summed over the exact pattern */
  int32_t ordering_method;  /* SYM_ORDER_NATURAL, SYM_ORDER_GIVEN, SYM_ORDER_METHOD_MD or _ND */
  int32_t reserved0;
  double ordering_flops_md; /* SYM_ORDER_AUTO: factor flops under minimum degree, else 0 */
  double ordering_flops_nd; /* SYM_ORDER_AUTO: factor flops under nested dissection, else 0 */
} sym_stats;

/* Fill *opt with the defaults (SYM_ORDER_GIVEN with a NULL perm means natural order). */
int sym_options_default(sym_options *opt);

/* Inspector with default options and the natural order (plus etree postorder). Same as
 * sym_analyze_perm(n, Ap, Ai, NULL, NULL, out). Host pointers. */
int sym_analyze(int64_t n, const int64_t *Ap, const int32_t *Ai, sym_handle *out);

/* Inspector (Sec. 3.2 of the paper; amalgamation and the level schedule are this library's
 * additions). perm (nullable, host, n entries) is a fill-reducing ordering: perm[k] is the
 * original index placed at position k. The final ordering is perm composed with the postorder
 * of the elimination tree. Steps: validate, permute, etree, postorder, column counts,
 * fundamental supernodes, amalgamation, supernodal row structure, descendant lists (the block
 * prune-set), relative row maps, level schedule, kernel task lists; then one upload of the
 * plan to the current device (unless SYM_FLAG_HOST_ONLY). Errors: SYM_ERR_INVALID for a bad
 * pattern or permutation, SYM_ERR_LIMIT when the forward solve's push buffer would hold 2^31
 * entries or more (see SYM_EXPORT_CONTRIB), SYM_ERR_OOM, SYM_ERR_CUDA. On error *out is NULL. */
int sym_analyze_perm(int64_t n, const int64_t *Ap, const int32_t *Ai, const int32_t *perm,
                     const sym_options *opt, sym_handle *out);

/* Inspector with one amalgamation rule per fundamental supernode (the learned schedule's
 * per-supernode choice; the paper tunes such thresholds by hand, Sec. 2.4 and Sec. 4.2). rules:
 * nrules records of 7 int32 {amalgamate, nrelax[3], zrelax_permille[3]} (amalgamate = 0 never
 * merges; otherwise the rule of sym_options). fund_rule: nfund rule indices, one per fundamental
 * supernode of this pattern under this ordering (SYM_EXPORT_FSUPER of a handle analyzed with the
 * same pattern, perm and ordering); a candidate merge of S into the next supernode follows the
 * rule of the fundamental supernode that holds the last column of S. opt's own amalgamation
 * fields are ignored. Errors as sym_analyze_perm, and SYM_ERR_INVALID for a bad rule, an index out
 * of range or an nfund that does not match. */
int sym_analyze_rules(int64_t n, const int64_t *Ap, const int32_t *Ai, const int32_t *perm,
                      const sym_options *opt, int32_t nrules, const int32_t *rules, int64_t nfund,
                      const int32_t *fund_rule, sym_handle *out);

/* Use this CUDA stream (a cudaStream_t passed as void*) for all later work of the handle. */
int sym_set_stream(sym_handle h, void *stream);

/* Launching. sym_factor* and sym_solve_multi capture their launch sequence in a CUDA graph on
 * first use (on a private stream) and replay it on the handle's stream while the device
 * pointers and sizes stay the same (a change re-captures). SYM_FLAG_NO_GRAPHS, or profiling,
 * launches kernel by kernel. */

/* Numeric factorization (Sec. 3.2: supernodal left-looking Cholesky; VS-Block turns each
 * supernode into a dense POTRF of its diagonal block and TRSMs of the rows below, and VI-Prune
 * restricts the update to the descendants in the prune-set). Ax: DEVICE pointer, Ap[n] float64
 * values in the order of the Ai given to the inspector. Enqueues the scatter of A into the
 * supernodal panels and the level-by-level update / POTRF / TRSM kernels on the handle's stream,
 * then waits for them and reads the pivot status. Returns SYM_ERR_NOT_SPD when a pivot is not
 * positive (or is NaN); sym_last_error_column then gives the first failing column in the
 * caller's numbering and the factor is not usable. Returns SYM_ERR_TIMEOUT (factor not usable)
 * when a tensor-core update of SYM_PREC_MIXED waited about a second for its MMAs in vain. */
int sym_factor(sym_handle h, const double *Ax);

/* As sym_factor but returns right after enqueueing (no wait, no status check). Call
 * sym_status afterwards to wait and read the pivot status. */
int sym_factor_async(sym_handle h, const double *Ax);

/* Batched refactorization (this library's addition: many matrices with the pattern of the handle
 * factored together, every kernel launch covering all of them, the launch sequence replayed as
 * one CUDA graph). Ax: DEVICE pointer to nbatch value arrays, matrix b at Ax + b * stride
 * (stride >= nnz(A)); 1 <= nbatch <= 65535. The handle grows its factor storage to nbatch
 * matrices on demand (one allocation, kept). Waits like sym_factor; SYM_ERR_NOT_SPD when any
 * matrix fails (sym_batch_error_columns gives every matrix's first failing column, or -1). */
int sym_factor_batch(sym_handle h, int32_t nbatch, const double *Ax, int64_t stride);

/* Per-matrix first failing columns (caller's numbering; -1 when fine) of the last factorization,
 * nbatch entries (1 after sym_factor). */
int sym_batch_error_columns(sym_handle h, int64_t *cols);

/* Solve for the first nbatch matrices of the last batch: matrix b's nrhs right-hand sides are
 * column-major at B + b * bstride (ld ldb), its solutions at X + b * xstride (ld ldx). DEVICE
 * pointers; bstride >= ldb * nrhs and xstride >= ldx * nrhs when nbatch > 1. FP64 factors solve
 * all matrices in the same launches; a mixed-precision handle refines each matrix in turn. */
int sym_solve_batch(sym_handle h, int32_t nbatch, int32_t nrhs, const double *B, int64_t ldb,
                    int64_t bstride, double *X, int64_t ldx, int64_t xstride);

/* Autotuner (this library's addition; the paper picks its variants by hand, Sec. 2.4): for a
 * batch of nbatch matrices (arguments as sym_factor_batch; nbatch = 1: one matrix, Ax as for
 * sym_factor), every factor launch that has two kernel forms is timed in both with CUDA events
 * over reps kernel-by-kernel factorizations of the given values, and the faster form is stored
 * in the plan for every later factorization of the handle (the captured graphs are rebuilt).
 * Forms: in a batch, FP64 updates run with the lanes of a warp on several matrices or one warp
 * per (tile, matrix) (small tiles, and full tiles with small entries) or one CTA per tile and
 * matrix (full tiles with large entries); small-tile POTRF, TRSM and TRTRI one warp per (tile,
 * matrix), four matrices per CTA, or one CTA per tile and matrix; for one
 * matrix, FP64 updates of tiles with many entries run on a thread-block cluster per tile or one
 * CTA per tile, FP32 updates of full tiles on the tensor cores or the SIMT pipes, and small-tile
 * POTRF and TRTRI one CTA or one warp per tile. A batch's levels of narrow supernodes
 * (SYM_EXPORT_BATCH_PANEL) are first timed as one fused launch against their separate POTRF,
 * TRSM and TRTRI launches (the sums of the level's launch times), the faster kept; the launches
 * of a level kept separate then have their forms tuned like the others. The
 * per-kernel profile totals are left as they were. *tuned: fused levels plus launches with two
 * forms; *changed: levels returned to separate launches plus launches now on their second form
 * (either pointer may be NULL). Errors as sym_factor_batch,
 * and SYM_ERR_INVALID for reps outside 1..100; the factor afterwards is that of the last run. */
int sym_autotune(sym_handle h, int32_t nbatch, const double *Ax, int64_t stride, int32_t reps, int32_t *tuned,
                 int32_t *changed);

/* Wait for the handle's stream and return the status of the last factorization. */
int sym_status(sym_handle h);

/* As sym_factor with Ax in host memory (copied to the device inside). */
int sym_factor_host(sym_handle h, const double *Ax);

/* Solve A x = b with the current factor (Sec. 3.1 supernodal forward substitution, then the
 * transposed backward sweep, which the paper does not spell out). b, x: DEVICE pointers of n
 * float64; they may alias. SYM_ERR_STATE before a successful sym_factor. */
int sym_solve(sym_handle h, const double *b, double *x);

/* nrhs right-hand sides, column-major: B (ldb >= n) and X (ldx >= n), DEVICE pointers. */
int sym_solve_multi(sym_handle h, int32_t nrhs, const double *B, int64_t ldb, double *X,
                    int64_t ldx);

/* As sym_solve_multi, but allocates nothing: for callers that may not call cudaMalloc (device
 * memory owned by their own pool or caching allocator, or loops that cannot take the device
 * synchronization cudaMalloc/cudaFree imply). The paper has no counterpart; it is a property of
 * this library's interface. The permuted work block (n * nrhs doubles) lives in a fixed array of
 * SYM_NOALLOC_MAX_WORK doubles (8 MiB) in the library's device memory, which every device that
 * loads the library holds until the process exits. Limits and behaviour:
 *   - n * nrhs > SYM_NOALLOC_MAX_WORK returns SYM_ERR_LIMIT before any work is issued;
 *   - the first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *     that device current; make that first call before any stream capture;
 *   - every call, on any handle and stream of a device, shares the one array: calls whose work
 *     overlaps on the GPU race and give wrong results, so serialize them (one stream, or events);
 *   - the array keeps the previous call's contents; the solve overwrites every element it reads,
 *     so no clearing is needed;
 *   - sym_profile does not time this entry point;
 *   - it needs an FP64 factor: a SYM_PREC_MIXED handle (whose solve refines in FP64 and needs
 *     more work memory) returns SYM_ERR_STATE, as does a call before a successful factorization
 *     or with another device current; these checks come before the array's address is looked up.
 * Other arguments, errors and results as sym_solve_multi (DEVICE pointers). */
#define SYM_NOALLOC_MAX_WORK 1048576
int sym_solve_multi_noalloc(sym_handle h, int32_t nrhs, const double *B, int64_t ldb, double *X,
                            int64_t ldx);

/* As sym_solve_multi with host pointers (copied inside). */
int sym_solve_host(sym_handle h, int32_t nrhs, const double *B, int64_t ldb, double *X,
                   int64_t ldx);

/* Mixed precision only: stopping rule of the FP64 refinement of sym_solve* (normwise backward
 * error <= tol for every right-hand side, at most max_iter conjugate-gradient iterations; each
 * iteration is one FP64 product with A and one FP32 solve with the factor). Not an operation of
 * the paper: its refinement counterpart is this library's mixed-precision addition. */
int sym_set_refinement(sym_handle h, double tol, int32_t max_iter);

/* Mixed precision only: iterations and final backward error of the last sym_solve* call.
 * sym_solve* returns SYM_ERR_NO_CONVERGENCE (with X holding the last iterate) when the limit is
 * reached above tolerance. */
int sym_refinement_info(sym_handle h, int32_t *iterations, double *backward_error);

/* Mixed precision only: the breakdown measure of the last factorization's FP32 factor. Its POTRF
 * kernels carry every pivot in FP64 (the diagonal entry as the external updates left it, minus
 * the squares of the tile's own column entries, subtracted in FP64; the reciprocal square root in
 * FP64; the column scaling in FP32), following the spec reading that the diagonal pivots
 * stay FP64 and that their ratio flags breakdown. For matrix `index` of the last batch (0 after
 * sym_factor): *min_ratio = min_k d_k / C_kk over the FP64 pivots d_k and the diagonal entries of
 * C = P A P^T, *column = that column (caller's numbering), and *breakdown = 1 when the ratio is
 * below the threshold (default 2^-16: cancellation has then taken 16 of FP32's 24 significand
 * bits from the pivot, so the factor may be a poor preconditioner and the matrix is close to
 * singular at FP32 precision), else 0. A flagged factor stays usable: the FP64 refinement still
 * runs and reports SYM_ERR_NO_CONVERGENCE if it cannot reach its tolerance. Output pointers may be
 * NULL. Errors: SYM_ERR_STATE for an FP64 handle or before any factorization, SYM_ERR_INVALID
 * for a bad index. */
int sym_pivot_info(sym_handle h, int32_t index, double *min_ratio, int64_t *column, int32_t *breakdown);

/* The breakdown threshold of sym_pivot_info (0 <= threshold <= 1). */
int sym_set_pivot_threshold(sym_handle h, double threshold);

/* Bounded waits of the tensor-core update (SYM_PREC_MIXED; no counterpart in the paper). Each
 * wait of a CTA on its MMAs gives up after limit_ns nanoseconds (1e3 .. 1e10; default 1e9); the
 * kernel then waits (with the same limit) for anything it still has in flight, frees its tensor
 * memory and records the failure, and the factorization returns SYM_ERR_TIMEOUT with the handle
 * still usable. withhold_mma = 1 is the failure-path test: the update issues no MMA and no
 * commit, so its first wait runs out and nothing is in flight when the tensor memory is freed;
 * 0 restores normal operation. Either change drops the captured factor graph. */
int sym_set_tc_wait(sym_handle h, uint64_t limit_ns, int32_t withhold_mma);

/* Sparse right-hand sides (Sec. 1.1 and Sec. 3.1 of the paper: decoupled sparse triangular
 * solve over the reach-set, with VI-Prune and VS-Block). For L y = P b with b nonzero only at
 * bidx (nnzb distinct indices, caller's numbering, host), sym_reach_analyze computes once per
 * pattern of b the set Reach_L(beta) of columns where y can be nonzero (the etree paths from the
 * nonzeros up) and a forward-solve schedule pruned to the supernodes holding them and to their
 * reached descendants. The reach handle depends on the pattern only: it stays valid across
 * refactorizations of its sym_handle, and must be freed before it. On a SYM_FLAG_HOST_ONLY handle
 * the reach is computed but cannot be solved with. Errors: SYM_ERR_INVALID for an index out of
 * range or repeated. */
typedef struct sym_reach_s *sym_reach;
int sym_reach_analyze(sym_handle h, int64_t nnzb, const int32_t *bidx, sym_reach *out);

/* Number of reached columns, and the reached columns in solve order (caller's numbering). */
int64_t sym_reach_size(sym_reach r);
int sym_reach_indices(sym_reach r, int32_t *idx);

/* Integer arrays of the reach set for checks: what = 0: reached columns (permuted numbering,
 * increasing); what = 1: reached supernodes. Returns the count; out may be NULL. */
int64_t sym_reach_export(sym_reach r, int32_t what, void *out);

/* Forward solve L y = P b for the sparse b: bvals (DEVICE, nnzb values in the order of bidx),
 * xvals (DEVICE, sym_reach_size values in the order of sym_reach_indices). Needs an FP64 factor
 * of the handle; only the reached supernodes are visited. */
int sym_solve_lower_sparse(sym_handle h, sym_reach r, const double *bvals, double *xvals);

void sym_reach_free(sym_reach r);

/* Cost model network (this library's addition for the learned schedule; the paper tunes its
 * thresholds by hand, Sec. 2.4 and Sec. 4.2). A multilayer perceptron
 *   y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3
 * with nin inputs and two hidden layers of `hidden` units, FP32, trained on the GPU by its own
 * forward, backward and Adam kernels on the mean squared error. Parameters are one flat vector:
 * W1 (hidden x nin, row-major), b1, W2 (hidden x hidden), b2, w3, b3. Row-major inputs X
 * (nrows x nin) and targets t (nrows) are DEVICE pointers; parameter and gradient copies are
 * host arrays. Initial weights are uniform in +-1/sqrt(fan-in) from a splitmix64 counter
 * stream of seed. Calls run on the legacy default stream and wait for their work. */
typedef struct sym_mlp_s *sym_mlp;
int sym_mlp_create(int32_t nin, int32_t hidden, uint64_t seed, sym_mlp *out);
int64_t sym_mlp_nparams(sym_mlp m);
int sym_mlp_set_params(sym_mlp m, const float *theta);
int sym_mlp_get_params(sym_mlp m, float *theta);
/* y (DEVICE, nrows) = network(X). */
int sym_mlp_predict(sym_mlp m, int64_t nrows, const float *X, float *y);
/* Gradient of the loss mean((y - t)^2) with respect to the parameters (host copy, may be
 * NULL) and the loss (host, may be NULL), at the current parameters. */
int sym_mlp_gradient(sym_mlp m, int64_t nrows, const float *X, const float *t, float *grad, float *loss);
/* steps full-batch Adam steps (beta1 0.9, beta2 0.999, eps 1e-8) at learning rate lr; the
 * final loss into *loss (host, may be NULL). */
int sym_mlp_train(sym_mlp m, int64_t nrows, const float *X, const float *t, int32_t steps, float lr, float *loss);
void sym_mlp_free(sym_mlp m);

/* Statistics of the analyzed pattern. */
int sym_info(sym_handle h, sym_stats *s);

/* First failing column (caller's numbering) of the last SYM_ERR_NOT_SPD, else -1. */
int sym_last_error_column(sym_handle h, int64_t *col);

/* Copy matrix index of the factored batch to host memory (storage_l doubles, widened from FP32
 * for a mixed-precision handle). */
int sym_get_batch_factor_host(sym_handle h, int32_t index, double *Lx_host);

/* Copy the factor to host memory in its supernodal panel layout (storage_l doubles; an FP32
 * factor is widened to double). For a batch: matrix 0. */
int sym_get_factor_host(sym_handle h, double *Lx_host);

/* Export an integer array of the symbolic plan (host copy) for checks against an independent
 * inspector. what = SYM_EXPORT_*; returns the element count (>= 0) or an error. When out is
 * NULL only the count is returned. Element types are listed per item. */
#define SYM_EXPORT_PERM 1        /* int32[n]: final ordering, perm[k] = original index */
#define SYM_EXPORT_PARENT 2      /* int32[n]: etree of the permuted matrix, -1 for roots */
#define SYM_EXPORT_COLCOUNT 3    /* int64[n]: |L_j| including the diagonal */
#define SYM_EXPORT_FSUPER 4      /* int32[nfund+1]: first column of each fundamental supernode */
#define SYM_EXPORT_SUPER 5       /* int32[nsuper+1]: first column of each supernode */
#define SYM_EXPORT_ROWPTR 6      /* int64[nsuper+1]: offsets of each supernode's row list */
#define SYM_EXPORT_ROWS 7        /* int32[]: sorted rows of each supernode (columns first) */
#define SYM_EXPORT_SPARENT 8     /* int32[nsuper]: supernodal tree parent, -1 for roots */
#define SYM_EXPORT_DESCPTR 9     /* int64[nsuper+1]: offsets of each descendant list */
#define SYM_EXPORT_DESC 10       /* int32[]: descendants K of each J, increasing */
#define SYM_EXPORT_DESCR0 11     /* int64[]: first position in rows(K) at or after first(J) */
#define SYM_EXPORT_DESCNIN 12    /* int32[]: rows of K that fall in cols(J) */
#define SYM_EXPORT_RELPTR 13     /* int64[npairs+1]: offsets of the relative maps */
#define SYM_EXPORT_REL 14        /* int32[]: position of rows(K)[r0+t] within rows(J) */
#define SYM_EXPORT_LEVEL 15      /* int32[nsuper]: level of each supernode */
#define SYM_EXPORT_LEVELPTR 16   /* int32[nlevels+1] */
#define SYM_EXPORT_LEVELLIST 17  /* int32[nsuper]: supernodes by level, increasing within one */
#define SYM_EXPORT_LXPTR 18      /* int64[nsuper+1]: offset of each panel in the factor storage */
/* The launch schedule and its task lists (raw records, for checks of the scheduler):
 * launches: int64 words {kind | level << 32, off, count, cluster | stream << 32, wait | tb << 32}
 * per launch (stream 1 = the factor's low-priority lookahead stream; wait = index of an earlier
 * launch it waits for, or -1; tb = 32 when all its tiles have at most 32 columns, for updates
 * also at most 32 rows, and run the small-tile kernels, else 0);
 * tasks: int32 words {a, b, c, d} per task (meaning per kind, see the SYM_KIND_* list);
 * update tasks: int64 words {J | bi << 32, bj, e0, e1}; update entries: int64 words
 * {K | r_lo << 32, c_lo | m << 32, n, relr, relc}. The count is in words. */
#define SYM_EXPORT_FACTOR_LAUNCHES 19
#define SYM_EXPORT_FWD_LAUNCHES 20
#define SYM_EXPORT_BWD_LAUNCHES 21
#define SYM_EXPORT_TASKS 22
#define SYM_EXPORT_UPD_TASKS 23
#define SYM_EXPORT_UPD_ENTRIES 24
/* Fused narrow levels: int32 words {role, pmax, ncmax, head} per factor launch. role 1: the POTRF
 * launch of a level whose supernodes all have at most 32 columns, which can factor each of their
 * panels (Cholesky of the diagonal block, triangular solve of the rows below it, inverse of the
 * diagonal block) in this one launch, with pmax the level's largest panel (rows x columns) and
 * ncmax its widest supernode; role 2: that level's TRSM and TRTRI launches, then skipped; role
 * 0: other launches. head: for roles 1 and 2 the index of the level's role-1 launch, else -1.
 * Batches run such a level fused where its panels fit the kernel's shared memory; a single
 * matrix where the level has at least 1216 supernodes; sym_autotune times both ways. */
#define SYM_EXPORT_BATCH_PANEL 27
/* The same for the forward and backward solve lists (SYM_EXPORT_FWD_LAUNCHES, _BWD_LAUNCHES):
 * role 1 on the step launch of a level whose supernodes all have at most 32 columns, on which
 * sym_solve_batch of FP64 factors runs the level's sums, steps and pushes (forward) or gathers
 * and steps (backward) in that one launch; role 2 on the level's other launches, then skipped. */
#define SYM_EXPORT_FWD_PANEL 28
#define SYM_EXPORT_BWD_PANEL 29
/* Forward solve by pushes: supernode J writes, per chunk ch of SOLVE_CW = 512 of its columns,
 * the products L_J(r, chunk) y_J(chunk) of its rows r below the diagonal block to a buffer t at
 * tx_J + ch (nrows_J - ncols_J) + (r - ncols_J), tx_J = sum over K < J of
 * (nrows_K - ncols_K) ceil(ncols_K / 512); column g then subtracts the entries of t listed in
 * contrib[contrib_ptr[g] .. contrib_ptr[g+1]) (ascending J, then ch). */
#define SYM_EXPORT_CONTRIB_PTR 25 /* int64[n+1] */
#define SYM_EXPORT_CONTRIB 26     /* int32[] */
int64_t sym_export(sym_handle h, int32_t what, void *out);

/* Per-kernel timing for measurement (no counterpart in the paper). With SYM_PROFILE_ON the
 * executor records a CUDA event on the handle's stream before the first launch and after every
 * launch of sym_factor* / sym_solve*; each sym_factor* and sym_solve* call then waits for its
 * work and adds the elapsed time of every launch to the totals of its kernel kind. OFF stops
 * recording (totals kept); RESET clears the totals. */
#define SYM_PROFILE_OFF 0
#define SYM_PROFILE_ON 1
#define SYM_PROFILE_RESET 2
int sym_profile(sym_handle h, int32_t mode);

/* Kernel kinds for sym_profile_read. */
#define SYM_KIND_SCATTER 0   /* zero the panels and scatter A (two launches counted as one) */
#define SYM_KIND_UPDATE 1    /* descendant updates of tiles */
#define SYM_KIND_POTRF 2     /* dense Cholesky of diagonal tiles */
#define SYM_KIND_TRSM 3      /* triangular solves of the tiles below a diagonal tile */
#define SYM_KIND_GEMM 4      /* trailing updates inside a supernode */
#define SYM_KIND_TRTRI 5     /* inverses of the diagonal tiles (for the solve) */
#define SYM_KIND_FGATHER 11  /* forward solve restricted to a reach set: gather from descendants */
#define SYM_KIND_FSTEP 12    /* forward solve: diagonal tile and updates inside a supernode */
#define SYM_KIND_FPUSH 13    /* forward solve: products of solved supernodes for the rows below */
#define SYM_KIND_FSUM 16     /* forward solve: columns subtract the pushed products */
#define SYM_KIND_BGATHER 14  /* backward solve: gather from the rows below */
#define SYM_KIND_BSTEP 15    /* backward solve: diagonal tile and updates inside a supernode */
#define SYM_KIND_PERM 17     /* solve: permutations in and out */
#define SYM_NUM_KINDS 18

/* Totals for one kernel kind since the last RESET: milliseconds, launches, and the algorithmic
 * flops those launches performed (useful multiply-adds x2 plus divisions and square roots; the
 * strict upper part of diagonal tiles excluded, explicit zeros of amalgamated panels included).
 * Any output pointer may be NULL. */
int sym_profile_read(sym_handle h, int32_t kind, double *ms, int64_t *launches, double *flops);

/* Milliseconds of every launch of the last profiled sym_factor* (which = 0) or sym_solve*
 * (which = 1) call, in execution order: for the factor, entry 0 is the zeroing and scatter of A
 * and entry 1 + i is launch i of SYM_EXPORT_FACTOR_LAUNCHES; for a solve, the launches of each
 * pass of up to 8 right-hand sides (the permutations, then the forward and backward lists).
 * Returns the count (0 before any profiled call); ms may be NULL to query it, else it receives
 * that many values. Errors: SYM_ERR_INVALID. */
int64_t sym_profile_launches(sym_handle h, int32_t which, double *ms);

/* Layout check of the tensor-core path (no counterpart in the paper): one CTA stages A (128 x 32)
 * and B (64 x 32), row-major float32 HOST arrays whose values TF32 represents exactly, in the
 * K-major core-matrix layout of the FP32 update, runs four kind::tf32 MMAs (M = 128, N = 64,
 * K = 8) with shared-memory descriptors of leading / stride byte offsets lbo / sbo (128 and 1024
 * in either order: the library's layout has lbo = 128, sbo = 1024), and writes D = A B^T
 * (128 x 64, row-major) to the HOST array D. Both orders keep every address the MMAs read inside
 * the staged operands. Errors: SYM_ERR_INVALID,
 * SYM_ERR_CUDA, SYM_ERR_OOM, SYM_ERR_TIMEOUT (the MMAs did not complete within about a second). */
int sym_tc_probe(const float *A, const float *B, float *D, uint32_t lbo, uint32_t sbo);

/* Measured FMA throughput of the current device in GFLOP/s (2 flops per FMA) for precision 64
 * (FP64 pipe) or 32 (FP32 pipe): register-resident FMA chains on every SM, best of three
 * launches of about 50 ms. The denominator of the roofline fraction of the ALU-bound kernels
 * (no counterpart in the paper). */
int sym_fma_peak(int32_t precision, double *gflops);

/* Text for an error code, and the message of the last failure on this thread. */
const char *sym_error_string(int code);
const char *sym_last_error_string(void);

/* Release the handle and everything it owns. NULL is allowed. */
void sym_free(sym_handle h);

#ifdef __cplusplus
}
#endif
#endif /* SYM_H_ */
