/*
 * mlbicgstab.h — C ABI of a GB300 (sm_103a) ML(n)BiCGStab solver library.
 *
 * ML(n)BiCGStab (M.-C. Yeung, "An introduction to ML(n)BiCGStab",
 * arXiv:1106.3678) solves A x = b for large sparse non-symmetric A using n
 * shadow vectors Q = [q_1 .. q_n].  This library implements the paper's
 * third algorithm, ML(n)BiCGStabt (Algorithm 4.1; Algorithm 7.1 with
 * M = I), whose per-iteration work is a sparse matrix-vector product fused
 * with shadow-vector inner products, plus AXPY-type recurrences indexed by
 * the index functions g_n, r_n of §2.  A^H appears only once per (A, Q), in
 * F = A^H Q(:,1:n-1) (Algorithm 4.1, step 2), which mlbicgstab_create
 * computes and keeps.
 *
 * Conventions shared by every entry point
 *   - Indices are 0-based (the paper's Matlab code is 1-based).
 *   - Real values are IEEE double.  Complex values are interleaved
 *     (re, im) double pairs, like C99 `double complex`.  Inner products
 *     conjugate their left argument: u^H v = sum conj(u_i) v_i.
 *   - Matrices are CSR: row_ptr[nrows+1] (int64, row_ptr[0] = 0,
 *     non-decreasing), col_idx[nnz] (int32 in [0, nrows)), values[nnz].
 *     Column indices need not be sorted; duplicates are summed.
 *   - Every function returns an API status (MLB_OK or MLB_ERR_*), which is
 *     separate from the solver flag of mlb_result (the paper's 0 / 1 / -1).
 *   - The library allocates and frees its own device memory.  It never
 *     takes ownership of caller pointers and never keeps them after a call
 *     returns.  A handle is not thread-safe: calls on one handle must not
 *     overlap.
 *   - No CPU fallback exists: without a CUDA device, create returns
 *     MLB_ERR_CUDA.
 */
#ifndef MLBICGSTAB_H
#define MLBICGSTAB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define MLB_OK 0
#define MLB_ERR_ARG 1         /* invalid argument (checked before any GPU work) */
#define MLB_ERR_CUDA 2        /* a CUDA runtime call failed (or no device) */
#define MLB_ERR_OOM 3         /* device or pinned host allocation failed */
#define MLB_ERR_TIMEOUT 4     /* a bounded device-side wait ran out; the
                                 kernel returned early and the context is
                                 still usable */
#define MLB_ERR_UNSUPPORTED 5 /* valid request the library does not handle */

/* ---- value types ------------------------------------------------------- */
#define MLB_F64 0   /* double */
#define MLB_F32 1   /* float (the FP32 copies of a refined handle) */
#define MLB_C128 2  /* complex double, interleaved (re, im) */
#define MLB_C64 3   /* complex float, interleaved (re, im) */

/* ---- precision modes --------------------------------------------------- */
/* Preconditioner M of Algorithm 7.1 (right preconditioning). */
#define MLB_PRECOND_NONE 0   /* M = I: Algorithm 4.1 */
#define MLB_PRECOND_JACOBI 1 /* M = diag(A) (every diagonal entry nonzero) */
#define MLB_PRECOND_ILU0 2   /* M = L U, the ILU(0) factors of A */
#define MLB_PRECOND_ILU0_MC 3 /* M = P^T L U P, the ILU(0) factors of
                                 P A P^T for a multicolour order P */

#define MLB_PREC_FP64 0     /* matrix, vectors and arithmetic in FP64 */
#define MLB_PREC_FP32_REFINED 1 /* inner ML(n)BiCGStab in FP32 (values,
                                   vectors, preconditioner factors,
                                   accumulation) inside an FP64 iterative
                                   refinement: residual b - A x, solution
                                   update and all recurrence coefficients
                                   in FP64.  The inner solve keeps its
                                   Krylov recurrences across refinement
                                   steps: reliable updates move its iterate
                                   into the FP64 solution and replace its
                                   residual by the FP64 true residual (see
                                   inner_tol).  It converges where FP32 can
                                   carry the (preconditioned) iteration;
                                   otherwise flag 1 with the solution of
                                   smallest true residual found. */

/* A sparse matrix in host memory: CSR, or BSR with 3x3 blocks.  The
 * library copies it; the caller's arrays may be freed after
 * mlbicgstab_create returns.
 *   block = 0 or 1: CSR (row_ptr over the nrows rows, col_idx columns,
 *   one value per entry).
 *   block = 3: BSR(3), the storage of systems with 3 unknowns per cell
 *   (e.g. reservoir models): nrows (a multiple of 3) scalar rows,
 *   row_ptr over the nrows/3 block rows, nnz blocks, col_idx block
 *   columns in [0, nrows/3), values 9 per block (row-major 3x3).  The
 *   product of real-valued matrices then streams one column index per 3
 *   values (a scalar CSR whose rows come in such triplets is stored the
 *   same way).  Handles of such matrices are not accepted by
 *   mlbicgstab_solve_batch or the fused-product entry points
 *   (MLB_ERR_UNSUPPORTED). */
typedef struct {
    int64_t nrows;          /* N scalar rows (square matrices only) */
    int64_t nnz;            /* stored entries (CSR) or blocks (BSR) */
    const int64_t *row_ptr; /* nrows + 1 (CSR) or nrows/3 + 1 (BSR) */
    const int32_t *col_idx; /* nnz (block) column indices */
    const void *values;     /* nnz (CSR) or 9 nnz (BSR) values of `dtype` */
    int32_t dtype;          /* MLB_F64 or MLB_C128 */
    int32_t block;          /* 0 or 1: CSR; 3: BSR with 3x3 blocks */
} mlb_matrix;

/* Options for mlbicgstab_create.  Zero-initialise, then set what you need;
 * mlbicgstab_default_options fills the defaults below. */
typedef struct {
    int32_t n;            /* number of shadow vectors, 1 <= n <= 64
                             (default 4; the paper suggests 4 or 8, §5.2) */
    int32_t precision;    /* MLB_PREC_FP64 (default) or MLB_PREC_FP32_REFINED */
    uint64_t q_seed;      /* seed of the shadow vectors when Q == NULL */
    const void *Q;        /* optional host N x n column-major shadow matrix
                             (dtype of A).  NULL: Q ~ N(0,1) entrywise from
                             q_seed, drawn by the counter-based generator
                             documented in mlbicgstab_get_Q */
    double kappa;         /* omega guard of Eq. 5.1; 0 (default) gives the
                             standard minimisation step */
    int32_t max_outer;    /* FP64: restarts from the current x while the
                             recursive residual met tol but the true one did
                             not.  Refined: maximum number of FP32 inner
                             calls; a new call (a restart of the inner
                             Krylov process from the current x) follows one
                             that stagnated or reached inner_maxit.
                             Default 10. */
    int32_t grid;         /* CTAs of the persistent solve kernel; 0 = auto
                             (all SMs x occupancy, fewer for small N) */
    double inner_tol;     /* refined mode, in (0, 1): reliable-update
                             factor.  At a block end, when the FP32
                             recursive residual has fallen below inner_tol
                             times its largest value since the last update
                             (or has met tol), the FP32 iterate is moved
                             into the FP64 solution and the FP32 residual
                             replaced by the FP64 true residual; the solve
                             ends when that true residual meets tol.
                             Default 1e-2.  An inner call also ends when its
                             residual has not reached a new minimum for
                             max(2000, iterations it took to reach the
                             current one) iterations. */
    int64_t inner_maxit;  /* refined mode: iteration cap of one inner call
                             (default 1e6; all inner iterations together
                             are capped by the maxit of the solve) */
    void *stream;         /* cudaStream_t for all work of this handle;
                             NULL = the legacy default stream */
    int64_t timeout_ns;   /* limit of every device-side wait (grid barrier
                             spin); default 2e9 (2 s) */
    int32_t precond;      /* MLB_PRECOND_NONE (default), MLB_PRECOND_JACOBI
                             or MLB_PRECOND_ILU0.
                             MLB_PRECOND_JACOBI: Algorithm 7.1 with
                             M = diag(A).  The handle
                             stores A M^{-1} (columns divided by the
                             diagonal), F = M^{-H} A^H Q (step 2), and each
                             solve maps x_0 to y_0 = M x_0 and the result
                             back to x = M^{-1} y, which is the algorithm's
                             x-recurrence along g^ = M^{-1} g (steps 6, 35,
                             39).  Stopping rule and residuals are those of
                             A x = b.
                             MLB_PRECOND_ILU0: M = L U, the ILU(0)
                             factors of A (the preconditioner of the
                             paper's experiments, §5; L unit lower and U
                             upper triangular in A's pattern with
                             (LU)_ij = a_ij there), computed on the host at
                             create.  Every product of the iteration is
                             A (M^{-1} v), M^{-1} by level-scheduled
                             triangular solves on the device; F = M^{-H}
                             A^H Q; the solve iterates on y = M x, mapped in
                             the kernel.  In refined mode the inner
                             FP32 solve applies FP32 copies of the
                             factors.  MLB_ERR_ARG when a row has no stored
                             diagonal or a pivot is zero.
                             MLB_PRECOND_ILU0_MC: the same with A's rows
                             and columns first reordered by colour (P A
                             P^T; the order of mlbicgstab_get_perm): greedy
                             colouring of A's symmetrised adjacency graph
                             in natural order, colour classes in colour
                             order.  The triangular solves then take one
                             level per colour (2 for a 7-point stencil)
                             instead of one per wavefront of the natural
                             order (382 at 128^3), at the price of a
                             weaker preconditioner (usually more
                             iterations).  Not the paper's natural-order
                             ILU(0).  The handle solves P A P^T y = P b
                             and returns x = P^T y; b, x0, x, Q and
                             mlbicgstab_get_Q stay in the caller's row
                             order (drawn Q entries keep their original
                             row index).  Handles with different
                             preconditioners may share one batch. */
    int32_t reserved0;    /* must be 0 */
} mlb_options;

/* Result of one solve.  flag/iter/err follow the paper's reference code
 * (§5, Appendix): flag 0 = converged (||r||/||b|| < tol on the recursive
 * residual), 1 = iteration limit, -1 = breakdown (c = 0, ||A u|| = 0 or
 * omega = 0, or a non-finite scalar). */
typedef struct {
    int32_t flag;
    int32_t j;            /* block index g_n(k) of the last iteration k */
    int32_t i;            /* in-block index r_n(k) (1..n) of the last k */
    int32_t status;       /* MLB_OK or MLB_ERR_TIMEOUT (device-side wait) */
    int64_t iter;         /* iterations k over all restarts / inner solves */
    int64_t spmv;         /* sparse matrix-vector products (FP64 + FP32) */
    int64_t outer;        /* restarts (FP64) or refinement steps (refined) */
    double err;           /* last recursive relative residual */
    double true_relres;   /* ||b - A x||_2 / ||b||_2 in FP64 at return
                             (||b|| replaced by 1 when b = 0) */
    double kernel_ms;     /* device time of the solve kernel(s) */
    double bytes;         /* algorithmic HBM bytes of the solve kernel(s):
                             each pass counted as its inputs read once and
                             its outputs written once */
    int64_t ops[5];       /* Table 4.3 operation counts of the last inner
                             call: matvec, dot, saxpy, scale (alpha v), norm */
    double flops;         /* algorithmic floating-point operations of the
                             solve kernel(s), real arithmetic: 2 per stored
                             matrix entry per product (and per ILU(0) factor
                             entry per M^{-1}), 2 per element per inner
                             product, AXPY or norm, 1 per scaling; complex
                             multiply-adds count 8 */
    int32_t ctas;         /* CTAs that solved the system (the grid of a
                             single solve; in a batch 1, or the team size) */
    int32_t reserved;
} mlb_result;

/* Facts about a handle. */
typedef struct {
    int64_t nrows, nnz;
    int32_t n, dtype, precision, grid, block;
    int32_t precond;      /* MLB_PRECOND_* of the handle */
    int64_t nnz_padded;   /* stored SELL-32 entries (>= nnz) */
    int64_t device_bytes; /* device memory held by the handle */
    int32_t n_active;     /* shadow vectors the next solve uses (<= n) */
    int32_t ilu_levels;   /* levels of the forward triangular solve of an
                             ILU(0) handle (one grid barrier each); 0
                             otherwise */
    double qd_kernel_ms;  /* device time of the last mlbicgstab_spmv_qdot
                             (CUDA events around its launch on the handle's
                             stream); 0 before the first call */
    int32_t entry_values; /* values per stored matrix entry of the
                             products: 1, or 3 (3x3-block rows with one
                             column index per three values) */
    int32_t reserved2;
} mlb_info;

/* Result of mlbicgstab_autotune. */
typedef struct {
    int32_t grid;         /* CTAs of the persistent solve kernel chosen */
    int32_t spt_cap;      /* cap on 32-row slices per SpMV tile chosen */
    double us_per_iter;   /* device time per iteration with the choice */
    double default_us_per_iter; /* the same before tuning */
    int32_t trials;       /* configurations timed (0 when from the cache) */
    int32_t from_cache;   /* 1: taken from the process-wide cache */
    int32_t qd_fused;     /* columns of Q fused into the epilogue of the
                             product of mlbicgstab_spmv_qdot chosen (1, 2
                             or 4); 0 when the handle has no such product
                             (a preconditioner, or 3x3-block storage) */
    int32_t reserved;
    double qd_us;         /* device time of one fused product with it */
    double qd_default_us; /* the same with the built-in rule */
} mlb_tune_result;

/* Launch configuration of a handle: what the autotuners choose, readable
 * and settable so that a choice can be kept across processes. */
typedef struct {
    int32_t grid;          /* CTAs of the persistent solve kernel, 1 to the
                              largest co-resident grid */
    int32_t spt_cap;       /* cap on 32-row slices per SpMV tile, 1..15 */
    int32_t batch_spt_cap; /* the same inside mlbicgstab_solve_batch, 0..15
                              (0: the product reads the matrix with plain
                              loads), or -1: spt_cap */
    int32_t batch_team;    /* CTAs per team for the large systems of a
                              batch whose first handle this is, 1..8 (1: no
                              teams); default 4 */
    int32_t qd_fused;      /* columns of Q fused into the epilogue of
                              mlbicgstab_spmv_qdot's product: 1, 2 or 4 (4
                              real only), or 0: the built-in rule (4 for
                              real n = 4; 1 for real FP64 values and
                              n > 4; else 2, or 1 when n = 1); a choice
                              above the active n falls back to the rule */
} mlb_tuning;

/* Result of mlbicgstab_autotune_batch. */
typedef struct {
    int32_t classes;      /* size classes of the batch (floor(log2 N),
                             round(nnz/N)) */
    int32_t trials;       /* batch launches timed (0 when all cached) */
    int32_t from_cache;   /* classes whose choice came from the cache */
    int32_t team;         /* CTAs per team chosen (batch_team of hs[0]) */
    double default_ms;    /* device time of the whole trial batch (see
                             mlbicgstab_autotune_batch) in one launch with
                             the settings the handles had before */
    double tuned_ms;      /* the same with the chosen settings */
} mlb_batch_tune_result;

/* Parameters of mlbicgstab_solve_sequence (automatic choice of n, §5). */
typedef struct {
    int32_t n0;           /* n for the first two systems */
    int32_t step;         /* search step of n (>= 0) */
    int32_t n_min;        /* n stays in [n_min, n_max]; n_min >= 1 and */
    int32_t n_max;        /* n_max <= the n every handle was created with */
} mlb_sequence_options;

typedef struct mlb_handle mlb_handle;

/* Fill `opt` with the defaults listed in mlb_options. */
void mlbicgstab_default_options(mlb_options *opt);

/*
 * Create a solver for the matrix A (host CSR).  Validates A (row_ptr
 * monotone, columns in range; MLB_ERR_ARG otherwise), copies it to the
 * device in SELL-32 form (rows in natural order, 32-row slices stored
 * column-major), draws or copies Q, and computes F = A^H Q(:,1:n-1)
 * (Algorithm 4.1, step 2; with M = I, Algorithm 7.1, step 2).
 *   AH   optional host CSR of A^H (for complex A, the conjugate transpose).
 *        NULL: the library forms A^H itself.  Only used for F.
 *   opt  NULL for defaults.
 * On success *h owns all device memory; release it with mlbicgstab_destroy.
 */
int mlbicgstab_create(mlb_handle **h, const mlb_matrix *A,
                      const mlb_matrix *AH, const mlb_options *opt);

/*
 * Solve A x = b (Algorithm 7.1, M as chosen at create; stopping rule of §5: stop when
 * ||r_k||/||b|| < tol after any update of r or u; at most `maxit` k-steps
 * in total).  The whole iteration runs in one persistent kernel: the
 * convergence and breakdown tests are taken on the device.
 *   b, x       N values each (dtype of A).  x holds x_0 on entry and the
 *              solution on return.  on_device = 0: host pointers (copied
 *              in and out inside the call); 1: device pointers, in memory
 *              of the handle's GPU or managed memory (MLB_ERR_ARG for
 *              another GPU's memory).
 *   err_hist   optional host array (NULL to skip): err_hist[k] = relative
 *              recursive residual after iteration k (k = 0: initial), for
 *              k < hist_cap, over the first inner call.
 * Blocks until the result is available.
 */
int mlbicgstab_solve(mlb_handle *h, const void *b, void *x, int32_t on_device,
                     double tol, int64_t maxit, mlb_result *res,
                     double *err_hist, int64_t hist_cap);

/*
 * Solve `count` independent systems, one handle each (created with the same
 * dtype, precision and device), in one persistent launch.  Estimated work
 * of a system: (nnz + N) N^(1/3) (the per-iteration cost times the growth
 * of iteration counts with N of discretised PDEs).  Systems of at least
 * 2048 rows per team CTA whose estimate exceeds 1/10 of the average work
 * per CTA (natural-order ILU(0) systems excepted: their triangular solves
 * take one barrier per level) are solved by teams of hs[0]'s batch_team
 * CTAs (mlb_tuning),
 * largest first, with team barriers and reductions (the arithmetic of a
 * single solve with grid = the team size); the other systems by one CTA
 * each, largest first, with CTA-wide barriers and shared-memory
 * reductions (the arithmetic of a single solve with grid = 1).  Each runs
 * the same method as mlbicgstab_solve (restarts and refinement included).
 *   b[s], x[s]  per-system pointers as in mlbicgstab_solve (on_device
 *               applies to all).  tol[s], maxit[s] per system.
 *   res         `count` results; kernel_ms is the time of the whole launch.
 * The stream of hs[0] is used; hs[0] keeps a workspace (items, order,
 * results) that grows to the largest batch it has run.  No residual
 * history is recorded.  Handles must not be used by other calls meanwhile.
 * Each system's SpMV tiles take its handle's batch cap on slices per tile
 * (set by mlbicgstab_autotune_batch), else the handle's own cap.
 */
int mlbicgstab_solve_batch(mlb_handle *const *hs, int32_t count,
                           const void *const *b, void *const *x,
                           int32_t on_device, const double *tol,
                           const int64_t *maxit, mlb_result *res);

/*
 * The work plan mlbicgstab_solve_batch uses (host only, no GPU work): for
 * `count` systems with N[s] rows, nnz[s] stored entries and preconditioner
 * precond[s] (MLB_PRECOND_*), teams of `team` CTAs (the batch's
 * batch_team) and `slots` co-resident CTAs (SMs x CTAs per SM of the batch
 * kernel), ctas[s] = CTAs that will solve system s (1, or the team size);
 * order = the team-solved systems (*nbig of them), then the others, each
 * list largest first; *teams = teams formed, *grid = CTAs launched.
 * MLB_ERR_ARG for a null pointer, count < 1, team < 1, slots < 1, N < 1 or
 * nnz < 0.
 */
int mlbicgstab_batch_plan(const int64_t *N, const int64_t *nnz, const int32_t *precond, int32_t count,
                          int32_t team, int32_t slots, int32_t *ctas, int32_t *order, int32_t *nbig,
                          int32_t *teams, int32_t *grid);

/*
 * Use the first n shadow vectors in the solves that follow
 * (1 <= n <= the n the handle was created with; MLB_ERR_ARG otherwise).
 * The handle's Q(:,1:n) and F(:,1:n-1) = A^H Q(:,1:n-1) are exactly the
 * Q and F of a handle created with this n (entries of the drawn Q depend
 * only on their row and column), so nothing is recomputed.
 */
int mlbicgstab_set_n(mlb_handle *h, int32_t n);

/*
 * The rule for choosing n in a sequence of systems (§5, "Choice of n":
 * Code #4 of the author's earlier work): with t_prev and t_cur the times of
 * the previous and the current solve, the next system uses n + step when
 * t_prev > t_cur and n - step otherwise, clamped to [n_min, n_max].
 * Returns the next n (or -1 when the arguments are invalid).
 */
int32_t mlbicgstab_next_n(int32_t n, double t_prev, double t_cur, int32_t step,
                          int32_t n_min, int32_t n_max);

/*
 * Solve a sequence of `count` systems one after another (system s with
 * handle hs[s]; a handle may repeat, e.g. one matrix with many right-hand
 * sides), choosing n by mlbicgstab_next_n: systems 0 and 1 use so->n0,
 * system s+1 (s >= 1) uses next_n(n_s, t_{s-1}, t_s), t being the device
 * time of each solve (mlb_result.kernel_ms).  Arguments as in
 * mlbicgstab_solve; n_used[s] receives the n of system s.  Every handle
 * is returned to the n it had before the call.  Stops at the first error.
 */
int mlbicgstab_solve_sequence(mlb_handle *const *hs, int32_t count,
                              const void *const *b, void *const *x,
                              int32_t on_device, const double *tol,
                              const int64_t *maxit,
                              const mlb_sequence_options *so,
                              mlb_result *res, int32_t *n_used);

/*
 * Autotuner (performance only; the paper has no counterpart).  Times
 * `iters` iterations of A x = 1 from x = 0 (host buffers, tol 0) for each
 * candidate configuration: CTA counts want, want/2, want/4, want/8 (want =
 * the CTAs that give each at least 512 16-byte chunks, at most all SMs)
 * and the current one, times slice caps 15, 12, 8, 4 per SpMV tile (rows
 * per tile = 32 x slices); keeps the fastest in the handle (later solves
 * and batches use it) and caches it for the process per (dtype,
 * precision, preconditioner, floor(log2 N), round(nnz/N)).  use_cache = 1
 * takes a cached choice without timing.  Later results change only in
 * rounding (reduction trees follow the CTA count).  Overwrites the
 * handle's device work buffers; blocks until done; MLB_ERR_ARG for iters
 * outside [1, 100000].
 */
int mlbicgstab_autotune(mlb_handle *h, int32_t iters, int32_t use_cache,
                        mlb_tune_result *out);
/* mlbicgstab_autotune also chooses, for a handle whose A has a fused
 * product (no preconditioner, scalar storage), how many columns of Q the
 * product's epilogue carries: it times 20 calls of mlbicgstab_spmv_qdot's
 * kernel (FP64, or the FP32 copies of a refined handle) for each of 1, 2
 * and 4 columns (4 for real data only; never more than the active n) and
 * keeps the fastest (qd_fused); later mlbicgstab_spmv_qdot and
 * mlbicgstab_spmv_qdot_async calls use it while n_active allows it.
 * Results change in rounding only (the sums' order follows the columns'
 * passes).  Allocates and frees two device vectors of N values. */

/*
 * Batch autotuner (performance only).  Its trial batches solve A x = 1 from
 * x = 0 for every system to `tol` (at most `maxit` iterations each): the
 * iteration counts of real solves, whose spread decides how the work
 * should be divided.  First the team size: the whole trial batch is run
 * with batch_team 1, 2, 4 and 8 (set on every handle; a batch takes
 * hs[0]'s), and the fastest kept.  Then the tile cap per size class
 * (floor(log2 N), round(nnz/N)): a trial batch of the class's systems
 * alone is run for each cap on slices per SpMV tile in {15, 12, 8, 4, 0}
 * (0: the product reads the matrix with plain loads instead of through
 * the tile ring), and the fastest set as the batch cap of the class's
 * handles (single solves keep the handle's own cap).  Choices are cached
 * for the process: the team size per (dtype, precision, preconditioner,
 * count, floor(log2 of the total N)), the caps per (dtype, precision,
 * preconditioner, class); use_cache = 1 takes cached choices without
 * running them.  Reports the device time of the whole trial batch before
 * and after.  The handles must satisfy mlbicgstab_solve_batch's rules;
 * their device work buffers are overwritten; blocks until done;
 * MLB_ERR_ARG for tol < 0, maxit outside [1, 10^7] or a bad list.
 */
int mlbicgstab_autotune_batch(mlb_handle *const *hs, int32_t count, double tol, int64_t maxit,
                              int32_t use_cache, mlb_batch_tune_result *out);

/* Read or set a handle's launch configuration (mlb_tuning).  Results
 * change in rounding only.  MLB_ERR_ARG for a value outside its range. */
int mlbicgstab_get_tuning(const mlb_handle *h, mlb_tuning *out);
int mlbicgstab_set_tuning(mlb_handle *h, const mlb_tuning *t);

/*
 * Fused hot operation: y = A x and d = Q^H y (all n shadow inner products,
 * a tall-skinny block reduction) in one pass over A — the per-iteration
 * product w = A g with c = q^H w of Algorithm 4.1 (step 32) generalised to
 * every q.  x, y: device arrays of N values (memory of the handle's GPU
 * or managed memory; MLB_ERR_ARG otherwise); d: host array of n_active
 * values (the handle's n unless mlbicgstab_set_n chose fewer columns).
 * Reductions are deterministic (fixed order).  Blocks until d is ready.
 * MLB_ERR_TIMEOUT if a wait inside the kernel gave up (y and d invalid).
 */
int mlbicgstab_spmv_qdot(mlb_handle *h, const void *x, void *y, void *d);
/* (MLB_ERR_UNSUPPORTED for a handle with a preconditioner: it stores
 * A M^{-1}, not A.) */

/*
 * Asynchronous form of mlbicgstab_spmv_qdot for pipelined callers: the same
 * fused y = A x, d = Q^H y, enqueued on the handle's stream with the
 * result left in device memory; the call returns without waiting.
 *   value_type  MLB_F64 (MLB_C128 for complex handles): the handle's FP64
 *               matrix and Q; x, y hold doubles (complex doubles).
 *               MLB_F32 (MLB_C64): the FP32 copies a MLB_PREC_FP32_REFINED
 *               handle keeps for its inner solve; x, y hold floats
 *               (complex floats), products and per-thread sums are FP32,
 *               sums across threads and CTAs FP64.  MLB_ERR_UNSUPPORTED
 *               for an FP64 handle.
 *   x, y        device arrays of N values of that type
 *   d           device array of n_active * k + 1 doubles (k = 1 real,
 *               2 complex): the inner products (complex as re, im), then a
 *               status word, 1.0 if a wait inside the kernel gave up (d
 *               and y are then invalid), else 0.0
 * Calls on one handle share its scratch and must not overlap on the GPU
 * (back-to-back calls on the handle's stream are ordered and fine).
 * MLB_ERR_ARG for a pointer that is not device memory of the handle's GPU.
 */
int mlbicgstab_spmv_qdot_async(mlb_handle *h, int32_t value_type, const void *x, void *y, void *d);

/*
 * Allocation-free variant of mlbicgstab_spmv_qdot: y = A x and d = Q^H y
 * with every array supplied by the caller in device memory and no handle.
 * The paper has no counterpart; it exists for callers that cannot allocate
 * device memory: code inside a framework whose memory pool owns the
 * device's memory budget, plug-ins whose host application forbids them to
 * allocate, and latency-critical loops that cannot afford the device-wide
 * synchronisation cudaMalloc/cudaFree may cause.  This call performs no
 * cudaMalloc, cudaFree or other allocation.
 *   nrows, nnz, row_ptr, col_idx, values  CSR of A in device memory
 *                (row_ptr int64, col_idx int32 in [0, nrows): the caller
 *                guarantees a valid CSR; it is not re-checked here)
 *   dtype        MLB_F64 or MLB_C128
 *   x            nrows values (device)
 *   Q            n columns of leading dimension ldq >= nrows (device)
 *   n            1 <= n <= 64; larger n returns MLB_ERR_ARG
 *   y            nrows values (device, written)
 *   d            n values (device, written)
 *   stream       cudaStream_t or NULL; the call returns once the work is
 *                enqueued (no host synchronisation)
 * Scratch: per-CTA partial sums live in one fixed 512 KiB array of this
 * library's device memory, held on every GPU that loads the library until
 * the process exits; the launch uses at most as many CTAs as fit in it.
 * Calls share that array: two calls that overlap on the GPU (on different
 * streams, or from different host threads) race and give wrong results.
 * The first call on a device looks up the array's device address (set-up);
 * make that first call before any stream capture.  Returns MLB_ERR_ARG for
 * invalid sizes, or for a pointer that is neither device memory of the
 * current device (cudaGetDevice) nor managed memory: memory of another GPU
 * is refused.  MLB_ERR_CUDA on launch failure.
 */
int mlbicgstab_spmv_qdot_noalloc(int64_t nrows, int64_t nnz,
                                 const int64_t *row_ptr,
                                 const int32_t *col_idx, const void *values,
                                 int32_t dtype, const void *x, const void *Q,
                                 int64_t ldq, int32_t n, void *y, void *d,
                                 void *stream);

/*
 * Copy Q (N x n, column-major, dtype of A) to host memory.  When Q was
 * drawn from q_seed, real entry e = col*N + row is normal number e and a
 * complex entry e takes normals 2e (re) and 2e+1 (im), where normal number
 * t is Box–Muller (cosine branch) of uniforms U(2t), U(2t+1) on (0,1],
 * U(s) = ((v >> 11) + 1) 2^-53 with v output number s of SplitMix64
 * (Steele, Lea & Flood 2014) seeded with q_seed.  The paper fixes no
 * generator (§5 uses Matlab's randn).
 */
int mlbicgstab_get_Q(const mlb_handle *h, void *host_out);

/* Row order of the handle's system: new row r is the caller's row
 * host_out[r] (N entries).  The multicolour order for MLB_PRECOND_ILU0_MC
 * handles, the identity otherwise.  The paper has no counterpart. */
int mlbicgstab_get_perm(const mlb_handle *h, int32_t *host_out);

/* Fill `info` for a handle. */
int mlbicgstab_info(const mlb_handle *h, mlb_info *info);

/* Release every resource of a handle (NULL is accepted). */
void mlbicgstab_destroy(mlb_handle *h);

/* Static text for a status code. */
const char *mlbicgstab_strerror(int code);

/*
 * Failure-detection self-test: launches the grid barrier the solve kernel
 * uses with one participant that never arrives, on `grid` CTAs, with a
 * wait limit of `timeout_ns`.  Every wait gives up after the limit and the
 * kernel returns; expected result MLB_ERR_TIMEOUT with the device still
 * usable.  The paper has no counterpart (library robustness only).
 */
int mlbicgstab_selftest_barrier_timeout(int32_t grid, int64_t timeout_ns);

#ifdef __cplusplus
}
#endif

#endif /* MLBICGSTAB_H */
