/*
 * ddps.h — C ABI of a single-GPU (sm_103a) DDPS solver.
 *
 * DDPS (Manguoglu, "A domain-decomposing parallel sparse linear system
 * solver", arXiv 1008.1700) solves a sparse system A x = f as follows.
 *   Sec. 3, Eq. (1)-(2) and Fig. 2 step 1: A is split by block rows into
 *     A = D + R, D = diag(A_11, ..., A_pp).
 *   Fig. 2 step 2: every diagonal block is factored, A_ii = L_i U_i (exact LU).
 *   Fig. 2 step 3 and the Sec. 3 dropping rule: R~ is R minus dropped entries.
 *   Fig. 2 steps 4-5: spikes G = D~^-1 R~, c = indices of G's nonzero columns.
 *   Fig. 2 step 6: a Krylov method (BiCGStab, Sec. 4) on A x = f with the
 *     preconditioner P = D~ + R~, applied by Fig. 3:
 *       6.1 g = D~^-1 y;  6.2 G^ = I(c,c) + G(c,c), g^ = g(c);
 *       6.3 solve G^ z^ = g^ (BiCGStab, tolerance eps_in);
 *       6.4-6.5 z = g - G(:,c) z^, computed here as z = D~^-1 (y - R~ z^).
 *
 * Conventions shared by every entry point:
 *   - Matrices are CSR with int32 row pointers and column indices (0-based,
 *     columns sorted inside a row, no duplicates) and float64 values.
 *   - A handle may hold a batch of independent systems: they are stacked into
 *     one block-diagonal matrix of order n = sum of the systems' orders, whose
 *     block rows are listed in block_ptr; sys_block_ptr says which blocks
 *     belong to which system.  No entry of A may couple two systems.  Krylov
 *     scalars, norms and convergence are kept per system.
 *   - Pointers documented "host" are read during the call only.  Pointers
 *     documented "device" must stay valid until the stream work they are used
 *     in has completed; the caller owns them.  The handle owns everything else
 *     (factors, spikes, workspace) and frees it in ddps_destroy.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Calls enqueue work on it; a call returns before the work has
 *     finished unless documented otherwise.
 *   - No exception crosses the ABI.  On failure an entry point returns a
 *     non-zero ddps_status and ddps_last_error(h) describes it.
 */
#ifndef DDPS_H
#define DDPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ddps_handle ddps_handle;

typedef enum {
  DDPS_OK = 0,
  DDPS_ERR_INVALID_ARG = 1,     /* bad size, pointer, pattern or option */
  DDPS_ERR_SINGULAR_BLOCK = 2,  /* a pivot of some A_ii fell under the threshold (Sec. 3 requires
                                   nonsingular diagonal blocks) */
  DDPS_ERR_NOT_CONVERGED = 3,   /* maxit_out reached: x holds the last iterate, info the residual */
  DDPS_ERR_OUT_OF_MEMORY = 4,   /* a device allocation failed */
  DDPS_ERR_CUDA = 5,            /* a CUDA runtime call failed */
  DDPS_ERR_TIMEOUT = 6,         /* a bounded device-side wait gave up */
  DDPS_ERR_STATE = 7            /* call order: e.g. solve before factor */
} ddps_status;

/* BF16X3 (spike products only): each fp32 operand is split into a bf16 high
 * part and a bf16 remainder and the product is hi*hi + hi*lo + lo*hi on the
 * tensor cores with fp32 accumulation (about 16 correct bits). */
typedef enum { DDPS_FP64 = 0, DDPS_FP32 = 1, DDPS_BF16 = 2, DDPS_BF16X3 = 3, DDPS_FP16 = 4 } ddps_precision;

/* Fig. 2 step 3.  COLUMN: the Sec. 3 rule — in block row R_i, column k is
 * dropped when ||R_i(:,k)||_inf <= drop_tol * max_j ||R_i(:,j)||_inf.
 * ABS: an entry r_ij is dropped when |r_ij| < drop_tol. */
typedef enum { DDPS_DROP_NONE = 0, DDPS_DROP_COLUMN = 1, DDPS_DROP_ABS = 2 } ddps_drop_mode;
/* How the reduced matrix G^ = I(c,c) + G(c,c) of Fig. 3 step 6.2 is applied.
 * EXPLICIT: Fig. 2 step 4 forms the spikes and stores G^ as dense arrays per
 * block (Sec. 3); every inner product streams them.
 * IMPLICIT: a variant that departs from Fig. 2 step 4: no spikes are formed
 * and G^ v = v + (D~^-1 (R~ v))(c) is computed with one R~ product and one
 * block solve (the kernels of 6.1) per inner product. */
typedef enum { DDPS_GHAT_EXPLICIT = 0, DDPS_GHAT_IMPLICIT = 1 } ddps_ghat_mode;
/* How Fig. 3 step 6.3 solves G^ z^ = g^ ("directly or iteratively").
 * ITERATIVE: unpreconditioned BiCGStab to tol_in (Sec. 4 settings), the
 * paper's choice in its experiments.
 * DIRECT: for partitions whose blocks form chains (every coupling column of
 * a block lies in the block before or after it in the same system, as for
 * z-slabs or grid-line blocks), G^ is block tridiagonal with identity
 * diagonal blocks; the factor phase forms its block LU (FP32) and every
 * application solves with it: no inner iterations (Sec. 3 direct mode when
 * nothing is dropped). */
typedef enum { DDPS_REDUCED_ITERATIVE = 0, DDPS_REDUCED_DIRECT = 1 } ddps_reduced_solver;
/* Fig. 2 step 2: the block factors "approximate or exact" (Sec. 3).
 * LU: exact multifrontal LU over a nested-dissection order of every block.
 * ILU0: incomplete LU with zero fill on the pattern of every block, in the
 * block's own row order; G = D~^-1 R~ then uses D~ = L~ U~, and the outer
 * Krylov iteration absorbs the approximation (P = D~ + R~ is no longer A
 * even without dropping).  Spike products run in factor_prec (SIMT). */
typedef enum { DDPS_FACTOR_LU = 0, DDPS_FACTOR_ILU0 = 1 } ddps_factor_kind;

typedef struct {
  int32_t drop_mode;      /* ddps_drop_mode */
  double drop_tol;        /* delta (COLUMN) or tau (ABS) */
  int32_t factor_prec;    /* FP64 or FP32: storage and arithmetic of the block factors (Fig. 2 step 2)
                             and of the block solves 6.1 / 6.5 */
  int32_t spike_prec;     /* operands of the spike products of Fig. 2 step 4: equal to factor_prec
                             (SIMT), or, with FP32 factors, BF16 / BF16X3 (tensor cores, fp32
                             accumulation) */
  int32_t ghat_prec;      /* FP64, FP32, FP16 or BF16 storage of G^ (Sec. 3: dense per-partition
                             arrays); FP16/BF16 products accumulate in FP32 */
  int32_t inner_prec;     /* FP64 or FP32 vectors of the inner BiCGStab on G^ (6.3) */
  double tol_out;         /* outer stop: ||f - A x||_inf <= tol_out ||f||_inf, per system */
  int32_t maxit_out;      /* outer iteration cap (Sec. 4: 1000) */
  double tol_in;          /* inner stop: ||g^ - G^ z^||_2 <= tol_in ||g^||_2 (Sec. 4: 1e-4) */
  int32_t maxit_in;       /* inner iteration cap (Sec. 4: 100) */
  double pivot_tol;       /* |u_kk| < pivot_tol * max|row k of A_ii| => DDPS_ERR_SINGULAR_BLOCK */
  int32_t leaf_size;      /* nested-dissection leaf size of the block ordering (0 = default) */
  int32_t rhs_chunk;      /* spike right-hand sides per pass (0 = chosen from free memory) */
  int32_t verbose;        /* 1: print analysis statistics to stderr */
  int32_t debug_wait_timeout; /* 1: the tensor-core spike products first wait (bounded, about
                                 4096 polls) on an mbarrier that nothing arrives at, so that the
                                 wait runs out and ddps_factor returns DDPS_ERR_TIMEOUT; tests the
                                 failure path.  0 in normal use. */
  int32_t fused_rows;     /* tensor-core spikes: a front with at most this many output rows of a
                             sweep (backward: its k pivots, forward: its order m) runs both
                             products of the sweep as one GEMM with a precomputed block
                             (0 = the largest supported, 512; -1 = never, every front takes the
                             two tile products) */
  int32_t ghat_mode;      /* ddps_ghat_mode; 0 = EXPLICIT is the paper's method */
  int32_t update_prec;    /* dense trailing updates of the block LU of large fronts (Fig. 2
                             step 2): FP64 or FP32 = SIMT in factor_prec (either value);
                             BF16X3 = with FP32 factors, blocks of 256 pivots whose update of
                             the rest of the front runs on the tensor cores (bf16 high part and
                             remainder, fp32 accumulation, about 16 correct bits per product) */
  int32_t reduced_solver; /* ddps_reduced_solver; DIRECT needs an explicit G^ (ghat_mode 0) and
                             a chain partition, else ddps_analyze returns DDPS_ERR_INVALID_ARG */
  int32_t use_graphs;     /* 1 (default): launch sequences that repeat unchanged (the factor
                             phase, chunks of inner iterations, a direct-mode preconditioner
                             application) are captured into CUDA graphs on a stream of the
                             handle at their first use and replayed afterwards; 0: plain
                             launches.  Graphs are not used while profiling is on. */
  int32_t persistent_solve; /* 1 (default): the block solves (6.1, 6.5) sweep the deep levels of
                             small fronts (at most 128 rows) in one persistent launch per sweep,
                             fronts ordered by per-front completion flags with bounded waits
                             (a wait that runs out makes ddps_solve return DDPS_ERR_TIMEOUT);
                             0: one launch per tree depth */
  int32_t factor_kind;    /* a ddps_factor_kind value; 0 = exact LU */
  int32_t autotune;       /* 1 (default): the first ddps_factor times every candidate launch shape
                             of each block-solve depth and sweep (warp per front, CTA per front,
                             clusters of 1-8 CTAs) on the handle's factors and keeps the fastest;
                             choices are cached per process and, when the environment variable
                             DDPS_TUNE_CACHE names a file, in that JSON file; 0: fixed rules */
  int32_t csr_kernel;     /* kernel of the products with A and R~: -1 (default) the autotuner's
                             choice (row blocks through shared memory when autotune is 0);
                             0 row blocks, 1 / 2: 4 / 8 lanes per row, 3: row blocks with
                             all of a block's loads issued at once, 4: 32-row groups per warp
                             copied asynchronously into shared memory; other values are
                             rejected */
} ddps_options;

typedef struct {
  double outer_iterations;   /* max over systems; half steps count 0.5 (Sec. 4 convention) */
  int32_t inner_iterations;  /* total inner BiCGStab iterations, all preconditioner applications */
  int32_t precond_applies;   /* Fig. 3 applications */
  int32_t converged;         /* 1 if every system met tol_out */
  int32_t guess_used;        /* 1 if a reduced initial guess was used (and accepted) */
  double relres_inf;         /* max over systems of ||f - A x||_inf / ||f||_inf (recomputed) */
  double first_inner_iters;  /* inner iterations of the first preconditioner application */
  double ms_solve;           /* wall time of the call, host clock */
} ddps_solve_info;

typedef struct {
  int64_t n, nnz, nsys, nblocks;
  int64_t m;                 /* |c|: order of the reduced system G^ */
  int64_t nnz_rt;            /* stored entries of R~ */
  int64_t nfronts, nlevels;  /* multifrontal tree of all blocks */
  int64_t factor_entries;    /* sum over fronts of m_f^2 (dense front storage) */
  int64_t factor_lu_entries; /* entries of L and U proper (what a solve streams) */
  int64_t ghat_entries;      /* sum over blocks of |c ∩ block| * |c_i| */
  int64_t max_front;         /* largest front order */
  int64_t max_rhs;           /* largest |c_i| (spike right-hand sides of one block) */
  int64_t device_bytes;      /* device memory held by the handle */
  double factor_flops;       /* partial-LU flops of all fronts */
  double spike_flops;        /* multi-RHS forward/backward flops for G^ */
  double direct_flops;       /* reduced_solver DIRECT: flops of the block LU of G^ per factor */
  int64_t direct_bytes;      /* reduced_solver DIRECT: FP32 matrix bytes one reduced solve reads */
} ddps_sizes;

/* Fills *opt with the paper's solver settings (Sec. 4: eps_in 1e-4, 100 inner
 * and 1000 outer iterations) and a 1e-10 outer tolerance, FP64 everywhere,
 * no dropping. */
void ddps_default_options(ddps_options* opt);

/* Symbolic phase: split A = D + R by block rows (Eq. (1)-(2)), apply the drop
 * rule (Fig. 2 step 3), find c (Fig. 2 step 5), order every A_ii by nested
 * dissection and lay out the multifrontal factors, the spikes and G^.
 * Sec. 3 notes that stages 1-5 need no right-hand side.
 *   n, nnz            order and stored entries of the stacked matrix
 *   rowptr, colind    host CSR pattern (n+1 and nnz entries)
 *   p, block_ptr      host, p+1 increasing row offsets, block_ptr[0]=0, block_ptr[p]=n
 *   nsys, sys_block_ptr  host, nsys+1 block offsets (NULL with nsys=1: one system)
 *   values            host float64[nnz]; required when opt->drop_mode != NONE (the
 *                     drop rule reads values), else may be NULL
 *   opt               host options (NULL = defaults)
 * The blocks are analysed on host threads (the environment variable
 * DDPS_ANALYZE_THREADS sets their number, default the CPUs the process may run
 * on, up to 64); the analysis is the same for every thread count.  The call returns
 * after all of them have finished.
 * On success *out owns the analysis and the device copies of the pattern. */
ddps_status ddps_analyze(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colind,
                         int32_t p, const int64_t* block_ptr, int32_t nsys,
                         const int32_t* sys_block_ptr, const double* values,
                         const ddps_options* opt, ddps_handle** out);

/* Numeric phase, Fig. 2 steps 1-4: scatter A's values into the factor fronts
 * and R~, factor every A_ii, form the spikes and store G^ = I + G(c,c).
 *   values  device float64[nnz], same pattern as at analysis
 * Synchronises `stream` once at the end to read the pivot check; returns
 * DDPS_ERR_SINGULAR_BLOCK (see ddps_last_error for block and row) when a
 * pivot fails the threshold. */
ddps_status ddps_factor(ddps_handle* h, const double* values, void* stream);

/* Same as ddps_factor with the values in host memory (host float64[nnz],
 * read during the call; pinned memory makes the copy asynchronous).  The
 * copy into the handle's value array is enqueued on `stream`. */
ddps_status ddps_factor_host(ddps_handle* h, const double* values_host, void* stream);

/* Fig. 2 step 6: right-preconditioned BiCGStab on A x = f with the DDPS
 * preconditioner, per-system scalars, stopping on the recomputed true
 * residual (tol_out, infinity norm, relative to ||f||_inf).
 *   f     device float64[n * nrhs]: nrhs right-hand sides, each n contiguous
 *         entries (column-major n x nrhs)
 *   x     device float64[n * nrhs] (output), same layout
 *   nrhs  number of right-hand sides (>= 1); they are solved one after the
 *         other with the same factors (the factor phase needs no right-hand
 *         side, Sec. 3)
 *   x0    device float64[n * nrhs] initial guesses, or NULL for x0 = 0; a
 *         guess that already meets tol_out is returned after no iteration
 *   info  host, may be NULL: iterations are the largest over the right-hand
 *         sides, inner iterations and applications the totals, relres_inf
 *         the worst, first_inner_iters that of the first right-hand side.
 * Synchronises `stream` (convergence is read on the host between iterations).
 * Returns DDPS_ERR_NOT_CONVERGED when some system misses tol_out within
 * maxit_out (x then holds the last iterate). */
ddps_status ddps_solve(ddps_handle* h, const double* f, double* x, int32_t nrhs, const double* x0,
                       void* stream, ddps_solve_info* info);

/* Same as ddps_solve with host buffers: copies f (and x0) to the device,
 * solves and copies x back (f, x, x0: host float64[n * nrhs]; x0 may be
 * NULL).  Synchronises. */
ddps_status ddps_solve_host(ddps_handle* h, const double* f_host, double* x_host, int32_t nrhs,
                            const double* x0_host, void* stream, ddps_solve_info* info);

/* Initial guess for the reduced unknowns z^ of the first preconditioner
 * application of the next solves (the hook a learned predictor fills).
 *   zhat0  device float64[m] in the order of c; NULL removes the guess.
 * The guess is used only if its reduced residual is smaller than that of
 * z^ = 0; the inner BiCGStab then runs to tol_in from it as usual. */
ddps_status ddps_set_reduced_guess(ddps_handle* h, const double* zhat0, void* stream);

/* Copies the reduced solution z^ and the reduced right-hand side g^ of the
 * first preconditioner application of the last solve (device float64[m]
 * each; either may be NULL).  Enqueued on `stream`. */
ddps_status ddps_get_reduced_solution(ddps_handle* h, double* zhat, double* ghat, void* stream);

/* Fig. 3 step 6.1 alone: g = D~^-1 y for all blocks (device float64[n] in/out). */
ddps_status ddps_block_solve(ddps_handle* h, const double* y, double* g, void* stream);

/* Same result as ddps_block_solve, for callers that cannot allocate device
 * memory when they need it (for example a program whose memory pool already
 * owns all free device memory, or whose policy allows device allocations
 * only at start-up).  The paper has no counterpart: this is a deployment
 * variant.  Its per-call scratch (the front vectors of the two sweeps) comes
 * from a fixed 16 MiB array compiled into the library, held by every GPU
 * that loads the library until the process exits, instead of the handle's
 * workspace; the call allocates nothing.
 *   y, g    device float64[n] (input, output)
 * Returns DDPS_ERR_INVALID_ARG when the analysed problem needs more scratch
 * than the array holds (n + the multifrontal update entries, times the
 * factor element size, must fit in 16 MiB).  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  The
 * address is cached per device and per context: after a device reset
 * (cudaDeviceReset) the first call in the new context looks it up again.
 * All calls share the one array: calls whose work overlaps on the GPU (other
 * streams, other handles, other threads) race on it and must be ordered by
 * the caller. */
ddps_status ddps_block_solve_noalloc(ddps_handle* h, const double* y, double* g, void* stream);

/* Fig. 3 steps 6.1-6.2: the reduced right-hand side g^ = (D~^-1 y)(c) that
 * the first preconditioner application of a solve with f = y would see
 * (y device float64[n], ghat device float64[m]).  A predictor of z^ can
 * use it as a feature before the solve starts. */
ddps_status ddps_reduced_rhs(ddps_handle* h, const double* y, double* ghat, void* stream);

/* Fig. 3 step 6.2 product: w = G^ v = v + G(c,c) v (device float64[m] in/out);
 * with ghat_mode IMPLICIT it is computed as v + (D~^-1 (R~ v))(c). */
ddps_status ddps_reduced_matvec(ddps_handle* h, const double* v, double* w, void* stream);

/* Fig. 3 step 6.3 alone: z^ = G^-1 g^ with the handle's reduced solver
 * (device float64[m] in/out, c order): DIRECT solves with the block LU of
 * the factor phase; ITERATIVE runs the inner BiCGStab to tol_in from z^ = 0
 * (synchronising `stream` between inner iterations). */
ddps_status ddps_reduced_solve(ddps_handle* h, const double* ghat, double* zhat, void* stream);

/* Fig. 3 in full: z = P^-1 y (device float64[n] in/out).  Runs the inner
 * solve from z^ = 0; synchronises `stream` between inner iterations. */
ddps_status ddps_precond_apply(ddps_handle* h, const double* y, double* z, void* stream);

/* y = A x with the analysed pattern and the last factored values
 * (device float64[n] in/out). */
ddps_status ddps_spmv(ddps_handle* h, const double* x, double* y, void* stream);

/* Sizes of the analysis (host struct). */
ddps_status ddps_get_sizes(const ddps_handle* h, ddps_sizes* s);

/* The autotuner's choices as a JSON text (per block-solve depth: fronts,
 * largest front, chosen shape per sweep and its time): at most cap-1 bytes
 * and a terminating zero are written to buf (host, may be NULL); *len (host,
 * may be NULL) receives the full length. */
ddps_status ddps_get_tuning(const ddps_handle* h, char* buf, int64_t cap, int64_t* len);

/* The interface set c (host int64[m], global row indices, ascending within
 * each system, systems in order). */
ddps_status ddps_get_interface(const ddps_handle* h, int64_t* c);

/* Layout of G^ for block b: rows q0..q1-1 of the reduced system (the rows of
 * the block that lie in c) and ncols coupling columns; cols (host int64[ncols],
 * may be NULL) receives their positions in c. */
ddps_status ddps_get_ghat_layout(const ddps_handle* h, int32_t b, int64_t* q0, int64_t* q1,
                                 int64_t* ncols, int64_t* cols);

/* Copies G(c ∩ block b, c_b) — the off-identity part of block b's rows of
 * G^ — row-major, converted to float64, into host memory dst
 * ((q1-q0) * ncols entries).  Synchronises `stream`.  DDPS_ERR_STATE when
 * G^ is implicit (ghat_mode IMPLICIT stores no spikes). */
ddps_status ddps_get_ghat_block(ddps_handle* h, int32_t b, double* dst, void* stream);

/* Number of kernels this handle has launched since ddps_analyze (host
 * counter, read without synchronising). */
int64_t ddps_launch_count(const ddps_handle* h);

/* Kernel classes timed by ddps_set_profiling. */
enum {
  DDPS_PROF_ASSEMBLE = 0,      /* scatter of A's values into the fronts, pivot thresholds */
  DDPS_PROF_EXTEND_ADD = 1,    /* child Schur complements added into parent fronts */
  DDPS_PROF_FRONT_LU = 2,      /* partial LU of the fronts (Fig. 2 step 2) */
  DDPS_PROF_SPIKE_FWD = 3,     /* multi-RHS forward substitution (Fig. 2 step 4) */
  DDPS_PROF_SPIKE_BWD = 4,     /* multi-RHS backward substitution (Fig. 2 step 4) */
  DDPS_PROF_GHAT_EXTRACT = 5,  /* rows of the spikes in c written into G^ */
  DDPS_PROF_BLOCK_SOLVE = 6,   /* g = D~^-1 y (6.1 and the retrieval) */
  DDPS_PROF_GHAT_MATVEC = 7,   /* w = G^ v (6.3) */
  DDPS_PROF_SPMV = 8,          /* y = A x (outer Krylov) */
  DDPS_PROF_DIRECT_FACTOR = 9, /* block LU of G^ (reduced_solver DIRECT) */
  DDPS_PROF_DIRECT_SOLVE = 10, /* z^ = G^-1 g^ with that LU (reduced_solver DIRECT) */
  DDPS_PROF_CLASSES = 11
};

/* Enables CUDA-event timing of the kernel classes whose bit (1 << class) is
 * set in mask (0 disables).  Every timed launch group is bracketed by an event
 * pair on the stream it runs on. */
ddps_status ddps_set_profiling(ddps_handle* h, int32_t mask);

/* Totals since the last reset: ms[c] (host double[DDPS_PROF_CLASSES]) and
 * count[c] (host int64[DDPS_PROF_CLASSES], launch groups timed); either may be
 * NULL.  Waits for the recorded events.  reset != 0 clears the totals. */
ddps_status ddps_get_profile(ddps_handle* h, double* ms, int64_t* count, int32_t reset);

/* Host-only symbolic analysis: runs the analysis of ddps_analyze without any
 * device work and reports its sizes (may be NULL), the new-to-old row
 * permutation of the nested-dissection orders (host int32[n], may be NULL)
 * and the interface set c (host int64 array with room for n entries, the
 * first sizes->m are written; may be NULL).  Arguments as ddps_analyze. */
ddps_status ddps_symbolic(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colind,
                          int32_t p, const int64_t* block_ptr, int32_t nsys,
                          const int32_t* sys_block_ptr, const double* values,
                          const ddps_options* opt, ddps_sizes* sizes, int32_t* perm, int64_t* c);

/* Frees the handle and all device memory it holds (NULL is a no-op). */
ddps_status ddps_destroy(ddps_handle* h);

/* Text of the last error on h (or of the last failed ddps_analyze when h is NULL). */
const char* ddps_last_error(const ddps_handle* h);
const char* ddps_status_string(ddps_status s);

/* ------------------------------------------------------------------------
 * Learned initial guess for 6.3: a multilayer perceptron with `layers`
 * hidden layers of width `hidden`, ReLU, linear output; loss
 * (1/2B) sum_b ||y_b - t_b||^2; Adam with bias correction.  The network has
 * no counterpart in the paper; it fills the initial-guess slot of the inner
 * iterative solve (6.3), whose result still has to meet tol_in.
 * Parameters are one float32 device array laid out
 *   [W1 (hidden x d_in) row-major, b1, W2 (hidden x hidden), b2, ...,
 *    W_out (d_out x hidden), b_out].
 * ------------------------------------------------------------------------ */

/* Number of float32 parameters. */
int64_t ddps_mlp_param_count(int32_t d_in, int32_t hidden, int32_t layers, int32_t d_out);

/* Bytes of device workspace the forward/backward calls need for batch B. */
int64_t ddps_mlp_workspace_bytes(int32_t d_in, int32_t hidden, int32_t layers, int32_t d_out,
                                 int32_t B);

/* Y = net(X): X device float32[B x d_in] row-major, Y device float32[B x d_out]. */
ddps_status ddps_mlp_forward(const float* params, int32_t d_in, int32_t hidden, int32_t layers,
                             int32_t d_out, const float* X, int32_t B, float* Y, void* workspace,
                             void* stream);

/* grads (device float32[param_count]) = d loss / d params for targets T
 * (device float32[B x d_out]); loss (device float32[1]) receives the loss. */
ddps_status ddps_mlp_backward(const float* params, int32_t d_in, int32_t hidden, int32_t layers,
                              int32_t d_out, const float* X, const float* T, int32_t B,
                              float* grads, float* loss, void* workspace, void* stream);

/* One Adam step in place over `count` parameters; m, v are device float32
 * moment buffers (zero before step 1); step is the 1-based step number. */
ddps_status ddps_mlp_adam(float* params, const float* grads, float* m, float* v, int64_t count,
                          float lr, float beta1, float beta2, float eps, int32_t step,
                          void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DDPS_H */
