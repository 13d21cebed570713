/*
 * bdfb.h - C ABI of libbdfb: batched variable-order BDF / Newton integration
 * of many independent small ODE systems on one NVIDIA B300 (sm_103a).
 *
 * The calls follow the integrator interface the paper keeps unchanged between
 * its CPU and GPU builds (Sec. 5): create / init / set tolerances /
 * integrate to tout / get stats.
 * The per-cell ("submodel") use case of Sec. 2 - many small independent
 * systems, each a diagonal block of one block-diagonal Jacobian (Fig. 1) - is
 * integrated with per-cell step control, Newton iteration and a direct solve
 * of each block of M = I - gamma J.  Vector kernels follow the streaming and
 * reduction operations of the NVECTOR class (Sec. 4).
 *
 * Conventions for every entry point:
 *  - Return value: BDFB_SUCCESS (0) or a negative BDFB_* code; nothing traps
 *    or aborts.  bdfb_strerror() gives a message.
 *  - Memory ownership follows the paper's SUNMemory ownership flag (Sec. 3):
 *    buffers passed in are owned by the caller and never freed by the
 *    library; memory the library allocates is owned by the context and freed
 *    by bdfb_destroy().
 *  - "device" pointers are CUDA device (or managed) addresses on the current
 *    device; "host" pointers are ordinary host memory.  Where a call takes a
 *    bdfb_mem flag the caller states which one it passes (Sec. 3 memory type).
 *  - All GPU work is issued on the stream set with bdfb_set_stream (default:
 *    the legacy default stream).  Vector operations are asynchronous; calls
 *    that return a scalar to the host synchronise that stream (Sec. 4.1).
 *  - Device arrays of doubles must be 8-byte aligned; the vector kernels take
 *    a faster path when all their arrays are 16-byte aligned.
 */
#ifndef BDFB_H
#define BDFB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
enum {
  BDFB_SUCCESS = 0,
  BDFB_TOO_MUCH_WORK = -1,   /* mxstep steps taken before tout */
  BDFB_ERR_FAILURE = -3,     /* error test failed 7 times in one step, or h underflow */
  BDFB_CONV_FAILURE = -4,    /* Newton failed 10 times in one step */
  BDFB_LSETUP_FAIL = -6,
  BDFB_LSOLVE_FAIL = -7,
  BDFB_RHSFUNC_FAIL = -8,
  BDFB_MEM_FAIL = -20,       /* device or host allocation failed */
  BDFB_CUDA_FAIL = -21,      /* a CUDA runtime call failed */
  BDFB_ILL_INPUT = -22       /* bad argument (null pointer, size, option, ...) */
};

typedef enum { BDFB_MEM_HOST = 0, BDFB_MEM_DEVICE = 1 } bdfb_mem;
typedef enum {
  BDFB_ROBERTSON = 0,
  BDFB_MASSACTION = 1,
  BDFB_BRUSSELATOR3D = 2,
  BDFB_BRUSSELATOR1D = 3,
  BDFB_MASSACTION_SHARED = 4
} bdfb_kind;

const char* bdfb_strerror(int code);
/* library version as an integer (major * 10000 + minor * 100 + patch) */
int bdfb_version(void);

/* ------------------------------------------------ NVECTOR operations (Sec. 4)
 * Length-n FP64 vectors in device memory; stream = cudaStream_t (NULL: default
 * stream).  Streaming operations are asynchronous.  Reductions write their
 * result to device memory (`out`, nv doubles) and need a caller-owned device
 * workspace of bdfb_nv_work_doubles(n, nv) doubles that is zero when first
 * used (the kernels leave it zero again); calls that share a workspace must
 * not overlap on the GPU.  n = 0 is valid (no work; reductions give 0). */

/* z = a x + b y  (N_VLinearSum; z may alias x or y) */
int bdfb_nv_linear_sum(int64_t n, double a, const double* x, double b, const double* y,
                       double* z, void* stream);
/* the support operations: z = c x (N_VScale), z = c (N_VConst), z = |x|
 * (N_VAbs), z = 1 / x (N_VInv), z = x + b (N_VAddConst), and the fused error
 * weights w = 1 / (rtol |y| + atol) (rtol >= 0, atol > 0); z may alias x */
int bdfb_nv_scale(int64_t n, double c, const double* x, double* z, void* stream);
int bdfb_nv_const(int64_t n, double c, double* z, void* stream);
int bdfb_nv_abs(int64_t n, const double* x, double* z, void* stream);
int bdfb_nv_inv(int64_t n, const double* x, double* z, void* stream);
int bdfb_nv_add_const(int64_t n, const double* x, double b, double* z, void* stream);
int bdfb_nv_error_weights(int64_t n, double rtol, double atol, const double* y, double* w, void* stream);
/* z = sum_{j<nv} c[j] x[j]; c is a host array, x a host array of nv device
 * pointers; 1 <= nv <= 16  (N_VLinearCombination; z may alias x[0]) */
int bdfb_nv_linear_combination(int64_t n, int nv, const double* c, const double* const* x,
                               double* z, void* stream);
/* z[j] = a[j] x + y[j], j < nv; a host array, y and z host arrays of device
 * pointers; 1 <= nv <= 16  (N_VScaleAddMulti; z[j] may alias y[j]) */
int bdfb_nv_scale_add_multi(int64_t n, int nv, const double* a, const double* x,
                            const double* const* y, double* const* z, void* stream);
/* out[j] = x . y[j], j < nv, 1 <= nv <= 16  (N_VDotProdMulti) */
int bdfb_nv_dot_prod_multi(int64_t n, int nv, const double* x, const double* const* y,
                           double* out, double* work, void* stream);
/* out[0] = sqrt(sum_i (x_i w_i)^2 / n)  (N_VWrmsNorm) */
int bdfb_nv_wrms_norm(int64_t n, const double* x, const double* w, double* out, double* work,
                      void* stream);
/* size (in doubles) of the reduction workspace for length n and nv results */
int64_t bdfb_nv_work_doubles(int64_t n, int nv);

/* out[j] = x . y[j] like bdfb_nv_dot_prod_multi, for callers that cannot
 * allocate device memory or hand the library a workspace: applications whose
 * own memory manager owns every device byte, and code that must avoid the
 * device synchronisation an allocation can trigger.  The paper has no
 * counterpart; it is an extension of this library.
 *  - Allocates nothing: its scratch is a fixed array of
 *    16 * 1024 + 2 doubles (128 KiB + 16 B) inside the library's device image,
 *    present on every GPU that loads the library until the process exits.
 *  - Limit: 1 <= nv <= bdfb_nv_noalloc_max_nv() (16); a larger nv returns
 *    BDFB_ILL_INPUT.  Any n >= 0.
 *  - The first call on a device looks up the scratch's device address (a
 *    runtime query, no allocation); make that first call before any stream
 *    capture on that device.  The address is cached for the life of the
 *    process: cudaDeviceReset on that device invalidates it, so do not call
 *    this entry point on a device after resetting it.
 *  - All calls on one device share the scratch: calls that overlap on the GPU
 *    (other streams or host threads) race, so serialise them.  Each call
 *    clears the scratch's arrival counter on `stream` before using it.
 *  - x, y[j] (host array of nv device pointers) and out (nv doubles) are
 *    caller-owned device memory; stream = cudaStream_t (NULL: default). */
int bdfb_nv_dot_prod_multi_noalloc(int64_t n, int nv, const double* x, const double* const* y,
                                   double* out, void* stream);
/* largest nv bdfb_nv_dot_prod_multi_noalloc accepts */
int64_t bdfb_nv_noalloc_max_nv(void);

/* --------------------------------------- batched dense LU of M = I - gamma J
 * nb independent n x n blocks, block b at a + b * n * n, row-major, FP64,
 * device memory (the block-diagonal matrix of Fig. 1 / Sec. 5).  Partial
 * pivoting, ties to the lowest row.  piv[b * n + k] = pivot row of step k.
 * info[b] = 0, or k + 1 when pivot k was exactly zero.  1 <= n <= 64. */
int bdfb_batched_lu_factor(int64_t nb, int n, double* a, int32_t* piv, int32_t* info,
                           void* stream);
/* solve M x = b in place for every block with the factors above */
int bdfb_batched_lu_solve(int64_t nb, int n, const double* lu, const int32_t* piv, double* b,
                          void* stream);
/* Mixed precision (FP32 factorisation, FP64 refinement): for every FP64
 * block a (not modified) solve a x = b: LU of the block in FP32, then
 * x += LU^{-1} r with the FP64 residual r = b - a x until the normwise
 * backward error |r|_inf / (|a|_inf |x|_inf + |b|_inf) <= 1e-12, at most 5
 * sweeps.  A block that does not reach 1e-12 in 5 sweeps (or whose FP32
 * factorisation meets a zero pivot) is factored and solved in FP64 by
 * partially pivoted LU instead, as the integrator does.  sweeps[blk] =
 * refinement sweeps used (1..5), 0 when the FP64 fallback solved the block,
 * -2 when the FP64 factorisation met an exactly zero pivot as well (x then
 * holds the last refined iterate).  1 <= n <= 64; all arrays device memory. */
int bdfb_batched_solve_mixed(int64_t nb, int n, const double* a, const double* b, double* x,
                             int32_t* sweeps, void* stream);

/* ------------------------------- shared-pattern block-sparse matrices
 * Block-diagonal matrices whose square blocks share one sparsity pattern
 * (Sec. 5: the submodel case's blocks keep one copy of the CSR row pointers
 * and column indices for all blocks).  bdfb_sparse_create analyses the
 * pattern once on the host: LU without pivoting, pivots taken in row order
 * (the paper's batched QR pivots neither), fill-in and elimination schedule.
 * Device values are entry-major: entry e of block b at v[e nb + b] (one
 * thread per block; a warp's accesses are 32 consecutive doubles).
 *  create:  n (1..2048), nnz, rowptr[n+1], colind[nnz] (host, 0-based, no
 *           duplicates, columns in any order); the diagonal joins the
 *           pattern.  BDFB_ILL_INPUT on a malformed pattern.  *out owns
 *           device copies of the schedule; free with bdfb_sparse_destroy.
 *  lu_nnz:  entries of the factor's pattern (with fill).
 *  load:    lu (device, lu_nnz x nb doubles) <- the blocks' values a
 *           (device, block-major: a[b nnz + e] in the CSR order of create),
 *           fill entries zero.
 *  factor:  every block in place: L unit lower (multipliers), U upper with
 *           its diagonal replaced by the reciprocal; info[b] (device, may be
 *           NULL) = 0 or k + 1 for a zero or non-finite pivot at step k.
 *  solve:   x <- M_b^{-1} x for every block, x device entry-major (x[i nb + b]).
 * All calls are asynchronous on `stream`. */
typedef struct bdfb_sparse bdfb_sparse;
int bdfb_sparse_create(int n, int nnz, const int32_t* rowptr, const int32_t* colind, bdfb_sparse** out);
void bdfb_sparse_destroy(bdfb_sparse* sp);
int64_t bdfb_sparse_lu_nnz(const bdfb_sparse* sp);
int bdfb_sparse_load(const bdfb_sparse* sp, int64_t nb, const double* a, double* lu, void* stream);
int bdfb_sparse_factor(const bdfb_sparse* sp, int64_t nb, double* lu, int32_t* info, void* stream);
int bdfb_sparse_solve(const bdfb_sparse* sp, int64_t nb, const double* lu, double* x, void* stream);

/* ---------------------------------------------------- per-cell problems
 * kind BDFB_ROBERTSON: k[3 c + {0,1,2}] = (k1, k2, k3) of cell c, n = 3.
 * kind BDFB_MASSACTION: cell c has n[c] species (1 <= n <= 56) stored at
 *   y[y_off[c] .. y_off[c+1]) and reactions rxn_off[c] .. rxn_off[c+1)
 *   (at most 2 * 56 per cell); reaction r consumes the distinct local species
 *   reactants[4 r .. 4 r + 3] and produces products[4 r .. 4 r + 3]
 *   (255 = empty slot) at rate k[r] * prod(y[reactants]).
 * kind BDFB_BRUSSELATOR3D: one coupled system (the Sec. 2 "full model" case):
 *   the Brusselator reaction terms of Sec. 7 with diffusion D lap() on a
 *   periodic nx^3 grid over [0,1)^3 (7-point Laplacian); k = {A, B, eps, D,
 *   nx} (5 doubles); ncell = nx^3; y is species-major, y[s nx^3 + (i nx + j)
 *   nx + l] for species s = u, v, w.  Integrated with one shared step size,
 *   global WRMS norms, Newton + GMRES (option "maxl", default 5, at most 16)
 *   left-preconditioned by the 3x3 reaction blocks; control on the host.
 *   Option "precision" 1 forms the preconditioner blocks and applies the
 *   Newton operator inside GMRES in FP32 (the right-hand side, the Newton
 *   residual, the Krylov basis and its orthogonalisation stay FP64: inexact
 *   Newton-Krylov with a matrix-vector product accurate to ~1e-7, far inside
 *   the linear tolerance); 0 (default) is FP64 throughout.  The same option
 *   selects this for BDFB_BRUSSELATOR1D's BDF path.
 * kind BDFB_BRUSSELATOR1D: the demonstration problem of Sec. 7 as one
 *   coupled system: the same reaction terms with advection -c d/dx (first-
 *   order upwind differences) on a periodic line of nx points over
 *   [0, len); k = {A, B, eps, c, len, nx} (6 doubles); ncell = nx; y is
 *   species-major, y[s nx + i] at x = i len / nx.  Integrated like
 *   BDFB_BRUSSELATOR3D (advection implicit inside the Newton operator), or,
 *   with option "imex" = 1 set before bdfb_init, by the paper's own
 *   integrator type: an IMEX additive Runge-Kutta method (ARK3(2)4L[2]SA of
 *   Kennedy and Carpenter) with the advection explicit and the reactions
 *   implicit, every implicit stage solved by Newton on the 3x3 point blocks
 *   (exact Jacobian at each iterate, one convergence test over the whole
 *   vector: the demonstration's task-local solver with one task per GPU);
 *   embedded error estimate, PID step control, last step clamped on tout.
 *   An integrate with "imex" = 1 before an init that followed it fails
 *   with BDFB_ILL_INPUT.  Option "precision" on this kind selects the IMEX
 *   path's arithmetic: 0 (default) FP64 throughout; 1 forms and solves the
 *   3x3 Newton blocks in FP32 and keeps FP32 norm weights, with the state,
 *   stage sums, reaction terms and Newton residual in FP64 (the iteration
 *   converges to the same FP64 residual test).  Option "device_loop" 1 runs
 *   the IMEX step loop to tout in one cooperative launch (grid-wide barriers
 *   in place of host round trips: every block takes the same decisions from
 *   the same sums); 0 drives it from the host; -1 (default) takes the
 *   former up to 2e6 points.
 * kind BDFB_MASSACTION_SHARED: ncell cells that share ONE network (the
 *   submodel case of Sec. 2 and Sec. 5 with one sparsity pattern for every
 *   block): n[0] species (1..255), reactions rxn_off[0] = 0 .. rxn_off[1]
 *   (at most 65535), reactants / products / k of that network (host memory
 *   only; y_off unused).  y is species-major, y[s ncell + c].  By default
 *   integrated as one grouped system (shared step size and order, error test
 *   over all species) with task-local Newton solves per cell on the shared
 *   sparse pattern of M = I - gamma J (bdfb_sparse's LU, one thread per
 *   cell).  Option "grouped" 0 (set before bdfb_init) integrates every cell
 *   with its own step size and order instead, one thread per cell running
 *   the per-cell integrator's step (the same readings as BDFB_MASSACTION)
 *   on the shared sparse LU; per-cell statuses then fill `status`.
 *   Options mxstep, qmax, interp, grouped and lsolver 0 (any other option
 *   returns BDFB_ILL_INPUT); (LU entries with fill, reactions and species)
 *   x ncell must stay below 2^30 (BDFB_ILL_INPUT otherwise: about 9e5
 *   cells of a 128-species banded network).  bdfb_get_cell_stats gives, grouped, one row: nst, nfe,
 *   nsetups, nni (summed over cells), ncfn, netf, LU entries with fill,
 *   entries of M's pattern; per cell, one row per cell as for
 *   BDFB_MASSACTION.
 * y_off / rxn_off have ncell + 1 entries starting at 0.  `mem` says where all
 * arrays live; bdfb_create copies everything it needs, so the caller may
 * free its arrays when bdfb_create returns. */
typedef struct {
  int32_t kind;              /* bdfb_kind */
  int32_t mem;               /* bdfb_mem of every array below */
  int64_t ncell;
  const int32_t* n;          /* [ncell] (mass action; NULL for Robertson) */
  const int64_t* y_off;      /* [ncell + 1] (NULL for Robertson: 3 c) */
  const int64_t* rxn_off;    /* [ncell + 1] (mass action) */
  const uint8_t* reactants;  /* [4 nrxn] */
  const uint8_t* products;   /* [4 nrxn] */
  const double* k;           /* [nrxn] or [3 ncell] */
} bdfb_problem;

typedef struct {
  int64_t ncell;
  int64_t nsteps, nfevals, nlinsetups, nniters, nncfails, netfails; /* sums over cells */
  int64_t max_steps, min_steps;                                     /* per-cell extremes */
  int64_t ncells_failed;                                            /* status != 0 */
  int64_t nrefine, nrefine_fallback;  /* mixed precision: refinement sweeps, FP64 refactorisations */
  double last_kernel_ms;              /* device time of the last integrate's kernels */
  int64_t nguess, nguess_fallback;    /* learned guesses taken; of those, Newton solves redone from 0 */
  int64_t graph_captures, graph_launches;  /* option "graph": captures made, replays launched */
} bdfb_stats;

typedef struct bdfb_ctx bdfb_ctx;

int bdfb_create(const bdfb_problem* prob, bdfb_ctx** out);
void bdfb_destroy(bdfb_ctx* ctx);
/* cudaStream_t for all later work of this context */
int bdfb_set_stream(bdfb_ctx* ctx, void* stream);
/* scalar relative and absolute tolerances (defaults 1e-6, 1e-10) */
int bdfb_set_tolerances(bdfb_ctx* ctx, double rtol, double atol);
/* Integer options:
 *  "mxstep"    steps allowed per cell per integrate call (default 100000)
 *  "mapping"   0 = automatic tiles by cell size (default), 32 = one warp per
 *              cell for every cell in input order (the plain form)
 *  "precision" 0 = FP64 factorisation (default), 1 = FP32 factorisation with
 *              FP64 iterative refinement to 1e-12 backward error for the
 *              cells of more than 32 species (where the factorisation
 *              dominates a step); smaller cells keep FP64 factors, which
 *              are faster there on B300, unless "mixed_small" is 1
 *  "mixed_small" 1 = precision 1 factors every cell in FP32 (mass action;
 *              default 0)
 *  "graph"     1 = capture integrate's launch sequence (counter reset, one
 *              persistent launch per kernel variant on forked streams, join)
 *              into a CUDA graph once and replay it; a call that differs only
 *              in tout patches tout into the graph, any other change
 *              (tolerances, options, schedule) recaptures
 *  "autotune"  1 = on the next integrate, and again after a precision change,
 *              time every kernel variant (bdfb_get_mapping) whose NMAX covers
 *              a size class (classes with one such variant are not timed) on
 *              a sample of that class (first 16384 cells, current state to
 *              tout, on scratch copies: the context's state is untouched)
 *              and run each class on the fastest (another variant must beat
 *              the class's own by 3%); mapping 0 only.  Variants differ in
 *              rounding order, so tuned runs agree with untuned ones to
 *              rounding, not bitwise.
 *  "qmax"      maximum BDF order, 1..5 (default 5)
 *  "predictor" 0 = Newton starts from a zero correction (default), 1 = from
 *              the learned guess of bdfb_load_mlp (every cell n <= 10, FP64
 *              factorisation; runs one warp per cell).  The unchanged Newton
 *              convergence test judges the guess.  A guess that would fail
 *              the local error test itself (E_q |guess| > 1) is dropped;
 *              when the Newton solve from a guess fails, or converges to a
 *              correction that fails the local error test, it is repeated
 *              from zero.  Both count in nguess_fallback, not as failures.
 *              The first Newton step from a nonzero guess skips the
 *              stale-matrix scaling so that linear invariants (sum y for
 *              mass action) are kept as with a zero start, and its
 *              convergence test uses the rate carried over from earlier
 *              solves only when the guess lies closer to the new iterate
 *              than zero does (else rate 1).
 *  "grouped"   1 = integrate all cells as ONE system (the grouping of many
 *              small systems into one, Sec. 2, with the demonstration
 *              problem's task-local Newton solver, Sec. 7): one step size
 *              and order for every cell, the local
 *              error test on the norm over all species, and a task-local
 *              Newton solve — each cell's block of the Newton matrix is
 *              factored and iterated to its own convergence test (the same
 *              test as per-cell mode, in that cell's norm) and the step's
 *              solve fails if any cell's does.  FP64 only, no predictor.
 *              The Jacobian is refreshed for every cell at once (gamma
 *              ratio 0.3 or 20 steps, as per-cell).  Setting it makes the
 *              next integrate start from the state of the last bdfb_init.
 *              Statistics: every cell counts every grouped step, RHS
 *              evaluation, setup and failure; nniters sums the cells'
 *              task-local iterations.
 *  "lsolver"   linear solver of the per-cell Newton systems M x = b:
 *              0 = batched dense LU with partial pivoting (default);
 *              1 = explicit inverse: each setup inverts every cell's M by
 *              Gauss-Jordan elimination with partial pivoting in FP64 (the
 *              task-local block inverse of the demonstration problem,
 *              Sec. 7, for any block size) and each Newton solve is one
 *              matrix-vector product.  Equal to LU in exact arithmetic;
 *              three times the setup flops, no dependent triangular chain
 *              in the solves.  With "precision" 1 the FP32 LU of that
 *              mode is used either way.  Not with "predictor", a recording
 *              or "grouped".  Grid and shared-network contexts accept 0
 *              only (GMRES, sparse LU).
 *  "interp"    0 = the last step is shortened to end exactly at tout and y
 *              is the state there (default); 1 = steps are never shortened
 *              for tout: the integrator steps until t_n >= tout and writes
 *              the history polynomial sum_{j<=q} z_j s^j, s = (tout - t_n)/h
 *              (the normal output mode of a Nordsieck BDF integrator,
 *              Sec. 3).  The next call continues from t_n; a tout inside
 *              the last step (tout <= t_n) is answered by interpolation
 *              alone, with no step (a tout before that step's start is
 *              extrapolated from the same polynomial, not refused).  Every BDF path takes it (cells,
 *              "grouped", BDFB_MASSACTION_SHARED, both grids); the line's
 *              "imex" path always ends its steps at tout.
 * "mapping" 32 runs every cell on the smallest one-warp-per-cell kernel all
 * cells fit (NMAX 16 — the predictor's kernel, FP64 only — 32 or 56). */
int bdfb_set_option(bdfb_ctx* ctx, const char* key, int64_t value);
/* set t0 and copy the initial state (packed by y_off); mem: where y0 lives */
int bdfb_init(bdfb_ctx* ctx, double t0, const double* y0, int32_t mem);
/* Advance every cell to tout (each with its own h and order), write the
 * states at tout to y (packed by y_off) and per-cell status codes to status
 * (may be NULL).  Returns the worst (most negative) cell status, or a call
 * error.  Cells that failed keep the state they reached.  Further calls
 * continue from tout (each call starts from a fresh Jacobian). */
int bdfb_integrate(bdfb_ctx* ctx, double tout, double* y, int32_t* status, int32_t mem);
int bdfb_get_stats(bdfb_ctx* ctx, bdfb_stats* out);
/* Per-operation timing of the grid integrator (BDFB_BRUSSELATOR3D, and
 * BDFB_BRUSSELATOR1D on its BDF path), the measurement behind the paper's
 * per-kernel bandwidth study (Sec. 6, Table 1).  Option "profile" 1 records
 * CUDA events around every vector operation and kernel of the step loop on
 * the context's stream (no extra synchronisation; the times are read when
 * each bdfb_integrate returns) and clears the sums; 0 stops.  out (host,
 * 3 * nkinds doubles, nkinds >= 14): for kind k, out[3k] = launches,
 * out[3k + 1] = summed event milliseconds, out[3k + 2] = summed algorithmic
 * gigabytes (the bytes the operation must move, N = unknowns, nv = vectors):
 *   0 WrmsNorm 16N; 1 DotProdMulti 8(nv+1)N; 2 LinearCombination 8(nv+1)N;
 *   3 LinearSum 24N; 4 prediction of z_0, z_1 8(q+3)N; 5 corrector and
 *   Pascal shift 8(2q+3)N; 6 history rescale 16qN; 7 error weights 24N;
 *   8 Newton update 40N; 9 unscaling product 24N; 10 right-hand side 16N;
 *   11 preconditioned GMRES operator 64N (52N with FP32 blocks); 12 3x3
 *   block setup 32N (20N); 13 preconditioning of the right-hand side 48N
 *   (36N).  Returns 14 (the number of kinds), or BDFB_ILL_INPUT (null
 *   pointers, nkinds < 14, or a context without a grid). */
int bdfb_get_op_profile(bdfb_ctx* ctx, double* out, int32_t nkinds);
/* per-cell counters, int64 [ncell][8] = nst, nfe, nsetups, nni, ncfn, netf, q, h-bits.
 * For BDFB_BRUSSELATOR3D one row for the whole system: nst, nfe, nsetups,
 * nni, ncfn, netf, GMRES iterations, GMRES solves that stopped at maxl.
 * Option "imex" (BDFB_BRUSSELATOR1D): one row nst, advection evaluations,
 * reaction evaluations, Newton iterations, ncfn, netf, 0, 0 (bdfb_get_stats:
 * nfevals = reaction evaluations, nlinsetups = nniters, since the 3x3 blocks
 * are formed at every iteration).
 * Option "grouped": every row holds the shared counters (nni: the mean over
 * cells of the summed task-local iterations), the order and the step size
 * the next step will try. */
int bdfb_get_cell_stats(bdfb_ctx* ctx, int64_t* out, int32_t mem);
/* Cell-to-lane mapping in use.  Size classes c = 0..4 hold cells with
 * max(n, ceil(reactions / 2)) <= 4, 8, 16, 32, 56.  Kernel variants v =
 * 0..7 are (lanes per cell G, largest cell NMAX) = (1, 4), (4, 8), (8, 16),
 * (16, 32), (32, 56) (the classes' own tilings), (32, 16) (one warp per cell;
 * the learned guess runs here), (32, 32) and (16, 16).  out (host, 15
 * int32): out[3c] = G, out[3c + 1] = NMAX of the variant class c runs on
 * (under the current options; the tuned one after autotuning), out[3c + 2] =
 * cells in class c (0: class empty, G = NMAX = 0).  trial_ms (host, 5 x 8
 * floats, or NULL): the autotuner's trial time of variant v on class c at
 * [8c + v] (0: not tried). */
int bdfb_get_mapping(bdfb_ctx* ctx, int32_t* out, float* trial_ms);

/* Phase timers of the per-cell step kernels, for profiling; no counterpart in
 * the paper.  A library built with the phase timers compiled in
 * (python -m paper_2011_12984_b300.build --phases, which writes
 * libbdfb_phases.so) charges the SM clock cycles of lane 0 of every warp to
 * the part of the BDF step it is in.  out (host, nphase >= 14 entries)
 * receives the cycles summed over all warps since the last reset, in the
 * order: step control and error weights; prediction; Jacobian and M;
 * factorisation pivoting (search, swap, column scaling); factorisation
 * trailing updates; right-hand side reaction rates; right-hand side species
 * sums; triangular solves; refinement residual (mixed precision); refinement
 * norms and conversions; Newton tests and updates; error test, correction
 * and step/order choice; failure handling; tile loads and stores.  reset != 0
 * zeroes the counters afterwards.  Synchronises the device.  Returns the
 * number of phases (14), or BDFB_ILL_INPUT from a library built without the
 * timers or for a short or null out. */
int bdfb_phase_cycles(uint64_t* out, int nphase, int reset);

/* ------------------------------------- learned Newton initial guess (MLP)
 * Not part of the paper: a 12 -> 64 -> 64 -> 10 ReLU network predicts the
 * Newton correction Delta of a step, in error-weight units (Delta_i ewt_i),
 * from the features x = ((log10 max(y_pred_i, 1e-20) + 10) / 10 for
 * i = 0..9 (zero past n), (log10|h| + 8) / 4, gamma / h).  Parameters:
 * 5642 FP32 values, W1[64][12], b1[64], W2[64][64], b2[64], W3[10][64],
 * b3[10] (W[out][in]).  Evaluation and training run
 * on BF16 tensor-core MMAs with FP32 accumulation; the master weights and
 * Adam moments stay FP32.  X is [rows][12], T and Y [rows][10], row-major
 * FP32; every pointer is device memory owned by the caller. */
int64_t bdfb_mlp_nparam(void);        /* 5642 */
int64_t bdfb_mlp_packed_bytes(void);  /* size of the packed BF16 operand form */
/* FP32 parameters -> packed form (BF16 weights in MMA layouts, FP32 biases) */
int bdfb_mlp_pack(const float* params, void* packed, void* stream);
/* Y = net(X) for nrows rows (nrows >= 0) */
int bdfb_mlp_forward(int64_t nrows, const float* X, const void* packed, float* Y, void* stream);
/* grad += d loss / d params and *loss += loss over nrows >= 1 rows, with
 * loss = mean over rows and the 10 outputs of (net(X) - T)^2; the caller
 * zeroes grad and *loss first */
int bdfb_mlp_loss_grad(int64_t nrows, const float* X, const float* T, const void* packed, float* grad,
                       float* loss, void* stream);
/* one Adam step (Kingma & Ba; b1 0.9, b2 0.999, eps 1e-8, bias-corrected
 * with step number t >= 1) on params with gradient grad; grad is zeroed */
int bdfb_mlp_adam(float* params, float* grad, float* m, float* v, int64_t t, float lr, void* stream);
/* nsteps Adam steps (b1 0.9, b2 0.999, eps 1e-8, learning rate lr) on
 * minibatches of `batch` consecutive rows, batch k = (t0 + step) mod
 * max(1, nrows / batch); t0 = Adam steps already taken (bias correction).
 * params, m, v (nparam FP32 each) are updated, packed is refreshed after
 * every step, grad (nparam FP32) is workspace, loss_hist[step] receives
 * each minibatch's loss. */
int bdfb_mlp_train(int64_t nrows, const float* X, const float* T, float* params, float* m, float* v,
                   void* packed, float* grad, float* loss_hist, int batch, int nsteps, int64_t t0,
                   float lr, void* stream);
/* use the packed network (device memory, 16-byte aligned, bytes ==
 * bdfb_mlp_packed_bytes(); must stay valid while the context uses it) for
 * the option "predictor"; NULL detaches it */
int bdfb_load_mlp(bdfb_ctx* ctx, const void* packed, int64_t bytes);
/* Recording for training: every accepted step of every cell (each cell
 * n <= 10, FP64 factorisation) appends its features x (12 floats) to x and
 * its converged correction Delta_i ewt_i (10 floats) to t at index
 * atomicAdd(count, 1) while that index is < cap; *count keeps counting past
 * cap.  x == NULL stops recording.  Recording runs the one-warp-per-cell
 * kernel. */
int bdfb_set_record(bdfb_ctx* ctx, float* x, float* t, int64_t cap, unsigned long long* count);

#ifdef __cplusplus
}
#endif
#endif /* BDFB_H */
