/*
 * oracle.h - plain, slow, obviously-correct CPU reference of the batched
 * BDF/Newton hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA library and
 * never calls it.
 *
 * Everything is IEEE double, compiled with -ffp-contract=off, single
 * threaded per call.  Each function cites the passage of the paper it
 * follows; where the paper is silent (it defers all integrator details to
 * the CVODE documentation, Sec. 1 and Sec. 5) the reading taken is stated
 * beside the code.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

/* Return / per-cell status codes (same numeric values as the library's). */
enum {
  OR_SUCCESS = 0,
  OR_TOO_MUCH_WORK = -1,
  OR_ERR_FAILURE = -3,
  OR_CONV_FAILURE = -4,
  OR_LSETUP_FAIL = -6,
  OR_LSOLVE_FAIL = -7,
  OR_RHSFUNC_FAIL = -8,
  OR_MEM_FAIL = -20,
  OR_ILL_INPUT = -22
};

#define OR_QMAX 5

/* ---------------- vector operations (Sec. 4: streaming / reduction) ---- */
void or_scale(int64_t n, double c, const double* x, double* z);
void or_const(int64_t n, double c, double* z);
void or_abs(int64_t n, const double* x, double* z);
void or_inv(int64_t n, const double* x, double* z);
void or_add_const(int64_t n, const double* x, double b, double* z);
void or_error_weights(int64_t n, double rtol, double atol, const double* y, double* w);
void or_linear_sum(int64_t n, double a, const double* x, double b, const double* y, double* z);
void or_linear_combination(int64_t n, int nv, const double* c, const double* const* x, double* z);
void or_scale_add_multi(int64_t n, int nv, const double* a, const double* x,
                        const double* const* y, double* const* z);
/* d[j] = x . y_j, compensated (Neumaier) sum; sabs[j] = sum |x_i y_ji| */
void or_dot_prod_multi(int64_t n, int nv, const double* x, const double* const* y,
                       double* d, double* sabs);
/* sqrt(sum (x_i w_i)^2 / n), compensated sum of squares */
double or_wrms_norm(int64_t n, const double* x, const double* w);

/* ---------------- dense LU with partial pivoting ------------------------ */
/* a: n x n row-major, overwritten by L\U; piv[k] = pivot row of step k.
 * Ties in |pivot| go to the lowest row index.  Returns 0, or k+1 when the
 * pivot of step k is exactly zero (factorisation stops there). */
int or_lu_factor(int n, double* a, int* piv);
void or_lu_solve(int n, const double* lu, const int* piv, double* b);

/* ---------------- generic BDF integrator -------------------------------- */
typedef struct {
  int64_t N;
  void* user;
  /* f = f(t, y); 0 ok, >0 recoverable, <0 unrecoverable */
  int (*rhs)(void* user, double t, const double* y, double* f);
  /* evaluate J at (t, y), form M = I - gamma J and prepare to solve with it */
  int (*lsetup)(void* user, double t, const double* y, double gamma);
  /* b <- M^{-1} b.  Direct solvers use the M of the last lsetup; iterative
   * solvers use the current gamma and the Jacobian at ycur, stopping when
   * the WRMS norm (weights ewt) of the preconditioned residual <= tol. */
  int (*lsolve)(void* user, double t, const double* ycur, double gamma,
                const double* ewt, double tol, double* b);
  int direct; /* 1: scale the correction by 2/(1+gamma/gamma_setup) */
  /* task-local Newton (demonstration problem's solver, Sec. 7) when nblock > 0:
   * the unknowns split into independent blocks [block_off[b], block_off[b+1])
   * and each block iterates to its own convergence test in its own WRMS norm;
   * the solve fails when any block's does.  lsolve must act block by block. */
  int64_t nblock;
  const int64_t* block_off;
} or_system;

typedef struct {
  double rtol, atol;
  int64_t mxstep;     /* steps per solve call (default 100000) */
  int qmax;           /* <= 5 */
  double fixed_h;     /* > 0: constant step, constant order fixed_q, no error test */
  int fixed_q;
  double h0;          /* > 0: initial step override */
  /* optional per-step trace: y_n and Delta_n after each accepted step */
  double* trace_y;
  double* trace_acor;
  int64_t trace_cap;
  /* optional exact starting history z_0..z_{fixed_q} (fixed-step runs), N each */
  const double* z_init;
  /* 1: step past tout and return the history polynomial's value at tout,
   * y(tout) = sum_j z_j ((tout - t_n) / h)^j (CVODE's normal mode); 0: the
   * last step lands on tout */
  int interp;
} or_options;

typedef struct {
  int64_t nst, nfe, nsetups, nni, ncfn, netf, nlfail;
  int qlast;
  double hlast, tcur;
} or_stats;

typedef struct or_bdf or_bdf;
or_bdf* or_bdf_create(const or_system* sys, const or_options* opt, double t0, const double* y0);
/* integrate to tout; y at tout (or at the point reached) copied to yout */
int or_bdf_solve(or_bdf* mem, double tout, double* yout);
void or_bdf_stats(const or_bdf* mem, or_stats* st);
/* the step-size and order choice after an accepted step from the test
 * quantities dsm = E_q |Delta|, dqm1 = E_{q-1} |z_q|, dqp1 = E_{q+1}
 * |Delta - Delta_prev|: returns 1 with the new order and step ratio, or 0
 * when h is kept */
int or_bdf_choose(int q, int qmax, int grown_once, double dsm, double dqm1, double dqp1, int* qnew,
                  double* eta);
void or_bdf_free(or_bdf* mem);
/* method constants for order q: l[0..q] (coefficients of prod_{i=1}^q (1 + x/i)),
 * out[0] = E_q, out[1] = E_{q-1} (from z_q), out[2] = E_{q+1} (from Delta - Delta_prev) */
void or_bdf_constants(int q, double* l, double* out);

/* ---------------- per-cell problems ------------------------------------- */
/* Robertson: k = (k1, k2, k3) */
void or_robertson_rhs(const double* k, const double* y, double* f);
void or_robertson_jac(const double* k, const double* y, double* J);
/* mass action: reaction r consumes reac[r*4 + i] (255 = none), produces prod[r*4+i] */
void or_massaction_rhs(int n, int nr, const uint8_t* reac, const uint8_t* prod,
                       const double* k, const double* y, double* f);
void or_massaction_jac(int n, int nr, const uint8_t* reac, const uint8_t* prod,
                       const double* k, const double* y, double* J);

typedef struct {
  int kind; /* 0 Robertson, 1 mass action */
  int64_t ncell;
  const int32_t* n;
  const int64_t* y_off;
  const int64_t* rxn_off;
  const uint8_t* reac;
  const uint8_t* prod;
  const double* k;
} or_cells;

/* Integrate cells [c0, c1) independently from t0 to tout (per-cell step
 * control: every cell owns its h, q and history, Sec. 2 submodel case).
 * y0/yout are packed by y_off; status[c]; stats[c*8 + {nst, nfe, nsetups,
 * nni, ncfn, netf, qlast, hlast}] when stats != NULL (hlast: the last step
 * size, its IEEE bits in the int64 slot). */
int or_cells_integrate(const or_cells* cells, int64_t c0, int64_t c1, double t0,
                       const double* y0, double tout, double rtol, double atol,
                       int64_t mxstep, double* yout, int32_t* status, int64_t* stats);
/* the same with the output mode of or_options.interp */
int or_cells_integrate_mode(const or_cells* cells, int64_t c0, int64_t c1, double t0,
                            const double* y0, double tout, double rtol, double atol,
                            int64_t mxstep, int interp, double* yout, int32_t* status,
                            int64_t* stats);

/* All cells [0, ncell) as ONE system (the grouping of Sec. 2): one step size,
 * order and error test over every species, block-diagonal Newton matrix with
 * one dense LU per cell, task-local Newton solves (or_system.nblock = ncell).
 * interp: the output mode of or_options.interp.
 * stats = {nst, nfe, nsetups, nni (summed over cells), ncfn, netf, qlast, hlast bits}. */
int or_cells_integrate_grouped(const or_cells* cells, double t0, const double* y0, double tout,
                               double rtol, double atol, int64_t mxstep, int interp,
                               double* yout, int64_t* stats);

/* y' = A y + sum_k C_k t^k, dense LU (pins of the BDF core) */
int or_linear_integrate(int64_t N, const double* A, int ncoef, const double* C, double t0,
                        const double* y0, double tout, const or_options* opt, double* yout,
                        int64_t* stats, int64_t* ntrace);

/* ---------------- Brusselator grids (grouped, GMRES) -------------------- */
/* dim 3: reaction-diffusion on a periodic nx^3 grid over [0,1)^3, 7-point
 * Laplacian with coefficient D.  dim 1: the paper's demo (Sec. 7),
 * advection-reaction on a periodic line of nx points over [0, len) with
 * first-order upwind differences for speed c.  Species-major u | v | w. */
typedef struct {
  int nx;
  double A, B, eps, D;
  int dim;
  double c, len;
} or_bruss;
void or_bruss_rhs(const or_bruss* p, const double* y, double* f);
void or_bruss_jv(const or_bruss* p, const double* y, const double* v, double* jv);
/* Integrate the whole grid as one system (shared h, global WRMS norms) with
 * Newton + GMRES(maxl) left-preconditioned by the 3x3 reaction blocks;
 * interp: the output mode of or_options.interp. */
int or_bruss_integrate(const or_bruss* p, double t0, const double* y0, double tout,
                       double rtol, double atol, int maxl, int64_t mxstep, int interp,
                       double* yout, int64_t* stats);
/* the two parts of the right-hand side and the reaction Jacobian of one
 * point (row-major 3x3): f = transport + reaction */
void or_bruss_transport(const or_bruss* p, const double* y, double* f);
void or_bruss_reaction(const or_bruss* p, const double* y, double* f);
void or_bruss_reaction_jac(const or_bruss* p, double u, double v, double w, double* J);
/* one GMRES solve of (I - gamma J(y)) x = b, preconditioner blocks at y,
 * as used inside the integrator; returns iterations; x overwrites b */
int or_bruss_gmres(const or_bruss* p, const double* y, double gamma, const double* ewt,
                   double tol, int maxl, double* b, double* resnorm);

/* ---------------- learned Newton initial guess (12 -> 64 -> 64 -> 10 MLP) ---- */
int or_mlp_nparam(void);
void or_mlp_forward(const double* p, int64_t nrows, const double* X, double* Y);
double or_mlp_loss_grad(const double* p, int64_t nrows, const double* X, const double* T, double* grad);
/* the same with BF16 operands (weights, inputs, hidden activations, dY, dH)
 * and exact accumulation: the learned guess's arithmetic */
double or_bf16_round(double x);
void or_mlp_forward_bf16(const double* p, int64_t nrows, const double* X, double* Y);
double or_mlp_loss_grad_bf16(const double* p, int64_t nrows, const double* X, const double* T, double* grad);
void or_adam_step(int64_t n, double* p, const double* g, double* m, double* v, int64_t t, double lr,
                  double b1, double b2, double eps);

/* ---------------- IMEX additive Runge-Kutta (ark.c) --------------------- */
/* y' = f_E(t, y) + f_I(t, y): f_E explicit, f_I implicit (the demonstration
 * problem's integrator, Sec. 7).  isolve: x <- (I - gamma J_I(t, y))^{-1} x. */
typedef struct {
  int64_t N;
  void* user;
  int (*fe)(void* user, double t, const double* y, double* f);
  int (*fi)(void* user, double t, const double* y, double* f);
  int (*isolve)(void* user, double t, const double* y, double gamma, double* x);
} or_imex_system;
typedef struct {
  double rtol, atol;
  int64_t mxstep;   /* steps per call (default 100000) */
  double fixed_h;   /* > 0: constant steps (the last one clamped to tout), no error control */
} or_ark_options;
typedef struct {
  int64_t nst, nfe, nfi, nni, ncfn, netf;
  double hlast, tcur;
} or_ark_stats;
/* the ARK3(2)4L[2]SA tables: c[4], AE[4x4], AI[4x4] row-major, b[4], bhat[4] */
void or_ark_table(double* c, double* AE, double* AI, double* b, double* bhat);
int or_ark_integrate(const or_imex_system* sys, const or_ark_options* opt, double t0,
                     const double* y0, double tout, double* yout, or_ark_stats* st);
/* the 1-D demonstration problem (dim 1): advection explicit, reaction
 * implicit with exact Newton on the 3x3 point blocks; stats = {nst, nfe,
 * nfi, nni, ncfn, netf, 0, 0} */
int or_bruss_ark_integrate(const or_bruss* p, double t0, const double* y0, double tout,
                           double rtol, double atol, int64_t mxstep, double* yout,
                           int64_t* stats);

#endif
