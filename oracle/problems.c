/*
 * problems.c - oracle right-hand sides, Jacobians and drivers.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Per-cell problems (Sec. 2, "submodel" use case: many small independent
 * systems, e.g. chemistry in each grid cell) are integrated one cell at a time
 * with their own step control and a dense LU of the cell's block of
 * M = I - gamma J (the block-diagonal structure of Fig. 1).  The Brusselator
 * (reaction terms of Sec. 7, with diffusion in place of advection) is one
 * coupled system integrated with Newton + GMRES, preconditioned by the 3x3
 * reaction blocks as in the Sec. 7 global-Newton configuration.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

/* ------------------------------------------------------------------------ */
/* Robertson kinetics                                                       */
/* ------------------------------------------------------------------------ */
void or_robertson_rhs(const double* k, const double* y, double* f) {
  f[0] = -k[0] * y[0] + k[2] * y[1] * y[2];
  f[1] = k[0] * y[0] - k[2] * y[1] * y[2] - k[1] * y[1] * y[1];
  f[2] = k[1] * y[1] * y[1];
}

void or_robertson_jac(const double* k, const double* y, double* J) {
  J[0] = -k[0];  J[1] = k[2] * y[2];                       J[2] = k[2] * y[1];
  J[3] = k[0];   J[4] = -k[2] * y[2] - 2.0 * k[1] * y[1];   J[5] = -k[2] * y[1];
  J[6] = 0.0;    J[7] = 2.0 * k[1] * y[1];                  J[8] = 0.0;
}

/* ------------------------------------------------------------------------ */
/* Mass action: rate_r = k_r prod_{s in R(r)} y_s; each reactant loses rate_r, */
/* each product gains it.                                                     */
/* ------------------------------------------------------------------------ */
void or_massaction_rhs(int n, int nr, const uint8_t* reac, const uint8_t* prod,
                       const double* k, const double* y, double* f) {
  for (int i = 0; i < n; ++i) f[i] = 0.0;
  for (int r = 0; r < nr; ++r) {
    double rate = k[r];
    for (int a = 0; a < 4; ++a)
      if (reac[r * 4 + a] != 255) rate *= y[reac[r * 4 + a]];
    for (int a = 0; a < 4; ++a)
      if (reac[r * 4 + a] != 255) f[reac[r * 4 + a]] -= rate;
    for (int a = 0; a < 4; ++a)
      if (prod[r * 4 + a] != 255) f[prod[r * 4 + a]] += rate;
  }
}

/* J[i*n + s] = d f_i / d y_s.  d rate_r / d y_s = k_r prod_{s' in R(r), s' != s} y_s'
 * (reactant lists hold distinct species). */
void or_massaction_jac(int n, int nr, const uint8_t* reac, const uint8_t* prod,
                       const double* k, const double* y, double* J) {
  for (int i = 0; i < n * n; ++i) J[i] = 0.0;
  for (int r = 0; r < nr; ++r) {
    for (int a = 0; a < 4; ++a) {
      int s = reac[r * 4 + a];
      if (s == 255) continue;
      double d = k[r];
      for (int b = 0; b < 4; ++b)
        if (b != a && reac[r * 4 + b] != 255) d *= y[reac[r * 4 + b]];
      for (int b = 0; b < 4; ++b)
        if (reac[r * 4 + b] != 255) J[reac[r * 4 + b] * n + s] -= d;
      for (int b = 0; b < 4; ++b)
        if (prod[r * 4 + b] != 255) J[prod[r * 4 + b] * n + s] += d;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* dense per-cell system                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
  int kind, n, nr;
  const double* k;
  const uint8_t *reac, *prod;
  double* J;
  double* M;
  int* piv;
} cell_user;

static int cell_rhs(void* u, double t, const double* y, double* f) {
  (void)t;
  cell_user* c = (cell_user*)u;
  if (c->kind == 0) or_robertson_rhs(c->k, y, f);
  else or_massaction_rhs(c->n, c->nr, c->reac, c->prod, c->k, y, f);
  for (int i = 0; i < c->n; ++i) if (!isfinite(f[i])) return 1;
  return 0;
}

static int cell_lsetup(void* u, double t, const double* y, double gamma) {
  (void)t;
  cell_user* c = (cell_user*)u;
  int n = c->n;
  if (c->kind == 0) or_robertson_jac(c->k, y, c->J);
  else or_massaction_jac(n, c->nr, c->reac, c->prod, c->k, y, c->J);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) c->M[i * n + j] = (i == j ? 1.0 : 0.0) - gamma * c->J[i * n + j];
  return or_lu_factor(n, c->M, c->piv) ? 1 : 0;
}

static int cell_lsolve(void* u, double t, const double* ycur, double gamma,
                       const double* ewt, double tol, double* b) {
  (void)t; (void)ycur; (void)gamma; (void)ewt; (void)tol;
  cell_user* c = (cell_user*)u;
  or_lu_solve(c->n, c->M, c->piv, b);
  return 0;
}

/* the data of cell c (buffers J, M, piv left to the caller) */
static void cell_user_of(const or_cells* cells, int64_t c, cell_user* u) {
  memset(u, 0, sizeof *u);
  u->kind = cells->kind;
  if (cells->kind == 0) {
    u->n = 3;
    u->k = cells->k + 3 * c;
  } else {
    u->n = cells->n[c];
    int64_t ro = cells->rxn_off[c];
    u->nr = (int)(cells->rxn_off[c + 1] - ro);
    u->k = cells->k + ro;
    u->reac = cells->reac + 4 * ro;
    u->prod = cells->prod + 4 * ro;
  }
}

int or_cells_integrate(const or_cells* cells, int64_t c0, int64_t c1, double t0,
                       const double* y0, double tout, double rtol, double atol,
                       int64_t mxstep, double* yout, int32_t* status, int64_t* stats) {
  return or_cells_integrate_mode(cells, c0, c1, t0, y0, tout, rtol, atol, mxstep, 0, yout, status, stats);
}

int or_cells_integrate_mode(const or_cells* cells, int64_t c0, int64_t c1, double t0,
                            const double* y0, double tout, double rtol, double atol,
                            int64_t mxstep, int interp, double* yout, int32_t* status,
                            int64_t* stats) {
  int worst = 0;
  for (int64_t c = c0; c < c1; ++c) {
    cell_user u;
    cell_user_of(cells, c, &u);
    int64_t yo = cells->y_off[c];
    u.J = (double*)malloc(sizeof(double) * u.n * u.n);
    u.M = (double*)malloc(sizeof(double) * u.n * u.n);
    u.piv = (int*)malloc(sizeof(int) * u.n);
    or_system sys = {u.n, &u, cell_rhs, cell_lsetup, cell_lsolve, 1, 0, NULL};
    or_options opt;
    memset(&opt, 0, sizeof opt);
    opt.rtol = rtol;
    opt.atol = atol;
    opt.mxstep = mxstep;
    opt.interp = interp;
    int ret;
    or_bdf* m = (u.J && u.M && u.piv) ? or_bdf_create(&sys, &opt, t0, y0 + yo) : NULL;
    if (!m) {
      ret = OR_MEM_FAIL;
    } else {
      ret = or_bdf_solve(m, tout, yout + yo);
      if (stats) {
        or_stats st;
        or_bdf_stats(m, &st);
        int64_t* s = stats + 8 * c;
        s[0] = st.nst; s[1] = st.nfe; s[2] = st.nsetups; s[3] = st.nni;
        s[4] = st.ncfn; s[5] = st.netf; s[6] = st.qlast;
        memcpy(&s[7], &st.hlast, sizeof st.hlast);   /* the last step size, as its bits */
      }
      or_bdf_free(m);
    }
    free(u.J); free(u.M); free(u.piv);
    if (status) status[c] = ret;
    if (ret < worst) worst = ret;
  }
  return worst;
}

/* ---- all cells as one system with task-local Newton solves -------------- */
typedef struct {
  int64_t ncell;
  const int64_t* y_off;
  cell_user* u;
} group_user;

static int group_rhs(void* p, double t, const double* y, double* f) {
  group_user* g = (group_user*)p;
  for (int64_t c = 0; c < g->ncell; ++c) cell_rhs(&g->u[c], t, y + g->y_off[c], f + g->y_off[c]);
  return 0;   /* non-finite entries fail their own block in the Newton iteration */
}

static int group_lsetup(void* p, double t, const double* y, double gamma) {
  group_user* g = (group_user*)p;
  int bad = 0;
  for (int64_t c = 0; c < g->ncell; ++c) bad |= cell_lsetup(&g->u[c], t, y + g->y_off[c], gamma);
  return bad ? 1 : 0;
}

static int group_lsolve(void* p, double t, const double* ycur, double gamma,
                        const double* ewt, double tol, double* b) {
  (void)t; (void)ycur; (void)gamma; (void)ewt; (void)tol;
  group_user* g = (group_user*)p;
  for (int64_t c = 0; c < g->ncell; ++c) or_lu_solve(g->u[c].n, g->u[c].M, g->u[c].piv, b + g->y_off[c]);
  return 0;
}

int or_cells_integrate_grouped(const or_cells* cells, double t0, const double* y0, double tout,
                               double rtol, double atol, int64_t mxstep, int interp,
                               double* yout, int64_t* stats) {
  const int64_t C = cells->ncell;
  if (C <= 0) return 0;
  group_user g;
  g.ncell = C;
  g.y_off = cells->y_off;
  g.u = (cell_user*)calloc((size_t)C, sizeof(cell_user));
  int ok = g.u != NULL;
  for (int64_t c = 0; ok && c < C; ++c) {
    cell_user_of(cells, c, &g.u[c]);
    const int n = g.u[c].n;
    g.u[c].J = (double*)malloc(sizeof(double) * n * n);
    g.u[c].M = (double*)malloc(sizeof(double) * n * n);
    g.u[c].piv = (int*)malloc(sizeof(int) * n);
    ok = g.u[c].J && g.u[c].M && g.u[c].piv;
  }
  int ret = OR_MEM_FAIL;
  if (ok) {
    or_system sys = {cells->y_off[C], &g, group_rhs, group_lsetup, group_lsolve, 1, C, cells->y_off};
    or_options opt;
    memset(&opt, 0, sizeof opt);
    opt.rtol = rtol;
    opt.atol = atol;
    opt.mxstep = mxstep;
    opt.interp = interp;
    or_bdf* m = or_bdf_create(&sys, &opt, t0, y0);
    if (m) {
      ret = or_bdf_solve(m, tout, yout);
      if (stats) {
        or_stats st;
        or_bdf_stats(m, &st);
        stats[0] = st.nst; stats[1] = st.nfe; stats[2] = st.nsetups; stats[3] = st.nni;
        stats[4] = st.ncfn; stats[5] = st.netf; stats[6] = st.qlast;
        memcpy(&stats[7], &st.hlast, sizeof st.hlast);
      }
      or_bdf_free(m);
    }
  }
  for (int64_t c = 0; g.u && c < C; ++c) { free(g.u[c].J); free(g.u[c].M); free(g.u[c].piv); }
  free(g.u);
  return ret;
}

/* ------------------------------------------------------------------------ */
/* linear test system y' = A y + sum_k C_k t^k (pins: closed forms, BDF      */
/* coefficient tables, local-error constants)                                */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t N;
  const double* A;
  int ncoef;
  const double* C;
  double* M;
  int* piv;
} lin_user;

static int lin_rhs(void* u, double t, const double* y, double* f) {
  lin_user* L = (lin_user*)u;
  int64_t N = L->N;
  for (int64_t i = 0; i < N; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < N; ++j) s += L->A[i * N + j] * y[j];
    double tk = 1.0;
    for (int k = 0; k < L->ncoef; ++k) { s += L->C[k * N + i] * tk; tk *= t; }
    f[i] = s;
  }
  return 0;
}
static int lin_lsetup(void* u, double t, const double* y, double gamma) {
  (void)t; (void)y;
  lin_user* L = (lin_user*)u;
  int64_t N = L->N;
  for (int64_t i = 0; i < N; ++i)
    for (int64_t j = 0; j < N; ++j) L->M[i * N + j] = (i == j ? 1.0 : 0.0) - gamma * L->A[i * N + j];
  return or_lu_factor((int)N, L->M, L->piv) ? 1 : 0;
}
static int lin_lsolve(void* u, double t, const double* ycur, double gamma,
                      const double* ewt, double tol, double* b) {
  (void)t; (void)ycur; (void)gamma; (void)ewt; (void)tol;
  lin_user* L = (lin_user*)u;
  or_lu_solve((int)L->N, L->M, L->piv, b);
  return 0;
}

int or_linear_integrate(int64_t N, const double* A, int ncoef, const double* C, double t0,
                        const double* y0, double tout, const or_options* opt, double* yout,
                        int64_t* stats, int64_t* ntrace) {
  lin_user L = {N, A, ncoef, C, (double*)malloc(sizeof(double) * N * N), (int*)malloc(sizeof(int) * N)};
  or_system sys = {N, &L, lin_rhs, lin_lsetup, lin_lsolve, 1, 0, NULL};
  or_bdf* m = or_bdf_create(&sys, opt, t0, y0);
  int ret = OR_MEM_FAIL;
  if (m && L.M && L.piv) {
    ret = or_bdf_solve(m, tout, yout);
    or_stats st;
    or_bdf_stats(m, &st);
    if (stats) {
      stats[0] = st.nst; stats[1] = st.nfe; stats[2] = st.nsetups; stats[3] = st.nni;
      stats[4] = st.ncfn; stats[5] = st.netf; stats[6] = st.qlast;
      memcpy(&stats[7], &st.hlast, sizeof st.hlast);
    }
    if (ntrace) *ntrace = opt->trace_cap < st.nst ? opt->trace_cap : st.nst;
  }
  or_bdf_free(m);
  free(L.M); free(L.piv);
  return ret;
}

/* ------------------------------------------------------------------------ */
/* Brusselator grids (species-major u | v | w), reaction terms of Sec. 7     */
/* u' = T u + A - (w+1) u + v u^2                                            */
/* v' = T v + w u - v u^2                                                    */
/* w' = T w + (B - w)/eps - w u                                              */
/* with the transport T = D lap on the periodic nx^3 grid (dim 3), or the    */
/* demo's advection T = -c d/dx by first-order upwind differences on the     */
/* periodic line of nx points (dim 1, Sec. 7)                                */
/* ------------------------------------------------------------------------ */
static int64_t wrapi(int64_t i, int64_t n) { return (i + n) % n; }

static double lap(const or_bruss* p, const double* a, int64_t i, int64_t j, int64_t k) {
  int64_t n = p->nx;
  double c = a[(i * n + j) * n + k];
  double s = a[(wrapi(i - 1, n) * n + j) * n + k] + a[(wrapi(i + 1, n) * n + j) * n + k] +
             a[(i * n + wrapi(j - 1, n)) * n + k] + a[(i * n + wrapi(j + 1, n)) * n + k] +
             a[(i * n + j) * n + wrapi(k - 1, n)] + a[(i * n + j) * n + wrapi(k + 1, n)];
  double dx = 1.0 / (double)n;
  return (s - 6.0 * c) / (dx * dx);
}

static int64_t bruss_npts(const or_bruss* p) {
  return p->dim == 1 ? (int64_t)p->nx : (int64_t)p->nx * p->nx * p->nx;
}

/* -c da/dx at point q of the line, upwind: backward difference for c >= 0,
 * forward difference for c < 0; dx = len / nx */
static double advect(const or_bruss* p, const double* a, int64_t q) {
  int64_t n = p->nx;
  double dx = p->len / (double)n;
  if (p->c >= 0.0) return -p->c * (a[q] - a[wrapi(q - 1, n)]) / dx;
  return -p->c * (a[wrapi(q + 1, n)] - a[q]) / dx;
}

/* the transport term of one species' field a at point q */
static double transport(const or_bruss* p, const double* a, int64_t q) {
  if (p->dim == 1) return advect(p, a, q);
  int64_t n = p->nx;
  int64_t i = q / (n * n), j = (q / n) % n, k = q % n;
  return p->D * lap(p, a, i, j, k);
}

/* reaction Jacobian of one point, row-major 3x3 */
static void bruss_jr(const or_bruss* p, double u, double v, double w, double* J) {
  J[0] = -(w + 1.0) + 2.0 * u * v;  J[1] = u * u;   J[2] = -u;
  J[3] = w - 2.0 * u * v;           J[4] = -u * u;  J[5] = u;
  J[6] = -w;                        J[7] = 0.0;     J[8] = -1.0 / p->eps - u;
}

void or_bruss_transport(const or_bruss* p, const double* y, double* f) {
  int64_t np = bruss_npts(p);
  for (int s = 0; s < 3; ++s)
    for (int64_t q = 0; q < np; ++q) f[s * np + q] = transport(p, y + s * np, q);
}

void or_bruss_reaction(const or_bruss* p, const double* y, double* f) {
  int64_t np = bruss_npts(p);
  const double *U = y, *V = y + np, *W = y + 2 * np;
  for (int64_t q = 0; q < np; ++q) {
    double u = U[q], v = V[q], w = W[q];
    f[q] = p->A - (w + 1.0) * u + v * u * u;
    f[np + q] = w * u - v * u * u;
    f[2 * np + q] = (p->B - w) / p->eps - w * u;
  }
}

void or_bruss_reaction_jac(const or_bruss* p, double u, double v, double w, double* J) {
  bruss_jr(p, u, v, w, J);
}

void or_bruss_rhs(const or_bruss* p, const double* y, double* f) {
  int64_t np = bruss_npts(p);
  const double *U = y, *V = y + np, *W = y + 2 * np;
  for (int64_t q = 0; q < np; ++q) {
    double u = U[q], v = V[q], w = W[q];
    f[q] = transport(p, U, q) + p->A - (w + 1.0) * u + v * u * u;
    f[np + q] = transport(p, V, q) + w * u - v * u * u;
    f[2 * np + q] = transport(p, W, q) + (p->B - w) / p->eps - w * u;
  }
}

void or_bruss_jv(const or_bruss* p, const double* y, const double* v, double* jv) {
  int64_t np = bruss_npts(p);
  for (int64_t q = 0; q < np; ++q) {
    double J[9];
    bruss_jr(p, y[q], y[np + q], y[2 * np + q], J);
    for (int s = 0; s < 3; ++s) {
      double acc = transport(p, v + s * np, q);
      for (int t = 0; t < 3; ++t) acc += J[s * 3 + t] * v[t * np + q];
      jv[s * np + q] = acc;
    }
  }
}

#define GM_MAX 32

typedef struct {
  const or_bruss* p;
  int maxl;
  double* plu;   /* per point LU of I - gamma_p J_R (9) */
  int* ppiv;     /* per point pivots (3) */
  double *V, *w, *u;
  int64_t nli, nlfail, npsetup;
} bruss_user;

static void bruss_psolve(bruss_user* B, double* v) {
  int64_t np = bruss_npts(B->p);
  for (int64_t q = 0; q < np; ++q) {
    double x[3] = {v[q], v[np + q], v[2 * np + q]};
    or_lu_solve(3, B->plu + 9 * q, B->ppiv + 3 * q, x);
    v[q] = x[0]; v[np + q] = x[1]; v[2 * np + q] = x[2];
  }
}

static int bruss_rhs_cb(void* u, double t, const double* y, double* f) {
  (void)t;
  bruss_user* B = (bruss_user*)u;
  or_bruss_rhs(B->p, y, f);
  return 0;
}

static int bruss_lsetup_cb(void* u, double t, const double* y, double gamma) {
  (void)t;
  bruss_user* B = (bruss_user*)u;
  int64_t np = bruss_npts(B->p);
  for (int64_t q = 0; q < np; ++q) {
    double J[9];
    bruss_jr(B->p, y[q], y[np + q], y[2 * np + q], J);
    double* M = B->plu + 9 * q;
    for (int a = 0; a < 9; ++a) M[a] = ((a % 4) == 0 ? 1.0 : 0.0) - gamma * J[a];
    if (or_lu_factor(3, M, B->ppiv + 3 * q)) return 1;
  }
  B->npsetup++;
  return 0;
}

/* GMRES on (I - gamma J(y)) x = b, left-preconditioned by the block solve,
 * residual measured in the WRMS norm (weights ewt) of the preconditioned
 * residual; classical Gram-Schmidt; no restarts.  Returns iterations used. */
static int gmres_core(bruss_user* B, const double* y, double gamma, const double* ewt,
                      double tol, double* b, double* resnorm, int* converged) {
  const or_bruss* p = B->p;
  int64_t np = bruss_npts(p), N = 3 * np;
  int maxl = B->maxl;
  double sqrtN = sqrt((double)N);
  double* V = B->V;        /* (maxl+1) x N */
  double* w = B->w;
  double* u = B->u;
  double H[(GM_MAX + 1) * GM_MAX];
  double g[GM_MAX + 1], cs[GM_MAX], sn[GM_MAX];
  memset(H, 0, sizeof H);
  /* r0 = P^{-1} b, v0 = S r0 */
  memcpy(u, b, sizeof(double) * N);
  bruss_psolve(B, u);
  for (int64_t i = 0; i < N; ++i) V[i] = ewt[i] * u[i];
  double beta = 0.0;
  for (int64_t i = 0; i < N; ++i) beta += V[i] * V[i];
  beta = sqrt(beta);
  *converged = 1;
  if (beta / sqrtN <= tol) {
    for (int64_t i = 0; i < N; ++i) b[i] = 0.0;
    *resnorm = beta / sqrtN;
    return 0;
  }
  for (int64_t i = 0; i < N; ++i) V[i] /= beta;
  for (int i = 0; i <= maxl; ++i) g[i] = 0.0;
  g[0] = beta;
  int k = 0;   /* number of Krylov vectors used */
  double res = beta;
  *converged = 0;
  for (int j = 0; j < maxl; ++j) {
    double* vj = V + (int64_t)j * N;
    for (int64_t i = 0; i < N; ++i) u[i] = vj[i] / ewt[i];
    or_bruss_jv(p, y, u, w);
    for (int64_t i = 0; i < N; ++i) w[i] = u[i] - gamma * w[i];
    bruss_psolve(B, w);
    for (int64_t i = 0; i < N; ++i) w[i] *= ewt[i];
    for (int i = 0; i <= j; ++i) {           /* classical Gram-Schmidt */
      const double* vi = V + (int64_t)i * N;
      double d = 0.0;
      for (int64_t a = 0; a < N; ++a) d += vi[a] * w[a];
      H[i * maxl + j] = d;
    }
    for (int i = 0; i <= j; ++i) {
      const double* vi = V + (int64_t)i * N;
      for (int64_t a = 0; a < N; ++a) w[a] -= H[i * maxl + j] * vi[a];
    }
    double hn = 0.0;
    for (int64_t a = 0; a < N; ++a) hn += w[a] * w[a];
    hn = sqrt(hn);
    H[(j + 1) * maxl + j] = hn;
    if (hn > 0.0)
      for (int64_t a = 0; a < N; ++a) V[(int64_t)(j + 1) * N + a] = w[a] / hn;
    for (int i = 0; i < j; ++i) {            /* previous Givens rotations */
      double h0 = H[i * maxl + j], h1 = H[(i + 1) * maxl + j];
      H[i * maxl + j] = cs[i] * h0 + sn[i] * h1;
      H[(i + 1) * maxl + j] = -sn[i] * h0 + cs[i] * h1;
    }
    double a0 = H[j * maxl + j], a1 = H[(j + 1) * maxl + j];
    double rr = sqrt(a0 * a0 + a1 * a1);
    cs[j] = rr > 0.0 ? a0 / rr : 1.0;
    sn[j] = rr > 0.0 ? a1 / rr : 0.0;
    H[j * maxl + j] = rr;
    H[(j + 1) * maxl + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    res = fabs(g[j + 1]);
    k = j + 1;
    if (res / sqrtN <= tol || hn == 0.0) { *converged = 1; break; }
  }
  double yv[GM_MAX];
  for (int i = k - 1; i >= 0; --i) {         /* back substitution */
    double s = g[i];
    for (int jj = i + 1; jj < k; ++jj) s -= H[i * maxl + jj] * yv[jj];
    yv[i] = s / H[i * maxl + i];
  }
  for (int64_t a = 0; a < N; ++a) {
    double s = 0.0;
    for (int i = 0; i < k; ++i) s += yv[i] * V[(int64_t)i * N + a];
    b[a] = s / ewt[a];
  }
  *resnorm = res / sqrtN;
  return k;
}

static int bruss_lsolve_cb(void* u, double t, const double* ycur, double gamma,
                           const double* ewt, double tol, double* b) {
  (void)t;
  bruss_user* B = (bruss_user*)u;
  double rn;
  int conv;
  int it = gmres_core(B, ycur, gamma, ewt, tol, b, &rn, &conv);
  B->nli += it;
  if (!conv) B->nlfail++;   /* inexact Newton: accept the iterate */
  return 0;
}

static int bruss_alloc(bruss_user* B, const or_bruss* p, int maxl) {
  int64_t np = bruss_npts(p), N = 3 * np;
  memset(B, 0, sizeof *B);
  B->p = p;
  B->maxl = maxl;
  B->plu = (double*)malloc(sizeof(double) * 9 * np);
  B->ppiv = (int*)malloc(sizeof(int) * 3 * np);
  B->V = (double*)malloc(sizeof(double) * (maxl + 1) * N);
  B->w = (double*)malloc(sizeof(double) * N);
  B->u = (double*)malloc(sizeof(double) * N);
  return (B->plu && B->ppiv && B->V && B->w && B->u) ? 0 : -1;
}
static void bruss_free(bruss_user* B) {
  free(B->plu); free(B->ppiv); free(B->V); free(B->w); free(B->u);
}

int or_bruss_gmres(const or_bruss* p, const double* y, double gamma, const double* ewt,
                   double tol, int maxl, double* b, double* resnorm) {
  bruss_user B;
  if (maxl < 1 || maxl > GM_MAX) return OR_ILL_INPUT;
  if (bruss_alloc(&B, p, maxl)) { bruss_free(&B); return OR_MEM_FAIL; }
  bruss_lsetup_cb(&B, 0.0, y, gamma);
  int conv;
  int it = gmres_core(&B, y, gamma, ewt, tol, b, resnorm, &conv);
  bruss_free(&B);
  return it;
}

int or_bruss_integrate(const or_bruss* p, double t0, const double* y0, double tout,
                       double rtol, double atol, int maxl, int64_t mxstep, int interp,
                       double* yout, int64_t* stats) {
  int64_t N = 3 * bruss_npts(p);
  bruss_user B;
  if (maxl < 1 || maxl > GM_MAX) return OR_ILL_INPUT;
  if (bruss_alloc(&B, p, maxl)) { bruss_free(&B); return OR_MEM_FAIL; }
  or_system sys = {N, &B, bruss_rhs_cb, bruss_lsetup_cb, bruss_lsolve_cb, 0, 0, NULL};
  or_options opt;
  memset(&opt, 0, sizeof opt);
  opt.rtol = rtol;
  opt.atol = atol;
  opt.mxstep = mxstep;
  opt.interp = interp;
  or_bdf* m = or_bdf_create(&sys, &opt, t0, y0);
  int ret = OR_MEM_FAIL;
  if (m) {
    ret = or_bdf_solve(m, tout, yout);
    or_stats st;
    or_bdf_stats(m, &st);
    if (stats) {
      stats[0] = st.nst; stats[1] = st.nfe; stats[2] = st.nsetups; stats[3] = st.nni;
      stats[4] = st.ncfn; stats[5] = st.netf; stats[6] = B.nli; stats[7] = B.nlfail;
    }
    or_bdf_free(m);
  }
  bruss_free(&B);
  return ret;
}
