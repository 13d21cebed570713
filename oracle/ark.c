/*
 * ark.c - oracle IMEX additive Runge-Kutta integrator (the demonstration
 * problem's time integrator, Sec. 7: the advection terms explicit, the stiff
 * reaction terms implicit).  TEST INFRASTRUCTURE ONLY (oracle.h).
 *
 * The paper names the integrator (an IMEX method of ARKODE) but gives no
 * method, tables or controller.  Readings taken:
 *
 *  method:   ARK3(2)4L[2]SA of Kennedy and Carpenter (Appl. Numer. Math. 44,
 *            2003): an explicit 4-stage table paired with a stiffly accurate
 *            ESDIRK table (diagonal gamma, explicit first stage), shared
 *            abscissae c and weights b (order 3) and embedded weights bhat
 *            (order 2).  The coefficients are the published rationals.
 *  stages:   z_1 = y_n; for i > 1, z_i solves
 *              z_i = a_i + h gamma f_I(z_i),
 *              a_i = y_n + h sum_{j<i} (AE_ij f_E(z_j) + AI_ij f_I(z_j));
 *            f_E and f_I are then evaluated at z_i.
 *  Newton:   from the predictor z = a_i + h gamma f_I(y_n) (the stage's
 *            implicit term guessed from the step's first stage; it took 2.0
 *            iterations per stage on the demonstration problem where the
 *            trivial predictor z = y_n took 2.8), delta = (I - h gamma J_I(z))^{-1}
 *            (a_i + h gamma f_I(z) - z) with the Jacobian of f_I at the
 *            current iterate (the demonstration problem's implicit part is
 *            pointwise, so the matrix is block diagonal and exact Newton costs
 *            one small solve per block); at most 3 iterations; rate
 *            R = max(0.3 R, |delta_m| / |delta_{m-1}|), converged when
 *            |delta_m| min(1, R) <= 0.1, diverged when
 *            |delta_m| > 2.3 |delta_{m-1}| (WRMS norms, weights of y_n).
 *  solution: y_{n+1} = y_n + h sum b_i (f_E(z_i) + f_I(z_i));
 *            error estimate h sum (b_i - bhat_i)(f_E(z_i) + f_I(z_i)),
 *            dsm = its WRMS norm (weights of y_n); accepted when dsm <= 1.
 *  control:  PID on e_k = 1.5 dsm_k (floored at 1e-10):
 *            eta = 0.96 e_n^{-0.58/3} e_{n-1}^{0.21/3} e_{n-2}^{-0.1/3}
 *            (missing history replaced by the newest value), eta in
 *            [0.1, 20] (1e4 after the first step), eta in [1, 1.5] -> 1;
 *            error-test failure: eta = 0.96 (1.5 dsm)^{-1/3} in [0.1, 0.9],
 *            <= 0.3 from the second failure in a step, 7 failures -> error;
 *            Newton failure: eta = 0.25, 10 failures -> error.
 *  h0:       the difference estimate of ||y''|| used by the BDF oracle,
 *            applied to f = f_E + f_I.
 *  output:   the last step is clamped to land on tout.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define S 4          /* stages */

void or_ark_table(double* c, double* AE, double* AI, double* b, double* bhat) {
  const double g = 1767732205903.0 / 4055673282236.0;
  double cc[S] = {0.0, 1767732205903.0 / 2027836641118.0, 3.0 / 5.0, 1.0};
  double ae[S][S] = {{0}}, ai[S][S] = {{0}};
  ae[1][0] = 1767732205903.0 / 2027836641118.0;
  ae[2][0] = 5535828885825.0 / 10492691773637.0;
  ae[2][1] = 788022342437.0 / 10882634858940.0;
  ae[3][0] = 6485989280629.0 / 16251701735622.0;
  ae[3][1] = -4246266847089.0 / 9704473918619.0;
  ae[3][2] = 10755448449292.0 / 10357097424841.0;
  ai[1][0] = g;
  ai[1][1] = g;
  ai[2][0] = 2746238789719.0 / 10658868560708.0;
  ai[2][1] = -640167445237.0 / 6845629431997.0;
  ai[2][2] = g;
  ai[3][0] = 1471266399579.0 / 7840856788654.0;
  ai[3][1] = -4482444167858.0 / 7529755066697.0;
  ai[3][2] = 11266239266428.0 / 11593286722821.0;
  ai[3][3] = g;
  double bb[S] = {ai[3][0], ai[3][1], ai[3][2], ai[3][3]};   /* stiffly accurate */
  double bh[S] = {2756255671327.0 / 12835298489170.0, -10771552573575.0 / 22201958757719.0,
                  9247589265047.0 / 10645013368117.0, 2193209047091.0 / 5459859503100.0};
  for (int i = 0; i < S; ++i) {
    c[i] = cc[i];
    b[i] = bb[i];
    bhat[i] = bh[i];
    for (int j = 0; j < S; ++j) { AE[i * S + j] = ae[i][j]; AI[i * S + j] = ai[i][j]; }
  }
}

typedef struct {
  double c[S], AE[S * S], AI[S * S], b[S], bh[S];
} tables;

static double wrms(int64_t N, const double* x, const double* w) { return or_wrms_norm(N, x, w); }

/* initial step: as the BDF oracle's (bdf.c initial_step), on f = f_E + f_I */
static int ark_h0(const or_imex_system* sys, const or_ark_options* opt, double t, const double* y,
                  double tout, const double* f0, double* ytmp, double* ftmp, double* fitmp,
                  const double* ewt, or_ark_stats* st, double* hout) {
  int64_t N = sys->N;
  double tdist = fabs(tout - t);
  double tround = 2.220446049250313e-16 * fmax(fabs(t), fabs(tout));
  double hlb = 100.0 * tround, hub = 0.1 * tdist, inv = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    double r = fabs(f0[i]) / (0.1 * fabs(y[i]) + opt->atol);
    if (r > inv) inv = r;
  }
  if (inv * hub > 1.0) hub = 1.0 / inv;
  if (hub < hlb) hub = hlb;
  double hg = sqrt(hlb * hub), hnew = hg;
  for (int it = 0; it < 4; ++it) {
    for (int64_t i = 0; i < N; ++i) ytmp[i] = y[i] + hg * f0[i];
    if (sys->fe(sys->user, t + hg, ytmp, ftmp) || sys->fi(sys->user, t + hg, ytmp, fitmp))
      return OR_RHSFUNC_FAIL;
    st->nfe++;
    st->nfi++;
    for (int64_t i = 0; i < N; ++i) ftmp[i] = (ftmp[i] + fitmp[i] - f0[i]) / hg;
    double ydd = wrms(N, ftmp, ewt);
    hnew = (ydd * hub * hub > 2.0) ? sqrt(2.0 / ydd) : sqrt(hg * hub);
    double rat = hnew / hg;
    if (it > 0 && rat > 0.5 && rat < 2.0) break;
    hg = hnew;
  }
  double h0 = 0.5 * hnew;
  if (h0 < hlb) h0 = hlb;
  if (h0 > hub) h0 = hub;
  *hout = (tout >= t) ? h0 : -h0;
  return 0;
}

/* the Newton solve of stage i; z holds the converged stage on success.
 * Returns 0 converged, 1 recoverable failure. */
static int stage_solve(const or_imex_system* sys, double tz, double hg, const double* a,
                       const double* fi0, const double* ewt, double* z, double* fi, double* r,
                       or_ark_stats* st) {
  int64_t N = sys->N;
  for (int64_t i = 0; i < N; ++i) z[i] = a[i] + hg * fi0[i];   /* predictor */
  double crate = 1.0, delp = 0.0;
  for (int m = 1; m <= 3; ++m) {
    int rf = sys->fi(sys->user, tz, z, fi);
    st->nfi++;
    if (rf) return 1;
    for (int64_t i = 0; i < N; ++i) {
      r[i] = a[i] + hg * fi[i] - z[i];
      if (!isfinite(r[i])) return 1;
    }
    if (sys->isolve(sys->user, tz, z, hg, r)) return 1;
    for (int64_t i = 0; i < N; ++i) z[i] += r[i];
    st->nni++;
    double del = wrms(N, r, ewt);
    if (!isfinite(del)) return 1;
    if (m > 1) {
      double rate = del / delp;
      crate = (0.3 * crate > rate) ? 0.3 * crate : rate;
    }
    if (del * (crate < 1.0 ? crate : 1.0) <= 0.1) return 0;
    if (m >= 2 && del > 2.3 * delp) return 1;
    delp = del;
  }
  return 1;
}

int or_ark_integrate(const or_imex_system* sys, const or_ark_options* opt, double t0,
                     const double* y0, double tout, double* yout, or_ark_stats* st) {
  int64_t N = sys->N;
  tables T;
  or_ark_table(T.c, T.AE, T.AI, T.b, T.bh);
  memset(st, 0, sizeof *st);
  int64_t mxstep = opt->mxstep > 0 ? opt->mxstep : 100000;
  double* y = (double*)malloc(sizeof(double) * N);
  double* ewt = (double*)malloc(sizeof(double) * N);
  double* fe = (double*)malloc(sizeof(double) * N * S);
  double* fi = (double*)malloc(sizeof(double) * N * S);
  double* a = (double*)malloc(sizeof(double) * N);
  double* z = (double*)malloc(sizeof(double) * N);
  double* r = (double*)malloc(sizeof(double) * N);
  double* tmp = (double*)malloc(sizeof(double) * N);
  double* ynew = (double*)malloc(sizeof(double) * N);
  int ret = 0;
  if (!y || !ewt || !fe || !fi || !a || !z || !r || !tmp || !ynew) { ret = OR_MEM_FAIL; goto done; }
  memcpy(y, y0, sizeof(double) * N);
  double t = t0, h = 0.0, e1 = 0.0, e2 = 0.0;
  int first = 1;
  if (tout == t) goto out;
  for (int64_t i = 0; i < N; ++i) ewt[i] = 1.0 / (opt->rtol * fabs(y[i]) + opt->atol);
  if (opt->fixed_h > 0.0) {
    h = (tout >= t) ? opt->fixed_h : -opt->fixed_h;
  } else {
    if (sys->fe(sys->user, t, y, fe) || sys->fi(sys->user, t, y, fi)) { ret = OR_RHSFUNC_FAIL; goto done; }
    st->nfe++;
    st->nfi++;
    for (int64_t i = 0; i < N; ++i) tmp[i] = fe[i] + fi[i];
    ret = ark_h0(sys, opt, t, y, tout, tmp, z, a, r, ewt, st, &h);
    if (ret) goto done;
  }
  for (int64_t nst = 0; (tout - t) * h > 0.0; ++nst) {
    if (nst >= mxstep) { ret = OR_TOO_MUCH_WORK; break; }
    for (int64_t i = 0; i < N; ++i) ewt[i] = 1.0 / (opt->rtol * fabs(y[i]) + opt->atol);
    int ncf = 0, nef = 0;
    for (;;) {                                   /* attempts of this step */
      int last = 0;
      double hs = h;
      if ((t + h - tout) * h >= 0.0) { hs = tout - t; last = 1; }
      if (t + hs == t) { ret = OR_ERR_FAILURE; goto out; }
      /* stage 1 */
      if (sys->fe(sys->user, t, y, fe) || sys->fi(sys->user, t, y, fi)) { ret = OR_RHSFUNC_FAIL; goto out; }
      st->nfe++;
      st->nfi++;
      int failed = 0;
      for (int i = 1; i < S && !failed; ++i) {
        for (int64_t k = 0; k < N; ++k) {
          double s = 0.0;
          for (int j = 0; j < i; ++j) s += T.AE[i * S + j] * fe[j * N + k] + T.AI[i * S + j] * fi[j * N + k];
          a[k] = y[k] + hs * s;
        }
        double tz = t + T.c[i] * hs;
        if (stage_solve(sys, tz, hs * T.AI[i * S + i], a, fi, ewt, z, fi + i * N, r, st)) { failed = 1; break; }
        if (sys->fe(sys->user, tz, z, fe + i * N) || sys->fi(sys->user, tz, z, fi + i * N)) { failed = 1; break; }
        st->nfe++;
        st->nfi++;
      }
      if (failed) {
        st->ncfn++;
        if (opt->fixed_h > 0.0 || ++ncf >= 10) { ret = OR_CONV_FAILURE; goto out; }
        h = hs * 0.25;
        continue;
      }
      for (int64_t k = 0; k < N; ++k) {
        double s = 0.0, e = 0.0;
        for (int i = 0; i < S; ++i) {
          double g = fe[i * N + k] + fi[i * N + k];
          s += T.b[i] * g;
          e += (T.b[i] - T.bh[i]) * g;
        }
        ynew[k] = y[k] + hs * s;
        tmp[k] = hs * e;
      }
      double dsm = wrms(N, tmp, ewt);
      if (opt->fixed_h <= 0.0 && !(dsm <= 1.0)) {
        st->netf++;
        if (++nef >= 7) { ret = OR_ERR_FAILURE; goto out; }
        double eta = 0.96 * pow(1.5 * dsm, -1.0 / 3.0);
        if (!(eta >= 0.1)) eta = 0.1;
        if (eta > 0.9) eta = 0.9;
        if (nef >= 2 && eta > 0.3) eta = 0.3;
        h = hs * eta;
        continue;
      }
      memcpy(y, ynew, sizeof(double) * N);
      t = last ? tout : t + hs;
      st->nst++;
      st->hlast = hs;
      if (opt->fixed_h <= 0.0) {
        double e0 = 1.5 * dsm;
        if (e0 < 1e-10) e0 = 1e-10;
        double p1 = e1 > 0.0 ? e1 : e0, p2 = e2 > 0.0 ? e2 : p1;
        double eta = 0.96 * pow(e0, -0.58 / 3.0) * pow(p1, 0.21 / 3.0) * pow(p2, -0.1 / 3.0);
        double cap = first ? 1.0e4 : 20.0;
        if (eta > cap) eta = cap;
        if (eta < 0.1) eta = 0.1;
        if (eta >= 1.0 && eta <= 1.5) eta = 1.0;
        e2 = p1;
        e1 = e0;
        h = hs * eta;
        first = 0;
      }
      break;
    }
  }
out:
  memcpy(yout, y, sizeof(double) * N);
  st->tcur = t;
done:
  free(y); free(ewt); free(fe); free(fi); free(a); free(z); free(r); free(tmp); free(ynew);
  return ret;
}

/* ---- the demonstration problem: f_E = advection, f_I = reaction -------- */
static int bruss_fe(void* u, double t, const double* y, double* f) {
  (void)t;
  const or_bruss* p = (const or_bruss*)u;
  or_bruss_transport(p, y, f);
  return 0;
}

static int bruss_fi(void* u, double t, const double* y, double* f) {
  (void)t;
  const or_bruss* p = (const or_bruss*)u;
  or_bruss_reaction(p, y, f);
  int64_t N = 3 * (int64_t)p->nx;
  for (int64_t i = 0; i < N; ++i) if (!isfinite(f[i])) return 1;
  return 0;
}

/* x <- (I - gamma J_R(y))^{-1} x, one pivoted 3x3 LU per point */
static int bruss_isolve(void* u, double t, const double* y, double gamma, double* x) {
  (void)t;
  const or_bruss* p = (const or_bruss*)u;
  int64_t np = p->nx;
  for (int64_t q = 0; q < np; ++q) {
    double M[9];
    int piv[3];
    or_bruss_reaction_jac(p, y[q], y[np + q], y[2 * np + q], M);
    for (int k = 0; k < 9; ++k) M[k] = ((k % 4) == 0 ? 1.0 : 0.0) - gamma * M[k];
    if (or_lu_factor(3, M, piv)) return 1;
    double b[3] = {x[q], x[np + q], x[2 * np + q]};
    or_lu_solve(3, M, piv, b);
    x[q] = b[0]; x[np + q] = b[1]; x[2 * np + q] = b[2];
  }
  return 0;
}

int or_bruss_ark_integrate(const or_bruss* p, double t0, const double* y0, double tout,
                           double rtol, double atol, int64_t mxstep, double* yout,
                           int64_t* stats) {
  if (p->dim != 1) return OR_ILL_INPUT;
  or_imex_system sys = {3 * (int64_t)p->nx, (void*)p, bruss_fe, bruss_fi, bruss_isolve};
  or_ark_options opt;
  memset(&opt, 0, sizeof opt);
  opt.rtol = rtol;
  opt.atol = atol;
  opt.mxstep = mxstep;
  or_ark_stats st;
  int ret = or_ark_integrate(&sys, &opt, t0, y0, tout, yout, &st);
  if (stats) {
    stats[0] = st.nst; stats[1] = st.nfe; stats[2] = st.nfi; stats[3] = st.nni;
    stats[4] = st.ncfn; stats[5] = st.netf; stats[6] = 0; stats[7] = 0;
  }
  return ret;
}
