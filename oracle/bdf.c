/*
 * bdf.c - oracle variable-order (1..5), variable-step BDF integrator with
 * Newton iteration, in Nordsieck form.  TEST INFRASTRUCTURE ONLY (oracle.h).
 *
 * The paper names the method (CVODE, an adaptive-order, adaptive-step
 * implicit linear multistep method, Sec. 1), its Newton nonlinear solver and
 * direct / Krylov linear solvers (Sec. 5), and the per-system Newton solve with
 * whole-step retry on failure (Sec. 7), but defers every formula to the CVODE
 * documentation.  The steps below are therefore the standard Nordsieck-form
 * BDF written from its mathematics, with these readings:
 *
 *  z = [z_0 .. z_q], z_j ~ h^j y^(j) / j!  (Nordsieck history)
 *  predict:      z_j <- sum_{k>=j} C(k, j) z_k              (Taylor shift by h)
 *  corrector:    z <- z + l Delta, with l_j the coefficients of
 *                Lambda(x) = prod_{i=1}^{q} (1 + x/i)  (l_0 = 1, l_1 = sum 1/i)
 *                so the new polynomial agrees with the old one at the q past
 *                points and has slope h f(t_n, y_n) at t_n;
 *  Newton:       G(Delta) = Delta - gamma f(t_n, z_0 + Delta) + z_1 / l_1,
 *                gamma = h / l_1, (I - gamma J) delta = -G, at most 3 iterations;
 *  error test:   dsm = E_q ||Delta||_WRMS <= 1, E_q = 1 / ((q+1) l_1(q));
 *  step changes: the history is rescaled z_j <- eta^j z_j and the
 *                constant-step coefficients above are kept (fixed-step
 *                interpolation); after every change of h or q both are held
 *                for q+1 steps, so the order-(q+1) estimate from
 *                Delta_n - Delta_{n-1} compares two steps of equal size.
 * Step-size heuristics (initial step, safety factors 6 / 6 / 10, eta limits,
 * Jacobian reuse) are the proposals recorded with each site below.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define ZCOLS (OR_QMAX + 2)

struct or_bdf {
  or_system sys;
  or_options opt;
  int64_t N;
  double t, h;
  int q, qwait;
  int started;           /* initial step chosen */
  int grown_once;        /* first step-size increase done (eta cap 1e4 before) */
  double *z, *zs, *ewt, *acor, *acor_prev, *y, *f, *b;
  double gamma, gammap, crate;
  double *bcrate, *bdelp; /* task-local Newton: per block rate and last |delta| */
  int8_t* bstate;         /* per block: 0 iterating, 1 converged, 2 failed */
  int64_t nst, nstlp;
  int force_setup, setup_done;
  or_stats st;
  int64_t ntrace;
};

/* ---- method constants ---------------------------------------------------- */
static void coef_l(int q, double* l) {
  for (int j = 0; j <= OR_QMAX + 1; ++j) l[j] = 0.0;
  l[0] = 1.0;
  for (int i = 1; i <= q; ++i)            /* multiply by (1 + x/i) */
    for (int j = i; j >= 1; --j) l[j] += l[j - 1] / (double)i;
}
static double ell1(int q) { double l[OR_QMAX + 2]; coef_l(q, l); return l[1]; }
static double factorial(int k) { double r = 1.0; for (int i = 2; i <= k; ++i) r *= i; return r; }

/* E_q: local error of order q per unit ||Delta|| (at constant step Delta equals
 * h^{q+1} y^{(q+1)} and the corrector error is h^{q+1} y^{(q+1)} / ((q+1) l_1));
 * E_{q-1}: order q-1 error per unit ||z_q|| (h^q y^(q) = q! z_q);
 * E_{q+1}: order q+1 error per unit ||Delta_n - Delta_{n-1}|| (~ h^{q+2} y^(q+2)). */
void or_bdf_constants(int q, double* l, double* out) {
  coef_l(q, l);
  out[0] = 1.0 / ((q + 1) * ell1(q));
  out[1] = q > 1 ? factorial(q - 1) / ell1(q - 1) : 0.0;
  out[2] = q < OR_QMAX ? 1.0 / ((q + 2) * ell1(q + 1)) : 0.0;
}

static double binom(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
  return r;
}

static double* Z(or_bdf* m, int j) { return m->z + (int64_t)j * m->N; }

static double wrms(or_bdf* m, const double* x) { return or_wrms_norm(m->N, x, m->ewt); }

static void set_ewt(or_bdf* m) {
  const double* y = Z(m, 0);
  for (int64_t i = 0; i < m->N; ++i) m->ewt[i] = 1.0 / (m->opt.rtol * fabs(y[i]) + m->opt.atol);
}

/* z_j <- sum_{k=j}^{q} C(k,j) z_k  (value of the history polynomial at t+h) */
static void predict(or_bdf* m) {
  int64_t N = m->N;
  double* tmp = m->b;
  for (int j = 0; j <= m->q; ++j) {
    for (int64_t i = 0; i < N; ++i) {
      double s = 0.0;
      for (int k = j; k <= m->q; ++k) s += binom(k, j) * Z(m, k)[i];
      tmp[i] = s;
    }
    memcpy(Z(m, j), tmp, sizeof(double) * N);
  }
}

static void rescale(or_bdf* m, double eta) {
  double f = 1.0;
  for (int j = 1; j <= m->q; ++j) {
    f *= eta;
    for (int64_t i = 0; i < m->N; ++i) Z(m, j)[i] *= f;
  }
  m->h *= eta;
}

static void save_z(or_bdf* m) { memcpy(m->zs, m->z, sizeof(double) * m->N * ZCOLS); }
static void restore_z(or_bdf* m) { memcpy(m->z, m->zs, sizeof(double) * m->N * ZCOLS); }

or_bdf* or_bdf_create(const or_system* sys, const or_options* opt, double t0, const double* y0) {
  or_bdf* m = (or_bdf*)calloc(1, sizeof(or_bdf));
  if (!m) return NULL;
  m->sys = *sys;
  m->opt = *opt;
  if (m->opt.mxstep <= 0) m->opt.mxstep = 100000;
  if (m->opt.qmax <= 0 || m->opt.qmax > OR_QMAX) m->opt.qmax = OR_QMAX;
  int64_t N = sys->N;
  m->N = N;
  m->z = (double*)calloc((size_t)(N * ZCOLS), sizeof(double));
  m->zs = (double*)calloc((size_t)(N * ZCOLS), sizeof(double));
  m->ewt = (double*)calloc((size_t)N, sizeof(double));
  m->acor = (double*)calloc((size_t)N, sizeof(double));
  m->acor_prev = (double*)calloc((size_t)N, sizeof(double));
  m->y = (double*)calloc((size_t)N, sizeof(double));
  m->f = (double*)calloc((size_t)N, sizeof(double));
  m->b = (double*)calloc((size_t)N, sizeof(double));
  const int64_t nb = sys->nblock > 0 ? sys->nblock : 0;
  m->bcrate = (double*)calloc((size_t)(nb + 1), sizeof(double));
  m->bdelp = (double*)calloc((size_t)(nb + 1), sizeof(double));
  m->bstate = (int8_t*)calloc((size_t)(nb + 1), 1);
  if (!m->z || !m->zs || !m->ewt || !m->acor || !m->acor_prev || !m->y || !m->f || !m->b ||
      !m->bcrate || !m->bdelp || !m->bstate) {
    or_bdf_free(m);
    return NULL;
  }
  memcpy(m->z, y0, sizeof(double) * N);
  m->t = t0;
  m->q = 1;
  return m;
}

void or_bdf_free(or_bdf* m) {
  if (!m) return;
  free(m->z); free(m->zs); free(m->ewt); free(m->acor); free(m->acor_prev);
  free(m->y); free(m->f); free(m->b);
  free(m->bcrate); free(m->bdelp); free(m->bstate);
  free(m);
}

void or_bdf_stats(const or_bdf* m, or_stats* st) {
  *st = m->st;
  st->nst = m->nst;
  st->tcur = m->t;
}

/* Initial step (reading; the paper is silent).  Upper bound: a tenth of the
 * interval and the step at which h |f_i| reaches 0.1 |y_i| + atol; then up
 * to four refinements of h ~ sqrt(2 / ||y''||), with y'' from a forward
 * difference of f along h f; h0 = half the result, within [100 eps t, upper]. */
static int initial_step(or_bdf* m, double tout, const double* f0) {
  int64_t N = m->N;
  const double* y0 = Z(m, 0);
  double tdist = fabs(tout - m->t);
  double tround = 2.220446049250313e-16 * fmax(fabs(m->t), fabs(tout));
  double hlb = 100.0 * tround;
  double hub = 0.1 * tdist;
  double inv = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    double r = fabs(f0[i]) / (0.1 * fabs(y0[i]) + m->opt.atol);
    if (r > inv) inv = r;
  }
  if (inv * hub > 1.0) hub = 1.0 / inv;
  if (hub < hlb) hub = hlb;
  double hg = sqrt(hlb * hub);
  double hnew = hg;
  for (int it = 0; it < 4; ++it) {
    int ok = 0;
    for (int tries = 0; tries < 4; ++tries) {
      for (int64_t i = 0; i < N; ++i) m->y[i] = y0[i] + hg * f0[i];
      int r = m->sys.rhs(m->sys.user, m->t + hg, m->y, m->f);
      m->st.nfe++;
      if (r < 0) return OR_RHSFUNC_FAIL;
      if (r == 0) { ok = 1; break; }
      hg *= 0.2;
    }
    if (!ok) return OR_RHSFUNC_FAIL;
    for (int64_t i = 0; i < N; ++i) m->b[i] = (m->f[i] - f0[i]) / hg;
    double ydd = wrms(m, m->b);
    hnew = (ydd * hub * hub > 2.0) ? sqrt(2.0 / ydd) : sqrt(hg * hub);
    double rat = hnew / hg;
    if (it > 0 && rat > 0.5 && rat < 2.0) break;
    hg = hnew;
  }
  double h0 = 0.5 * hnew;
  if (h0 < hlb) h0 = hlb;
  if (h0 > hub) h0 = hub;
  m->h = (tout >= m->t) ? h0 : -h0;
  return 0;
}

/* Newton iteration on G(Delta) = 0 for the predicted history in z.
 * Returns 0 converged (acor = Delta, *acnrm = ||Delta||), 1 recoverable
 * failure, < 0 fatal.  M = I - gamma J is refreshed (reading; CVODE-like
 * reuse) on the first step, when asked after a failure, when gamma moved
 * more than 30% from the gamma of the last setup, and every 20 steps; with a
 * stale M the correction is scaled by 2 / (1 + gamma / gamma_setup).  A
 * failed iteration with a stale M is retried once with a fresh one.
 * Convergence: with rate R = max(0.3 R_prev, |delta_m| / |delta_{m-1}|),
 * converged when |delta_m| min(1, R) E_q <= 0.1 (a tenth of the error-test
 * bound); diverged when |delta_m| > 2 |delta_{m-1}|. */
static int newton_local(or_bdf* m, double tnew, double Eq, double* acnrm);

static int newton(or_bdf* m, double tnew, double Eq, double* acnrm) {
  if (m->sys.nblock > 0) return newton_local(m, tnew, Eq, acnrm);
  int64_t N = m->N;
  double l1 = ell1(m->q);
  const double* z0 = Z(m, 0);
  const double* z1 = Z(m, 1);
  int tried_fresh = 0;
  for (;;) {
    int jcur = 0;
    if (!m->setup_done || m->force_setup || fabs(m->gamma / m->gammap - 1.0) > 0.3 ||
        m->nst >= m->nstlp + 20) {
      int r = m->sys.lsetup(m->sys.user, tnew, z0, m->gamma);
      m->st.nsetups++;
      m->gammap = m->gamma;
      m->crate = 1.0;
      m->nstlp = m->nst;
      m->force_setup = 0;
      m->setup_done = 1;
      jcur = 1;
      if (r < 0) return OR_LSETUP_FAIL;
      if (r > 0) return 1;
    }
    for (int64_t i = 0; i < N; ++i) { m->acor[i] = 0.0; m->y[i] = z0[i]; }
    double delp = 0.0;
    int conv = 0;
    for (int it = 1; it <= 3; ++it) {
      int r = m->sys.rhs(m->sys.user, tnew, m->y, m->f);
      m->st.nfe++;
      if (r < 0) return OR_RHSFUNC_FAIL;
      if (r > 0) break;
      for (int64_t i = 0; i < N; ++i) m->b[i] = m->gamma * m->f[i] - z1[i] / l1 - m->acor[i];
      double tol = 0.05 * 0.1 / Eq;
      r = m->sys.lsolve(m->sys.user, tnew, m->y, m->gamma, m->ewt, tol, m->b);
      if (r < 0) return OR_LSOLVE_FAIL;
      if (r > 0) break;
      if (m->sys.direct && m->gamma != m->gammap) {
        double s = 2.0 / (1.0 + m->gamma / m->gammap);
        for (int64_t i = 0; i < N; ++i) m->b[i] *= s;
      }
      double del = wrms(m, m->b);
      for (int64_t i = 0; i < N; ++i) { m->acor[i] += m->b[i]; m->y[i] = z0[i] + m->acor[i]; }
      m->st.nni++;
      if (it > 1) {
        double rate = del / delp;
        m->crate = (0.3 * m->crate > rate) ? 0.3 * m->crate : rate;
      }
      double dcon = del * (m->crate < 1.0 ? m->crate : 1.0) * Eq / 0.1;
      if (dcon <= 1.0) {
        *acnrm = (it == 1) ? del : wrms(m, m->acor);
        conv = 1;
        break;
      }
      if (it >= 2 && del > 2.0 * delp) break;
      delp = del;
    }
    if (conv) return 0;
    if (!jcur && !tried_fresh) { m->force_setup = 1; tried_fresh = 1; continue; }
    return 1;
  }
}

/* Task-local Newton (sys.nblock > 0).  The Jacobian refresh rule, gamma and
 * the stale-M scaling are those of newton() and shared by all blocks; each
 * block b then runs the iteration of newton() on its own entries: its own
 * rate R_b, its own |delta| (WRMS over the block's n_b entries), its own
 * convergence and divergence tests, and it stops changing once converged.  A
 * block whose f is not finite fails.  The solve succeeds when every block
 * has converged (then *acnrm = ||Delta|| over all N); otherwise a stale M is
 * refreshed once, as in newton(), and the step fails after that. */
static int newton_local(or_bdf* m, double tnew, double Eq, double* acnrm) {
  const int64_t N = m->N, nb = m->sys.nblock;
  const int64_t* off = m->sys.block_off;
  double l1 = ell1(m->q);
  const double* z0 = Z(m, 0);
  const double* z1 = Z(m, 1);
  int tried_fresh = 0;
  for (;;) {
    int jcur = 0;
    if (!m->setup_done || m->force_setup || fabs(m->gamma / m->gammap - 1.0) > 0.3 ||
        m->nst >= m->nstlp + 20) {
      int r = m->sys.lsetup(m->sys.user, tnew, z0, m->gamma);
      m->st.nsetups++;
      m->gammap = m->gamma;
      for (int64_t k = 0; k < nb; ++k) m->bcrate[k] = 1.0;
      m->nstlp = m->nst;
      m->force_setup = 0;
      m->setup_done = 1;
      jcur = 1;
      if (r < 0) return OR_LSETUP_FAIL;
      if (r > 0) return 1;
    }
    for (int64_t i = 0; i < N; ++i) { m->acor[i] = 0.0; m->y[i] = z0[i]; }
    for (int64_t k = 0; k < nb; ++k) { m->bstate[k] = 0; m->bdelp[k] = 0.0; }
    int64_t active = nb, failed = 0;
    for (int it = 1; it <= 3 && active > 0; ++it) {
      int r = m->sys.rhs(m->sys.user, tnew, m->y, m->f);
      m->st.nfe++;
      if (r < 0) return OR_RHSFUNC_FAIL;
      for (int64_t i = 0; i < N; ++i) m->b[i] = m->gamma * m->f[i] - z1[i] / l1 - m->acor[i];
      r = m->sys.lsolve(m->sys.user, tnew, m->y, m->gamma, m->ewt, 0.05 * 0.1 / Eq, m->b);
      if (r < 0) return OR_LSOLVE_FAIL;
      const double s = (m->sys.direct && m->gamma != m->gammap) ? 2.0 / (1.0 + m->gamma / m->gammap) : 1.0;
      for (int64_t k = 0; k < nb; ++k) {
        if (m->bstate[k] != 0) continue;
        const int64_t i0 = off[k], i1 = off[k + 1];
        int finite = r == 0;
        for (int64_t i = i0; i < i1; ++i) finite = finite && isfinite(m->f[i]);
        if (!finite) { m->bstate[k] = 2; --active; ++failed; continue; }
        double ss = 0.0;
        for (int64_t i = i0; i < i1; ++i) {
          const double d = m->b[i] * s;
          ss += (d * m->ewt[i]) * (d * m->ewt[i]);
          m->acor[i] += d;
          m->y[i] = z0[i] + m->acor[i];
        }
        const double del = sqrt(ss / (double)(i1 - i0));
        m->st.nni++;
        if (it > 1) {
          double rate = del / m->bdelp[k];
          m->bcrate[k] = (0.3 * m->bcrate[k] > rate) ? 0.3 * m->bcrate[k] : rate;
        }
        double dcon = del * (m->bcrate[k] < 1.0 ? m->bcrate[k] : 1.0) * Eq / 0.1;
        if (dcon <= 1.0) { m->bstate[k] = 1; --active; continue; }
        if ((it >= 2 && del > 2.0 * m->bdelp[k]) || it == 3) { m->bstate[k] = 2; --active; ++failed; continue; }
        m->bdelp[k] = del;
      }
    }
    if (!failed && active == 0) {
      *acnrm = wrms(m, m->acor);
      return 0;
    }
    if (!jcur && !tried_fresh) { m->force_setup = 1; tried_fresh = 1; continue; }
    return 1;
  }
}

/* The step-size and order choice from the three test quantities (reading:
 * safety factors 6 for orders q and q-1, 10 for q+1; change only when the
 * best eta >= 1.5; eta <= 1e4 before the first increase, <= 10 after; ties
 * keep q, then prefer q-1).  dsm = E_q |Delta|, dqm1 = E_{q-1} |z_q| (used
 * when q > 1), dqp1 = E_{q+1} |Delta - Delta_prev| (used when q < qmax).
 * Returns 1 and sets *qnew, *eta when h (and maybe q) changes, else 0. */
int or_bdf_choose(int q, int qmax, int grown_once, double dsm, double dqm1, double dqp1, int* qnew,
                  double* eta) {
  double eq = 1.0 / (pow(6.0 * dsm, 1.0 / (q + 1)) + 1e-6);
  double eqm1 = 0.0, eqp1 = 0.0;
  if (q > 1) eqm1 = 1.0 / (pow(6.0 * dqm1, 1.0 / q) + 1e-6);
  if (q < qmax) eqp1 = 1.0 / (pow(10.0 * dqp1, 1.0 / (q + 2)) + 1e-6);
  double etam = eq;
  int qn = q;
  if (eqm1 > etam) { etam = eqm1; qn = q - 1; }
  if (eqp1 > etam) { etam = eqp1; qn = q + 1; }
  if (etam < 1.5) return 0;
  double cap = grown_once ? 10.0 : 1.0e4;
  if (etam > cap) etam = cap;
  *qnew = qn;
  *eta = etam;
  return 1;
}

/* choose step size and order after an accepted step (or_bdf_choose on the
 * step's norms), every q+1 steps after a change and after every step that
 * kept h */
static void select_next(or_bdf* m, double dsm) {
  if (--m->qwait > 0) return;
  int q = m->q;
  double l[OR_QMAX + 2], E[3];
  or_bdf_constants(q, l, E);
  double dqm1 = 0.0, dqp1 = 0.0;
  if (q > 1) dqm1 = E[1] * wrms(m, Z(m, q));
  if (q < m->opt.qmax) {
    for (int64_t i = 0; i < m->N; ++i) m->b[i] = m->acor[i] - m->acor_prev[i];
    dqp1 = E[2] * wrms(m, m->b);
  }
  int qn = q;
  double etam = 1.0;
  if (!or_bdf_choose(q, m->opt.qmax, m->grown_once, dsm, dqm1, dqp1, &qn, &etam)) {
    m->qwait = 1;
    return;
  }
  m->grown_once = 1;
  if (qn == q + 1) {
    double fq = factorial(q + 1);
    for (int64_t i = 0; i < m->N; ++i) Z(m, q + 1)[i] = m->acor[i] / fq;
    m->q = q + 1;
  } else if (qn == q - 1) {
    for (int64_t i = 0; i < m->N; ++i) Z(m, q)[i] = 0.0;
    m->q = q - 1;
  }
  rescale(m, etam);
  m->qwait = m->q + 1;
}

/* one accepted step towards tout; *reached set when the step ended on tout */
static int step(or_bdf* m, double tout, int* reached) {
  int64_t N = m->N;
  int ncf = 0, nef = 0;
  int fixed = m->opt.fixed_h > 0.0;
  for (;;) {
    int last = 0;
    if (!fixed && !m->opt.interp && (m->t + m->h - tout) * m->h >= 0.0) {
      last = 1;
      if (m->t + m->h != tout) { rescale(m, (tout - m->t) / m->h); m->qwait = m->q + 1; }
    }
    if (m->t + m->h == m->t) return OR_ERR_FAILURE;
    double l[OR_QMAX + 2], E[3];
    or_bdf_constants(m->q, l, E);
    save_z(m);
    predict(m);
    double tnew = last ? tout : m->t + m->h;
    m->gamma = m->h / l[1];
    double acnrm = 0.0;
    int r = newton(m, tnew, E[0], &acnrm);
    if (r < 0) { restore_z(m); return r; }
    if (r == 1) {
      restore_z(m);
      ncf++;
      m->st.ncfn++;
      if (ncf >= 10 || fixed) return OR_CONV_FAILURE;
      rescale(m, 0.25);
      m->qwait = m->q + 1;
      m->force_setup = 1;
      continue;
    }
    double dsm = acnrm * E[0];
    if (!fixed && !(dsm <= 1.0)) {
      restore_z(m);
      nef++;
      m->st.netf++;
      if (nef >= 7) return OR_ERR_FAILURE;
      if (nef < 3) {
        double eta = 1.0 / (pow(6.0 * dsm, 1.0 / (m->q + 1)) + 1e-6);
        if (!(eta >= 0.1)) eta = 0.1;
        if (nef >= 2 && eta > 0.2) eta = 0.2;
        rescale(m, eta);
        m->qwait = m->q + 1;
      } else {
        /* third failure: restart at order 1 with h/10 and a fresh slope */
        for (int j = 2; j <= OR_QMAX + 1; ++j)
          for (int64_t i = 0; i < N; ++i) Z(m, j)[i] = 0.0;
        m->q = 1;
        m->h *= 0.1;
        int rr = m->sys.rhs(m->sys.user, m->t, Z(m, 0), m->f);
        m->st.nfe++;
        if (rr != 0) return OR_RHSFUNC_FAIL;
        for (int64_t i = 0; i < N; ++i) Z(m, 1)[i] = m->h * m->f[i];
        m->qwait = 2;
      }
      continue;
    }
    /* accept: z <- z + l Delta */
    for (int j = 0; j <= m->q; ++j)
      for (int64_t i = 0; i < N; ++i) Z(m, j)[i] += l[j] * m->acor[i];
    m->t = tnew;
    m->nst++;
    m->st.hlast = m->h;
    m->st.qlast = m->q;
    if (m->opt.trace_y && m->ntrace < m->opt.trace_cap) {
      memcpy(m->opt.trace_y + m->ntrace * N, Z(m, 0), sizeof(double) * N);
      if (m->opt.trace_acor) memcpy(m->opt.trace_acor + m->ntrace * N, m->acor, sizeof(double) * N);
      m->ntrace++;
    }
    if (!fixed) select_next(m, dsm);
    memcpy(m->acor_prev, m->acor, sizeof(double) * N);
    *reached = last;
    return 0;
  }
}

int or_bdf_solve(or_bdf* m, double tout, double* yout) {
  int64_t N = m->N;
  int ret = 0;
  if (tout == m->t) {            /* nothing to integrate; the first step waits for tout != t0 */
    memcpy(yout, Z(m, 0), sizeof(double) * N);
    return 0;
  }
  if (!m->started) {
    set_ewt(m);
    int r = m->sys.rhs(m->sys.user, m->t, Z(m, 0), m->f);
    m->st.nfe++;
    if (r != 0) { ret = OR_RHSFUNC_FAIL; goto done; }
    double* f0 = (double*)malloc(sizeof(double) * N);
    if (!f0) { ret = OR_MEM_FAIL; goto done; }
    memcpy(f0, m->f, sizeof(double) * N);
    if (m->opt.fixed_h > 0.0) m->h = (tout >= m->t) ? m->opt.fixed_h : -m->opt.fixed_h;
    else if (m->opt.h0 > 0.0) m->h = (tout >= m->t) ? m->opt.h0 : -m->opt.h0;
    else r = initial_step(m, tout, f0);
    if (r == 0)
      for (int64_t i = 0; i < N; ++i) Z(m, 1)[i] = m->h * f0[i];
    free(f0);
    if (r != 0) { ret = r; goto done; }
    m->q = (m->opt.fixed_h > 0.0 && m->opt.fixed_q > 0) ? m->opt.fixed_q : 1;
    if (m->opt.fixed_h > 0.0 && m->opt.z_init)
      memcpy(m->z, m->opt.z_init, sizeof(double) * N * (m->q + 1));
    m->qwait = m->q + 1;
    m->started = 1;
  }
  int64_t nst0 = m->nst;
  if (m->opt.fixed_h > 0.0) {
    /* constant-step run: as many steps of fixed_h as fit in [t, tout] */
    while ((tout - m->t) * m->h > 0.5 * m->h * m->h) {
      set_ewt(m);
      int reached = 0;
      ret = step(m, tout, &reached);
      if (ret) break;
    }
  } else {
    while ((tout - m->t) * m->h > 0.0) {
      if (m->nst - nst0 >= m->opt.mxstep) { ret = OR_TOO_MUCH_WORK; break; }
      set_ewt(m);
      int reached = 0;
      ret = step(m, tout, &reached);
      if (ret) break;
      if (reached) { m->t = tout; break; }
    }
  }
done:
  if (m->opt.interp && ret == 0 && m->started && m->t != tout) {
    /* the history polynomial at tout (Horner in s = (tout - t_n) / h) */
    double s = (tout - m->t) / m->h;
    for (int64_t i = 0; i < N; ++i) {
      double v = Z(m, m->q)[i];
      for (int j = m->q - 1; j >= 0; --j) v = v * s + Z(m, j)[i];
      yout[i] = v;
    }
  } else {
    memcpy(yout, Z(m, 0), sizeof(double) * N);
  }
  m->st.tcur = m->t;
  return ret;
}
