/*
 * linalg.c - oracle vector operations and dense LU.  TEST INFRASTRUCTURE ONLY
 * (see oracle.h).
 *
 * Vector operations follow the definitions of the fused NVECTOR operations
 * (Sec. 4: streaming operations such as N_VLinearSum and reductions such as
 * norms and dot products, whose scalar result returns to the host).  Each is
 * the definition written out element by element; reductions use Neumaier's
 * compensated summation so their result is accurate to about one rounding.
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

/* Neumaier (improved Kahan-Babuska) running sum */
typedef struct { double s, c; } nsum;
static void nadd(nsum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}
static double nget(const nsum* a) { return a->s + a->c; }

/* z = a x + b y */
/* the elementwise support operations of the vector class (Sec. 4): one
 * correctly rounded IEEE operation per element (two for the error weights) */
void or_scale(int64_t n, double c, const double* x, double* z) {
  for (int64_t i = 0; i < n; ++i) z[i] = c * x[i];
}
void or_const(int64_t n, double c, double* z) {
  for (int64_t i = 0; i < n; ++i) z[i] = c;
}
void or_abs(int64_t n, const double* x, double* z) {
  for (int64_t i = 0; i < n; ++i) z[i] = fabs(x[i]);
}
void or_inv(int64_t n, const double* x, double* z) {
  for (int64_t i = 0; i < n; ++i) z[i] = 1.0 / x[i];
}
void or_add_const(int64_t n, const double* x, double b, double* z) {
  for (int64_t i = 0; i < n; ++i) z[i] = x[i] + b;
}
/* error weights ewt_i = 1 / (rtol |y_i| + atol) */
void or_error_weights(int64_t n, double rtol, double atol, const double* y, double* w) {
  for (int64_t i = 0; i < n; ++i) w[i] = 1.0 / (rtol * fabs(y[i]) + atol);
}

void or_linear_sum(int64_t n, double a, const double* x, double b, const double* y, double* z) {
  for (int64_t i = 0; i < n; ++i) z[i] = a * x[i] + b * y[i];
}

/* z = sum_j c_j x_j  (N_VLinearCombination) */
void or_linear_combination(int64_t n, int nv, const double* c, const double* const* x, double* z) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < nv; ++j) s += c[j] * x[j][i];
    z[i] = s;
  }
}

/* z_j = a_j x + y_j  (N_VScaleAddMulti) */
void or_scale_add_multi(int64_t n, int nv, const double* a, const double* x,
                        const double* const* y, double* const* z) {
  for (int j = 0; j < nv; ++j)
    for (int64_t i = 0; i < n; ++i) z[j][i] = a[j] * x[i] + y[j][i];
}

/* d_j = x . y_j  (N_VDotProdMulti) */
void or_dot_prod_multi(int64_t n, int nv, const double* x, const double* const* y,
                       double* d, double* sabs) {
  for (int j = 0; j < nv; ++j) {
    nsum s = {0.0, 0.0}, a = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) {
      double p = x[i] * y[j][i];
      nadd(&s, p);
      nadd(&a, fabs(p));
    }
    d[j] = nget(&s);
    if (sabs) sabs[j] = nget(&a);
  }
}

/* sqrt( sum_i (x_i w_i)^2 / n )  (N_VWrmsNorm) */
double or_wrms_norm(int64_t n, const double* x, const double* w) {
  nsum s = {0.0, 0.0};
  for (int64_t i = 0; i < n; ++i) {
    double p = x[i] * w[i];
    nadd(&s, p * p);
  }
  return n > 0 ? sqrt(nget(&s) / (double)n) : 0.0;
}

/* Gaussian elimination with partial pivoting, P A = L U, row-major.
 * The paper factors the block-diagonal M = I - gamma J block by block
 * (Sec. 5, batched solver over blocks sharing one structure; Sec. 7, per-point
 * 3x3 block solves); this is the textbook dense algorithm for one block. */
int or_lu_factor(int n, double* a, int* piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(a[k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double v = fabs(a[i * n + k]);
      if (v > best) { best = v; p = i; }   /* strict: ties keep the lowest row */
    }
    piv[k] = p;
    if (best == 0.0) return k + 1;
    if (p != k)
      for (int j = 0; j < n; ++j) { double t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t; }
    for (int i = k + 1; i < n; ++i) {
      double l = a[i * n + k] / a[k * n + k];
      a[i * n + k] = l;
      for (int j = k + 1; j < n; ++j) a[i * n + j] -= l * a[k * n + j];
    }
  }
  return 0;
}

void or_lu_solve(int n, const double* lu, const int* piv, double* b) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k) { double t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
  for (int i = 0; i < n; ++i) {          /* L y = P b, unit lower */
    double s = b[i];
    for (int j = 0; j < i; ++j) s -= lu[i * n + j] * b[j];
    b[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {     /* U x = y */
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= lu[i * n + j] * b[j];
    b[i] = s / lu[i * n + i];
  }
}
