/*
 * mlp.c - oracle of the learned Newton initial guess: a 12 -> 64 -> 64 -> 10
 * multilayer perceptron with ReLU hidden layers, mean-squared-error loss,
 * its gradient by backpropagation, and the Adam update.  Plain FP64 loops.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper has no learned component; this network is the one the build
 * adds to predict the Newton correction.  Parameter layout (5642 values):
 *   W1[64][12], b1[64], W2[64][64], b2[64], W3[10][64], b3[10]
 * with W[out][in], so layer l computes h_out = sum_in W[out][in] h_in + b[out].
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

#define NI 12
#define NH 64
#define NO 10
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + NH * NI)
#define OFF_W2 (OFF_B1 + NH)
#define OFF_B2 (OFF_W2 + NH * NH)
#define OFF_W3 (OFF_B2 + NH)
#define OFF_B3 (OFF_W3 + NO * NH)
#define NPARAM (OFF_B3 + NO)

int or_mlp_nparam(void) { return NPARAM; }

static void layer(const double* W, const double* b, int nin, int nout, const double* x, double* y, int relu) {
  for (int o = 0; o < nout; ++o) {
    double s = b[o];
    for (int i = 0; i < nin; ++i) s += W[o * nin + i] * x[i];
    y[o] = (relu && s < 0.0) ? 0.0 : s;
  }
}

/* Y[r][0..9] for rows r < nrows of X[r][0..11] */
void or_mlp_forward(const double* p, int64_t nrows, const double* X, double* Y) {
  double h1[NH], h2[NH];
  for (int64_t r = 0; r < nrows; ++r) {
    layer(p + OFF_W1, p + OFF_B1, NI, NH, X + r * NI, h1, 1);
    layer(p + OFF_W2, p + OFF_B2, NH, NH, h1, h2, 1);
    layer(p + OFF_W3, p + OFF_B3, NH, NO, h2, Y + r * NO, 0);
  }
}

/* loss = mean over rows and outputs of (Y - T)^2; grad (NPARAM) = d loss / d p */
double or_mlp_loss_grad(const double* p, int64_t nrows, const double* X, const double* T, double* grad) {
  memset(grad, 0, sizeof(double) * NPARAM);
  double loss = 0.0;
  const double scale = 1.0 / ((double)nrows * NO);
  double h1[NH], h2[NH], y[NO], dy[NO], dh2[NH], dh1[NH];
  for (int64_t r = 0; r < nrows; ++r) {
    const double* x = X + r * NI;
    layer(p + OFF_W1, p + OFF_B1, NI, NH, x, h1, 1);
    layer(p + OFF_W2, p + OFF_B2, NH, NH, h1, h2, 1);
    layer(p + OFF_W3, p + OFF_B3, NH, NO, h2, y, 0);
    for (int o = 0; o < NO; ++o) {
      const double e = y[o] - T[r * NO + o];
      loss += e * e * scale;
      dy[o] = 2.0 * e * scale;
    }
    /* layer 3 */
    for (int o = 0; o < NO; ++o) {
      grad[OFF_B3 + o] += dy[o];
      for (int i = 0; i < NH; ++i) grad[OFF_W3 + o * NH + i] += dy[o] * h2[i];
    }
    for (int i = 0; i < NH; ++i) {
      double s = 0.0;
      for (int o = 0; o < NO; ++o) s += p[OFF_W3 + o * NH + i] * dy[o];
      dh2[i] = h2[i] > 0.0 ? s : 0.0;
    }
    /* layer 2 */
    for (int o = 0; o < NH; ++o) {
      grad[OFF_B2 + o] += dh2[o];
      for (int i = 0; i < NH; ++i) grad[OFF_W2 + o * NH + i] += dh2[o] * h1[i];
    }
    for (int i = 0; i < NH; ++i) {
      double s = 0.0;
      for (int o = 0; o < NH; ++o) s += p[OFF_W2 + o * NH + i] * dh2[o];
      dh1[i] = h1[i] > 0.0 ? s : 0.0;
    }
    /* layer 1 */
    for (int o = 0; o < NH; ++o) {
      grad[OFF_B1 + o] += dh1[o];
      for (int i = 0; i < NI; ++i) grad[OFF_W1 + o * NI + i] += dh1[o] * x[i];
    }
  }
  return loss;
}

/* one Adam step (Kingma & Ba 2015) at step number t >= 1 */
void or_adam_step(int64_t n, double* p, const double* g, double* m, double* v, int64_t t, double lr,
                  double b1, double b2, double eps) {
  const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
  }
}
