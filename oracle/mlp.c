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

/* BF16 rounding (bfloat16: 8 significant bits, the FP32 exponent range):
 * round to nearest, ties to even, from the definition -- x = m 2^e with
 * 0.5 <= |m| < 1, keep m 2^8 rounded to an integer (nearbyint rounds ties to
 * even in the default rounding mode).  Zero, infinities and NaN pass. */
double or_bf16_round(double x) {
  if (x == 0.0 || !isfinite(x)) return x;
  int e;
  const double m = frexp(x, &e);
  return ldexp(nearbyint(ldexp(m, 8)), e - 8);
}

/* the operands of the network's products, as the BF16 method sees them:
 * exact (q = 0) or rounded to BF16 (q = 1) */
static double opnd(double x, int q) { return q ? or_bf16_round(x) : x; }

static void layer(const double* W, const double* b, int nin, int nout, const double* x, double* y, int relu,
                  int q) {
  for (int o = 0; o < nout; ++o) {
    double s = b[o];
    for (int i = 0; i < nin; ++i) s += opnd(W[o * nin + i], q) * x[i];
    y[o] = (relu && s < 0.0) ? 0.0 : s;
  }
}

/* the forward pass of one row: h1, h2 (as the next layer's operands) and y */
static void forward_row(const double* p, const double* xin, double* x, double* h1, double* h2, double* y, int q) {
  for (int i = 0; i < NI; ++i) x[i] = opnd(xin[i], q);
  layer(p + OFF_W1, p + OFF_B1, NI, NH, x, h1, 1, q);
  for (int i = 0; i < NH; ++i) h1[i] = opnd(h1[i], q);
  layer(p + OFF_W2, p + OFF_B2, NH, NH, h1, h2, 1, q);
  for (int i = 0; i < NH; ++i) h2[i] = opnd(h2[i], q);
  layer(p + OFF_W3, p + OFF_B3, NH, NO, h2, y, 0, q);
}

static void forward(const double* p, int64_t nrows, const double* X, double* Y, int q) {
  double x[NI], h1[NH], h2[NH];
  for (int64_t r = 0; r < nrows; ++r) forward_row(p, X + r * NI, x, h1, h2, Y + r * NO, q);
}

/* Y[r][0..9] for rows r < nrows of X[r][0..11] */
void or_mlp_forward(const double* p, int64_t nrows, const double* X, double* Y) { forward(p, nrows, X, Y, 0); }

/* The same network computed with BF16 operands and exact accumulation (the
 * learned guess's arithmetic: BF16 weights with higher-precision
 * accumulation): every product's operands -- the weights, the inputs and the
 * hidden activations (after bias and ReLU) -- are rounded to BF16; biases and
 * outputs are not. */
void or_mlp_forward_bf16(const double* p, int64_t nrows, const double* X, double* Y) {
  forward(p, nrows, X, Y, 1);
}

static double loss_grad(const double* p, int64_t nrows, const double* X, const double* T, double* grad, int q) {
  memset(grad, 0, sizeof(double) * NPARAM);
  double loss = 0.0;
  const double scale = 1.0 / ((double)nrows * NO);
  double xq[NI], h1[NH], h2[NH], y[NO], dy[NO], dh2[NH], dh1[NH];
  for (int64_t r = 0; r < nrows; ++r) {
    const double* x = xq;
    forward_row(p, X + r * NI, xq, h1, h2, y, q);
    for (int o = 0; o < NO; ++o) {
      const double e = y[o] - T[r * NO + o];
      loss += e * e * scale;
      dy[o] = opnd(2.0 * e * scale, q);
    }
    /* layer 3 */
    for (int o = 0; o < NO; ++o) {
      grad[OFF_B3 + o] += dy[o];
      for (int i = 0; i < NH; ++i) grad[OFF_W3 + o * NH + i] += dy[o] * h2[i];
    }
    for (int i = 0; i < NH; ++i) {
      double s = 0.0;
      for (int o = 0; o < NO; ++o) s += opnd(p[OFF_W3 + o * NH + i], q) * dy[o];
      dh2[i] = opnd(h2[i] > 0.0 ? s : 0.0, q);
    }
    /* layer 2 */
    for (int o = 0; o < NH; ++o) {
      grad[OFF_B2 + o] += dh2[o];
      for (int i = 0; i < NH; ++i) grad[OFF_W2 + o * NH + i] += dh2[o] * h1[i];
    }
    for (int i = 0; i < NH; ++i) {
      double s = 0.0;
      for (int o = 0; o < NH; ++o) s += opnd(p[OFF_W2 + o * NH + i], q) * dh2[o];
      dh1[i] = opnd(h1[i] > 0.0 ? s : 0.0, q);
    }
    /* layer 1 */
    for (int o = 0; o < NH; ++o) {
      grad[OFF_B1 + o] += dh1[o];
      for (int i = 0; i < NI; ++i) grad[OFF_W1 + o * NI + i] += dh1[o] * x[i];
    }
  }
  return loss;
}

/* loss = mean over rows and outputs of (Y - T)^2; grad (NPARAM) = d loss / d p */
double or_mlp_loss_grad(const double* p, int64_t nrows, const double* X, const double* T, double* grad) {
  return loss_grad(p, nrows, X, T, grad, 0);
}

/* The loss and gradient as back-propagation computes them with BF16
 * operands: the forward pass of or_mlp_forward_bf16 (h1, h2 and x as BF16
 * operands), the output gradient dY = 2 (Y - T) / (rows 10) rounded to BF16,
 * the back-propagated dH2 = [h2 > 0] W3^T dY and dH1 = [h1 > 0] W2^T dH2
 * rounded to BF16 after the mask, BF16 weights in those products; the
 * gradients are the exact sums of products of these operands. */
double or_mlp_loss_grad_bf16(const double* p, int64_t nrows, const double* X, const double* T, double* grad) {
  return loss_grad(p, nrows, X, T, grad, 1);
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
