// grid.cu - the grouped ("full model", Sec. 2) integrator: the Brusselator
// reaction terms of Sec. 7 with diffusion on a periodic nx^3 grid, integrated
// as ONE coupled system (shared step size, global FP64 WRMS norms) by
// variable-order BDF with Newton, the linear systems solved by GMRES built
// on the NVECTOR kernels (Sec. 5: Krylov solvers need only vector
// operations) and left-preconditioned by the 3x3 reaction blocks (the
// block-Jacobi preconditioner of the Sec. 7 global-Newton configuration,
// each block inverted in closed form like the paper's symbolically generated
// Gauss-Jordan inverse).
//
// Control runs on the host, as in the paper (Sec. 2: the integrator's
// decisions are taken on the CPU); every vector operation is a B300 kernel and
// every reduction returns one scalar to the host (Sec. 4.1).  Fused kernels
// cut the passes over the ~400 MB vectors of a 256^3 grid: the Nordsieck
// prediction only materialises z_0 and z_1, the corrector applies the Pascal
// shift and the update in one pass, and one kernel applies the scaled,
// preconditioned Newton operator (stencil, reaction Jacobian, 3x3 inverse).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "grid.cuh"

namespace bdfb {

constexpr int GQMAX = 5;
constexpr int GT = 256;         // threads per block of the grid kernels
constexpr int MAXL_MAX = 16;

struct GZ {
  double* z[GQMAX + 1];
};

static int gblocks(int64_t n) {
  int64_t b = (n + GT - 1) / GT;
  const int64_t cap = (int64_t)sm_count() * 8;
  return (int)std::max<int64_t>(1, std::min(b, cap));
}

__device__ __forceinline__ int64_t wrapi(int64_t i, int64_t n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Stencil kernels run on a 3-D launch: x threads along the contiguous index
// l, blockIdx.y = j, blockIdx.z = i (no integer division per point).
struct Pt {
  int64_t p, o[6];
};
__device__ __forceinline__ bool stencil_point(int nx, Pt& P) {
  const int64_t n = nx;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return false;
  const int64_t j = blockIdx.y, i = blockIdx.z;
  P.p = (i * n + j) * n + l;
  P.o[0] = (wrapi(i - 1, n) * n + j) * n + l;
  P.o[1] = (wrapi(i + 1, n) * n + j) * n + l;
  P.o[2] = (i * n + wrapi(j - 1, n)) * n + l;
  P.o[3] = (i * n + wrapi(j + 1, n)) * n + l;
  P.o[4] = (i * n + j) * n + wrapi(l - 1, n);
  P.o[5] = (i * n + j) * n + wrapi(l + 1, n);
  return true;
}

static dim3 stencil_grid(int nx) { return dim3((unsigned)((nx + 127) / 128), (unsigned)nx, (unsigned)nx); }
constexpr int ST_X = 128;

// f = D lap(y) + reaction(y), species-major u | v | w; reps = 1/eps
__global__ void k_bruss_rhs(int nx, double A, double B, double reps, double D, const double* __restrict__ y,
                            double* __restrict__ f) {
  Pt P;
  if (!stencil_point(nx, P)) return;
  const int64_t n = nx, np = n * n * n, p = P.p;
  const double c = D * (double)(n * n);     // D / dx^2
  double lap[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const double* a = y + s * np;
    const double sum = ((a[P.o[0]] + a[P.o[1]]) + (a[P.o[2]] + a[P.o[3]])) + (a[P.o[4]] + a[P.o[5]]);
    lap[s] = c * (sum - 6.0 * a[p]);
  }
  const double u = y[p], v = y[np + p], w = y[2 * np + p];
  f[p] = lap[0] + A - (w + 1.0) * u + v * u * u;
  f[np + p] = lap[1] + w * u - v * u * u;
  f[2 * np + p] = lap[2] + (B - w) * reps - w * u;
}

// 1-D advection-reaction line (the demo problem of Sec. 7): -c da/dx by
// first-order upwind differences on a periodic line of np points; cdx = c / dx
__device__ __forceinline__ double upwind(const double* a, int64_t q, int64_t np, double cdx) {
  if (cdx >= 0.0) return -cdx * (a[q] - a[q == 0 ? np - 1 : q - 1]);
  return -cdx * (a[q + 1 == np ? 0 : q + 1] - a[q]);
}

// f = -c da/dx + reaction(y), species-major u | v | w; reps = 1/eps
__global__ void k_bruss1_rhs(int64_t np, double A, double B, double reps, double cdx, const double* __restrict__ y,
                             double* __restrict__ f) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < np; q += (int64_t)gridDim.x * blockDim.x) {
    const double u = y[q], v = y[np + q], w = y[2 * np + q];
    f[q] = upwind(y, q, np, cdx) + A - (w + 1.0) * u + v * u * u;
    f[np + q] = upwind(y + np, q, np, cdx) + w * u - v * u * u;
    f[2 * np + q] = upwind(y + 2 * np, q, np, cdx) + (B - w) * reps - w * u;
  }
}

// reaction Jacobian of one point (row-major 3x3); reps = 1/eps
__device__ __forceinline__ void bruss_jr(double reps, double u, double v, double w, double* J) {
  J[0] = -(w + 1.0) + 2.0 * u * v; J[1] = u * u;   J[2] = -u;
  J[3] = w - 2.0 * u * v;          J[4] = -u * u;  J[5] = u;
  J[6] = -w;                       J[7] = 0.0;     J[8] = -reps - u;
}

// the reaction Jacobian in FP32 (precision 1: the preconditioner and the
// Newton operator inside GMRES)
__device__ __forceinline__ void bruss_jr32(float reps, float u, float v, float w, float* J) {
  J[0] = -(w + 1.0f) + 2.0f * u * v; J[1] = u * u;   J[2] = -u;
  J[3] = w - 2.0f * u * v;           J[4] = -u * u;  J[5] = u;
  J[6] = -w;                         J[7] = 0.0f;    J[8] = -reps - u;
}

template <typename T> __device__ __forceinline__ T ld(const double* p) { return *p; }
template <> __device__ __forceinline__ float ld<float>(const double* p) { return to_f32(*p); }

// Pinv = (I - gamma J_R(y))^{-1} per point, by the adjugate formula, in T
// (double: precision 0; float: precision 1, the preconditioner in FP32)
template <typename T>
__global__ void k_bruss_psetup(int64_t np, double reps, double gamma, const double* __restrict__ y,
                               T* __restrict__ Pinv, int* __restrict__ singular) {
  const T gm = (T)gamma;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    T J[9];
    if constexpr (sizeof(T) == 8) bruss_jr(reps, y[p], y[np + p], y[2 * np + p], J);
    else bruss_jr32((float)reps, ld<T>(y + p), ld<T>(y + np + p), ld<T>(y + 2 * np + p), J);
    const T a = (T)1 - gm * J[0], b = -gm * J[1], c = -gm * J[2];
    const T d = -gm * J[3], e = (T)1 - gm * J[4], f = -gm * J[5];
    const T g = -gm * J[6], h = -gm * J[7], i = (T)1 - gm * J[8];
    const T A0 = e * i - f * h, A1 = c * h - b * i, A2 = b * f - c * e;
    const T B0 = f * g - d * i, B1 = a * i - c * g, B2 = c * d - a * f;
    const T C0 = d * h - e * g, C1 = b * g - a * h, C2 = a * e - b * d;
    const T det = a * A0 + b * B0 + c * C0;
    if (!(det != (T)0) || !isfinite(det)) { *singular = 1; continue; }
    const T r = (T)1 / det;
    T* P = Pinv + 9 * p;
    P[0] = A0 * r; P[1] = A1 * r; P[2] = A2 * r;
    P[3] = B0 * r; P[4] = B1 * r; P[5] = B2 * r;
    P[6] = C0 * r; P[7] = C1 * r; P[8] = C2 * r;
  }
}

// w = S P^{-1} (u - gamma (D lap(u) + J_R(y) u)),  u = S^{-1} v, S = diag(ewt);
// S^{-1} = diag(sc) with sc = rtol |y| + atol, so unscaling is a product
template <typename T>
__global__ void k_bruss_apply(int nx, double D, double reps, double gamma, const double* __restrict__ v,
                              const double* __restrict__ ewt, const double* __restrict__ sc,
                              const double* __restrict__ y, const T* __restrict__ Pinv,
                              double* __restrict__ w) {
  Pt Q;
  if (!stencil_point(nx, Q)) return;
  const int64_t n = nx, np = n * n * n, p = Q.p;
  const T c = (T)(D * (double)(n * n));
  const T gm = (T)gamma;
  T u[3], lap[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const double* vs = v + s * np;
    const double* ss = sc + s * np;
    u[s] = ld<T>(vs + p) * ld<T>(ss + p);
    T sum = (T)0;
#pragma unroll
    for (int t = 0; t < 6; ++t) sum += ld<T>(vs + Q.o[t]) * ld<T>(ss + Q.o[t]);
    lap[s] = c * (sum - (T)6 * u[s]);
  }
  T J[9];
  if constexpr (sizeof(T) == 8) bruss_jr(reps, y[p], y[np + p], y[2 * np + p], J);
  else bruss_jr32((float)reps, ld<T>(y + p), ld<T>(y + np + p), ld<T>(y + 2 * np + p), J);
  T a[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) a[s] = u[s] - gm * (lap[s] + J[3 * s] * u[0] + J[3 * s + 1] * u[1] + J[3 * s + 2] * u[2]);
  const T* P = Pinv + 9 * p;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const T o = ld<T>(ewt + s * np + p) * (P[3 * s] * a[0] + P[3 * s + 1] * a[1] + P[3 * s + 2] * a[2]);
    if constexpr (sizeof(T) == 8) w[s * np + p] = o;
    else w[s * np + p] = to_f64(o);
  }
}

// the same operator on the 1-D line, advection in place of diffusion
template <typename T>
__global__ void k_bruss1_apply(int64_t np, double cdx, double reps, double gamma, const double* __restrict__ v,
                               const double* __restrict__ ewt, const double* __restrict__ sc,
                               const double* __restrict__ y, const T* __restrict__ Pinv,
                               double* __restrict__ w) {
  const T cx = (T)cdx, gm = (T)gamma;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pl = p == 0 ? np - 1 : p - 1, pr = p + 1 == np ? 0 : p + 1;
    T u[3], adv[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const double* vs = v + s * np;
      const double* ss = sc + s * np;
      u[s] = ld<T>(vs + p) * ld<T>(ss + p);
      adv[s] = cdx >= 0.0 ? -cx * (u[s] - ld<T>(vs + pl) * ld<T>(ss + pl))
                          : -cx * (ld<T>(vs + pr) * ld<T>(ss + pr) - u[s]);
    }
    T J[9];
    if constexpr (sizeof(T) == 8) bruss_jr(reps, y[p], y[np + p], y[2 * np + p], J);
    else bruss_jr32((float)reps, ld<T>(y + p), ld<T>(y + np + p), ld<T>(y + 2 * np + p), J);
    T a[3];
#pragma unroll
    for (int s = 0; s < 3; ++s)
      a[s] = u[s] - gm * (adv[s] + J[3 * s] * u[0] + J[3 * s + 1] * u[1] + J[3 * s + 2] * u[2]);
    const T* P = Pinv + 9 * p;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const T o = ld<T>(ewt + s * np + p) * (P[3 * s] * a[0] + P[3 * s + 1] * a[1] + P[3 * s + 2] * a[2]);
      if constexpr (sizeof(T) == 8) w[s * np + p] = o;
      else w[s * np + p] = to_f64(o);
    }
  }
}

// v = S P^{-1} b
template <typename T>
__global__ void k_prec_scale(int64_t np, const double* __restrict__ b, const T* __restrict__ Pinv,
                             const double* __restrict__ ewt, double* __restrict__ v) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    const T b0 = ld<T>(b + p), b1 = ld<T>(b + np + p), b2 = ld<T>(b + 2 * np + p);
    const T* P = Pinv + 9 * p;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const T o = ld<T>(ewt + s * np + p) * (P[3 * s] * b0 + P[3 * s + 1] * b1 + P[3 * s + 2] * b2);
      if constexpr (sizeof(T) == 8) v[s * np + p] = o;
      else v[s * np + p] = to_f64(o);
    }
  }
}


// ewt = 1 / sc and sc = rtol |y| + atol (sc undoes the scaling by a product)
__global__ void k_ewt(int64_t N, double rtol, double atol, const double* __restrict__ y, double* __restrict__ e,
                      double* __restrict__ sc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double s = rtol * fabs(y[i]) + atol;
    sc[i] = s;
    e[i] = recip_nr(s);
  }
}

// y(tout) = sum_{j <= q} z_j s^j, s = (tout - t_n) / h (Horner)
__global__ void k_interp(int64_t N, int q, GZ Z, double s, double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double v = Z.z[q][i];
    for (int j = q - 1; j >= 0; --j) v = v * s + Z.z[j][i];
    out[i] = v;
  }
}

// acor += delta; y = zp0 + acor (one pass for the Newton update)
__global__ void k_newton_update(int64_t N, const double* __restrict__ delta, double* __restrict__ acor,
                                const double* __restrict__ zp0, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = acor[i] + delta[i];
    acor[i] = a;
    y[i] = zp0[i] + a;
  }
}

__global__ void k_mul(int64_t N, const double* __restrict__ x, const double* __restrict__ d, double* __restrict__ o) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = x[i] * d[i];
}

// per-block maxima of |f_i| / (0.1 |y_i| + atol) (initial-step bound)
__global__ void k_ratio_max(int64_t N, double atol, const double* __restrict__ f, const double* __restrict__ y,
                            double* __restrict__ part) {
  double m = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(f[i]) / (0.1 * fabs(y[i]) + atol));
  __shared__ double sh[GT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(FULL_MASK, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < GT / 32; ++w) m = fmax(m, sh[w]);
    part[blockIdx.x] = fmax(m, sh[0]);
  }
}

// predicted z_0 and z_1 (Pascal sums of the history), z left untouched:
// with the suffix sums s_j = z_j + s_{j+1} (j = q..1), z_0 + s_1 is the
// predicted z_0 and s_1 + ... + s_q = sum_k k z_k the predicted z_1 (2q
// additions per element, no multiplications)
template <int Q>
__global__ void k_predict01(int64_t N, GZ Z, double* __restrict__ zp0, double* __restrict__ zp1) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double zz[Q + 1];
#pragma unroll
    for (int k = 0; k <= Q; ++k) zz[k] = Z.z[k][i];
    double s = zz[Q], s1 = zz[Q];
#pragma unroll
    for (int k = Q - 1; k >= 1; --k) {
      s += zz[k];
      s1 += s;
    }
    zp0[i] = zz[0] + s;
    zp1[i] = s1;
  }
}

struct GL {
  double l[GQMAX + 1];
};

// accept: z_j <- sum_{k>=j} C(k,j) z_k + l_j acor, all j <= Q in one pass
template <int Q>
__global__ void k_accept(int64_t N, GZ Z, GL L, const double* __restrict__ acor) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double zz[Q + 1];
#pragma unroll
    for (int k = 0; k <= Q; ++k) zz[k] = Z.z[k][i];
    // Pascal shift in place: for k = 1..Q, for j = Q..k: zz[j-1] += zz[j]
#pragma unroll
    for (int k = 1; k <= Q; ++k)
#pragma unroll
      for (int j = Q; j >= k; --j) zz[j - 1] += zz[j];
    const double a = acor[i];
#pragma unroll
    for (int j = 0; j <= Q; ++j) Z.z[j][i] = fma(L.l[j], a, zz[j]);
  }
}

__global__ void k_rescale(int64_t N, int q, GZ Z, double eta) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double f = 1.0;
    for (int j = 1; j <= q; ++j) {
      f *= eta;
      Z.z[j][i] *= f;
    }
  }
}

struct GridBDF {
  int nx = 0;
  int dim = 3;                // 3: nx^3 diffusion grid; 1: nx-point advection line
  int64_t np = 0, N = 0;
  double A = 1, B = 3, eps = 5e-6, D = 1e-2;
  double cdx = 0.0;           // dim 1: c / dx
  bool external = false;      // rhs and Newton solve supplied from outside
  GridExternal ext = {};
  double rtol = 1e-6, atol = 1e-10;
  int maxl = 5;
  int prec = 0;               // 1: preconditioner and GMRES operator in FP32
  int interp = 0;             // 1: step past tout, output the history polynomial at tout
  int64_t mxstep = 100000;
  int qmax = GQMAX;
  cudaStream_t s = nullptr;
  // device vectors
  double* z[GQMAX + 2] = {};
  double *ewt = nullptr, *acor = nullptr, *acorp = nullptr, *y = nullptr, *f = nullptr, *b = nullptr;
  double* sc = nullptr;       // rtol |y| + atol = 1 / ewt
  double reps = 0.0;          // 1 / eps
  double *zp0 = nullptr, *zp1 = nullptr, *tmp = nullptr, *w = nullptr, *Pinv = nullptr;
  double* V[MAXL_MAX + 1] = {};
  double* work = nullptr;     // reduction workspace
  double* dres = nullptr;     // device results
  double* hres = nullptr;     // pinned host results
  int* dsing = nullptr;
  double* part = nullptr;     // per-block maxima
  // integrator state
  double t = 0, h = 0, gamma = 0, gammap = 0, crate = 1;
  int q = 1, qwait = 2;
  bool started = false, grown = false, setup_done = false, force_setup = false;
  int64_t nst = 0, nstlp = 0;
  int64_t nfe = 0, nsetups = 0, nni = 0, ncfn = 0, netf = 0, nli = 0, nlfail = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float last_ms = 0;
  double l[GQMAX + 2][GQMAX + 2] = {}, E[GQMAX + 2][3] = {}, qfact[GQMAX + 3] = {};
  // option "profile": events around every vector operation and kernel of the
  // step loop, with its algorithmic bytes, summed per kind (grid_profile)
  bool prof = false;
  std::vector<cudaEvent_t> pev;
  std::vector<int> pkind;
  std::vector<double> pbytes;
  size_t pused = 0;
  int64_t pcalls[GOP_N] = {};
  double pms[GOP_N] = {}, pgb[GOP_N] = {};
};

// one timed operation: events recorded on the step loop's stream before and
// after (no synchronisation; the times are read when the call ends).  Each
// scope reserves its own pair of events, and each wraps one launch only.
struct GTimed {
  GridBDF* g;
  size_t idx = 0;
  bool on = false;
  GTimed(GridBDF* g_, int kind, double bytes) : g(g_) {
    if (!g->prof) return;
    while (g->pused + 2 > g->pev.size()) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      g->pev.push_back(e);
    }
    idx = g->pused;
    g->pused += 2;
    g->pkind.push_back(kind);
    g->pbytes.push_back(bytes);
    on = cudaEventRecord(g->pev[idx], g->s) == cudaSuccess;
  }
  ~GTimed() {
    if (on) cudaEventRecord(g->pev[idx + 1], g->s);
  }
};

// fold the recorded events of a finished call into the per-kind sums
static void prof_flush(GridBDF* g) {
  for (size_t i = 0; i < g->pkind.size() && 2 * i + 1 < g->pused; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, g->pev[2 * i], g->pev[2 * i + 1]) != cudaSuccess) continue;
    g->pcalls[g->pkind[i]]++;
    g->pms[g->pkind[i]] += ms;
    g->pgb[g->pkind[i]] += g->pbytes[i] * 1e-9;
  }
  g->pkind.clear();
  g->pbytes.clear();
  g->pused = 0;
}

static double ell1(const GridBDF* g, int q) { return g->l[q][1]; }

static void make_tables(GridBDF* g) {
  for (int q = 1; q <= GQMAX; ++q) {
    double l[GQMAX + 2] = {0};
    l[0] = 1.0;
    for (int i = 1; i <= q; ++i)
      for (int j = i; j >= 1; --j) l[j] += l[j - 1] / (double)i;
    for (int j = 0; j <= q; ++j) g->l[q][j] = l[j];
  }
  g->qfact[0] = 1.0;
  for (int k = 1; k <= GQMAX + 1; ++k) g->qfact[k] = g->qfact[k - 1] * k;
  for (int q = 1; q <= GQMAX; ++q) {
    g->E[q][0] = 1.0 / ((q + 1) * g->l[q][1]);
    g->E[q][1] = q > 1 ? g->qfact[q - 1] / g->l[q - 1][1] : 0.0;
    double l1 = 0.0;
    for (int i = 1; i <= q + 1; ++i) l1 += 1.0 / i;
    g->E[q][2] = q < GQMAX ? 1.0 / ((q + 2) * l1) : 0.0;
  }
}

#define GCHK(call)                         \
  do {                                     \
    int r_ = (call);                       \
    if (r_) return r_;                     \
  } while (0)

// ---- reductions returning to the host (Sec. 4.1: a reduction synchronises)
static int g_wrms(GridBDF* g, const double* x, double* out) {
  {
    GTimed t(g, GOP_WRMS, 16.0 * g->N);
    GCHK(bdfb_nv_wrms_norm(g->N, x, g->ewt, g->dres, g->work, g->s));
  }
  BDFB_CUDA(cudaMemcpyAsync(g->hres, g->dres, sizeof(double), cudaMemcpyDeviceToHost, g->s));
  BDFB_CUDA(cudaStreamSynchronize(g->s));
  *out = g->hres[0];
  return 0;
}

static int g_dots(GridBDF* g, const double* x, const double* const* ys, int nv, double* out) {
  {
    GTimed t(g, GOP_DOTS, 8.0 * (nv + 1) * g->N);
    GCHK(bdfb_nv_dot_prod_multi(g->N, nv, x, ys, g->dres, g->work, g->s));
  }
  BDFB_CUDA(cudaMemcpyAsync(g->hres, g->dres, nv * sizeof(double), cudaMemcpyDeviceToHost, g->s));
  BDFB_CUDA(cudaStreamSynchronize(g->s));
  std::memcpy(out, g->hres, nv * sizeof(double));
  return 0;
}

static int g_rhs(GridBDF* g, const double* y, double* f) {
  if (g->external) {
    const int r = g->ext.rhs(g->ext.user, y, f, g->s);
    if (r) return r;
  } else {
    GTimed t(g, GOP_RHS, 16.0 * g->N);
    if (g->dim == 1)
      k_bruss1_rhs<<<gblocks(g->np), GT, 0, g->s>>>(g->np, g->A, g->B, g->reps, g->cdx, y, f);
    else
      k_bruss_rhs<<<stencil_grid(g->nx), ST_X, 0, g->s>>>(g->nx, g->A, g->B, g->reps, g->D, y, f);
  }
  BDFB_CUDA(cudaGetLastError());
  g->nfe++;
  return 0;
}

static int g_ewt(GridBDF* g) {
  {
    GTimed t(g, GOP_EWT, 24.0 * g->N);
    k_ewt<<<gblocks(g->N), GT, 0, g->s>>>(g->N, g->rtol, g->atol, g->z[0], g->ewt, g->sc);
  }
  BDFB_CUDA(cudaGetLastError());
  return 0;
}

static GZ zcols(GridBDF* g) {
  GZ Z;
  for (int j = 0; j <= GQMAX; ++j) Z.z[j] = g->z[j];
  return Z;
}

static int g_rescale(GridBDF* g, double eta) {
  {
    GTimed t(g, GOP_RESCALE, 16.0 * g->q * g->N);
    k_rescale<<<gblocks(g->N), GT, 0, g->s>>>(g->N, g->q, zcols(g), eta);
  }
  BDFB_CUDA(cudaGetLastError());
  g->h *= eta;
  return 0;
}

// GMRES on (I - gamma J(ycur)) x = b, left-preconditioned by the 3x3 blocks,
// scaled by ewt, classical Gram-Schmidt, no restart; x overwrites b.
static int g_gmres(GridBDF* g, const double* ycur, double tol) {
  const int64_t N = g->N;
  const int maxl = g->maxl;
  const double sqrtN = std::sqrt((double)N);
  double H[(MAXL_MAX + 1) * MAXL_MAX] = {0};
  double gv[MAXL_MAX + 1] = {0}, cs[MAXL_MAX] = {0}, sn[MAXL_MAX] = {0}, yv[MAXL_MAX] = {0};
  {
    GTimed t(g, GOP_PSCALE, (g->prec ? 36.0 : 48.0) * N);   // b, ewt, v; 3x3 blocks (FP32 or FP64)
    if (g->prec) k_prec_scale<float><<<gblocks(g->np), GT, 0, g->s>>>(g->np, g->b, (const float*)g->Pinv, g->ewt, g->V[0]);
    else k_prec_scale<double><<<gblocks(g->np), GT, 0, g->s>>>(g->np, g->b, g->Pinv, g->ewt, g->V[0]);
  }
  BDFB_CUDA(cudaGetLastError());
  // The basis is stored unnormalised: basis vector i is sig[i] V[i], the
  // scales kept on the host and folded into the coefficients of the next
  // linear combination, so no pass over the vectors only rescales one.
  double sig[MAXL_MAX + 1] = {0};
  double beta2;
  const double* v0 = g->V[0];
  GCHK(g_dots(g, g->V[0], &v0, 1, &beta2));
  const double beta = std::sqrt(beta2);
  if (beta / sqrtN <= tol) {
    BDFB_CUDA(cudaMemsetAsync(g->b, 0, N * sizeof(double), g->s));
    return 0;
  }
  sig[0] = 1.0 / beta;
  gv[0] = beta;
  int k = 0;
  bool conv = false;
  for (int j = 0; j < maxl; ++j) {
    const float* P32 = (const float*)g->Pinv;
    {
    // v, ewt, sc, y and w, plus the 3x3 blocks (FP32 or FP64)
    GTimed t(g, GOP_APPLY, (g->prec ? 52.0 : 64.0) * N);
    if (g->dim == 1 && g->prec)
      k_bruss1_apply<float><<<gblocks(g->np), GT, 0, g->s>>>(g->np, g->cdx, g->reps, g->gamma, g->V[j], g->ewt,
                                                             g->sc, ycur, P32, g->w);
    else if (g->dim == 1)
      k_bruss1_apply<double><<<gblocks(g->np), GT, 0, g->s>>>(g->np, g->cdx, g->reps, g->gamma, g->V[j], g->ewt,
                                                              g->sc, ycur, g->Pinv, g->w);
    else if (g->prec)
      k_bruss_apply<float><<<stencil_grid(g->nx), ST_X, 0, g->s>>>(g->nx, g->D, g->reps, g->gamma, g->V[j],
                                                                   g->ewt, g->sc, ycur, P32, g->w);
    else
      k_bruss_apply<double><<<stencil_grid(g->nx), ST_X, 0, g->s>>>(g->nx, g->D, g->reps, g->gamma, g->V[j],
                                                                    g->ewt, g->sc, ycur, g->Pinv, g->w);
    }
    BDFB_CUDA(cudaGetLastError());
    // w = sig[j] A V[j]: h_ij = (w, basis_i) = sig[j] sig[i] (A V[j], V[i]);
    // classical Gram-Schmidt into V[j + 1]: sig[j] (A V[j] - sum c_i V[i])
    // with c_i = h_ij sig[i] / sig[j]
    double hcol[MAXL_MAX + 1];
    GCHK(g_dots(g, g->w, g->V, j + 1, hcol));
    for (int i = 0; i <= j; ++i) hcol[i] *= sig[j] * sig[i];
    {
      const double* xs[MAXL_MAX + 2];
      double c[MAXL_MAX + 2];
      xs[0] = g->w;
      c[0] = 1.0;
      for (int i = 0; i <= j; ++i) { xs[i + 1] = g->V[i]; c[i + 1] = -hcol[i] * sig[i] / sig[j]; }
      GTimed t(g, GOP_LINCOMB, 8.0 * (j + 3) * N);
      GCHK(bdfb_nv_linear_combination(N, j + 2, c, xs, g->V[j + 1], g->s));
    }
    for (int i = 0; i <= j; ++i) H[i * maxl + j] = hcol[i];
    double hn2;
    const double* wp = g->V[j + 1];
    GCHK(g_dots(g, g->V[j + 1], &wp, 1, &hn2));
    const double hn = sig[j] * std::sqrt(hn2);
    H[(j + 1) * maxl + j] = hn;
    sig[j + 1] = hn > 0.0 ? sig[j] / hn : 0.0;
    for (int i = 0; i < j; ++i) {
      const double h0 = H[i * maxl + j], h1 = H[(i + 1) * maxl + j];
      H[i * maxl + j] = cs[i] * h0 + sn[i] * h1;
      H[(i + 1) * maxl + j] = -sn[i] * h0 + cs[i] * h1;
    }
    const double a0 = H[j * maxl + j], a1 = H[(j + 1) * maxl + j];
    const double rr = std::sqrt(a0 * a0 + a1 * a1);
    cs[j] = rr > 0.0 ? a0 / rr : 1.0;
    sn[j] = rr > 0.0 ? a1 / rr : 0.0;
    H[j * maxl + j] = rr;
    H[(j + 1) * maxl + j] = 0.0;
    gv[j + 1] = -sn[j] * gv[j];
    gv[j] = cs[j] * gv[j];
    k = j + 1;
    g->nli++;
    if (std::fabs(gv[j + 1]) / sqrtN <= tol || hn == 0.0) { conv = true; break; }
  }
  if (!conv) g->nlfail++;        // inexact Newton: keep the iterate
  for (int i = k - 1; i >= 0; --i) {
    double sacc = gv[i];
    for (int jj = i + 1; jj < k; ++jj) sacc -= H[i * maxl + jj] * yv[jj];
    yv[i] = sacc / H[i * maxl + i];
  }
  {
    const double* xs[MAXL_MAX];
    double c[MAXL_MAX];
    for (int i = 0; i < k; ++i) { xs[i] = g->V[i]; c[i] = yv[i] * sig[i]; }
    GTimed t(g, GOP_LINCOMB, 8.0 * (k + 1) * N);
    GCHK(bdfb_nv_linear_combination(N, k, c, xs, g->tmp, g->s));
  }
  {
    GTimed t(g, GOP_MUL, 24.0 * N);
    k_mul<<<gblocks(N), GT, 0, g->s>>>(N, g->tmp, g->sc, g->b);     // x = S^{-1} (V y)
  }
  BDFB_CUDA(cudaGetLastError());
  return 0;
}

static int g_psetup(GridBDF* g, const double* y) {
  BDFB_CUDA(cudaMemsetAsync(g->dsing, 0, sizeof(int), g->s));
  {
    GTimed t(g, GOP_PSETUP, (g->prec ? 20.0 : 32.0) * g->N);   // y; the 3x3 blocks (FP32 or FP64)
    if (g->prec)
      k_bruss_psetup<float><<<gblocks(g->np), GT, 0, g->s>>>(g->np, g->reps, g->gamma, y, (float*)g->Pinv, g->dsing);
    else
      k_bruss_psetup<double><<<gblocks(g->np), GT, 0, g->s>>>(g->np, g->reps, g->gamma, y, g->Pinv, g->dsing);
  }
  BDFB_CUDA(cudaGetLastError());
  int sing = 0;
  BDFB_CUDA(cudaMemcpyAsync(&sing, g->dsing, sizeof(int), cudaMemcpyDeviceToHost, g->s));
  BDFB_CUDA(cudaStreamSynchronize(g->s));
  return sing ? 1 : 0;
}

// Newton iteration; 0 converged (*acnrm = |acor|), 1 recoverable failure, <0 error
// grouped task-local Newton: one global setup decision, the solves per part
// outside; any part that fails fails the whole step (retried once with fresh
// Jacobians when they were stale, then h / 4 by the caller)
static int g_newton_external(GridBDF* g, double Eq, double* acnrm) {
  bool tried_fresh = false;
  for (;;) {
    bool setup = false;
    if (!g->setup_done || g->force_setup || std::fabs(g->gamma / g->gammap - 1.0) > 0.3 ||
        g->nst >= g->nstlp + 20) {
      setup = true;
      g->nsetups++;
      g->gammap = g->gamma;
      g->nstlp = g->nst;
      g->force_setup = false;
      g->setup_done = true;
    }
    int failed = 0;
    int64_t iters = 0, sweeps = 0;
    const int r = g->ext.solve(g->ext.user, g->zp0, g->zp1, g->ewt, g->gamma, g->gammap, 1.0 / ell1(g, g->q), Eq,
                               setup ? 1 : 0, g->acor, &failed, &iters, &sweeps, g->s);
    if (r) return r;
    g->nni += iters;
    g->nfe += sweeps;
    if (!failed) {
      GCHK(g_wrms(g, g->acor, acnrm));
      GTimed t(g, GOP_LINSUM, 24.0 * g->N);
      GCHK(bdfb_nv_linear_sum(g->N, 1.0, g->zp0, 1.0, g->acor, g->y, g->s));
      return 0;
    }
    if (!setup && !tried_fresh) { g->force_setup = true; tried_fresh = true; continue; }
    return 1;
  }
}

static int g_newton(GridBDF* g, double Eq, double* acnrm) {
  if (g->external) return g_newton_external(g, Eq, acnrm);
  const int64_t N = g->N;
  const double l1 = ell1(g, g->q);
  bool tried_fresh = false;
  for (;;) {
    bool jcur = false;
    if (!g->setup_done || g->force_setup || std::fabs(g->gamma / g->gammap - 1.0) > 0.3 ||
        g->nst >= g->nstlp + 20) {
      int r = g_psetup(g, g->zp0);
      if (r < 0) return r;
      g->nsetups++;
      g->gammap = g->gamma;
      g->crate = 1.0;
      g->nstlp = g->nst;
      g->force_setup = false;
      g->setup_done = true;
      jcur = true;
      if (r > 0) return 1;
    }
    BDFB_CUDA(cudaMemsetAsync(g->acor, 0, N * sizeof(double), g->s));
    BDFB_CUDA(cudaMemcpyAsync(g->y, g->zp0, N * sizeof(double), cudaMemcpyDeviceToDevice, g->s));
    double delp = 0.0;
    bool conv = false;
    for (int it = 1; it <= 3; ++it) {
      GCHK(g_rhs(g, g->y, g->f));
      const double* xs[3] = {g->f, g->zp1, g->acor};
      const double c[3] = {g->gamma, -1.0 / l1, -1.0};
      {
        GTimed t(g, GOP_LINCOMB, 32.0 * N);
        GCHK(bdfb_nv_linear_combination(N, 3, c, xs, g->b, g->s));
      }
      GCHK(g_gmres(g, g->y, 0.05 * 0.1 / Eq));
      double del;
      GCHK(g_wrms(g, g->b, &del));
      {
        GTimed t(g, GOP_NEWTON, 40.0 * N);
        k_newton_update<<<gblocks(N), GT, 0, g->s>>>(N, g->b, g->acor, g->zp0, g->y);
      }
      BDFB_CUDA(cudaGetLastError());
      g->nni++;
      if (!std::isfinite(del)) break;
      if (it > 1) g->crate = std::max(0.3 * g->crate, del / delp);
      const double dcon = del * std::min(1.0, g->crate) * Eq / 0.1;
      if (dcon <= 1.0) {
        if (it == 1) *acnrm = del;
        else GCHK(g_wrms(g, g->acor, acnrm));
        conv = true;
        break;
      }
      if (it >= 2 && del > 2.0 * delp) break;
      delp = del;
    }
    if (conv) return 0;
    if (!jcur && !tried_fresh) { g->force_setup = true; tried_fresh = true; continue; }
    return 1;
  }
}

static int g_predict(GridBDF* g) {
  {
    GTimed t(g, GOP_PREDICT, 8.0 * (g->q + 3) * g->N);
    switch (g->q) {
      case 1: k_predict01<1><<<gblocks(g->N), GT, 0, g->s>>>(g->N, zcols(g), g->zp0, g->zp1); break;
      case 2: k_predict01<2><<<gblocks(g->N), GT, 0, g->s>>>(g->N, zcols(g), g->zp0, g->zp1); break;
      case 3: k_predict01<3><<<gblocks(g->N), GT, 0, g->s>>>(g->N, zcols(g), g->zp0, g->zp1); break;
      case 4: k_predict01<4><<<gblocks(g->N), GT, 0, g->s>>>(g->N, zcols(g), g->zp0, g->zp1); break;
      default: k_predict01<5><<<gblocks(g->N), GT, 0, g->s>>>(g->N, zcols(g), g->zp0, g->zp1); break;
    }
  }
  BDFB_CUDA(cudaGetLastError());
  return 0;
}

static int g_select(GridBDF* g, double dsm) {
  if (--g->qwait > 0) return 0;
  const int q = g->q;
  const double eq = 1.0 / (std::pow(6.0 * dsm, 1.0 / (q + 1)) + 1e-6);
  double eqm1 = 0.0, eqp1 = 0.0;
  if (q > 1) {
    double nz;
    GCHK(g_wrms(g, g->z[q], &nz));
    eqm1 = 1.0 / (std::pow(6.0 * g->E[q][1] * nz, 1.0 / q) + 1e-6);
  }
  if (q < g->qmax) {
    {
      GTimed t(g, GOP_LINSUM, 24.0 * g->N);
      GCHK(bdfb_nv_linear_sum(g->N, 1.0, g->acor, -1.0, g->acorp, g->tmp, g->s));
    }
    double nd;
    GCHK(g_wrms(g, g->tmp, &nd));
    eqp1 = 1.0 / (std::pow(10.0 * g->E[q][2] * nd, 1.0 / (q + 2)) + 1e-6);
  }
  double etam = eq;
  int qn = q;
  if (eqm1 > etam) { etam = eqm1; qn = q - 1; }
  if (eqp1 > etam) { etam = eqp1; qn = q + 1; }
  if (etam < 1.5) { g->qwait = 1; return 0; }
  const double cap = g->grown ? 10.0 : 1.0e4;
  if (etam > cap) etam = cap;
  g->grown = true;
  if (qn == q + 1) {
    GCHK(bdfb_nv_linear_sum(g->N, 1.0 / g->qfact[q + 1], g->acor, 0.0, g->acor, g->z[q + 1], g->s));
    g->q = q + 1;
  } else if (qn == q - 1) {
    BDFB_CUDA(cudaMemsetAsync(g->z[q], 0, g->N * sizeof(double), g->s));
    g->q = q - 1;
  }
  GCHK(g_rescale(g, etam));
  g->qwait = g->q + 1;
  return 0;
}

// one accepted step (mirrors the per-cell step: clamp to tout, predict,
// Newton with its failure handling, error test with its failure handling,
// accept, step / order selection)
static int g_step(GridBDF* g, double tout, bool* reached) {
  const int64_t N = g->N;
  int ncf = 0, nef = 0;
  for (;;) {
    bool last = false;
    if (!g->interp && (g->t + g->h - tout) * g->h >= 0.0) {
      last = true;
      if (g->t + g->h != tout) { GCHK(g_rescale(g, (tout - g->t) / g->h)); g->qwait = g->q + 1; }
    }
    if (g->t + g->h == g->t) return BDFB_ERR_FAILURE;
    const double Eq = g->E[g->q][0];
    GCHK(g_predict(g));
    const double tnew = last ? tout : g->t + g->h;
    g->gamma = g->h / ell1(g, g->q);
    double acnrm = 0.0;
    int r = g_newton(g, Eq, &acnrm);
    if (r < 0) return r;
    if (r == 1) {
      ncf++;
      g->ncfn++;
      if (ncf >= 10) return BDFB_CONV_FAILURE;
      GCHK(g_rescale(g, 0.25));
      g->qwait = g->q + 1;
      g->force_setup = true;
      continue;
    }
    const double dsm = acnrm * Eq;
    if (!(dsm <= 1.0)) {
      nef++;
      g->netf++;
      if (nef >= 7) return BDFB_ERR_FAILURE;
      if (nef < 3) {
        double eta = 1.0 / (std::pow(6.0 * dsm, 1.0 / (g->q + 1)) + 1e-6);
        if (!(eta >= 0.1)) eta = 0.1;
        if (nef >= 2 && eta > 0.2) eta = 0.2;
        GCHK(g_rescale(g, eta));
        g->qwait = g->q + 1;
      } else {
        for (int j = 2; j <= GQMAX; ++j) BDFB_CUDA(cudaMemsetAsync(g->z[j], 0, N * sizeof(double), g->s));
        g->q = 1;
        g->h *= 0.1;
        GCHK(g_rhs(g, g->z[0], g->f));
        GCHK(bdfb_nv_linear_sum(N, g->h, g->f, 0.0, g->f, g->z[1], g->s));
        g->qwait = 2;
      }
      continue;
    }
    GL L;
    for (int j = 0; j <= GQMAX; ++j) L.l[j] = j <= g->q ? g->l[g->q][j] : 0.0;
    {
      GTimed t(g, GOP_ACCEPT, 8.0 * (2 * g->q + 3) * N);   // z_0..z_q read and written, acor read
      switch (g->q) {
        case 1: k_accept<1><<<gblocks(N), GT, 0, g->s>>>(N, zcols(g), L, g->acor); break;
        case 2: k_accept<2><<<gblocks(N), GT, 0, g->s>>>(N, zcols(g), L, g->acor); break;
        case 3: k_accept<3><<<gblocks(N), GT, 0, g->s>>>(N, zcols(g), L, g->acor); break;
        case 4: k_accept<4><<<gblocks(N), GT, 0, g->s>>>(N, zcols(g), L, g->acor); break;
        default: k_accept<5><<<gblocks(N), GT, 0, g->s>>>(N, zcols(g), L, g->acor); break;
      }
    }
    BDFB_CUDA(cudaGetLastError());
    g->t = tnew;
    g->nst++;
    GCHK(g_select(g, dsm));
    std::swap(g->acor, g->acorp);      // keep Delta_n as the previous correction
    *reached = last;
    return 0;
  }
}

static int g_initial_step(GridBDF* g, double tout) {
  const int64_t N = g->N;
  GCHK(g_ewt(g));
  GCHK(g_rhs(g, g->z[0], g->f));
  BDFB_CUDA(cudaMemcpyAsync(g->acorp, g->f, N * sizeof(double), cudaMemcpyDeviceToDevice, g->s));  // f0
  const double tdist = std::fabs(tout - g->t);
  const double hlb = 100.0 * 2.220446049250313e-16 * std::max(std::fabs(g->t), std::fabs(tout));
  double hub = 0.1 * tdist;
  const int nb = gblocks(N);
  k_ratio_max<<<nb, GT, 0, g->s>>>(N, g->atol, g->acorp, g->z[0], g->part);
  BDFB_CUDA(cudaGetLastError());
  std::vector<double> part(nb);
  BDFB_CUDA(cudaMemcpyAsync(part.data(), g->part, nb * sizeof(double), cudaMemcpyDeviceToHost, g->s));
  BDFB_CUDA(cudaStreamSynchronize(g->s));
  double inv = 0.0;
  for (double v : part) inv = std::max(inv, v);
  if (inv * hub > 1.0) hub = 1.0 / inv;
  if (hub < hlb) hub = hlb;
  double hg = std::sqrt(hlb * hub), hnew = hg;
  for (int it = 0; it < 4; ++it) {
    GCHK(bdfb_nv_linear_sum(N, 1.0, g->z[0], hg, g->acorp, g->y, g->s));
    GCHK(g_rhs(g, g->y, g->f));
    GCHK(bdfb_nv_linear_sum(N, 1.0 / hg, g->f, -1.0 / hg, g->acorp, g->b, g->s));
    double ydd;
    GCHK(g_wrms(g, g->b, &ydd));
    hnew = (ydd * hub * hub > 2.0) ? std::sqrt(2.0 / ydd) : std::sqrt(hg * hub);
    const double rat = hnew / hg;
    if (it > 0 && rat > 0.5 && rat < 2.0) break;
    hg = hnew;
  }
  double h0 = 0.5 * hnew;
  if (h0 < hlb) h0 = hlb;
  if (h0 > hub) h0 = hub;
  g->h = tout >= g->t ? h0 : -h0;
  GCHK(bdfb_nv_linear_sum(N, g->h, g->acorp, 0.0, g->acorp, g->z[1], g->s));
  BDFB_CUDA(cudaMemsetAsync(g->acorp, 0, N * sizeof(double), g->s));
  g->q = 1;
  g->qwait = 2;
  g->started = true;
  return 0;
}

int grid_create(int nx, double A, double B, double eps, double D, GridBDF** out) {
  return grid_create_line_or_cube(3, nx, A, B, eps, D, 0.0, 1.0, out);
}

int grid_create_line_or_cube(int dim, int64_t nx, double A, double B, double eps, double D, double c,
                             double len, GridBDF** out) {
  if ((dim != 1 && dim != 3) || nx < 2 || (dim == 3 && nx > 2048) || (dim == 1 && nx > (int64_t)1 << 30) ||
      !(eps > 0.0) || !std::isfinite(c) || !(len > 0.0))
    return BDFB_ILL_INPUT;
  GridBDF* g = new (std::nothrow) GridBDF();
  if (!g) return BDFB_MEM_FAIL;
  g->nx = (int)nx;
  g->dim = dim;
  g->np = dim == 1 ? nx : nx * nx * nx;
  g->N = 3 * g->np;
  g->A = A; g->B = B; g->eps = eps; g->D = D;
  g->cdx = dim == 1 ? c / (len / (double)nx) : 0.0;
  g->reps = 1.0 / eps;
  make_tables(g);
  const size_t vb = g->N * sizeof(double);
  bool ok = true;
  auto alloc = [&](double** p, size_t bytes) {
    if (ok && cudaMalloc(p, bytes) != cudaSuccess) { *p = nullptr; ok = false; }
  };
  for (int j = 0; j <= GQMAX + 1; ++j) alloc(&g->z[j], vb);
  alloc(&g->ewt, vb); alloc(&g->sc, vb); alloc(&g->acor, vb); alloc(&g->acorp, vb); alloc(&g->y, vb); alloc(&g->f, vb);
  alloc(&g->b, vb); alloc(&g->zp0, vb); alloc(&g->zp1, vb); alloc(&g->tmp, vb); alloc(&g->w, vb);
  alloc(&g->Pinv, 9 * g->np * sizeof(double));
  for (int i = 0; i <= MAXL_MAX; ++i) g->V[i] = nullptr;
  alloc(&g->work, bdfb_nv_work_doubles(g->N, MAXL_MAX) * sizeof(double));
  alloc(&g->dres, (MAXL_MAX + 2) * sizeof(double));
  alloc(&g->part, (size_t)sm_count() * 8 * sizeof(double));
  if (ok && cudaMalloc(&g->dsing, sizeof(int)) != cudaSuccess) ok = false;
  if (ok && cudaMallocHost(&g->hres, (MAXL_MAX + 2) * sizeof(double)) != cudaSuccess) ok = false;
  if (ok && cudaMemset(g->work, 0, bdfb_nv_work_doubles(g->N, MAXL_MAX) * sizeof(double)) != cudaSuccess) ok = false;
  if (ok && (cudaEventCreate(&g->e0) != cudaSuccess || cudaEventCreate(&g->e1) != cudaSuccess)) ok = false;
  if (ok) ok = grid_set_option(g, "maxl", 5) == 0;
  if (!ok) {
    grid_destroy(g);
    return BDFB_MEM_FAIL;
  }
  *out = g;
  return 0;
}

int grid_create_external(int64_t N, GridExternal ext, GridBDF** out) {
  if (N < 1 || !ext.rhs || !ext.solve) return BDFB_ILL_INPUT;
  GridBDF* g = new (std::nothrow) GridBDF();
  if (!g) return BDFB_MEM_FAIL;
  g->external = true;
  g->ext = ext;
  g->nx = 0;
  g->dim = 0;
  g->np = N;
  g->N = N;
  make_tables(g);
  const size_t vb = g->N * sizeof(double);
  bool ok = true;
  auto alloc = [&](double** p, size_t bytes) {
    if (ok && cudaMalloc(p, bytes) != cudaSuccess) { *p = nullptr; ok = false; }
  };
  for (int j = 0; j <= GQMAX + 1; ++j) alloc(&g->z[j], vb);
  alloc(&g->ewt, vb); alloc(&g->sc, vb); alloc(&g->acor, vb); alloc(&g->acorp, vb); alloc(&g->y, vb); alloc(&g->f, vb);
  alloc(&g->b, vb); alloc(&g->zp0, vb); alloc(&g->zp1, vb); alloc(&g->tmp, vb); alloc(&g->w, vb);
  alloc(&g->work, bdfb_nv_work_doubles(g->N, MAXL_MAX) * sizeof(double));
  alloc(&g->dres, (MAXL_MAX + 2) * sizeof(double));
  alloc(&g->part, (size_t)sm_count() * 8 * sizeof(double));
  if (ok && cudaMalloc(&g->dsing, sizeof(int)) != cudaSuccess) ok = false;
  if (ok && cudaMallocHost(&g->hres, (MAXL_MAX + 2) * sizeof(double)) != cudaSuccess) ok = false;
  if (ok && cudaMemset(g->work, 0, bdfb_nv_work_doubles(g->N, MAXL_MAX) * sizeof(double)) != cudaSuccess) ok = false;
  if (ok && (cudaEventCreate(&g->e0) != cudaSuccess || cudaEventCreate(&g->e1) != cudaSuccess)) ok = false;
  if (!ok) {
    grid_destroy(g);
    return BDFB_MEM_FAIL;
  }
  *out = g;
  return 0;
}

void grid_destroy(GridBDF* g) {
  if (!g) return;
  for (int j = 0; j <= GQMAX + 1; ++j) cudaFree(g->z[j]);
  cudaFree(g->ewt); cudaFree(g->sc); cudaFree(g->acor); cudaFree(g->acorp); cudaFree(g->y); cudaFree(g->f);
  cudaFree(g->b); cudaFree(g->zp0); cudaFree(g->zp1); cudaFree(g->tmp); cudaFree(g->w); cudaFree(g->Pinv);
  for (int i = 0; i <= MAXL_MAX; ++i) cudaFree(g->V[i]);
  cudaFree(g->work); cudaFree(g->dres); cudaFree(g->part); cudaFree(g->dsing);
  if (g->hres) cudaFreeHost(g->hres);
  if (g->e0) cudaEventDestroy(g->e0);
  if (g->e1) cudaEventDestroy(g->e1);
  delete g;
}

void grid_set_stream(GridBDF* g, cudaStream_t s) { g->s = s; }
void grid_set_tolerances(GridBDF* g, double rtol, double atol) { g->rtol = rtol; g->atol = atol; }

int grid_set_option(GridBDF* g, const char* key, int64_t v) {
  if (!std::strcmp(key, "maxl")) {
    if (v < 1 || v > MAXL_MAX) return BDFB_ILL_INPUT;
    for (int i = 0; i <= v; ++i)
      if (!g->V[i] && cudaMalloc(&g->V[i], g->N * sizeof(double)) != cudaSuccess) {
        g->V[i] = nullptr;
        return BDFB_MEM_FAIL;
      }
    g->maxl = (int)v;
  } else if (!std::strcmp(key, "mxstep")) {
    if (v < 1) return BDFB_ILL_INPUT;
    g->mxstep = v;
  } else if (!std::strcmp(key, "qmax")) {
    if (v < 1 || v > GQMAX) return BDFB_ILL_INPUT;
    g->qmax = (int)v;
  } else if (!std::strcmp(key, "interp")) {
    if (v != 0 && v != 1) return BDFB_ILL_INPUT;
    g->interp = (int)v;
  } else if (!std::strcmp(key, "profile")) {
    if (v != 0 && v != 1) return BDFB_ILL_INPUT;
    g->prof = v != 0;
    for (int k = 0; k < GOP_N; ++k) { g->pcalls[k] = 0; g->pms[k] = 0.0; g->pgb[k] = 0.0; }
  } else if (!std::strcmp(key, "precision") && !g->external) {
    if (v != 0 && v != 1) return BDFB_ILL_INPUT;
    g->prec = (int)v;
    g->force_setup = true;      // the preconditioner's storage type changes
  } else {
    return BDFB_ILL_INPUT;
  }
  return 0;
}

int grid_init(GridBDF* g, double t0, const double* y0, int mem) {
  for (int j = 0; j <= GQMAX + 1; ++j) BDFB_CUDA(cudaMemsetAsync(g->z[j], 0, g->N * sizeof(double), g->s));
  BDFB_CUDA(cudaMemsetAsync(g->acorp, 0, g->N * sizeof(double), g->s));
  BDFB_CUDA(cudaMemcpyAsync(g->z[0], y0, g->N * sizeof(double),
                            mem == BDFB_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, g->s));
  BDFB_CUDA(cudaStreamSynchronize(g->s));
  g->t = t0;
  g->h = 0;
  g->q = 1;
  g->qwait = 2;
  g->started = g->grown = g->setup_done = g->force_setup = false;
  g->crate = 1.0;
  g->nst = g->nstlp = 0;
  g->nfe = g->nsetups = g->nni = g->ncfn = g->netf = g->nli = g->nlfail = 0;
  return 0;
}

int grid_integrate(GridBDF* g, double tout, double* y, int mem) {
  int ret = 0;
  BDFB_CUDA(cudaEventRecord(g->e0, g->s));
  if (tout != g->t) {
    if (!g->started) ret = g_initial_step(g, tout);
    const int64_t nst0 = g->nst;
    while (!ret && (tout - g->t) * g->h > 0.0) {
      if (g->nst - nst0 >= g->mxstep) { ret = BDFB_TOO_MUCH_WORK; break; }
      GCHK(g_ewt(g));
      bool reached = false;
      ret = g_step(g, tout, &reached);
      if (ret) break;
      if (reached) { g->t = tout; break; }
    }
  }
  BDFB_CUDA(cudaEventRecord(g->e1, g->s));
  const double* src = g->z[0];
  if (g->interp && !ret && g->started && g->t != tout) {
    k_interp<<<gblocks(g->N), GT, 0, g->s>>>(g->N, g->q, zcols(g), (tout - g->t) / g->h, g->tmp);
    BDFB_CUDA(cudaGetLastError());
    src = g->tmp;
  }
  if (y)
    BDFB_CUDA(cudaMemcpyAsync(y, src, g->N * sizeof(double),
                              mem == BDFB_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, g->s));
  BDFB_CUDA(cudaStreamSynchronize(g->s));
  cudaEventElapsedTime(&g->last_ms, g->e0, g->e1);
  if (g->prof) prof_flush(g);
  return ret;
}

void grid_profile(GridBDF* g, double* out) {
  for (int k = 0; k < GOP_N; ++k) {
    out[3 * k] = (double)g->pcalls[k];
    out[3 * k + 1] = g->pms[k];
    out[3 * k + 2] = g->pgb[k];
  }
}

void grid_stats(GridBDF* g, int64_t out[8], double* last_ms) {
  out[0] = g->nst; out[1] = g->nfe; out[2] = g->nsetups; out[3] = g->nni;
  out[4] = g->ncfn; out[5] = g->netf; out[6] = g->nli; out[7] = g->nlfail;
  *last_ms = g->last_ms;
}

void grid_next_step(GridBDF* g, int* q, double* h) {
  *q = g->q;
  *h = g->h;
}

}  // namespace bdfb
