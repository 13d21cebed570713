// sparse.cu - shared-pattern block-diagonal matrices (Sec. 5: the blocks of
// the submodel case share one sparsity pattern, so one copy of the CSR index
// arrays serves every block) with a batched sparse LU, and the grouped
// integrator of many cells that share one sparse mass-action network.
//
// B300 design: one thread per block, values stored entry-major
// (entry e of block b at v[e nb + b]).  The symbolic factorisation (fill-in
// of LU without pivoting in the given order, and the elimination schedule)
// is computed once on the host; every thread then runs the same schedule on
// its own block, so the warp never diverges and every load and store of a
// warp touches 32 consecutive doubles.  The paper's batched sparse QR needs
// no pivoting; LU here takes the pivots in order too (M = I - gamma J has a
// unit diagonal plus gamma times the Jacobian's; a zero pivot is reported
// and fails the Newton solve, which repeats the step with a smaller h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "cellcore.cuh"
#include "grid.cuh"
#include "sparse.cuh"

namespace bdfb {

namespace {

constexpr int ST = 128;                // threads per block of the per-cell kernels
constexpr int SP_NMAX = 2048;          // largest block dimension

// Symbolic LU of one pattern (no pivoting, natural order) and the schedules
// the kernels run.  Entries of the factor's pattern are numbered row-major.
struct Symb {
  int n = 0, nnz = 0;
  std::vector<int> pos;                           // n*n -> entry or -1
  std::vector<int> diag;                          // [n]
  std::vector<int> lptr, lpos, uptr, upos, tptr, tgt;
  std::vector<int> rlptr, rlpos, rlcol, ruptr, rupos, rucol;
};

Symb symbolic(int n, const std::vector<uint8_t>& A) {
  std::vector<uint8_t> P = A;
  for (int i = 0; i < n; ++i) P[(size_t)i * n + i] = 1;
  for (int k = 0; k < n; ++k)
    for (int i = k + 1; i < n; ++i) {
      if (!P[(size_t)i * n + k]) continue;
      for (int j = k + 1; j < n; ++j)
        if (P[(size_t)k * n + j]) P[(size_t)i * n + j] = 1;
    }
  Symb S;
  S.n = n;
  S.pos.assign((size_t)n * n, -1);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (P[(size_t)i * n + j]) S.pos[(size_t)i * n + j] = S.nnz++;
  S.diag.resize(n);
  for (int k = 0; k < n; ++k) S.diag[k] = S.pos[(size_t)k * n + k];
  S.lptr.push_back(0); S.uptr.push_back(0); S.tptr.push_back(0);
  for (int k = 0; k < n; ++k) {
    std::vector<int> L, U;
    for (int i = k + 1; i < n; ++i)
      if (P[(size_t)i * n + k]) L.push_back(i);
    for (int j = k + 1; j < n; ++j)
      if (P[(size_t)k * n + j]) U.push_back(j);
    for (int i : L) S.lpos.push_back(S.pos[(size_t)i * n + k]);
    for (int j : U) S.upos.push_back(S.pos[(size_t)k * n + j]);
    for (int i : L)
      for (int j : U) S.tgt.push_back(S.pos[(size_t)i * n + j]);   // present by construction of the fill
    S.lptr.push_back((int)S.lpos.size());
    S.uptr.push_back((int)S.upos.size());
    S.tptr.push_back((int)S.tgt.size());
  }
  S.rlptr.push_back(0); S.ruptr.push_back(0);
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < i; ++j)
      if (P[(size_t)i * n + j]) { S.rlpos.push_back(S.pos[(size_t)i * n + j]); S.rlcol.push_back(j); }
    for (int j = i + 1; j < n; ++j)
      if (P[(size_t)i * n + j]) { S.rupos.push_back(S.pos[(size_t)i * n + j]); S.rucol.push_back(j); }
    S.rlptr.push_back((int)S.rlpos.size());
    S.ruptr.push_back((int)S.rupos.size());
  }
  return S;
}

// device copies of the schedules
struct LUDev {
  int n, nnz;
  const int *diag, *lptr, *lpos, *uptr, *upos, *tptr, *tgt;
  const int *rlptr, *rlpos, *rlcol, *ruptr, *rupos, *rucol;
};

template <typename T>
int upload(T** d, const std::vector<T>& h) {
  *d = nullptr;
  const size_t bytes = std::max<size_t>(1, h.size()) * sizeof(T);
  BDFB_CUDA(cudaMalloc(d, bytes));
  if (!h.empty()) BDFB_CUDA(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return 0;
}

struct LUOwn {
  LUDev D = {};
  std::vector<void*> bufs;
  ~LUOwn() {
    for (void* p : bufs) cudaFree(p);
  }
  int make(const Symb& S) {
    D.n = S.n;
    D.nnz = S.nnz;
    int* p = nullptr;
#define UP(field, vec)                         \
  do {                                         \
    int r_ = upload(&p, S.vec);                \
    if (r_) return r_;                         \
    bufs.push_back(p);                         \
    D.field = p;                               \
  } while (0)
    UP(diag, diag); UP(lptr, lptr); UP(lpos, lpos); UP(uptr, uptr); UP(upos, upos); UP(tptr, tptr); UP(tgt, tgt);
    UP(rlptr, rlptr); UP(rlpos, rlpos); UP(rlcol, rlcol); UP(ruptr, ruptr); UP(rupos, rupos); UP(rucol, rucol);
#undef UP
    return 0;
  }
};

// LU of block c in place: L unit lower (multipliers), U upper with its
// diagonal replaced by the reciprocal.  Returns 0 or k + 1 for a zero or
// non-finite pivot at step k.
__device__ __forceinline__ int lu_factor_sp(const LUDev& L, int64_t nb, double* __restrict__ v, int64_t c) {
  for (int k = 0; k < L.n; ++k) {
    double* dk = v + (int64_t)L.diag[k] * nb + c;
    const double piv = *dk;
    if (!(piv != 0.0) || !isfinite(piv)) return k + 1;
    const double inv = 1.0 / piv;
    *dk = inv;
    const int l0 = L.lptr[k], l1 = L.lptr[k + 1], u0 = L.uptr[k], u1 = L.uptr[k + 1];
    const int nu = u1 - u0;
    const int* t = L.tgt + L.tptr[k];
    for (int a = l0; a < l1; ++a) {
      double* lp = v + (int64_t)L.lpos[a] * nb + c;
      const double m = *lp * inv;
      *lp = m;
      const int* ta = t + (a - l0) * nu;
      for (int b = 0; b < nu; ++b) {
        double* tp = v + (int64_t)ta[b] * nb + c;
        *tp -= m * v[(int64_t)L.upos[u0 + b] * nb + c];
      }
    }
  }
  return 0;
}

// x <- (LU)^{-1} x for block c; x entry-major [n][nb]
__device__ __forceinline__ void lu_solve_sp(const LUDev& L, int64_t nb, const double* __restrict__ v,
                                            double* __restrict__ x, int64_t c) {
  for (int i = 0; i < L.n; ++i) {
    double s = x[(int64_t)i * nb + c];
#pragma unroll 4
    for (int e = L.rlptr[i]; e < L.rlptr[i + 1]; ++e) s -= v[(int64_t)L.rlpos[e] * nb + c] * x[(int64_t)L.rlcol[e] * nb + c];
    x[(int64_t)i * nb + c] = s;
  }
  for (int i = L.n - 1; i >= 0; --i) {
    double s = x[(int64_t)i * nb + c];
#pragma unroll 4
    for (int e = L.ruptr[i]; e < L.ruptr[i + 1]; ++e) s -= v[(int64_t)L.rupos[e] * nb + c] * x[(int64_t)L.rucol[e] * nb + c];
    x[(int64_t)i * nb + c] = s * v[(int64_t)L.diag[i] * nb + c];
  }
}

// ---- standalone batched matrices
__global__ void __launch_bounds__(ST) k_sp_zero(int64_t total, double* v) {
  for (int64_t i = (int64_t)blockIdx.x * ST + threadIdx.x; i < total; i += (int64_t)gridDim.x * ST) v[i] = 0.0;
}

// lu[map[e] nb + b] = a[b nnz + e], one thread per (b, e) (reads coalesced)
__global__ void __launch_bounds__(ST) k_sp_load(int64_t nb, int nnz, const int* __restrict__ map,
                                                const double* __restrict__ a, double* __restrict__ lu) {
  const int64_t total = nb * nnz;
  for (int64_t i = (int64_t)blockIdx.x * ST + threadIdx.x; i < total; i += (int64_t)gridDim.x * ST) {
    const int64_t b = i / nnz;
    const int e = (int)(i - b * nnz);
    lu[(int64_t)map[e] * nb + b] = a[i];
  }
}

__global__ void __launch_bounds__(ST) k_sp_factor(LUDev L, int64_t nb, double* lu, int32_t* info) {
  const int64_t c = (int64_t)blockIdx.x * ST + threadIdx.x;
  if (c >= nb) return;
  const int r = lu_factor_sp(L, nb, lu, c);
  if (info) info[c] = r;
}

__global__ void __launch_bounds__(ST) k_sp_solve(LUDev L, int64_t nb, const double* lu, double* x) {
  const int64_t c = (int64_t)blockIdx.x * ST + threadIdx.x;
  if (c >= nb) return;
  lu_solve_sp(L, nb, lu, x, c);
}

// ---- a network shared by every cell
// Every table below holds offsets already multiplied by the cell count nb
// (entry e of cell c at v[e nb + c]): the kernels add them to per-cell base
// pointers, so an access costs one address add.  The context checks that
// every offset fits an int32.
struct NetDev {
  int n, R;
  int64_t nb;                  // cells
  const int* reac;             // [4 R] reactant offsets s nb, -1 = empty slot
  const double* k;             // [R]
  const int* inc_off;          // [n + 1] species-major incidence lists
  const int* inc;              // (r nb) << 1 | produced, reaction order, consumption first
  const int* jac_off;          // [4 R + 1] scatter lists of d rate_r / d y_(reactant a)
  const int* jac_pos;          // LU entry offsets
  const int8_t* jac_sgn;       // +1: the species is a reactant (M += gamma d), -1: a product
  int nnz;                     // LU entries (with fill)
  const int *diag, *lptr, *lpos, *uptr, *upos, *tptr, *tgt;   // factor schedule (offsets)
  const int *rlptr, *rlpos, *rlcol, *ruptr, *rupos, *rucol;   // solve schedule (offsets)
  // banded factors (every entry within BW of the diagonal): offset of
  // (i, i - d) at bl[i BW + d - 1], of (i, i + d) at bu[i BW + d - 1], -1 if absent
  const int* bl;
  const int* bu;
};

constexpr int BW = 8;          // widest band the register-window solve takes

// LU of cell c in place (v = the cell's base pointer): L unit lower, U upper
// with its diagonal replaced by the reciprocal; 0 or k + 1 for a zero or
// non-finite pivot at step k
__device__ __forceinline__ int net_factor(const NetDev& D, double* __restrict__ v) {
  for (int k = 0; k < D.n; ++k) {
    double* dk = v + D.diag[k];
    const double piv = *dk;
    if (!(piv != 0.0) || !isfinite(piv)) return k + 1;
    const double inv = 1.0 / piv;
    *dk = inv;
    const int l0 = D.lptr[k], l1 = D.lptr[k + 1], u0 = D.uptr[k], u1 = D.uptr[k + 1];
    const int nu = u1 - u0;
    const int* t = D.tgt + D.tptr[k];
    for (int a = l0; a < l1; ++a) {
      double* lp = v + D.lpos[a];
      const double m = *lp * inv;
      *lp = m;
      const int* ta = t + (a - l0) * nu;
#pragma unroll 4
      for (int b = 0; b < nu; ++b) v[ta[b]] -= m * v[D.upos[u0 + b]];
    }
  }
  return 0;
}

// x <- (LU)^{-1} x for one cell (v, x: the cell's base pointers)
__device__ __forceinline__ void net_solve(const NetDev& D, const double* __restrict__ v, double* __restrict__ x) {
  const int64_t nb = D.nb;
  for (int i = 0; i < D.n; ++i) {
    double s = x[i * nb];
#pragma unroll 4
    for (int e = D.rlptr[i]; e < D.rlptr[i + 1]; ++e) s -= v[D.rlpos[e]] * x[D.rlcol[e]];
    x[i * nb] = s;
  }
  for (int i = D.n - 1; i >= 0; --i) {
    double s = x[i * nb];
#pragma unroll 4
    for (int e = D.ruptr[i]; e < D.ruptr[i + 1]; ++e) s -= v[D.rupos[e]] * x[D.rucol[e]];
    x[i * nb] = s * v[D.diag[i]];
  }
}

// The same solves for a banded factor with the last BW solved values in
// registers: each row's dependence on the rows above (below) it runs through
// registers, and every load of the row (its right-hand side and factor
// entries) is independent of that chain.  Rows go in chunks of BW so that
// every register index is static.
__device__ __forceinline__ void net_solve_band(const NetDev& D, const double* __restrict__ v,
                                               double* __restrict__ x) {
  const int n = D.n;
  const int64_t nb = D.nb;
  double ring[BW];
#pragma unroll
  for (int t = 0; t < BW; ++t) ring[t] = 0.0;
  for (int i0 = 0; i0 < n; i0 += BW) {
#pragma unroll
    for (int t = 0; t < BW; ++t) {
      const int i = i0 + t;
      if (i < n) {
        double s = x[i * nb];
        const int* bl = D.bl + i * BW;
#pragma unroll
        for (int d = 1; d <= BW; ++d) {
          const int p = bl[d - 1];
          if (p >= 0) s -= v[p] * ring[(t - d + BW) % BW];
        }
        ring[t] = s;
        x[i * nb] = s;
      }
    }
  }
  for (int j0 = 0; j0 < n; j0 += BW) {           // rows i = n - 1 - (j0 + t)
#pragma unroll
    for (int t = 0; t < BW; ++t) {
      const int i = n - 1 - (j0 + t);
      if (i >= 0) {
        double s = x[i * nb];                      // the forward value of row i
        const int* bu = D.bu + i * BW;
#pragma unroll
        for (int d = 1; d <= BW; ++d) {
          const int p = bu[d - 1];
          if (p >= 0) s -= v[p] * ring[(t - d + BW) % BW];
        }
        s *= v[D.diag[i]];
        ring[t] = s;
        x[i * nb] = s;
      }
    }
  }
}

__device__ __forceinline__ void net_rates(const NetDev& D, const double* __restrict__ y, double* __restrict__ rates) {
  const int64_t nb = D.nb;
#pragma unroll 4
  for (int r = 0; r < D.R; ++r) {
    double v = D.k[r];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int o = D.reac[4 * r + a];
      if (o >= 0) v *= y[o];
    }
    rates[r * nb] = v;
  }
}

// f_s of species s from the rates (reaction order, consumption first)
__device__ __forceinline__ double net_fs(const NetDev& D, const double* __restrict__ rates, int s) {
  double acc = 0.0;
#pragma unroll 4
  for (int e = D.inc_off[s]; e < D.inc_off[s + 1]; ++e) {
    const int ent = D.inc[e];
    const double v = rates[ent >> 1];
    acc = (ent & 1) ? acc + v : acc - v;
  }
  return acc;
}

// M = I - gamma J(y) in the LU pattern of one cell, then its LU
__device__ __forceinline__ int net_setup(const NetDev& D, const double* __restrict__ y, double gamma,
                                         double* __restrict__ lu) {
  const int64_t nb = D.nb;
  for (int e = 0; e < D.nnz; ++e) lu[e * nb] = 0.0;
  for (int k = 0; k < D.n; ++k) lu[D.diag[k]] = 1.0;
  for (int r = 0; r < D.R; ++r) {
    const int* ro = D.reac + 4 * r;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (ro[a] < 0) continue;
      double d = D.k[r];
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (b != a && ro[b] >= 0) d *= y[ro[b]];
      const double gd = gamma * d;
      for (int e = D.jac_off[4 * r + a]; e < D.jac_off[4 * r + a + 1]; ++e) {
        double* p = lu + D.jac_pos[e];
        *p = D.jac_sgn[e] > 0 ? *p + gd : *p - gd;
      }
    }
  }
  return net_factor(D, lu);
}

__global__ void __launch_bounds__(ST) k_net_rhs(NetDev D, const double* __restrict__ y, double* __restrict__ f,
                                                double* __restrict__ rates) {
  const int64_t c = (int64_t)blockIdx.x * ST + threadIdx.x;
  if (c >= D.nb) return;
  net_rates(D, y + c, rates + c);
  for (int s = 0; s < D.n; ++s) f[s * D.nb + c] = net_fs(D, rates + c, s);
}

struct NewtonArgs {
  const double *zp0, *zp1, *ewt;
  double gamma, gammap, rl1, Eq;
  int setup;
  double* acor;
  double* crate;               // per cell, kept between solves
  int* failed;
  unsigned long long* iters;   // [0] completed iterations (sum), [1] RHS sweeps (max)
};

// Task-local Newton solve of every cell (the grouped mode's solve): each
// cell iterates on its own block to its own test, as the per-cell
// integrator's Newton: rate R = max(0.3 R, |d_m| / |d_{m-1}|), converged when
// |d_m| min(1, R) E_q <= 0.1, diverged when |d_m| > 2 |d_{m-1}|, <= 3
// iterations; a stale M scales the correction by 2 / (1 + gamma / gamma_p).
__global__ void __launch_bounds__(ST) k_net_newton(NetDev D, NewtonArgs A, double* __restrict__ lu,
                                                   double* __restrict__ rates, double* __restrict__ yv,
                                                   double* __restrict__ xv) {
  const int64_t c = (int64_t)blockIdx.x * ST + threadIdx.x;
  if (c >= D.nb) return;
  const int64_t nb = D.nb;
  const int n = D.n;
  const double* z0 = A.zp0 + c;
  const double* z1 = A.zp1 + c;
  const double* ew = A.ewt + c;
  double* ac = A.acor + c;
  double* luc = lu + c;
  double* rc = rates + c;
  double* yc = yv + c;
  double* xc = xv + c;
  double crate = A.crate[c];
  if (A.setup) {
    crate = 1.0;
    if (net_setup(D, z0, A.gamma, luc)) {
      A.crate[c] = crate;
      atomicOr(A.failed, 1);
      return;
    }
  }
  for (int s = 0; s < n; ++s) ac[s * nb] = 0.0;
  const double rn = 1.0 / (double)n;
  const double eq2 = A.Eq * A.Eq * 100.0;
  const double scst = A.gamma != A.gammap ? 2.0 / (1.0 + A.gamma / A.gammap) : 1.0;
  double delp2 = 0.0;
  bool conv = false;
  int it = 1, nit = 0;
  for (; it <= 3; ++it) {
    for (int s = 0; s < n; ++s) yc[s * nb] = z0[s * nb] + ac[s * nb];
    net_rates(D, yc, rc);
    bool fin = true;
    for (int s = 0; s < n; ++s) {              // x = gamma f - z1 / l1 - acor
      const double f = net_fs(D, rc, s);
      fin = fin && isfinite(f);
      xc[s * nb] = A.gamma * f - z1[s * nb] * A.rl1 - ac[s * nb];
    }
    if (!fin) break;
    ++nit;
    if (D.bl) net_solve_band(D, luc, xc);
    else net_solve(D, luc, xc);
    double del2 = 0.0;
    for (int s = 0; s < n; ++s) {
      double x = xc[s * nb];
      if (A.gamma != A.gammap) x *= scst;
      const double e = x * ew[s * nb];
      del2 += e * e;
      ac[s * nb] += x;
    }
    del2 *= rn;
    if (it > 1) crate = fmax(0.3 * crate, sqrt(del2 / delp2));
    const double cr = fmin(1.0, crate);
    if (del2 * cr * cr * eq2 <= 1.0) { conv = true; break; }
    if (it >= 2 && del2 > 4.0 * delp2) break;
    delp2 = del2;
  }
  A.crate[c] = crate;
  atomicAdd(A.iters, (unsigned long long)nit);
  atomicMax(A.iters + 1, (unsigned long long)(it > 3 ? 3 : it));
  if (!conv) atomicOr(A.failed, 1);
}


// ---------------------------------------------- per-cell step control
// Every cell of the shared network integrated with its own step size and
// order by one thread (the per-cell mode of the other cell workloads, on the
// shared sparse pattern): the BDF/Newton step of the per-cell integrator --
// prediction, Jacobian reuse, Newton with the rate test and a stale-M retry,
// local error test, accept, step and order choice -- over the cell's
// entry-major vectors, with M = I - gamma J factored by the shared sparse LU.
// Threads of a warp run their cells' steps in lockstep where their control
// agrees and serialise where it does not (a setup or a second Newton
// iteration of one cell); every access of a warp touches 32 consecutive
// doubles.
struct NetCellState {
  double t, h, gammap, crate, hlast;   // crate: the squared Newton rate R^2
  int32_t q, qwait, nst, nstlp;
  int32_t nfe, nsetups, nni, ncfn;
  int32_t netf, flags, status, qlast;
};
enum { NF_STARTED = 1, NF_GROWN = 2 };

struct NetCellArgs {
  NetDev D;
  double *z, *zs;                      // (QMAX + 1) n nb: plane j, species s at (j n + s) nb
  double *acor, *acorp, *ewt;          // n nb
  double *y, *x;                       // n nb scratch
  double *lu, *rates;
  NetCellState* st;
  int32_t* status;                     // per cell (may be null)
  double* yout;                        // interpolated output (interp), n nb
  int* worst;
  double tout, rtol, atol;
  int32_t mxstep, qmax, interp;
  Consts K;
};

struct NetCell {
  double t, h, gamma, gammap, crate, hlast;
  int q, qwait, nst, nstlp, nfe, nsetups, nni, ncfn, netf, qlast, flags, status;
  int nst0, ncf, nef, setup_done, force_setup, tried_fresh, newstep, last, retry;
};

// the cell's vectors: base pointers already offset by the cell
struct NetV {
  double *z, *zs, *acor, *acorp, *ewt, *y, *x, *lu, *rates;
  int64_t nb;
  int n;
  __device__ __forceinline__ double& Z(int j, int s) const { return z[((int64_t)j * n + s) * nb]; }
  __device__ __forceinline__ double& ZS(int j, int s) const { return zs[((int64_t)j * n + s) * nb]; }
  __device__ __forceinline__ double& at(double* a, int s) const { return a[(int64_t)s * nb]; }
};

// sum (x_s w_s)^2 over the cell's species, times rn
__device__ __forceinline__ double net_wrms2(const NetV& V, const double* a, double rn) {
  double s2 = 0.0;
  for (int s = 0; s < V.n; ++s) {
    const double v = a[(int64_t)s * V.nb] * V.ewt[(int64_t)s * V.nb];
    s2 = fma(v, v, s2);
  }
  return s2 * rn;
}

// f(y) into out (rates into V.rates); false when an entry is not finite
__device__ __forceinline__ bool net_f(const NetDev& D, const NetV& V, const double* y, double* out) {
  net_rates(D, y, V.rates);
  bool fin = true;
  for (int s = 0; s < V.n; ++s) {
    const double f = net_fs(D, V.rates, s);
    fin = fin && finite_bits(f);
    out[(int64_t)s * V.nb] = f;
  }
  return fin;
}

// error weights by the Newton-Raphson reciprocal (four FP64 FMAs where a
// division issues many more)
__device__ __forceinline__ void net_set_ewt(const NetCellArgs& A, const NetV& V) {
  for (int s = 0; s < V.n; ++s) V.at(V.ewt, s) = recip_nr(A.rtol * fabs(V.Z(0, s)) + A.atol);
}

__device__ __forceinline__ void net_rescale(const NetV& V, NetCell& C, double eta) {
  for (int s = 0; s < V.n; ++s) {
    double f = 1.0;
    for (int j = 1; j <= C.q; ++j) {
      f *= eta;
      V.Z(j, s) *= f;
    }
  }
  C.h *= eta;
}

__device__ __forceinline__ void net_restore(const NetV& V, const NetCell& C) {
  for (int s = 0; s < V.n; ++s)
    for (int j = 0; j <= C.q; ++j) V.Z(j, s) = V.ZS(j, s);
}

// saved copy of z_0..z_Q, then the prediction in place (registers per species)
template <int Q>
__device__ __forceinline__ void net_predict(const NetV& V) {
  for (int s = 0; s < V.n; ++s) {
    double zz[Q + 1];
#pragma unroll
    for (int j = 0; j <= Q; ++j) {
      zz[j] = V.Z(j, s);
      V.ZS(j, s) = zz[j];
    }
#pragma unroll
    for (int k = 1; k <= Q; ++k)
#pragma unroll
      for (int j = Q; j >= k; --j) zz[j - 1] += zz[j];
#pragma unroll
    for (int j = 0; j <= Q; ++j) V.Z(j, s) = zz[j];
  }
}

// initial step and history (the per-cell integrator's reading); 0 or a code
__device__ int net_start(const NetCellArgs& A, const NetV& V, NetCell& C) {
  const NetDev& D = A.D;
  const int n = V.n;
  net_set_ewt(A, V);
  if (!net_f(D, V, V.z, V.acor)) return BDFB_RHSFUNC_FAIL;          // f0 in acor
  C.nfe++;
  const double tdist = fabs(A.tout - C.t);
  const double tround = 2.220446049250313e-16 * fmax(fabs(C.t), fabs(A.tout));
  const double hlb = 100.0 * tround;
  double hub = 0.1 * tdist;
  double inv = 0.0;
  for (int s = 0; s < n; ++s) inv = fmax(inv, fabs(V.at(V.acor, s)) / (0.1 * fabs(V.Z(0, s)) + A.atol));
  if (inv * hub > 1.0) hub = 1.0 / inv;
  if (hub < hlb) hub = hlb;
  double hg = sqrt(hlb * hub), hnew = hg;
  const double rn = 1.0 / (double)n;
  for (int it = 0; it < 4; ++it) {
    bool ok = false;
    for (int tries = 0; tries < 4; ++tries) {
      for (int s = 0; s < n; ++s) V.at(V.y, s) = V.Z(0, s) + hg * V.at(V.acor, s);
      ok = net_f(D, V, V.y, V.x);
      C.nfe++;
      if (ok) break;
      hg *= 0.2;
    }
    if (!ok) return BDFB_RHSFUNC_FAIL;
    for (int s = 0; s < n; ++s) V.at(V.x, s) = (V.at(V.x, s) - V.at(V.acor, s)) / hg;
    const double ydd = sqrt(net_wrms2(V, V.x, rn));
    hnew = (ydd * hub * hub > 2.0) ? sqrt(2.0 / ydd) : sqrt(hg * hub);
    const double rat = hnew / hg;
    if (it > 0 && rat > 0.5 && rat < 2.0) break;
    hg = hnew;
  }
  double h0 = 0.5 * hnew;
  if (h0 < hlb) h0 = hlb;
  if (h0 > hub) h0 = hub;
  C.h = (A.tout >= C.t) ? h0 : -h0;
  for (int s = 0; s < n; ++s) {
    V.Z(1, s) = C.h * V.at(V.acor, s);
    for (int j = 2; j <= QMAX; ++j) V.Z(j, s) = 0.0;
  }
  C.q = 1;
  C.qwait = 2;
  C.flags |= NF_STARTED;
  return 0;
}

// step size and order after an accepted step: the per-cell integrator's rules
// (FP32 candidates, FP64 near ties and the FP64 applied ratio)
__device__ __forceinline__ void net_select(const NetCellArgs& A, const NetV& V, NetCell& C, double dsm2, double rn) {
  if (--C.qwait > 0) return;
  const int q = C.q;
  const bool hm = q > 1, hp = q < A.qmax;
  const double xq = dsm2;
  double xm = 0.0, xp = 0.0;
  if (hm) {
    double s2 = 0.0;
    for (int s = 0; s < V.n; ++s) {
      const double v = V.Z(q, s) * V.at(V.ewt, s);
      s2 = fma(v, v, s2);
    }
    xm = s2 * (rn * A.K.E2[q][1]);
  }
  if (hp) {
    double s2 = 0.0;
    for (int s = 0; s < V.n; ++s) {
      const double v = (V.at(V.acor, s) - V.at(V.acorp, s)) * V.at(V.ewt, s);
      s2 = fma(v, v, s2);
    }
    xp = s2 * (rn * A.K.E2[q][2]);
  }
  const float fq = eta_f(xq, 36.0f, 0.5f / (q + 1));
  const float fm = hm ? eta_f(xm, 36.0f, 0.5f / q) : 0.0f;
  const float fp = hp ? eta_f(xp, 100.0f, 0.5f / (q + 2)) : 0.0f;
  auto near = [](float a, float b) { return fabsf(a - b) <= 1.0e-5f * fmaxf(a, b); };
  const bool tie = near(fq, 1.5f) || (hm && (near(fm, fq) || near(fm, 1.5f))) ||
                   (hp && (near(fp, fq) || near(fp, 1.5f) || (hm && near(fp, fm))));
  double etam;
  int qn = q;
  const double cap = (C.flags & NF_GROWN) ? 10.0 : 1.0e4;
  if (tie) {
    etam = eta64(xq, 36.0, 2 * (q + 1));
    const double em = hm ? eta64(xm, 36.0, 2 * q) : 0.0;
    const double ep = hp ? eta64(xp, 100.0, 2 * (q + 2)) : 0.0;
    if (em > etam) { etam = em; qn = q - 1; }
    if (ep > etam) { etam = ep; qn = q + 1; }
    if (etam < 1.5) { C.qwait = 1; return; }
  } else {
    float fbest = fq;
    if (fm > fbest) { fbest = fm; qn = q - 1; }
    if (fp > fbest) { fbest = fp; qn = q + 1; }
    if (fbest < 1.5f) { C.qwait = 1; return; }
    etam = fbest >= ((C.flags & NF_GROWN) ? 10.0f : 1.0e4f) * 1.00001f ? cap
           : (qn == q ? eta64(xq, 36.0, 2 * (q + 1)) : (qn < q ? eta64(xm, 36.0, 2 * q) : eta64(xp, 100.0, 2 * (q + 2))));
  }
  if (etam > cap) etam = cap;
  C.flags |= NF_GROWN;
  if (qn == q + 1) {
    for (int s = 0; s < V.n; ++s) V.Z(q + 1, s) = V.at(V.acor, s) / A.K.qfact[q + 1];
    C.q = q + 1;
  } else if (qn == q - 1) {
    for (int s = 0; s < V.n; ++s) V.Z(q, s) = 0.0;
    C.q = q - 1;
  }
  net_rescale(V, C, etam);
  C.qwait = C.q + 1;
}

// one step attempt; true when the cell is finished (tout reached or a
// failure status set)
__device__ __forceinline__ bool net_attempt(const NetCellArgs& A, const NetV& V, NetCell& C) {
  const NetDev& D = A.D;
  const int n = V.n;
  const double rn = 1.0 / (double)n;
  if (!(C.flags & NF_STARTED)) {
    if (A.tout == C.t) { C.status = 0; return true; }
    const int r = net_start(A, V, C);
    if (r) { C.status = r; return true; }
    C.newstep = 1;
  }
  if (C.newstep) {
    if ((A.tout - C.t) * C.h <= 0.0) { C.status = 0; return true; }
    if (C.nst - C.nst0 >= A.mxstep) { C.status = BDFB_TOO_MUCH_WORK; return true; }
    net_set_ewt(A, V);
    C.ncf = 0;
    C.nef = 0;
    C.newstep = 0;
    C.retry = 0;
  }
  if (!C.retry) {
    C.last = 0;
    if (!A.interp && (C.t + C.h - A.tout) * C.h >= 0.0) {
      C.last = 1;
      if (C.t + C.h != A.tout) { net_rescale(V, C, (A.tout - C.t) / C.h); C.qwait = C.q + 1; }
    }
  }
  C.retry = 0;
  if (C.t + C.h == C.t) { C.status = BDFB_ERR_FAILURE; return true; }
  const int q = C.q;
  // save, then predict: z_{j-1} += z_j repeatedly (Pascal triangle)
  switch (q) {
    case 1: net_predict<1>(V); break;
    case 2: net_predict<2>(V); break;
    case 3: net_predict<3>(V); break;
    case 4: net_predict<4>(V); break;
    default: net_predict<5>(V); break;
  }
  const double tnew = C.last ? A.tout : C.t + C.h;
  const double rl1 = A.K.rl1[q];
  const double Eq = A.K.E[q][0];
  C.gamma = C.h * rl1;
  // ---- linear setup
  int jcur = 0;
  bool fail = false;
  const double dgam = C.gamma - C.gammap;
  if (!C.setup_done || C.force_setup || fabs(dgam) > 0.3 * fabs(C.gammap) || C.nst >= C.nstlp + 20) {
    const int info = net_setup(D, V.z, C.gamma, V.lu);
    C.nsetups++;
    C.gammap = C.gamma;
    C.crate = 1.0;
    C.nstlp = C.nst;
    C.force_setup = 0;
    C.setup_done = 1;
    jcur = 1;
    if (info) { fail = true; C.setup_done = 0; }
  }
  // ---- Newton iteration (norms compared squared, in FP64)
  const bool stale = C.gamma != C.gammap;
  const double scst = stale ? 2.0 * C.gammap / (C.gammap + C.gamma) : 1.0;
  double acnrm2 = 0.0;
  bool conv = false;
  if (!fail) {
    for (int s = 0; s < n; ++s) V.at(V.acor, s) = 0.0;
    double delp2 = 0.0;
    const double eq2 = Eq * Eq * 100.0;   // (E_q / 0.1)^2
    for (int it = 1; it <= 3; ++it) {
      for (int s = 0; s < n; ++s) V.at(V.y, s) = V.Z(0, s) + V.at(V.acor, s);
      const bool fin = net_f(D, V, V.y, V.x);
      C.nfe++;
      if (!fin) break;
      for (int s = 0; s < n; ++s)
        V.at(V.x, s) = C.gamma * V.at(V.x, s) - V.Z(1, s) * rl1 - V.at(V.acor, s);
      if (D.bl) net_solve_band(D, V.lu, V.x);
      else net_solve(D, V.lu, V.x);
      double del2 = 0.0;
      for (int s = 0; s < n; ++s) {
        double d = V.at(V.x, s);
        if (stale) d *= scst;
        const double e = d * V.at(V.ewt, s);
        del2 = fma(e, e, del2);
        V.at(V.acor, s) += d;
      }
      del2 *= rn;
      C.nni++;
      if (it > 1) {                                  // R^2 = max(0.09 R_prev^2, del2 / delp2)
        const double r2 = 0.09 * C.crate;
        C.crate = r2 * delp2 >= del2 ? r2 : del2 / delp2;
      }
      if (del2 * fmin(1.0, C.crate) * eq2 <= 1.0) {  // |del| min(1, R) E_q / 0.1 <= 1
        acnrm2 = it == 1 ? del2 : net_wrms2(V, V.acor, rn);
        conv = true;
        break;
      }
      if (it >= 2 && del2 > 4.0 * delp2) break;       // |del| > 2 |del_prev|: diverging
      delp2 = del2;
    }
    if (!conv) fail = true;
  }
  if (fail) {
    net_restore(V, C);
    if (!jcur && !C.tried_fresh && C.setup_done) {   // stale M: retry once with a fresh one
      C.force_setup = 1;
      C.tried_fresh = 1;
      C.retry = 1;
      return false;
    }
    C.tried_fresh = 0;
    C.ncf++;
    C.ncfn++;
    if (C.ncf >= 10) { C.status = BDFB_CONV_FAILURE; return true; }
    net_rescale(V, C, 0.25);
    C.qwait = C.q + 1;
    C.force_setup = 1;
    return false;
  }
  C.tried_fresh = 0;
  // ---- local error test
  const double dsm2 = acnrm2 * Eq * Eq;
  if (!(dsm2 <= 1.0)) {
    net_restore(V, C);
    C.nef++;
    C.netf++;
    if (C.nef >= 7) { C.status = BDFB_ERR_FAILURE; return true; }
    if (C.nef < 3) {
      double eta = eta64(dsm2, 36.0, 2 * (q + 1));
      if (!(eta >= 0.1)) eta = 0.1;
      if (C.nef >= 2 && eta > 0.2) eta = 0.2;
      net_rescale(V, C, eta);
      C.qwait = C.q + 1;
    } else {                                         // third failure: order 1, h / 10, fresh slope
      for (int s = 0; s < n; ++s)
        for (int j = 2; j <= QMAX; ++j) V.Z(j, s) = 0.0;
      C.q = 1;
      C.h *= 0.1;
      const bool fin = net_f(D, V, V.z, V.x);
      C.nfe++;
      if (!fin) { C.status = BDFB_RHSFUNC_FAIL; return true; }
      for (int s = 0; s < n; ++s) V.Z(1, s) = C.h * V.at(V.x, s);
      C.qwait = 2;
    }
    return false;
  }
  // ---- accept
  for (int s = 0; s < n; ++s) {
    const double a = V.at(V.acor, s);
    for (int j = 0; j <= q; ++j) V.Z(j, s) = fma(A.K.l[q][j], a, V.Z(j, s));
  }
  C.t = tnew;
  C.nst++;
  C.hlast = C.h;
  C.qlast = q;
  net_select(A, V, C, dsm2, rn);
  for (int s = 0; s < n; ++s) V.at(V.acorp, s) = V.at(V.acor, s);
  C.newstep = 1;
  if (C.last) { C.t = A.tout; C.status = 0; return true; }
  return false;
}

// 6 resident blocks per SM (80 registers, 44 bytes spilled) measured faster
// than 8 (64 registers, 280 bytes spilled) and 5 (no spills, fewer threads)
__global__ void __launch_bounds__(ST, 6) k_net_cells(const __grid_constant__ NetCellArgs A) {
  const int64_t c = (int64_t)blockIdx.x * ST + threadIdx.x;
  const int64_t nb = A.D.nb;
  if (c >= nb) return;
  NetV V;
  V.nb = nb;
  V.n = A.D.n;
  V.z = A.z + c; V.zs = A.zs + c; V.acor = A.acor + c; V.acorp = A.acorp + c; V.ewt = A.ewt + c;
  V.y = A.y + c; V.x = A.x + c; V.lu = A.lu + c; V.rates = A.rates + c;
  const NetCellState s = A.st[c];
  NetCell C;
  C.t = s.t; C.h = s.h; C.gammap = s.gammap; C.crate = s.crate; C.hlast = s.hlast;
  C.q = s.q; C.qwait = s.qwait; C.nst = s.nst; C.nstlp = s.nstlp; C.nfe = s.nfe; C.nsetups = s.nsetups;
  C.nni = s.nni; C.ncfn = s.ncfn; C.netf = s.netf; C.flags = s.flags; C.qlast = s.qlast; C.status = 0;
  C.nst0 = C.nst; C.setup_done = 0; C.force_setup = 0; C.tried_fresh = 0; C.gamma = 0.0;
  C.newstep = 1; C.retry = 0; C.last = 0; C.ncf = 0; C.nef = 0;
  while (!net_attempt(A, V, C)) {
  }
  if (A.yout) {
    // the history polynomial at tout, sum_j z_j s^j with s = (tout - t) / h,
    // for a cell past tout; otherwise its current state
    const bool pol = A.interp && C.status == 0 && (C.flags & NF_STARTED) && C.t != A.tout;
    const double sv = pol ? (A.tout - C.t) / C.h : 0.0;
    for (int sp = 0; sp < V.n; ++sp) {
      double v = V.Z(0, sp);
      if (pol) {
        v = V.Z(C.q, sp);
        for (int j = C.q - 1; j >= 0; --j) v = v * sv + V.Z(j, sp);
      }
      A.yout[(int64_t)sp * nb + c] = v;
    }
  }
  NetCellState o;
  o.t = C.t; o.h = C.h; o.gammap = C.gammap; o.crate = C.crate; o.hlast = C.hlast;
  o.q = C.q; o.qwait = C.qwait; o.nst = C.nst; o.nstlp = C.nstlp; o.nfe = C.nfe; o.nsetups = C.nsetups;
  o.nni = C.nni; o.ncfn = C.ncfn; o.netf = C.netf; o.flags = C.flags; o.status = C.status; o.qlast = C.qlast;
  A.st[c] = o;
  if (A.status) A.status[c] = C.status;
  if (C.status < 0) atomicMin(A.worst, C.status);
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + ST - 1) / ST, 1 << 30)); }

}  // namespace

// ------------------------------------------------------------ C ABI: matrices
}  // namespace bdfb

struct bdfb_sparse {
  bdfb::Symb S;
  bdfb::LUOwn own;
  int n = 0, nnz_in = 0;
  int* dmap = nullptr;         // input CSR entry -> LU entry
};

extern "C" int bdfb_sparse_create(int n, int nnz, const int32_t* rowptr, const int32_t* colind,
                                  bdfb_sparse** out) {
  using namespace bdfb;
  if (!out || n < 1 || n > SP_NMAX || nnz < 0 || !rowptr || (nnz > 0 && !colind)) return BDFB_ILL_INPUT;
  *out = nullptr;
  if (rowptr[0] != 0 || rowptr[n] != nnz) return BDFB_ILL_INPUT;
  std::vector<uint8_t> A((size_t)n * n, 0);
  for (int i = 0; i < n; ++i) {
    if (rowptr[i + 1] < rowptr[i]) return BDFB_ILL_INPUT;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int j = colind[e];
      if (j < 0 || j >= n || A[(size_t)i * n + j]) return BDFB_ILL_INPUT;   // range, duplicates
      A[(size_t)i * n + j] = 1;
    }
  }
  bdfb_sparse* sp = new (std::nothrow) bdfb_sparse();
  if (!sp) return BDFB_MEM_FAIL;
  sp->S = symbolic(n, A);
  sp->n = n;
  sp->nnz_in = nnz;
  std::vector<int> map(std::max(nnz, 1));
  for (int i = 0; i < n; ++i)
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) map[e] = sp->S.pos[(size_t)i * n + colind[e]];
  int r = sp->own.make(sp->S);
  if (!r) r = upload(&sp->dmap, map);
  if (r) {
    cudaFree(sp->dmap);
    delete sp;
    return r;
  }
  *out = sp;
  return BDFB_SUCCESS;
}

extern "C" void bdfb_sparse_destroy(bdfb_sparse* sp) {
  if (!sp) return;
  cudaFree(sp->dmap);
  delete sp;
}

extern "C" int64_t bdfb_sparse_lu_nnz(const bdfb_sparse* sp) { return sp ? sp->S.nnz : BDFB_ILL_INPUT; }

extern "C" int bdfb_sparse_load(const bdfb_sparse* sp, int64_t nb, const double* a, double* lu, void* stream) {
  using namespace bdfb;
  if (!sp || nb < 0 || (nb > 0 && (!a || !lu))) return BDFB_ILL_INPUT;
  if (nb == 0) return BDFB_SUCCESS;
  cudaStream_t s = as_stream(stream);
  const int64_t tot = nb * sp->S.nnz;
  const int g = (int)std::min<int64_t>((tot + ST - 1) / ST, (int64_t)sm_count() * 16);
  k_sp_zero<<<g, ST, 0, s>>>(tot, lu);
  if (sp->nnz_in > 0) {
    const int64_t tin = nb * sp->nnz_in;
    const int gi = (int)std::min<int64_t>((tin + ST - 1) / ST, (int64_t)sm_count() * 16);
    k_sp_load<<<gi, ST, 0, s>>>(nb, sp->nnz_in, sp->dmap, a, lu);
  }
  BDFB_CUDA(cudaGetLastError());
  return BDFB_SUCCESS;
}

extern "C" int bdfb_sparse_factor(const bdfb_sparse* sp, int64_t nb, double* lu, int32_t* info, void* stream) {
  using namespace bdfb;
  if (!sp || nb < 0 || (nb > 0 && !lu)) return BDFB_ILL_INPUT;
  if (nb == 0) return BDFB_SUCCESS;
  k_sp_factor<<<grid_for(nb), ST, 0, as_stream(stream)>>>(sp->own.D, nb, lu, info);
  BDFB_CUDA(cudaGetLastError());
  return BDFB_SUCCESS;
}

extern "C" int bdfb_sparse_solve(const bdfb_sparse* sp, int64_t nb, const double* lu, double* x, void* stream) {
  using namespace bdfb;
  if (!sp || nb < 0 || (nb > 0 && (!lu || !x))) return BDFB_ILL_INPUT;
  if (nb == 0) return BDFB_SUCCESS;
  k_sp_solve<<<grid_for(nb), ST, 0, as_stream(stream)>>>(sp->own.D, nb, lu, x);
  BDFB_CUDA(cudaGetLastError());
  return BDFB_SUCCESS;
}

// ------------------------------------------------- cells sharing one network
namespace bdfb {

struct SharedInt {
  NetDev D = {};
  std::vector<void*> bufs;
  int nnz_m = 0;               // entries of M's own pattern
  double *lu = nullptr, *rates = nullptr, *yv = nullptr, *xv = nullptr, *crate = nullptr;
  int* dflag = nullptr;
  unsigned long long* diters = nullptr;
  GridBDF* gg = nullptr;
  cudaStream_t s = nullptr;
  // per-cell step control (option "grouped" 0): history, saved history,
  // corrections, weights, states; allocated on first use
  bool percell = false, pc_alloc = false;
  double *z = nullptr, *zs = nullptr, *acor = nullptr, *acorp = nullptr, *ewt = nullptr, *yout = nullptr;
  NetCellState* st = nullptr;
  int32_t* dstatus = nullptr;
  int* dworst = nullptr;
  double rtol = 1e-6, atol = 1e-10;
  int64_t mxstep = 100000;
  int qmax = QMAX, interp = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float last_ms = 0.f;
  ~SharedInt() {
    grid_destroy(gg);
    for (void* p : bufs) cudaFree(p);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
  template <typename T>
  int up(const T** d, const std::vector<T>& h) {
    T* p = nullptr;
    const int r = upload(&p, h);
    if (!r) bufs.push_back(p);
    *d = p;
    return r;
  }
};

static int net_rhs_cb(void* user, const double* y, double* f, cudaStream_t s) {
  SharedInt* S = static_cast<SharedInt*>(user);
  k_net_rhs<<<grid_for(S->D.nb), ST, 0, s>>>(S->D, y, f, S->rates);
  BDFB_CUDA(cudaGetLastError());
  return 0;
}

static int net_solve_cb(void* user, const double* zp0, const double* zp1, const double* ewt, double gamma,
                        double gammap, double rl1, double Eq, int setup, double* acor, int* failed,
                        int64_t* iters, int64_t* sweeps, cudaStream_t s) {
  SharedInt* S = static_cast<SharedInt*>(user);
  NewtonArgs A;
  A.zp0 = zp0; A.zp1 = zp1; A.ewt = ewt;
  A.gamma = gamma; A.gammap = gammap; A.rl1 = rl1; A.Eq = Eq;
  A.setup = setup;
  A.acor = acor;
  A.crate = S->crate;
  A.failed = S->dflag;
  A.iters = S->diters;
  BDFB_CUDA(cudaMemsetAsync(S->dflag, 0, sizeof(int), s));
  BDFB_CUDA(cudaMemsetAsync(S->diters, 0, 2 * sizeof(unsigned long long), s));
  k_net_newton<<<grid_for(S->D.nb), ST, 0, s>>>(S->D, A, S->lu, S->rates, S->yv, S->xv);
  BDFB_CUDA(cudaGetLastError());
  int fl = 0;
  unsigned long long it[2] = {0, 0};
  BDFB_CUDA(cudaMemcpyAsync(&fl, S->dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
  BDFB_CUDA(cudaMemcpyAsync(it, S->diters, sizeof it, cudaMemcpyDeviceToHost, s));
  BDFB_CUDA(cudaStreamSynchronize(s));
  *failed = fl;
  *iters = (int64_t)it[0];
  *sweeps = (int64_t)it[1];
  return 0;
}

int shared_create(const bdfb_problem* prob, SharedInt** out) {
  *out = nullptr;
  if (prob->mem != BDFB_MEM_HOST || !prob->n || !prob->rxn_off || !prob->reactants || !prob->products ||
      prob->ncell < 1)
    return BDFB_ILL_INPUT;
  const int n = prob->n[0];
  const int64_t R64 = prob->rxn_off[1] - prob->rxn_off[0];
  if (prob->rxn_off[0] != 0 || n < 1 || n > 255 || R64 < 0 || R64 > 65535) return BDFB_ILL_INPUT;
  const int R = (int)R64;
  const int64_t nb = prob->ncell;
  // network, pattern of J (rows: affected species, columns: reactants)
  std::vector<uint8_t> A((size_t)n * n, 0);
  std::vector<std::vector<int>> incs(n);
  for (int r = 0; r < R; ++r) {
    const uint8_t* ra = prob->reactants + 4 * r;
    const uint8_t* pa = prob->products + 4 * r;
    for (int a = 0; a < 4; ++a) {
      if ((ra[a] != 255 && ra[a] >= n) || (pa[a] != 255 && pa[a] >= n)) return BDFB_ILL_INPUT;
      for (int b = 0; b < a; ++b)
        if ((ra[a] != 255 && ra[a] == ra[b]) || (pa[a] != 255 && pa[a] == pa[b])) return BDFB_ILL_INPUT;
    }
    for (int a = 0; a < 4; ++a) {
      if (ra[a] == 255) continue;
      for (int b = 0; b < 4; ++b) {
        if (ra[b] != 255) A[(size_t)ra[b] * n + ra[a]] = 1;
        if (pa[b] != 255) A[(size_t)pa[b] * n + ra[a]] = 1;
      }
    }
    for (int a = 0; a < 4; ++a)
      if (ra[a] != 255) incs[ra[a]].push_back(r << 1);
    for (int a = 0; a < 4; ++a)
      if (pa[a] != 255) incs[pa[a]].push_back((r << 1) | 1);
  }
  const Symb sy = symbolic(n, A);
  // every table holds offsets times nb: they must fit an int32 (the rate
  // offsets keep one more bit for the production flag)
  const int64_t lim = (int64_t)1 << 30;
  if ((int64_t)sy.nnz * nb >= lim || (int64_t)std::max(R, 1) * nb >= lim || (int64_t)n * nb >= lim)
    return BDFB_ILL_INPUT;
  auto sc = [nb](int v) { return v < 0 ? -1 : (int)((int64_t)v * nb); };
  auto scv = [&](const std::vector<int>& v) {
    std::vector<int> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = sc(v[i]);
    return o;
  };
  std::vector<int> reac(4 * (size_t)std::max(R, 1), -1);
  for (int r = 0; r < R; ++r)
    for (int a = 0; a < 4; ++a) {
      const uint8_t s2 = prob->reactants[4 * r + a];
      reac[4 * (size_t)r + a] = s2 == 255 ? -1 : sc(s2);
    }
  std::vector<int> inc_off(n + 1, 0), inc;
  for (int s2 = 0; s2 < n; ++s2) {
    for (int ent : incs[s2]) inc.push_back((int)(((int64_t)(ent >> 1) * nb) << 1) | (ent & 1));
    inc_off[s2 + 1] = (int)inc.size();
  }
  // Jacobian scatter lists in reaction order
  std::vector<int> jac_off(4 * (size_t)R + 1, 0), jac_pos;
  std::vector<int8_t> jac_sgn;
  for (int rr = 0; rr < R; ++rr) {
    const uint8_t* ra = prob->reactants + 4 * rr;
    const uint8_t* pa = prob->products + 4 * rr;
    for (int a = 0; a < 4; ++a) {
      if (ra[a] != 255)
        for (int b = 0; b < 4; ++b) {
          if (ra[b] != 255) { jac_pos.push_back(sc(sy.pos[(size_t)ra[b] * n + ra[a]])); jac_sgn.push_back(1); }
          if (pa[b] != 255) { jac_pos.push_back(sc(sy.pos[(size_t)pa[b] * n + ra[a]])); jac_sgn.push_back(-1); }
        }
      jac_off[4 * (size_t)rr + a + 1] = (int)jac_pos.size();
    }
  }
  // band tables when every factor entry lies within BW of the diagonal
  bool banded = true;
  for (int i = 0; i < n && banded; ++i)
    for (int j = 0; j < n; ++j)
      if (sy.pos[(size_t)i * n + j] >= 0 && std::abs(i - j) > BW) { banded = false; break; }
  std::vector<int> bl, bu;
  if (banded) {
    bl.assign((size_t)n * BW, -1);
    bu.assign((size_t)n * BW, -1);
    for (int i = 0; i < n; ++i)
      for (int d = 1; d <= BW; ++d) {
        if (i - d >= 0) bl[(size_t)i * BW + d - 1] = sc(sy.pos[(size_t)i * n + i - d]);
        if (i + d < n) bu[(size_t)i * BW + d - 1] = sc(sy.pos[(size_t)i * n + i + d]);
      }
  }
  SharedInt* S = new (std::nothrow) SharedInt();
  if (!S) return BDFB_MEM_FAIL;
  for (uint8_t v : A) S->nnz_m += v != 0;
  NetDev& D = S->D;
  D.n = n;
  D.R = R;
  D.nb = nb;
  D.nnz = sy.nnz;
  int r = 0;
  const std::vector<double> k(prob->k, prob->k + R);
  if (!r) r = S->up(&D.reac, reac);
  if (!r) r = S->up(&D.k, k);
  if (!r) r = S->up(&D.inc_off, inc_off);
  if (!r) r = S->up(&D.inc, inc);
  if (!r) r = S->up(&D.jac_off, jac_off);
  if (!r) r = S->up(&D.jac_pos, jac_pos);
  if (!r) r = S->up(&D.jac_sgn, jac_sgn);
  if (!r) r = S->up(&D.diag, scv(sy.diag));
  if (!r) r = S->up(&D.lptr, sy.lptr);
  if (!r) r = S->up(&D.lpos, scv(sy.lpos));
  if (!r) r = S->up(&D.uptr, sy.uptr);
  if (!r) r = S->up(&D.upos, scv(sy.upos));
  if (!r) r = S->up(&D.tptr, sy.tptr);
  if (!r) r = S->up(&D.tgt, scv(sy.tgt));
  if (!r) r = S->up(&D.rlptr, sy.rlptr);
  if (!r) r = S->up(&D.rlpos, scv(sy.rlpos));
  if (!r) r = S->up(&D.rlcol, scv(sy.rlcol));
  if (!r) r = S->up(&D.ruptr, sy.ruptr);
  if (!r) r = S->up(&D.rupos, scv(sy.rupos));
  if (!r) r = S->up(&D.rucol, scv(sy.rucol));
  if (!r && banded) r = S->up(&D.bl, bl);
  if (!r && banded) r = S->up(&D.bu, bu);
  if (!banded) D.bl = D.bu = nullptr;
  auto alloc = [&](double** p, size_t count) {
    if (r) return;
    if (cudaMalloc(p, std::max<size_t>(count, 1) * sizeof(double)) != cudaSuccess) { *p = nullptr; r = BDFB_MEM_FAIL; return; }
    S->bufs.push_back(*p);
  };
  alloc(&S->lu, (size_t)sy.nnz * nb);
  alloc(&S->rates, (size_t)std::max(R, 1) * nb);
  alloc(&S->yv, (size_t)n * nb);
  alloc(&S->xv, (size_t)n * nb);
  alloc(&S->crate, (size_t)nb);
  if (!r && cudaMalloc(&S->dflag, sizeof(int)) != cudaSuccess) r = BDFB_MEM_FAIL;
  if (!r) S->bufs.push_back(S->dflag);
  if (!r && cudaMalloc(&S->diters, 2 * sizeof(unsigned long long)) != cudaSuccess) r = BDFB_MEM_FAIL;
  if (!r) S->bufs.push_back(S->diters);
  GridExternal ext;
  ext.user = S;
  ext.rhs = net_rhs_cb;
  ext.solve = net_solve_cb;
  if (!r) r = grid_create_external((int64_t)n * nb, ext, &S->gg);
  if (r) {
    delete S;
    return r;
  }
  *out = S;
  return 0;
}

void shared_destroy(SharedInt* S) { delete S; }

void shared_set_stream(SharedInt* S, cudaStream_t s) {
  S->s = s;
  grid_set_stream(S->gg, s);
}

void shared_set_tolerances(SharedInt* S, double rtol, double atol) {
  S->rtol = rtol;
  S->atol = atol;
  grid_set_tolerances(S->gg, rtol, atol);
}

static int percell_alloc(SharedInt* S) {
  if (S->pc_alloc) return 0;
  const NetDev& D = S->D;
  const size_t nv = (size_t)D.n * D.nb;
  auto alloc = [&](void** p, size_t bytes) -> int {
    if (cudaMalloc(p, std::max<size_t>(bytes, 1)) != cudaSuccess) { *p = nullptr; return BDFB_MEM_FAIL; }
    S->bufs.push_back(*p);
    return 0;
  };
  int r = alloc((void**)&S->z, (QMAX + 1) * nv * sizeof(double));
  if (!r) r = alloc((void**)&S->zs, (QMAX + 1) * nv * sizeof(double));
  if (!r) r = alloc((void**)&S->acor, nv * sizeof(double));
  if (!r) r = alloc((void**)&S->acorp, nv * sizeof(double));
  if (!r) r = alloc((void**)&S->ewt, nv * sizeof(double));
  if (!r) r = alloc((void**)&S->yout, nv * sizeof(double));
  if (!r) r = alloc((void**)&S->st, (size_t)D.nb * sizeof(NetCellState));
  if (!r) r = alloc((void**)&S->dstatus, (size_t)D.nb * sizeof(int32_t));
  if (!r) r = alloc((void**)&S->dworst, sizeof(int));
  if (!r && (cudaEventCreate(&S->e0) != cudaSuccess || cudaEventCreate(&S->e1) != cudaSuccess)) r = BDFB_CUDA_FAIL;
  if (r) return r;
  S->pc_alloc = true;
  return 0;
}

int shared_set_option(SharedInt* S, const char* key, int64_t v) {
  if (!std::strcmp(key, "grouped")) {
    if (v != 0 && v != 1) return BDFB_ILL_INPUT;
    if (v == 0) {
      const int r = percell_alloc(S);
      if (r) return r;
    }
    S->percell = v == 0;
    return 0;
  }
  if (!std::strcmp(key, "mxstep") && v >= 1) S->mxstep = v;
  if (!std::strcmp(key, "qmax") && v >= 1 && v <= QMAX) S->qmax = (int)v;
  if (!std::strcmp(key, "interp") && (v == 0 || v == 1)) S->interp = (int)v;
  if (!std::strcmp(key, "mxstep") || !std::strcmp(key, "qmax") || !std::strcmp(key, "interp"))
    return grid_set_option(S->gg, key, v);
  return BDFB_ILL_INPUT;
}

bool shared_percell(const SharedInt* S) { return S->percell; }

int shared_init(SharedInt* S, double t0, const double* y0, int mem) {
  const int r = grid_init(S->gg, t0, y0, mem);
  if (r || !S->pc_alloc) return r;
  // per-cell state: history plane 0 = y0 (species-major, as the grouped state)
  const NetDev& D = S->D;
  const size_t nv = (size_t)D.n * D.nb;
  BDFB_CUDA(cudaMemsetAsync(S->z, 0, (QMAX + 1) * nv * sizeof(double), S->s));
  BDFB_CUDA(cudaMemsetAsync(S->acorp, 0, nv * sizeof(double), S->s));
  BDFB_CUDA(cudaMemcpyAsync(S->z, y0, nv * sizeof(double),
                            mem == BDFB_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, S->s));
  std::vector<NetCellState> st((size_t)D.nb);
  for (auto& c : st) {
    std::memset(&c, 0, sizeof c);
    c.t = t0;
    c.q = 1;
    c.crate = 1.0;
  }
  BDFB_CUDA(cudaMemcpyAsync(S->st, st.data(), st.size() * sizeof(NetCellState), cudaMemcpyHostToDevice, S->s));
  BDFB_CUDA(cudaStreamSynchronize(S->s));
  return 0;
}

int shared_integrate(SharedInt* S, double tout, double* y, int mem) { return grid_integrate(S->gg, tout, y, mem); }

// per-cell mode: every cell to tout with its own step size and order;
// per-cell statuses to status (may be null); returns the worst status
int shared_integrate_cells(SharedInt* S, double tout, double* y, int32_t* status, int mem) {
  const NetDev& D = S->D;
  const size_t nv = (size_t)D.n * D.nb;
  NetCellArgs A;
  std::memset(&A, 0, sizeof A);
  A.D = D;
  A.z = S->z; A.zs = S->zs; A.acor = S->acor; A.acorp = S->acorp; A.ewt = S->ewt;
  A.y = S->yv; A.x = S->xv; A.lu = S->lu; A.rates = S->rates;
  A.st = S->st;
  A.status = S->dstatus;
  A.yout = S->yout;
  A.worst = S->dworst;
  A.tout = tout; A.rtol = S->rtol; A.atol = S->atol;
  A.mxstep = (int32_t)std::min<int64_t>(S->mxstep, 0x7fffffff);
  A.qmax = S->qmax;
  A.interp = S->interp;
  static const Consts K = make_consts();
  A.K = K;
  BDFB_CUDA(cudaMemsetAsync(S->dworst, 0, sizeof(int), S->s));
  BDFB_CUDA(cudaEventRecord(S->e0, S->s));
  k_net_cells<<<grid_for(D.nb), ST, 0, S->s>>>(A);
  BDFB_CUDA(cudaGetLastError());
  BDFB_CUDA(cudaEventRecord(S->e1, S->s));
  const cudaMemcpyKind kind = mem == BDFB_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (y) BDFB_CUDA(cudaMemcpyAsync(y, S->yout, nv * sizeof(double), kind, S->s));
  if (status) BDFB_CUDA(cudaMemcpyAsync(status, S->dstatus, D.nb * sizeof(int32_t), kind, S->s));
  int worst = 0;
  BDFB_CUDA(cudaMemcpyAsync(&worst, S->dworst, sizeof(int), cudaMemcpyDeviceToHost, S->s));
  BDFB_CUDA(cudaStreamSynchronize(S->s));
  cudaEventElapsedTime(&S->last_ms, S->e0, S->e1);
  return worst;
}

// per-cell mode: rows nst, nfe, nsetups, nni, ncfn, netf, qlast, hlast bits
int shared_cell_stats(SharedInt* S, std::vector<int64_t>& rows, double* last_ms) {
  const int64_t nb = S->D.nb;
  std::vector<NetCellState> st((size_t)nb);
  BDFB_CUDA(cudaMemcpy(st.data(), S->st, nb * sizeof(NetCellState), cudaMemcpyDeviceToHost));
  rows.assign(8 * (size_t)nb, 0);
  for (int64_t c = 0; c < nb; ++c) {
    const NetCellState& s = st[c];
    int64_t* o = rows.data() + 8 * c;
    int64_t hb;
    std::memcpy(&hb, &s.hlast, sizeof hb);
    o[0] = s.nst; o[1] = s.nfe; o[2] = s.nsetups; o[3] = s.nni;
    o[4] = s.ncfn; o[5] = s.netf; o[6] = s.qlast; o[7] = hb;
  }
  *last_ms = S->last_ms;
  return 0;
}

void shared_stats(SharedInt* S, int64_t out[8], double* last_ms, int* q, double* h) {
  grid_stats(S->gg, out, last_ms);
  out[6] = S->D.nnz;
  out[7] = S->nnz_m;
  grid_next_step(S->gg, q, h);
}

}  // namespace bdfb
