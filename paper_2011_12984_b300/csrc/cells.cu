// cells.cu - persistent batched BDF / Newton integration of independent cells.
//
// The paper's submodel use case (Sec. 2): many small independent ODE systems,
// one per grid cell, whose Jacobian is block diagonal (Fig. 1); each block is
// solved directly (Sec. 5 batched block solver; Sec. 7 task-local Newton with
// per-block solves, a failed solve repeating the step with a smaller h).
// Here every cell keeps its own step size and order, and one persistent launch
// integrates all cells to tout: warps take tiles of cells from an atomic
// counter; a tile is 32/G cells of one size class handled by groups of G
// lanes (cellcore.cuh).  The BDF step is the fixed-leading-coefficient
// Nordsieck form with constant-step coefficients and history rescaling:
//   predict z <- z A (Pascal), Newton on
//   G(D) = D - gamma f(t, z0 + D) + z1 / l1 with M = I - gamma J,
//   error test E_q ||D|| <= 1, accept z <- z + l D, then choose h and q.
// Nothing in the kernel waits on another warp; every loop is bounded.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "cellcore.cuh"
#include "mixed.cuh"
#include "ark.cuh"
#include "grid.cuh"
#include "mlp.cuh"
#include "sparse.cuh"

namespace bdfb {

constexpr int NCLASS = 5;
constexpr int CLS_G[NCLASS] = {1, 4, 8, 16, 32};
constexpr int CLS_NMAX[NCLASS] = {4, 8, 16, 32, 56};
constexpr int NMAX_ALL = 56;



struct CellState {
  double t, h, gammap, crate, hlast;   // crate: the squared Newton rate R^2
  int32_t q, qwait, nst, nstlp;
  int32_t nfe, nsetups, nni, ncfn;
  int32_t netf, flags, status, qlast;
  int32_t nrefine, nrefine_fb, nguess, nguess_fb;
};
enum { F_STARTED = 1, F_GROWN = 2 };

struct TileDesc {
  int32_t cls, first, count, pad;
};

struct Params {
  int kind;
  int qmax;
  int64_t ny;                 // total species
  const int32_t* n;
  const int64_t* y_off;
  const int64_t* rxn_off;
  const uint32_t* reac;
  const double* k;
  const int32_t* inc_off;
  const uint16_t* inc;
  const uint32_t* gsched;     // per species slot: gather schedules of the cells of > 32 species, or null
  const TileDesc* tiles;
  const int32_t* tile_cells;
  int ntiles;
  unsigned* tile_counter;
  int* worst;
  CellState* st;
  double* z;                  // 6 planes of ny doubles; plane 0 = y
  double* acorp;              // ny
  int32_t* status;            // per cell (may be null)
  double tout, rtol, atol;
  int32_t mxstep;
  Consts K;
  // learned Newton initial guess (one-warp-per-cell kernel only)
  const void* mlp;            // packed network, or null: Newton starts from 0
  float* rec_x;               // recording of (features, converged correction)
  float* rec_t;               //   pairs of accepted steps, or null
  int64_t rec_cap;
  unsigned long long* rec_count;
  // output mode: 0 the last step lands on tout (y = history plane 0); 1 the
  // cells step past tout and yout receives the history polynomial at tout
  int interp;
  double* yout;
};

template <int G>
__device__ __forceinline__ double gmax(const Grp<G>& g, double v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(g.mask, v, o, G));
  return v;
}

template <int G, int NMAX>
struct Cell {
  static constexpr int NPL = (NMAX + G - 1) / G;
  double z[QMAX + 1][NPL];
  double zsave[NMAX >= 56 ? QMAX + 1 : 1][NPL];   // saved history (CellSmem::ZREG kernels)
  double acor[NPL], acorp[NPL], ewt[NPL], f[NPL], b[NPL];
  double t, h, gamma, gammap, crate, hlast, rn;   // rn = 1/n
  int q, qwait, nst, nstlp, nfe, nsetups, nni, ncfn, netf, qlast, flags, status;
  int nst0, ncf, nef, setup_done, force_setup, tried_fresh, newstep, last, retry;
  int nref, nref_fb, fp64mode;   // mixed precision: refinement sweeps, FP64 fallbacks, M in FP64
  double mnorm;                  // |M|_inf of the current setup (mixed precision)
  int nguess, nguess_fb;         // learned guesses taken, guesses abandoned for a zero start
  int lastit;                    // Newton iterations of the last converged solve (gates the guess)
};

// The order-dependent loops are dispatched on q (group-uniform) to bodies
// unrolled for that order, so no predicated-off FP64 work is issued for the
// columns above q.
template <int Q, int NPL>
__device__ __forceinline__ void rescale_q(double (&z)[QMAX + 1][NPL], double eta) {
  double fct = 1.0;
#pragma unroll
  for (int j = 1; j <= Q; ++j) {
    fct *= eta;
#pragma unroll
    for (int p = 0; p < NPL; ++p) z[j][p] *= fct;
  }
}

// z_{j-1} += z_j for k = 1..Q, j = Q..k (multiplication by the Pascal matrix)
template <int Q, int NPL>
__device__ __forceinline__ void pascal_q(double (&z)[QMAX + 1][NPL]) {
#pragma unroll
  for (int k = 1; k <= Q; ++k)
#pragma unroll
    for (int j = Q; j >= k; --j)
#pragma unroll
      for (int p = 0; p < NPL; ++p) z[j - 1][p] += z[j][p];
}

// z_j += l_j acor, j = 0..Q
template <int Q, int NPL>
__device__ __forceinline__ void correct_q(double (&z)[QMAX + 1][NPL], const double* l, const double (&acor)[NPL]) {
#pragma unroll
  for (int j = 0; j <= Q; ++j) {
    const double lj = l[j];
#pragma unroll
    for (int p = 0; p < NPL; ++p) z[j][p] = fma(lj, acor[p], z[j][p]);
  }
}

#define BDFB_DISPATCH_Q(q, call) \
  switch (q) {                   \
    case 1: call(1); break;      \
    case 2: call(2); break;      \
    case 3: call(3); break;      \
    case 4: call(4); break;      \
    default: call(5); break;     \
  }

template <int G, int NMAX>
__device__ __forceinline__ void rescale(Cell<G, NMAX>& C, double eta) {
  constexpr int NPL = Cell<G, NMAX>::NPL;
#define BDFB_RESCALE(Q) rescale_q<Q, NPL>(C.z, eta)
  BDFB_DISPATCH_Q(C.q, BDFB_RESCALE)
#undef BDFB_RESCALE
  C.h *= eta;
}

template <int G, int NMAX>
__device__ __forceinline__ void set_ewt(const Grp<G>& g, const Params& P, int n, Cell<G, NMAX>& C) {
#pragma unroll
  for (int p = 0; p < Cell<G, NMAX>::NPL; ++p) {
    const int i = g.rank + G * p;
    // the Newton-Raphson reciprocal: four FP64 FMAs where a division issues more
    C.ewt[p] = i < n ? recip_nr(P.rtol * fabs(C.z[0][p]) + P.atol) : 0.0;
  }
}

// initial step and history (reading shared with the oracle: h0 from a
// difference estimate of ||y''|| within [100 eps t, min(0.1 |tout - t|,
// 0.1 (|y| + atol) / |f|)]).  Returns 0 or an error code.
template <int G, int NMAX, int PREC>
__device__ __forceinline__ int start_cell(const Grp<G>& g, const Params& P, const CellDesc& cd,
                                          CellSmem<NMAX, PREC>& S, Cell<G, NMAX>& C) {
  constexpr int NPL = Cell<G, NMAX>::NPL;
  const int n = cd.n;
  set_ewt(g, P, n, C);
  double y[NPL];
#pragma unroll
  for (int p = 0; p < NPL; ++p) y[p] = C.z[0][p];
  rhs<G, NPL, NMAX>(g, cd, S, y, C.acor);          // f0 kept in acor
  C.nfe++;
  if (!all_finite(g, n, C.acor)) return BDFB_RHSFUNC_FAIL;
  const double tdist = fabs(P.tout - C.t);
  const double tround = 2.220446049250313e-16 * fmax(fabs(C.t), fabs(P.tout));
  const double hlb = 100.0 * tround;
  double hub = 0.1 * tdist;
  double inv = 0.0;
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    if (i < n) inv = fmax(inv, fabs(C.acor[p]) / (0.1 * fabs(C.z[0][p]) + P.atol));
  }
  inv = gmax(g, inv);
  if (inv * hub > 1.0) hub = 1.0 / inv;
  if (hub < hlb) hub = hlb;
  double hg = sqrt(hlb * hub), hnew = hg;
  for (int it = 0; it < 4; ++it) {
    bool ok = false;
    for (int tries = 0; tries < 4; ++tries) {
#pragma unroll
      for (int p = 0; p < NPL; ++p) y[p] = C.z[0][p] + hg * C.acor[p];
      rhs<G, NPL, NMAX>(g, cd, S, y, C.f);
      C.nfe++;
      if (all_finite(g, n, C.f)) { ok = true; break; }
      hg *= 0.2;
    }
    if (!ok) return BDFB_RHSFUNC_FAIL;
#pragma unroll
    for (int p = 0; p < NPL; ++p) C.b[p] = (C.f[p] - C.acor[p]) / hg;
    const double ydd = wrms(g, n, C.b, C.ewt);
    hnew = (ydd * hub * hub > 2.0) ? sqrt(2.0 / ydd) : sqrt(hg * hub);
    const double rat = hnew / hg;
    if (it > 0 && rat > 0.5 && rat < 2.0) break;
    hg = hnew;
  }
  double h0 = 0.5 * hnew;
  if (h0 < hlb) h0 = hlb;
  if (h0 > hub) h0 = hub;
  C.h = (P.tout >= C.t) ? h0 : -h0;
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    C.z[1][p] = C.h * C.acor[p];
#pragma unroll
    for (int j = 2; j <= QMAX; ++j) C.z[j][p] = 0.0;
  }
  C.q = 1;
  C.qwait = 2;
  C.flags |= F_STARTED;
  return 0;
}

// choose h and q after an accepted step (same rules as the oracle: safety
// 6 / 6 / 10, change only if the best eta >= 1.5, eta <= 1e4 before the first
// increase and <= 10 after, ties keep q then prefer q - 1).  The candidates are
// formed and compared in FP32 (eta_f: no FP64 instruction); where two of them,
// or the best and the 1.5 threshold, lie within 1e-5 of each other (far above
// the FP32 error) all are formed to FP64 accuracy (eta64) and compared in
// FP64, so the choice is the one FP64 arithmetic makes; the eta applied is
// always the FP64 one.
__device__ __forceinline__ bool near_tie(float a, float b) { return fabsf(a - b) <= 1.0e-5f * fmaxf(a, b); }

template <int G, int NMAX>
__device__ __forceinline__ void select_next(const Grp<G>& g, const Params& P, int n, double rn,
                                            Cell<G, NMAX>& C, double dsm2) {
  constexpr int NPL = Cell<G, NMAX>::NPL;
  if (--C.qwait > 0) return;
  const int q = C.q;
  const bool hm = q > 1, hp = q < P.qmax;
  // squared test quantities of orders q, q - 1 (E_{q-1} |z_q|), q + 1
  // (E_{q+1} |Delta - Delta_prev|); eta = 1 / ((safety^2 x)^(1/k) + 1e-6)
  const double xq = dsm2;
  double xm = 0.0, xp = 0.0;
  if (hm) {
    double zq[NPL];
#pragma unroll
    for (int p = 0; p < NPL; ++p) {
      double v = 0.0;
#pragma unroll
      for (int j = 2; j <= QMAX; ++j)
        if (j == q) v = C.z[j][p];
      zq[p] = v;
    }
    xm = wrms2(g, n, rn * P.K.E2[q][1], zq, C.ewt);
  }
  if (hp) {
#pragma unroll
    for (int p = 0; p < NPL; ++p) C.b[p] = C.acor[p] - C.acorp[p];
    xp = wrms2(g, n, rn * P.K.E2[q][2], C.b, C.ewt);
  }
  const float fq = eta_f(xq, 36.0f, 0.5f / (q + 1));
  const float fm = hm ? eta_f(xm, 36.0f, 0.5f / q) : 0.0f;
  const float fp = hp ? eta_f(xp, 100.0f, 0.5f / (q + 2)) : 0.0f;
  const bool tie = near_tie(fq, 1.5f) || (hm && (near_tie(fm, fq) || near_tie(fm, 1.5f))) ||
                   (hp && (near_tie(fp, fq) || near_tie(fp, 1.5f) || (hm && near_tie(fp, fm))));
  double etam;
  int qn = q;
  const double cap = (C.flags & F_GROWN) ? 10.0 : 1.0e4;
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
    etam = fbest >= ((C.flags & F_GROWN) ? 10.0f : 1.0e4f) * 1.00001f ? cap
           : (qn == q ? eta64(xq, 36.0, 2 * (q + 1)) : (qn < q ? eta64(xm, 36.0, 2 * q) : eta64(xp, 100.0, 2 * (q + 2))));
  }
  if (etam > cap) etam = cap;
  C.flags |= F_GROWN;
  if (qn == q + 1) {
    const double fq = P.K.qfact[q + 1];
#pragma unroll
    for (int j = 2; j <= QMAX; ++j)
      if (j == q + 1) {
#pragma unroll
        for (int p = 0; p < NPL; ++p) C.z[j][p] = C.acor[p] / fq;
      }
    C.q = q + 1;
  } else if (qn == q - 1) {
#pragma unroll
    for (int j = 2; j <= QMAX; ++j)
      if (j == q) {
#pragma unroll
        for (int p = 0; p < NPL; ++p) C.z[j][p] = 0.0;
      }
    C.q = q - 1;
  }
  rescale(C, etam);
  C.qwait = C.q + 1;
}

template <int G, int NMAX, int PREC>
__device__ __forceinline__ void restore_z(const Grp<G>& g, int n, const CellSmem<NMAX, PREC>& S,
                                          Cell<G, NMAX>& C, const double* zg) {
  if constexpr (CellSmem<NMAX, PREC>::ZREG) {
#pragma unroll
    for (int p = 0; p < Cell<G, NMAX>::NPL; ++p)
#pragma unroll
      for (int j = 0; j <= QMAX; ++j) C.z[j][p] = C.zsave[j][p];
  } else if constexpr (CellSmem<NMAX, PREC>::ZGLOB) {
#pragma unroll
    for (int p = 0; p < Cell<G, NMAX>::NPL; ++p) {
      const int i = g.rank + G * p;
      if (i < n) {
#pragma unroll
        for (int j = 0; j <= QMAX; ++j) C.z[j][p] = zg[j * NMAX + i];
      }
    }
  } else {
#pragma unroll
    for (int p = 0; p < Cell<G, NMAX>::NPL; ++p) {
      const int i = g.rank + G * p;
      if (i < n) {
#pragma unroll
        for (int j = 0; j <= QMAX; ++j) C.z[j][p] = S.zs[j][i];
      }
    }
  }
}

// Input feature of the learned guess held by this lane (one warp per cell,
// species i on lane i): lanes 0..9 the predicted state on a log scale,
// (log10 max(y_pred, 1e-20) + 10) / 10 (zero past n), lane 10
// (log10 |h| + 8) / 4, lane 11 gamma / h = 1 / l_1.
__device__ __forceinline__ float mlp_feature(int lane, int n, double ypred, double h, double rl1) {
  if (lane < MLP_NO) return lane < n ? (log10f(fmaxf((float)ypred, 1e-20f)) + 10.f) * 0.1f : 0.f;
  if (lane == MLP_NO) return (log10f(fabsf((float)h)) + 8.f) * 0.25f;
  if (lane == MLP_NO + 1) return (float)rl1;
  return 0.f;
}

// Newton initial correction from the network: row 0 of a 16-row MMA tile
// holds this cell's features; the output (Delta in error-weight units) is
// un-scaled by ewt.  A non-finite output starts that component from zero.
__device__ __forceinline__ double mlp_guess(const void* mlp, float feat, int n, double ewt) {
  const int lane = threadIdx.x & 31, c = lane & 3;
  const float x0 = __shfl_sync(FULL_MASK, feat, 2 * c), x1 = __shfl_sync(FULL_MASK, feat, 2 * c + 1);
  const float x8 = __shfl_sync(FULL_MASK, feat, 2 * c + 8), x9 = __shfl_sync(FULL_MASK, feat, 2 * c + 9);
  uint32_t a[4] = {0u, 0u, 0u, 0u};
  if (lane < 4) { a[0] = pack_bf16(x0, x1); a[2] = pack_bf16(x8, x9); }
  float out[2][4];
  mlp_tile_forward(mlp_view(mlp), a, out);
  // row 0, column i sits on lane (i mod 8) / 2 of n-tile i / 8, element i & 1
  const int src = (lane & 7) >> 1;
  const float s00 = __shfl_sync(FULL_MASK, out[0][0], src), s01 = __shfl_sync(FULL_MASK, out[0][1], src);
  const float s10 = __shfl_sync(FULL_MASK, out[1][0], src), s11 = __shfl_sync(FULL_MASK, out[1][1], src);
  const float v = lane < 8 ? ((lane & 1) ? s01 : s00) : ((lane & 1) ? s11 : s10);
  const double d = lane < n && lane < MLP_NO ? (double)v / ewt : 0.0;
  return isfinite(d) ? d : 0.0;
}

// One step attempt.  Returns true when the cell is finished (tout reached or
// a failure status set).  LEARN (one warp per cell, n <= 10): Newton may
// start from the network's guess and a recording of the accepted steps'
// (features, converged correction) pairs may be kept.
template <int G, int NMAX, int PREC, int LEARN = 0>
__device__ __forceinline__ bool attempt(const Grp<G>& g, const Params& P, const CellDesc& cd,
                                        CellSmem<NMAX, PREC>& S, Cell<G, NMAX>& C,
                                        double (*Mg)[NMAX + 1]) {
  constexpr int NPL = Cell<G, NMAX>::NPL;
  static_assert(!LEARN || (G == 32 && NPL == 1 && PREC == 0), "learned guess: one warp per cell, FP64");
  const int n = cd.n;
  ph_mark(PH_CTRL);
  // the saved history of the kernels that keep it in the global workspace
  // (after the fallback matrix); without a workspace nothing has changed yet
  double* zg = nullptr;
  if constexpr (CellSmem<NMAX, PREC>::ZGLOB) {
    if (Mg == nullptr) { C.status = BDFB_MEM_FAIL; return true; }
    zg = reinterpret_cast<double*>(Mg) + NMAX * (NMAX + 1);
  }
  if (!(C.flags & F_STARTED)) {
    if (P.tout == C.t) { C.status = 0; return true; }   // first step waits for tout != t0
    const int r = start_cell(g, P, cd, S, C);
    if (r) { C.status = r; return true; }
    C.newstep = 1;
  }
  if (C.newstep) {
    if ((P.tout - C.t) * C.h <= 0.0) { C.status = 0; return true; }
    if (C.nst - C.nst0 >= P.mxstep) { C.status = BDFB_TOO_MUCH_WORK; return true; }
    set_ewt(g, P, n, C);
    C.ncf = 0;
    C.nef = 0;
    C.newstep = 0;
    C.retry = 0;
  }
  if (!C.retry) {
    C.last = 0;
    if (!P.interp && (C.t + C.h - P.tout) * C.h >= 0.0) {
      C.last = 1;
      if (C.t + C.h != P.tout) { rescale(C, (P.tout - C.t) / C.h); C.qwait = C.q + 1; }
    }
  }
  C.retry = 0;
  if (C.t + C.h == C.t) { C.status = BDFB_ERR_FAILURE; return true; }
  const int q = C.q;
  ph_mark(PH_PRED);
  // save and predict: z_{j-1} += z_j repeatedly (Pascal triangle)
  if constexpr (CellSmem<NMAX, PREC>::ZREG) {
#pragma unroll
    for (int p = 0; p < NPL; ++p)
#pragma unroll
      for (int j = 0; j <= QMAX; ++j) C.zsave[j][p] = C.z[j][p];
  } else if constexpr (CellSmem<NMAX, PREC>::ZGLOB) {
#pragma unroll
    for (int p = 0; p < NPL; ++p) {
      const int i = g.rank + G * p;
      if (i < n) {
#pragma unroll
        for (int j = 0; j <= QMAX; ++j) zg[j * NMAX + i] = C.z[j][p];
      }
    }
  } else {
#pragma unroll
    for (int p = 0; p < NPL; ++p) {
      const int i = g.rank + G * p;
      if (i < n) {
#pragma unroll
        for (int j = 0; j <= QMAX; ++j) S.zs[j][i] = C.z[j][p];
      }
    }
  }
#define BDFB_PASCAL(Q) pascal_q<Q, NPL>(C.z)
  BDFB_DISPATCH_Q(q, BDFB_PASCAL)
#undef BDFB_PASCAL
  const double tnew = C.last ? P.tout : C.t + C.h;
  const double rl1 = P.K.rl1[q];
  const double Eq = P.K.E[q][0];
  C.gamma = C.h * rl1;
  // ---- linear setup
  int jcur = 0;
  bool fail = false;
  // |gamma / gamma_setup - 1| > 0.3 tested without a division
  const double dgam = C.gamma - C.gammap;
  if (!C.setup_done || C.force_setup || fabs(dgam) > 0.3 * fabs(C.gammap) || C.nst >= C.nstlp + 20) {
    ph_mark(PH_JAC);
    double y[NPL];
#pragma unroll
    for (int p = 0; p < NPL; ++p) y[p] = C.z[0][p];
    int info;
    if constexpr (PREC == 1) {
      // FP32 LU of M (its pivot reciprocals in the float view of dinv);
      // FP64 reaction derivatives kept for the refinement residual
      reaction_derivs<G, NPL, NMAX>(g, cd, S, y);
      C.mnorm = form_M32<G, NPL, NMAX>(g, cd, S, C.gamma);
      ph_mark(PH_LU_PIV);
      info = lu_factor<G, NMAX, float, true>(g, S.M, reinterpret_cast<float*>(S.dinv), S.perm, n);
      C.fp64mode = 0;
    } else {
      bool direct = true;
      if constexpr (CellSmem<NMAX, PREC>::DR) {
        if (cd.kind == BDFB_MASSACTION) {
          // each reaction's derivatives once (scaled by -gamma), then
          // gathered into the rows; the largest cells keep them in their
          // warp's global workspace (Mg points there)
          double (*drg)[2 * NMAX] = reinterpret_cast<double (*)[2 * NMAX]>(Mg);
          if (CellSmem<NMAX, PREC>::DRG && !drg) { C.status = BDFB_MEM_FAIL; return true; }
          reaction_derivs<G, NPL, NMAX>(g, cd, S, y, -C.gamma, drg);
          form_M64_scaled<G, NPL, NMAX>(g, cd, S, S.M, drg);
          direct = false;
        }
      }
      if (direct) form_M<G, NPL, NMAX>(g, cd, S, y, C.gamma);
      ph_mark(PH_LU_PIV);
      if constexpr (PREC == 2)   // explicit inverse: each Newton solve is one product
        info = gj_inverse<G, NMAX, double>(g, S.M, S.perm, S.ybuf, n);
      else
        info = lu_factor<G, NMAX, double, true>(g, S.M, S.dinv, S.perm, n);
    }
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
  ph_mark(PH_NEWT);
  // a stale M's step scaling 2 / (1 + gamma / gamma_setup), once per attempt
  const double scst = C.gamma != C.gammap ? 2.0 * C.gammap / (C.gammap + C.gamma) : 1.0;
  double acnrm2 = 0.0;
  bool conv = false;
  float feat = 0.f;
  if constexpr (LEARN) feat = mlp_feature(g.rank, n, C.z[0][0], C.h, rl1);
  if (!fail) {
    // pass 0 starts from the network's guess when one is loaded; if that
    // Newton solve fails, pass 1 repeats it from zero (not a step failure)
    bool guess = false;
    // the guess is consulted only after a zero-start solve that needed two
    // or more iterations: where the zero start converges in one (most
    // steps), no start can save an iteration, and an imperfect one costs one
    if constexpr (LEARN) guess = P.mlp != nullptr && C.lastit >= 2;
    const double crate0 = C.crate;
    for (int pass = 0; pass < 2 && !conv; ++pass) {
      bool nzguess = false;     // this pass starts from a nonzero guess
      if (pass == 1) {
        if (!guess) break;
        guess = false;
        C.nguess_fb++;
        C.crate = crate0;
      }
      if constexpr (LEARN) {
        if (guess) {
          C.nguess++;
          C.acor[0] = mlp_guess(P.mlp, feat, n, C.ewt[0]);
          // trust region: a correction that would fail the local error test
          // (E_q |Delta| > 1) cannot be the accepted one; such a guess is dropped
          if (!(wrms2(g, n, C.rn, C.acor, C.ewt) * Eq * Eq <= 1.0)) {
            C.acor[0] = 0.0;
            guess = false;
            C.nguess_fb++;
          }
          nzguess = __any_sync(FULL_MASK, C.acor[0] != 0.0);
        }
      }
      if (!guess) {
#pragma unroll
        for (int p = 0; p < NPL; ++p) C.acor[p] = 0.0;
      }
      double delp2 = 0.0;
      const double eq2 = Eq * Eq * 100.0;   // (E_q / 0.1)^2
      for (int it = 1; it <= 3; ++it) {
        double y[NPL];
#pragma unroll
        for (int p = 0; p < NPL; ++p) y[p] = C.z[0][p] + C.acor[p];
        rhs<G, NPL, NMAX>(g, cd, S, y, C.f);
        C.nfe++;
        if (!all_finite(g, n, C.f)) break;
#pragma unroll
        for (int p = 0; p < NPL; ++p) C.b[p] = C.gamma * C.f[p] - C.z[1][p] * rl1 - C.acor[p];
        ph_mark(PH_TRI);
        if constexpr (PREC == 1) {
          bool solved = false;
          if (!C.fp64mode) {
            double bs[NPL];
#pragma unroll
            for (int p = 0; p < NPL; ++p) bs[p] = C.b[p];
            const int sw = refined_solve<G, NPL, NMAX>(g, cd, S, C.gammap, C.mnorm, C.b);
            C.nref += sw > 0 ? sw : MAXREF;
            if (sw > 0) {
              solved = true;
            } else {
              // refinement stalled: factor this setup's M in FP64 instead (in
              // the cell's global workspace) until the next setup
              if (Mg == nullptr) { restore_z(g, n, S, C, zg); C.status = BDFB_MEM_FAIL; return true; }  // never write through null
              C.nref_fb++;
              form_M64_from_dr<G, NPL, NMAX>(g, cd, S, C.gammap, Mg);
              if (lu_factor1<G, NMAX, double, true>(g, Mg, S.dinv, S.perm, n)) {
                C.setup_done = 0;
                break;                      // singular: counts as a Newton failure
              }
              C.fp64mode = 1;
#pragma unroll
              for (int p = 0; p < NPL; ++p) C.b[p] = bs[p];
            }
          }
          if (!solved) lu_solve<G, NPL, NMAX, double, true>(g, Mg, S.dinv, S.perm, S.ybuf, n, C.b);
        } else if constexpr (PREC == 2) {
          apply_inverse<G, NPL, NMAX, double>(g, S.M, S.ybuf, n, C.b, C.b);
        } else {
          lu_solve<G, NPL, NMAX, double, true>(g, S.M, S.dinv, S.perm, S.ybuf, n, C.b);
        }
        ph_mark(PH_NEWT);
        // a stale M's step scaling, except on the first step from a nonzero
        // guess: unscaled, that step gives w.Delta = -w.z1 / l1 for every w
        // with w^T J = 0 (w^T M = w^T), so the linear invariants of the ODE
        // come out as from a zero start; a scaled one would keep a share of
        // the guess's error in them
        if (C.gamma != C.gammap && !(nzguess && it == 1)) {
#pragma unroll
          for (int p = 0; p < NPL; ++p) C.b[p] *= scst;
        }
        const double del2 = wrms2(g, n, C.rn, C.b, C.ewt);
#pragma unroll
        for (int p = 0; p < NPL; ++p) C.acor[p] += C.b[p];
        C.nni++;
        // the rate R = max(0.3 R_prev, |del| / |del_prev|) is carried squared
        // (crate holds R^2; the division only when the ratio wins)
        if (it > 1) {
          const double r2 = 0.09 * C.crate;
          C.crate = r2 * delp2 >= del2 ? r2 : del2 / delp2;
        }
        // the rate carried over from earlier solves holds between the zero
        // start and the solution; a guessed start is tested with it only when
        // the guess lies closer to the new iterate than zero does
        // (|del| <= |Delta|), else with rate 1
        double cr2 = fmin(1.0, C.crate);
        if (nzguess && it == 1 && !(del2 <= wrms2(g, n, C.rn, C.acor, C.ewt))) cr2 = 1.0;
        if (del2 * cr2 * eq2 <= 1.0) {           // |del| min(1, R) E_q / 0.1 <= 1
          acnrm2 = (it == 1 && !guess) ? del2 : wrms2(g, n, C.rn, C.acor, C.ewt);
          conv = true;
          C.lastit = guess ? 0 : it;   // only a zero start's count re-arms the guess
          break;
        }
        if (it >= 2 && del2 > 4.0 * delp2) break;  // |del| > 2 |del_prev|: diverging
        delp2 = del2;
      }
      // a guessed start whose converged correction fails the local error
      // test is redone from zero too: the test then judges the plain solve
      if (conv && guess && !(acnrm2 * Eq * Eq <= 1.0)) conv = false;
    }
    if (!conv) fail = true;
  }
  if (fail) {
    ph_mark(PH_FAIL);
    restore_z(g, n, S, C, zg);
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
    rescale(C, 0.25);
    C.qwait = C.q + 1;
    C.force_setup = 1;
    return false;
  }
  C.tried_fresh = 0;
  ph_mark(PH_ACCEPT);
  // ---- local error test
  const double dsm2 = acnrm2 * Eq * Eq;    // (E_q ||Delta||)^2
  if (!(dsm2 <= 1.0)) {
    ph_mark(PH_FAIL);
    restore_z(g, n, S, C, zg);
    C.nef++;
    C.netf++;
    if (C.nef >= 7) { C.status = BDFB_ERR_FAILURE; return true; }
    if (C.nef < 3) {
      double eta = eta64(dsm2, 36.0, 2 * (q + 1));
      if (!(eta >= 0.1)) eta = 0.1;
      if (C.nef >= 2 && eta > 0.2) eta = 0.2;
      rescale(C, eta);
      C.qwait = C.q + 1;
    } else {
      // third failure: order 1, h / 10, fresh slope
#pragma unroll
      for (int j = 2; j <= QMAX; ++j)
#pragma unroll
        for (int p = 0; p < NPL; ++p) C.z[j][p] = 0.0;
      C.q = 1;
      C.h *= 0.1;
      double y[NPL];
#pragma unroll
      for (int p = 0; p < NPL; ++p) y[p] = C.z[0][p];
      rhs<G, NPL, NMAX>(g, cd, S, y, C.f);
      C.nfe++;
      if (!all_finite(g, n, C.f)) { C.status = BDFB_RHSFUNC_FAIL; return true; }
#pragma unroll
      for (int p = 0; p < NPL; ++p) C.z[1][p] = C.h * C.f[p];
      C.qwait = 2;
    }
    return false;
  }
  // ---- accept
  if constexpr (LEARN) {
    if (P.rec_x) {
      unsigned long long idx = 0;
      if (g.rank == 0) idx = atomicAdd(P.rec_count, 1ull);
      idx = __shfl_sync(FULL_MASK, idx, 0);
      if (idx < (unsigned long long)P.rec_cap) {
        if (g.rank < MLP_NI) P.rec_x[idx * MLP_NI + g.rank] = feat;
        if (g.rank < MLP_NO) P.rec_t[idx * MLP_NO + g.rank] = g.rank < n ? (float)(C.acor[0] * C.ewt[0]) : 0.f;
      }
    }
  }
#define BDFB_CORRECT(Q) correct_q<Q, NPL>(C.z, P.K.l[q], C.acor)
  BDFB_DISPATCH_Q(q, BDFB_CORRECT)
#undef BDFB_CORRECT
  C.t = tnew;
  C.nst++;
  C.hlast = C.h;
  C.qlast = q;
  select_next(g, P, n, C.rn, C, dsm2);
#pragma unroll
  for (int p = 0; p < NPL; ++p) C.acorp[p] = C.acor[p];
  C.newstep = 1;
  if (C.last) { C.t = P.tout; C.status = 0; return true; }
  return false;
}

// doubles of one group's slice of the per-warp global workspace: mixed
// precision, the FP64 fallback matrix and, for the largest cells, the saved
// history (ZCOLS x NMAX); FP64, the largest cells' reaction derivatives
__host__ __device__ constexpr int64_t group_ws_doubles(int nmax, int pr) {
  return pr == 1 ? (int64_t)nmax * (nmax + 1) + (nmax >= 56 ? (int64_t)ZCOLS * nmax : 0)
                 : (nmax >= 56 ? 8LL * nmax : 0);
}

// fb: this warp's slice of the FP64 fallback workspace (mixed precision;
// (32 / G) matrices of NMAX x (NMAX + 1) doubles), else null
// Cells [c0, c1) of P.tile_cells on this warp: every group of G lanes takes
// the next cell from `counter` as soon as its own cell is finished, not when
// the warp's last cell is, so cells of unequal step counts that share a warp
// leave no group idle until the range is exhausted.
template <int G, int NMAX, int PREC, int LEARN = 0>
__device__ __forceinline__ void run_cells(const Params& P, int c0, int c1, unsigned* counter, char* smem,
                                          double* fb) {
  constexpr int NPL = Cell<G, NMAX>::NPL;
  Grp<G> g;
  const int gid = (threadIdx.x & 31) / G;
  CellSmem<NMAX, PREC>& S = reinterpret_cast<CellSmem<NMAX, PREC>*>(smem)[gid];
  // mixed precision: this group's FP64 fallback matrix (then, for the
  // largest cells, its saved history); the largest FP64 cells: their
  // derivative workspace (the same pointer)
  constexpr int64_t WS = group_ws_doubles(NMAX, PREC);
  double (*Mg)[NMAX + 1] = fb ? reinterpret_cast<double (*)[NMAX + 1]>(fb + (int64_t)gid * WS) : nullptr;
  bool active = false, more = true;
  int64_t c = 0;
  CellDesc cd;
  Cell<G, NMAX> C;
  ph_start(PH_TILE);
  int64_t yo = 0;
  for (;;) {
    if (!active && more) {
      int pos = 0;
      if (g.rank == 0) pos = c0 + (int)atomicAdd(counter, 1u);
      pos = g.bcast(pos, 0);
      more = pos < c1;
      if (more) {
        active = true;
        c = P.tile_cells[pos];
        if (P.kind == BDFB_ROBERTSON) {
          cd.n = 3;
          cd.nr = 0;
          cd.k = P.k + 3 * c;
          cd.reac = nullptr;
          cd.inc_off = nullptr;
          cd.inc = nullptr;
          cd.gs = nullptr;
          yo = 3 * c;
        } else {
          cd.n = P.n[c];
          yo = P.y_off[c];
          const int64_t ro = P.rxn_off[c];
          cd.nr = (int)(P.rxn_off[c + 1] - ro);
          cd.k = P.k + ro;
          cd.reac = P.reac + ro;
          cd.inc_off = P.inc_off + yo;
          cd.inc = P.inc;
          cd.gs = (P.gsched && cd.n > 32) ? P.gsched + yo : nullptr;
        }
        cd.kind = P.kind;
        const CellState s = P.st[c];
        C.t = s.t; C.h = s.h; C.gammap = s.gammap; C.crate = s.crate; C.hlast = s.hlast;
        C.q = s.q; C.qwait = s.qwait; C.nst = s.nst; C.nstlp = s.nstlp;
        C.nfe = s.nfe; C.nsetups = s.nsetups; C.nni = s.nni; C.ncfn = s.ncfn;
        C.netf = s.netf; C.flags = s.flags; C.status = 0; C.qlast = s.qlast;
        C.nst0 = C.nst; C.setup_done = 0; C.force_setup = 0; C.tried_fresh = 0;
        C.rn = 1.0 / (double)cd.n;
        C.nref = s.nrefine; C.nref_fb = s.nrefine_fb; C.fp64mode = 0; C.mnorm = 0.0;
        C.nguess = s.nguess; C.nguess_fb = s.nguess_fb; C.lastit = 0;
        C.newstep = 1; C.retry = 0; C.last = 0; C.ncf = 0; C.nef = 0; C.gamma = 0.0;
#pragma unroll
        for (int p = 0; p < NPL; ++p) {
          const int i = g.rank + G * p;
          const bool in = i < cd.n;
#pragma unroll
          for (int j = 0; j <= QMAX; ++j) C.z[j][p] = in ? P.z[(int64_t)j * P.ny + yo + i] : 0.0;
          C.acorp[p] = in ? P.acorp[yo + i] : 0.0;
          C.acor[p] = 0.0;
          C.ewt[p] = 0.0;
        }
      }
    }
    if (!__any_sync(FULL_MASK, active)) break;
    if (active && attempt<G, NMAX, PREC, LEARN>(g, P, cd, S, C, Mg)) {
      ph_mark(PH_TILE);
      active = false;
#pragma unroll
      for (int p = 0; p < NPL; ++p) {
        const int i = g.rank + G * p;
        if (i < cd.n) {
#pragma unroll
          for (int j = 0; j <= QMAX; ++j) P.z[(int64_t)j * P.ny + yo + i] = C.z[j][p];
          P.acorp[yo + i] = C.acorp[p];
          if (P.yout) {
            // the history polynomial at tout, sum_j z_j s^j with s = (tout - t) / h
            // (Horner), for a cell past tout; otherwise its current state
            double v = C.z[0][p];
            if (P.interp && C.status == 0 && (C.flags & F_STARTED) && C.t != P.tout) {
              const double sv = (P.tout - C.t) / C.h;
              v = C.z[QMAX][p];
#pragma unroll
              for (int j = QMAX - 1; j >= 0; --j) v = j < C.q ? v * sv + C.z[j][p] : C.z[j][p];
            }
            P.yout[yo + i] = v;
          }
        }
      }
      if (g.rank == 0) {
        CellState s;
        s.t = C.t; s.h = C.h; s.gammap = C.gammap; s.crate = C.crate; s.hlast = C.hlast;
        s.q = C.q; s.qwait = C.qwait; s.nst = C.nst; s.nstlp = C.nstlp;
        s.nfe = C.nfe; s.nsetups = C.nsetups; s.nni = C.nni; s.ncfn = C.ncfn;
        s.netf = C.netf; s.flags = C.flags; s.status = C.status; s.qlast = C.qlast;
        s.nrefine = C.nref; s.nrefine_fb = C.nref_fb; s.nguess = C.nguess; s.nguess_fb = C.nguess_fb;
        P.st[c] = s;
        if (P.status) P.status[c] = C.status;
        if (C.status < 0) atomicMin(P.worst, C.status);
      }
    }
  }
  ph_mark(PH_TILE);
}

// Kernel variants (cell-to-lane mappings): G lanes per cell for cells of at
// most NMAX species.  0..4 are the size classes' own tilings; 5 is one warp
// per cell of up to 16 species carrying the learned guess and the recording;
// 6 is one warp per cell of up to 32 species; 7 is 16 lanes per cell of up
// to 16 species.  A cell runs on any variant whose NMAX covers it; launches
// go largest NMAX first.
constexpr int NVAR = NCLASS + 3;
constexpr int VAR_W16 = NCLASS, VAR_W32 = NCLASS + 1, VAR_H16 = NCLASS + 2;
constexpr int VAR_G[NVAR] = {1, 4, 8, 16, 32, 32, 32, 16};
constexpr int VAR_NMAX[NVAR] = {4, 8, 16, 32, 56, 16, 32, 16};
constexpr int VAR_LEARN[NVAR] = {0, 0, 0, 0, 0, 1, 0, 0};
constexpr int VAR_ORDER[NVAR] = {4, 3, VAR_W32, VAR_W16, VAR_H16, 2, 1, 0};
// warps per SM each variant should keep resident (the shared-memory limit of
// the largest ones): bounds the registers ptxas may use
constexpr int VAR_MINB[NVAR] = {12, 12, 12, 8, 8, 12, 12, 14};   // (16, 16) at 14: 5 % faster than 12
// mixed precision: M in FP32 halves the shared memory, so registers bound the
// residency of the two largest tilings (the largest cells' saved history in
// the global workspace lets 12 warps fit)
constexpr int var_minb(int v, int prec) { return prec == 1 && v == 4 ? 12 : prec == 1 && v == 3 ? 10 : VAR_MINB[v]; }
static_assert(CLS_G[0] == VAR_G[0] && CLS_NMAX[4] == VAR_NMAX[4], "variants 0..4 are the class tilings");

// doubles of global workspace one warp of variant v needs: mixed precision,
// the FP64 fallback matrices of its cells; the FP64 kernels of the largest
// cells, their reaction derivatives (4 reactant slots x 2 NMAX reactions);
// others none
constexpr int64_t workspace_doubles_per_warp(int v, int pr) {
  return (int64_t)(32 / VAR_G[v]) * group_ws_doubles(VAR_NMAX[v], pr);
}
template <int V, int PREC>
struct VarWs {
  static constexpr int64_t value = workspace_doubles_per_warp(V, PREC);
};

template <int V, int PREC>
struct VarSmem {
  static constexpr int bytes = (32 / VAR_G[V]) * (int)sizeof(CellSmem<VAR_NMAX[V], PREC>);
};

// Persistent kernel of one variant: the cells of the tiles [t0, t1) (one
// contiguous range of P.tile_cells), each group of G lanes taking the next
// cell from `counter` until none is left.  PREC 0: FP64 LU
// factorisation; PREC 1: FP32 LU with FP64 refinement; PREC 2: FP64
// Gauss-Jordan inverse (Newton solves by one matrix-vector product).
template <int V, int PREC>
__global__ void __launch_bounds__(32, var_minb(V, PREC)) k_cells(const __grid_constant__ Params P, int t0, int t1,
                                                           unsigned* counter, double* fbws) {
  extern __shared__ __align__(16) char smem[];
  constexpr int64_t FB = VarWs<V, PREC>::value;
  double* fb = fbws ? fbws + (int64_t)blockIdx.x * FB : nullptr;
  if (t1 <= t0) return;
  const int c0 = P.tiles[t0].first;
  const TileDesc last = P.tiles[t1 - 1];
  run_cells<VAR_G[V], VAR_NMAX[V], PREC, VAR_LEARN[V]>(P, c0, last.first + last.count, counter, smem, fb);
}


typedef void (*cells_kernel_t)(const Params, int, int, unsigned*, double*);
constexpr int NKPREC = 3;   // kernel rows: FP64 LU, FP32 LU + refinement, FP64 inverse
static const cells_kernel_t CELLS_KERNELS[NKPREC][NVAR] = {
    {k_cells<0, 0>, k_cells<1, 0>, k_cells<2, 0>, k_cells<3, 0>, k_cells<4, 0>, k_cells<5, 0>, k_cells<6, 0>,
     k_cells<7, 0>},
    {k_cells<0, 1>, k_cells<1, 1>, k_cells<2, 1>, k_cells<3, 1>, k_cells<4, 1>, nullptr, k_cells<6, 1>,
     k_cells<7, 1>},
    {k_cells<0, 2>, k_cells<1, 2>, k_cells<2, 2>, k_cells<3, 2>, k_cells<4, 2>, nullptr, k_cells<6, 2>,
     k_cells<7, 2>}};
static const int CELLS_SMEM[NKPREC][NVAR] = {
    {VarSmem<0, 0>::bytes, VarSmem<1, 0>::bytes, VarSmem<2, 0>::bytes, VarSmem<3, 0>::bytes, VarSmem<4, 0>::bytes,
     VarSmem<5, 0>::bytes, VarSmem<6, 0>::bytes, VarSmem<7, 0>::bytes},
    {VarSmem<0, 1>::bytes, VarSmem<1, 1>::bytes, VarSmem<2, 1>::bytes, VarSmem<3, 1>::bytes, VarSmem<4, 1>::bytes,
     0, VarSmem<6, 1>::bytes, VarSmem<7, 1>::bytes},
    {VarSmem<0, 2>::bytes, VarSmem<1, 2>::bytes, VarSmem<2, 2>::bytes, VarSmem<3, 2>::bytes, VarSmem<4, 2>::bytes,
     0, VarSmem<6, 2>::bytes, VarSmem<7, 2>::bytes}};
static cells_kernel_t var_kernel(int pr, int v) { return CELLS_KERNELS[pr][v]; }
static int var_smem(int pr, int v) { return CELLS_SMEM[pr][v]; }

// ------------------------------------------- grouped task-local Newton mode
// The cells as ONE system (shared h and q, global error norms; the control of
// the grid integrator drives it) solved the way of the paper's demo (Sec. 7):
// every cell runs its own Newton iteration with its own convergence test and
// a direct solve of its block, and if any cell fails the whole step is
// retried with a smaller step size.  Jacobian LU factors persist between the
// host-driven steps in global memory (lu: n x n per cell, row-major).
struct GroupParams {
  Params P;                      // cell data, tiles of the size-class schedule
  int mode;                      // 0: Newton solve, 1: right-hand side
  int setup;                     // fresh Jacobians at zp0 first
  double gamma, gammap, rl1, Eq;
  const double* zp0;             // predicted state / RHS input (mode 1)
  const double* zp1;
  const double* ewt;
  double* out;                   // Newton: converged correction; RHS: f
  double* lu;                    // per-cell factors, offsets lu_off
  const int64_t* lu_off;
  double* dinv;                  // per species
  int16_t* perm;                 // per species
  double* crate;                 // per cell: the squared Newton rate R^2
  int* failed;
  unsigned long long* iters;     // [0] completed iterations (sum), [1] RHS evaluations (max)
};

template <int G, int NMAX>
__device__ __forceinline__ void group_cell(const Grp<G>& g, const GroupParams& GP, CellSmem<NMAX, 0>& S,
                                           int64_t c) {
  constexpr int NPL = (NMAX + G - 1) / G;
  const Params& P = GP.P;
  CellDesc cd;
  int64_t yo;
  if (P.kind == BDFB_ROBERTSON) {
    cd.n = 3; cd.nr = 0; cd.k = P.k + 3 * c; cd.reac = nullptr; cd.inc_off = nullptr; cd.inc = nullptr;
    cd.gs = nullptr;
    yo = 3 * c;
  } else {
    cd.n = P.n[c];
    yo = P.y_off[c];
    const int64_t ro = P.rxn_off[c];
    cd.nr = (int)(P.rxn_off[c + 1] - ro);
    cd.k = P.k + ro;
    cd.reac = P.reac + ro;
    cd.inc_off = P.inc_off + yo;
    cd.inc = P.inc;
    cd.gs = nullptr;
  }
  cd.kind = P.kind;
  const int n = cd.n;
  double z0[NPL], z1[NPL], w[NPL];
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    const bool in = i < n;
    z0[p] = in ? GP.zp0[yo + i] : 0.0;
    z1[p] = in && GP.mode == 0 ? GP.zp1[yo + i] : 0.0;
    w[p] = in && GP.mode == 0 ? GP.ewt[yo + i] : 0.0;
  }
  if (GP.mode == 1) {
    double f[NPL];
    rhs<G, NPL, NMAX>(g, cd, S, z0, f);
#pragma unroll
    for (int p = 0; p < NPL; ++p) {
      const int i = g.rank + G * p;
      if (i < n) GP.out[yo + i] = f[p];
    }
    return;
  }
  double* lu = GP.lu + GP.lu_off[c];
  double crate = GP.crate[c];
  if (GP.setup) {
    bool direct = true;
    if constexpr (CellSmem<NMAX, 0>::DR && !CellSmem<NMAX, 0>::DRG) {
      if (cd.kind == BDFB_MASSACTION) {
        reaction_derivs<G, NPL, NMAX>(g, cd, S, z0, -GP.gamma);
        form_M64_scaled<G, NPL, NMAX>(g, cd, S, S.M);
        direct = false;
      }
    }
    if (direct) form_M<G, NPL, NMAX>(g, cd, S, z0, GP.gamma);
    int info = lu_factor<G, NMAX, double, true>(g, S.M, S.dinv, S.perm, n);
    crate = 1.0;
    if (info) {                   // singular block: the step fails
      if (g.rank == 0) atomicOr(GP.failed, 1);
      if (g.rank == 0) GP.crate[c] = crate;
      return;
    }
    for (int e = g.rank; e < n * n; e += G) lu[e] = S.M[e / n][e % n];
    for (int i = g.rank; i < n; i += G) { GP.dinv[yo + i] = S.dinv[i]; GP.perm[yo + i] = S.perm[i]; }
  } else {
    for (int e = g.rank; e < n * n; e += G) S.M[e / n][e % n] = lu[e];
    for (int i = g.rank; i < n; i += G) { S.dinv[i] = GP.dinv[yo + i]; S.perm[i] = GP.perm[yo + i]; }
  }
  g.sync();
  const double rn = 1.0 / (double)n;
  const double eq2 = GP.Eq * GP.Eq * 100.0;
  const double scst = GP.gamma != GP.gammap ? 2.0 / (1.0 + GP.gamma / GP.gammap) : 1.0;
  double acor[NPL], f[NPL], b[NPL];
#pragma unroll
  for (int p = 0; p < NPL; ++p) acor[p] = 0.0;
  double delp2 = 0.0;
  bool conv = false;
  int it = 1, nit = 0;
  for (; it <= 3; ++it) {
    double y[NPL];
#pragma unroll
    for (int p = 0; p < NPL; ++p) y[p] = z0[p] + acor[p];
    rhs<G, NPL, NMAX>(g, cd, S, y, f);
    if (!all_finite(g, n, f)) break;
    ++nit;
#pragma unroll
    for (int p = 0; p < NPL; ++p) b[p] = GP.gamma * f[p] - z1[p] * GP.rl1 - acor[p];
    lu_solve<G, NPL, NMAX, double, true>(g, S.M, S.dinv, S.perm, S.ybuf, n, b);
    if (GP.gamma != GP.gammap) {
#pragma unroll
      for (int p = 0; p < NPL; ++p) b[p] *= scst;
    }
    const double del2 = wrms2(g, n, rn, b, w);
#pragma unroll
    for (int p = 0; p < NPL; ++p) acor[p] += b[p];
    if (it > 1) {                 // R^2 = max(0.09 R_prev^2, del2 / delp2)
      const double r2 = 0.09 * crate;
      crate = r2 * delp2 >= del2 ? r2 : del2 / delp2;
    }
    if (del2 * fmin(1.0, crate) * eq2 <= 1.0) { conv = true; break; }
    if (it >= 2 && del2 > 4.0 * delp2) break;
    delp2 = del2;
  }
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    if (i < n) GP.out[yo + i] = acor[p];
  }
  if (g.rank == 0) {
    GP.crate[c] = crate;
    atomicAdd(GP.iters, (unsigned long long)nit);
    atomicMax(GP.iters + 1, (unsigned long long)(it > 3 ? 3 : it));
    if (!conv) atomicOr(GP.failed, 1);
  }
}

template <int V>
__global__ void __launch_bounds__(32, VAR_MINB[V]) k_group(const __grid_constant__ GroupParams GP, int t0, int t1,
                                                           unsigned* counter) {
  static_assert(V < NCLASS, "grouped mode runs on the size classes' own tilings");
  constexpr int G = VAR_G[V], NMAX = VAR_NMAX[V];
  extern __shared__ __align__(16) char smem[];
  const int lane = threadIdx.x & 31;
  Grp<G> g;
  const int gid = lane / G;
  CellSmem<NMAX, 0>& S = reinterpret_cast<CellSmem<NMAX, 0>*>(smem)[gid];
  for (;;) {
    int t = 0;
    if (lane == 0) t = t0 + (int)atomicAdd(counter, 1u);
    t = __shfl_sync(FULL_MASK, t, 0);
    if (t >= t1) break;
    const TileDesc td = GP.P.tiles[t];
    if (gid < td.count) group_cell<G, NMAX>(g, GP, S, GP.P.tile_cells[td.first + gid]);
    __syncwarp();
  }
}

typedef void (*group_kernel_t)(const GroupParams, int, int, unsigned*);
static const group_kernel_t GROUP_KERNELS[NCLASS] = {k_group<0>, k_group<1>, k_group<2>, k_group<3>, k_group<4>};

// ------------------------------------------------- standalone batched LU
constexpr int LU_NMAX = 64;

__global__ void __launch_bounds__(32) k_lu_factor(int64_t nb, int n, double* a, int32_t* piv,
                                                  int32_t* info) {
  extern __shared__ __align__(16) char smem[];
  auto& S = *reinterpret_cast<CellSmem<LU_NMAX>*>(smem);
  int16_t* pk = reinterpret_cast<int16_t*>(smem + sizeof(CellSmem<LU_NMAX>));
  Grp<32> g;
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    double* A = a + b * n * n;
    for (int e = g.rank; e < n * n; e += 32) S.M[e / n][e % n] = A[e];
    g.sync();
    for (int e = g.rank; e < n; e += 32) pk[e] = (int16_t)e;
    g.sync();
    const int r = lu_factor<32, LU_NMAX, double>(g, S.M, S.dinv, S.perm, n, pk);
    for (int e = g.rank; e < n * n; e += 32) A[e] = S.M[e / n][e % n];
    for (int e = g.rank; e < n; e += 32) piv[b * n + e] = pk[e];
    if (g.rank == 0) info[b] = r;
    g.sync();
  }
}

__global__ void __launch_bounds__(32) k_lu_solve(int64_t nb, int n, const double* lu,
                                                 const int32_t* piv, double* bvec) {
  extern __shared__ __align__(16) char smem[];
  auto& S = *reinterpret_cast<CellSmem<LU_NMAX>*>(smem);
  Grp<32> g;
  constexpr int NPL = 2;
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    const double* A = lu + b * n * n;
    for (int e = g.rank; e < n * n; e += 32) S.M[e / n][e % n] = A[e];
    for (int e = g.rank; e < n; e += 32) S.dinv[e] = 1.0 / A[e * n + e];
    if (g.rank == 0) {                       // compose the row swaps into a permutation
      for (int e = 0; e < n; ++e) S.perm[e] = (int16_t)e;
      for (int e = 0; e < n; ++e) {
        const int p = piv[b * n + e];
        const int16_t t = S.perm[e];
        S.perm[e] = S.perm[p];
        S.perm[p] = t;
      }
    }
    g.sync();
    double x[NPL];
#pragma unroll
    for (int p = 0; p < NPL; ++p) {
      const int i = g.rank + 32 * p;
      x[p] = i < n ? bvec[b * n + i] : 0.0;
    }
    lu_solve<32, NPL, LU_NMAX, double>(g, S.M, S.dinv, S.perm, S.ybuf, n, x);
#pragma unroll
    for (int p = 0; p < NPL; ++p) {
      const int i = g.rank + 32 * p;
      if (i < n) bvec[b * n + i] = x[p];
    }
    g.sync();
  }
}

// Mixed-precision solve of dense blocks, the same scheme as the integrator's:
// FP32 LU of each block, FP64 dense residual r = b - A x, x += (LU32)^{-1} r
// until |r|/(|A| |x| + |b|) <= 1e-12 (at most MAXREF sweeps);
// a block that does not get there is solved by FP64 LU (sweeps[b] = 0), and
// sweeps[b] = -2 only when that factorisation meets a zero pivot too.
__global__ void __launch_bounds__(32) k_solve_mixed(int64_t nb, int n, const double* a,
                                                   const double* bvec, double* xout, int32_t* sweeps) {
  extern __shared__ __align__(16) char smem[];
  auto& S = *reinterpret_cast<CellSmem<LU_NMAX, 1>*>(smem);
  double (*A)[LU_NMAX + 1] = reinterpret_cast<double (*)[LU_NMAX + 1]>(smem + sizeof(CellSmem<LU_NMAX, 1>));
  float (*M32)[LU_NMAX + 1] = reinterpret_cast<float (*)[LU_NMAX + 1]>(&S.M[0][0]);
  Grp<32> g;
  constexpr int NPL = 2;
  for (int64_t blk = blockIdx.x; blk < nb; blk += gridDim.x) {
    const double* Ab = a + blk * n * n;
    for (int e = g.rank; e < n * n; e += 32) {
      const double v = Ab[e];
      A[e / n][e % n] = v;
      M32[e / n][e % n] = (float)v;
    }
    g.sync();
    double anorm = 0.0;
#pragma unroll
    for (int p = 0; p < NPL; ++p) {
      const int i = g.rank + 32 * p;
      if (i < n) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += fabs(A[i][j]);
        anorm = fmax(anorm, s);
      }
    }
    anorm = gmaxd(g, anorm);
    float* dinv32 = reinterpret_cast<float*>(S.dinv);
    const int info = lu_factor<32, LU_NMAX, float, true>(g, M32, dinv32, S.perm, n);
    double b[NPL], x[NPL], r[NPL];
    double bn = 0.0;
#pragma unroll
    for (int p = 0; p < NPL; ++p) {
      const int i = g.rank + 32 * p;
      b[p] = i < n ? bvec[blk * n + i] : 0.0;
      x[p] = 0.0;
      r[p] = b[p];
      bn = fmax(bn, fabs(b[p]));
    }
    bn = gmaxd(g, bn);
    int sw = -1;
    for (int it = 1; it <= MAXREF && !info; ++it) {
      float c32[NPL];
#pragma unroll
      for (int p = 0; p < NPL; ++p) c32[p] = (float)r[p];
      lu_solve<32, NPL, LU_NMAX, float, true, float>(g, M32, dinv32, S.perm, reinterpret_cast<float*>(S.ybuf), n,
                                                     c32);
#pragma unroll
      for (int p = 0; p < NPL; ++p) x[p] += (double)c32[p];
      g.sync();
#pragma unroll
      for (int p = 0; p < NPL; ++p) {
        const int i = g.rank + 32 * p;
        if (i < n) S.rates[i] = x[p];
      }
      g.sync();
      double rn = 0.0, xn = 0.0;
#pragma unroll
      for (int p = 0; p < NPL; ++p) {
        const int i = g.rank + 32 * p;
        if (i < n) {
          double s = b[p];
          for (int j = 0; j < n; ++j) s = fma(-A[i][j], S.rates[j], s);
          r[p] = s;
          rn = fmax(rn, fabs(s));
          xn = fmax(xn, fabs(x[p]));
        }
      }
      rn = gmaxd(g, rn);
      xn = gmaxd(g, xn);
      if (rn <= BERR_TOL * (anorm * xn + bn)) { sw = it; break; }
    }
    if (sw < 0) {
      // refinement stalled (or the FP32 factorisation met a zero pivot): the
      // block is factored and solved in FP64 instead, as the integrator does
      g.sync();
      if (lu_factor<32, LU_NMAX, double>(g, A, S.dinv, S.perm, n) == 0) {
#pragma unroll
        for (int p = 0; p < NPL; ++p) x[p] = b[p];
        lu_solve<32, NPL, LU_NMAX, double>(g, A, S.dinv, S.perm, S.ybuf, n, x);
        sw = 0;
      } else {
        sw = -2;
      }
    }
#pragma unroll
    for (int p = 0; p < NPL; ++p) {
      const int i = g.rank + 32 * p;
      if (i < n) xout[blk * n + i] = x[p];
    }
    if (g.rank == 0) sweeps[blk] = sw;
    g.sync();
  }
}



}  // namespace bdfb

using namespace bdfb;

// ---------------------------------------------------------------- context
struct Sched {
  TileDesc* d_tiles = nullptr;
  int32_t* d_tcells = nullptr;
  int ntiles = 0;
  int vbeg[NVAR] = {}, vend[NVAR] = {};   // tile range of each variant
};

struct bdfb_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int kind = 0;
  int64_t ncell = 0, ny = 0, nrxn = 0;
  std::vector<int32_t> h_n;
  std::vector<int64_t> h_yoff;
  int32_t* d_n = nullptr;
  int64_t* d_yoff = nullptr;
  int64_t* d_rxnoff = nullptr;
  uint32_t* d_reac = nullptr;
  double* d_k = nullptr;
  int32_t* d_incoff = nullptr;
  uint16_t* d_inc = nullptr;
  uint32_t* d_gsched = nullptr;   // gather schedules (cells of more than 32 species), or null
  CellState* d_state = nullptr;
  double* d_z = nullptr;
  double* d_acorp = nullptr;
  // schedules: [0] size-class tiles, [1] one cell per warp in input order,
  // [2] size classes on the variants the autotuner picked
  Sched sched[3];
  int sched_gen = 0;               // bumped whenever a schedule is rebuilt
  std::vector<int8_t> h_cls;       // size class of every cell
  unsigned* d_counter = nullptr;   // [v] tile counter of variant v, [NVAR] worst status (int)
  int autotune = 0;                // option "autotune"
  int tuned_prec = -1;             // precision the tuned schedule was made for (-1: none)
  int tuned_var[NCLASS] = {};      // variant picked for each size class
  float tune_ms[NCLASS][NVAR] = {};  // trial times, 0 = not tried
  // CUDA graph of the launch sequence (option "graph")
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t cgraph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  Params gkey;                     // Params of the capture with tout = 0
  int gkey_gen = -1, gkey_m = -1, gkey_single = -1, gkey_rows = -1;
  int64_t graph_launches = 0, graph_captures = 0;
  int32_t* d_status = nullptr;
  double rtol = 1e-6, atol = 1e-10;
  int64_t mxstep = 100000;
  int mapping = 0, precision = 0, graph = 0, qmax = QMAX;
  int lsolver = 0;            // 1: FP64 Gauss-Jordan inverse instead of LU
  int mixed_small = 0;        // precision 1: cells of at most 32 species get FP32 factors too
  double t0 = 0.0;
  bool initialized = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evfork = nullptr;
  cudaEvent_t evjoin[NVAR] = {};
  double* d_fbws[NKPREC][NVAR] = {};   // global workspace per kernel row and variant (lazy)
  cudaStream_t cstream[NVAR] = {};  // one per variant, forked from `stream`
  float last_ms = 0.f;
  int pgrid[NKPREC][NVAR] = {};   // persistent grid size [kernel row][variant]
  GridBDF* grid = nullptr;    // BDFB_BRUSSELATOR3D / 1D: the grouped grid integrator
  ArkLine* ark = nullptr;     // BDFB_BRUSSELATOR1D with option "imex": the IMEX ARK integrator
  SharedInt* shared = nullptr;  // BDFB_MASSACTION_SHARED: grouped cells on one sparse network
  int imex = 0;
  int line_prec = 0;          // "precision" of the IMEX path
  int line_dloop = -1;        // "device_loop" of the IMEX path (-1: by size)
  double line_par[6] = {};    // A, B, eps, c, length, nx of the 1-D line
  // option "grouped": the cells as one system with task-local Newton solves
  int grouped = 0;
  // option "interp": output by interpolation past tout; the output buffer
  int interp = 0;
  double* d_yout = nullptr;
  bool gfresh = true;         // the grouped integrator needs the state of bdfb_init
  GridBDF* gg = nullptr;
  double* d_glu = nullptr;    // per-cell LU factors (n x n each)
  int64_t* d_gluoff = nullptr;
  double* d_gdinv = nullptr;
  int16_t* d_gperm = nullptr;
  double* d_gcrate = nullptr;
  int* d_gflag = nullptr;
  unsigned long long* d_giters = nullptr;
  int gpgrid[NCLASS] = {};
  int maxn = 0;               // largest cell
  bool fits_w16 = false;      // every cell fits the NMAX 16 shared-memory layout
  bool fits_w32 = false;      // every cell fits the NMAX 32 shared-memory layout
  int predictor = 0;          // 1: Newton starts from the learned guess
  const void* mlp = nullptr;  // packed network (caller-owned device memory)
  float* rec_x = nullptr;     // recording buffers (caller-owned device memory)
  float* rec_t = nullptr;
  int64_t rec_cap = 0;
  unsigned long long* rec_count = nullptr;
};

static void free_ctx(bdfb_ctx* c) {
  if (!c) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(c->device);
  grid_destroy(c->grid);
  ark_destroy(c->ark);
  shared_destroy(c->shared);
  grid_destroy(c->gg);
  cudaFree(c->d_glu); cudaFree(c->d_gluoff); cudaFree(c->d_gdinv); cudaFree(c->d_gperm);
  cudaFree(c->d_gcrate); cudaFree(c->d_gflag); cudaFree(c->d_giters);
  cudaFree(c->d_n); cudaFree(c->d_yoff); cudaFree(c->d_rxnoff); cudaFree(c->d_reac);
  cudaFree(c->d_k); cudaFree(c->d_incoff); cudaFree(c->d_inc); cudaFree(c->d_gsched); cudaFree(c->d_state);
  cudaFree(c->d_z); cudaFree(c->d_acorp); cudaFree(c->d_counter); cudaFree(c->d_status); cudaFree(c->d_yout);
  for (int pr = 0; pr < NKPREC; ++pr)
    for (int k = 0; k < NVAR; ++k) cudaFree(c->d_fbws[pr][k]);
  for (int m = 0; m < 3; ++m) { cudaFree(c->sched[m].d_tiles); cudaFree(c->sched[m].d_tcells); }
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->cgraph) cudaGraphDestroy(c->cgraph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->evfork) cudaEventDestroy(c->evfork);
  for (int k = 0; k < NVAR; ++k) {
    if (c->evjoin[k]) cudaEventDestroy(c->evjoin[k]);
    if (c->cstream[k]) cudaStreamDestroy(c->cstream[k]);
  }
  cudaSetDevice(prev);
  delete c;
}

template <typename T>
static int dev_alloc_copy(T** dst, const T* src, size_t count) {
  if (count == 0) count = 1;
  BDFB_CUDA(cudaMalloc(dst, count * sizeof(T)));
  if (src) BDFB_CUDA(cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice));
  return 0;
}

// copy `count` elements from caller memory (host or device) into a host vector
template <typename T>
static int fetch(std::vector<T>& out, const T* src, size_t count, int mem) {
  out.resize(count);
  if (count == 0) return 0;
  if (!src) return BDFB_ILL_INPUT;
  if (mem == BDFB_MEM_DEVICE) {
    BDFB_CUDA(cudaMemcpy(out.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(out.data(), src, count * sizeof(T));
  }
  return 0;
}

// events, per-class streams and persistent grid sizes (resident warps per SM
// x SM count) of every class kernel
static int setup_launch(bdfb_ctx* c) {
  BDFB_CUDA(cudaEventCreate(&c->ev0));
  BDFB_CUDA(cudaEventCreate(&c->ev1));
  BDFB_CUDA(cudaEventCreateWithFlags(&c->evfork, cudaEventDisableTiming));
  BDFB_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  for (int k = 0; k < NVAR; ++k) {
    BDFB_CUDA(cudaEventCreateWithFlags(&c->evjoin[k], cudaEventDisableTiming));
    BDFB_CUDA(cudaStreamCreateWithFlags(&c->cstream[k], cudaStreamNonBlocking));
    for (int pr = 0; pr < NKPREC; ++pr) {
      const cells_kernel_t kf = var_kernel(pr, k);
      if (!kf) continue;
      BDFB_CUDA(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, var_smem(pr, k)));
      int per_sm = 0;
      BDFB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kf, 32, var_smem(pr, k)));
      c->pgrid[pr][k] = std::max(1, per_sm) * sm_count();
    }
  }
  return 0;
}

// Tiles of the cells in `order`, grouped by variant in launch order (the
// caller sorts `order` so that each variant's cells are contiguous): 32 / G
// cells of one variant per tile, or one cell per tile when `single`.
static void make_tiles(const std::vector<int32_t>& order, const std::vector<int8_t>& var, bool single,
                       std::vector<TileDesc>& tiles, std::vector<int32_t>& tcells, int* vbeg, int* vend) {
  tiles.clear();
  tcells.clear();
  for (int v = 0; v < NVAR; ++v) { vbeg[v] = 0; vend[v] = 0; }
  size_t i = 0;
  while (i < order.size()) {
    const int v = var[order[i]];
    const int cpt = single ? 1 : 32 / VAR_G[v];
    TileDesc td;
    td.cls = v;
    td.first = (int32_t)tcells.size();
    td.count = 0;
    td.pad = 0;
    while (i < order.size() && var[order[i]] == v && td.count < cpt) {
      tcells.push_back(order[i]);
      ++td.count;
      ++i;
    }
    const int t = (int)tiles.size();
    if (vend[v] == 0) vbeg[v] = t;
    vend[v] = t + 1;
    tiles.push_back(td);
  }
}

// cells grouped by variant in launch order, larger cells first within one
static std::vector<int32_t> launch_order(const std::vector<int8_t>& var, const std::vector<int32_t>& n,
                                         const std::vector<int32_t>& cells) {
  int rank[NVAR];
  for (int k = 0; k < NVAR; ++k) rank[VAR_ORDER[k]] = k;
  std::vector<int32_t> order(cells);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    if (var[a] != var[b]) return rank[var[a]] < rank[var[b]];
    return n[a] > n[b];
  });
  return order;
}

static int upload_sched(bdfb_ctx* c, int m, const std::vector<int32_t>& order, const std::vector<int8_t>& var,
                        bool single) {
  std::vector<TileDesc> tiles;
  std::vector<int32_t> tcells;
  Sched& S = c->sched[m];
  make_tiles(order, var, single, tiles, tcells, S.vbeg, S.vend);
  cudaFree(S.d_tiles);
  cudaFree(S.d_tcells);
  S.d_tiles = nullptr;
  S.d_tcells = nullptr;
  S.ntiles = (int)tiles.size();
  c->sched_gen++;
  int r = dev_alloc_copy(&S.d_tiles, tiles.data(), tiles.size());
  if (r) return r;
  return dev_alloc_copy(&S.d_tcells, tcells.data(), tcells.size());
}

static int class_of(int n, int nr) {
  const int need = std::max(n, (nr + 1) / 2);
  for (int c = 0; c < NCLASS; ++c)
    if (need <= CLS_NMAX[c]) return c;
  return -1;
}

#define TRY(x)                  \
  do {                          \
    int r_ = (x);               \
    if (r_) { free_ctx(c); return r_; } \
  } while (0)

extern "C" int bdfb_create(const bdfb_problem* prob, bdfb_ctx** out) {
  if (!prob || !out) return BDFB_ILL_INPUT;
  *out = nullptr;
  if (prob->ncell < 0 ||
      (prob->kind != BDFB_ROBERTSON && prob->kind != BDFB_MASSACTION && prob->kind != BDFB_BRUSSELATOR3D &&
       prob->kind != BDFB_BRUSSELATOR1D && prob->kind != BDFB_MASSACTION_SHARED) ||
      (prob->mem != BDFB_MEM_HOST && prob->mem != BDFB_MEM_DEVICE) || !prob->k)
    return BDFB_ILL_INPUT;
  bdfb_ctx* c = new (std::nothrow) bdfb_ctx();
  if (!c) return BDFB_MEM_FAIL;
  cudaGetDevice(&c->device);
  c->kind = prob->kind;
  c->ncell = prob->ncell;
  if (prob->kind == BDFB_MASSACTION_SHARED) {   // grouped cells on one sparse network
    TRY(shared_create(prob, &c->shared));
    c->ny = (int64_t)prob->n[0] * prob->ncell;
    BDFB_CUDA(cudaEventCreate(&c->ev0));
    BDFB_CUDA(cudaEventCreate(&c->ev1));
    *out = c;
    return BDFB_SUCCESS;
  }
  if (prob->kind == BDFB_BRUSSELATOR3D) {   // one coupled system on a grid
    std::vector<double> par;
    TRY(fetch(par, prob->k, 5, prob->mem));
    const int nx = (int)par[4];
    if ((double)nx != par[4] || (int64_t)nx * nx * nx != prob->ncell) { free_ctx(c); return BDFB_ILL_INPUT; }
    TRY(grid_create(nx, par[0], par[1], par[2], par[3], &c->grid));
    c->ny = 3 * prob->ncell;
    BDFB_CUDA(cudaEventCreate(&c->ev0));
    BDFB_CUDA(cudaEventCreate(&c->ev1));
    *out = c;
    return BDFB_SUCCESS;
  }
  if (prob->kind == BDFB_BRUSSELATOR1D) {   // the demo's advection-reaction line
    std::vector<double> par;
    TRY(fetch(par, prob->k, 6, prob->mem));
    const int64_t nx = (int64_t)par[5];
    if ((double)nx != par[5] || nx != prob->ncell) { free_ctx(c); return BDFB_ILL_INPUT; }
    TRY(grid_create_line_or_cube(1, nx, par[0], par[1], par[2], 0.0, par[3], par[4], &c->grid));
    for (int i = 0; i < 6; ++i) c->line_par[i] = par[i];
    c->ny = 3 * prob->ncell;
    BDFB_CUDA(cudaEventCreate(&c->ev0));
    BDFB_CUDA(cudaEventCreate(&c->ev1));
    *out = c;
    return BDFB_SUCCESS;
  }
  const int64_t C = prob->ncell;
  std::vector<int32_t> n;
  std::vector<int64_t> yoff, roff;
  std::vector<uint8_t> reac, prod;
  std::vector<double> k;
  std::vector<int32_t> cls(C);
  if (prob->kind == BDFB_ROBERTSON) {
    n.assign(C, 3);
    yoff.resize(C + 1);
    for (int64_t i = 0; i <= C; ++i) yoff[i] = 3 * i;
    TRY(fetch(k, prob->k, 3 * C, prob->mem));
    for (int64_t i = 0; i < C; ++i) cls[i] = 0;
  } else {
    if (!prob->n || !prob->y_off || !prob->rxn_off || !prob->reactants || !prob->products) {
      free_ctx(c);
      return BDFB_ILL_INPUT;
    }
    TRY(fetch(n, prob->n, C, prob->mem));
    TRY(fetch(yoff, prob->y_off, C + 1, prob->mem));
    TRY(fetch(roff, prob->rxn_off, C + 1, prob->mem));
    if (yoff[0] != 0 || roff[0] != 0) { free_ctx(c); return BDFB_ILL_INPUT; }
    for (int64_t i = 0; i < C; ++i) {
      const int64_t nr = roff[i + 1] - roff[i];
      if (n[i] < 1 || n[i] > NMAX_ALL || yoff[i + 1] - yoff[i] != n[i] || nr < 0 ||
          nr > 2 * NMAX_ALL) {
        free_ctx(c);
        return BDFB_ILL_INPUT;
      }
      cls[i] = class_of(n[i], (int)nr);
    }
    const int64_t nrxn = roff[C];
    TRY(fetch(reac, prob->reactants, 4 * nrxn, prob->mem));
    TRY(fetch(prod, prob->products, 4 * nrxn, prob->mem));
    TRY(fetch(k, prob->k, nrxn, prob->mem));
    c->nrxn = nrxn;
  }
  c->ny = yoff[C];
  for (int64_t i = 0; i < C; ++i) c->maxn = std::max(c->maxn, n[i]);
  c->fits_w16 = true;
  c->fits_w32 = true;
  for (int64_t i = 0; i < C; ++i) {
    if (cls[i] > 2) c->fits_w16 = false;    // class 2 has NMAX 16
    if (cls[i] > 3) c->fits_w32 = false;    // class 3 has NMAX 32
  }
  c->h_n = n;
  c->h_yoff = yoff;
  if (prob->kind == BDFB_MASSACTION) {
    // validate species and build the species-major incidence lists (reaction
    // order; a reaction's consumption entry before its production entry)
    std::vector<int32_t> incoff(c->ny + 1, 0);
    std::vector<uint32_t> reac32(c->nrxn);
    for (int64_t cc = 0; cc < C; ++cc) {
      const int nn = n[cc];
      for (int64_t r = roff[cc]; r < roff[cc + 1]; ++r) {
        uint32_t w = 0;
        for (int a = 0; a < 4; ++a) {
          const uint8_t s = reac[4 * r + a], p = prod[4 * r + a];
          if ((s != 255 && s >= nn) || (p != 255 && p >= nn)) { free_ctx(c); return BDFB_ILL_INPUT; }
          for (int b2 = 0; b2 < a; ++b2)
            if (s != 255 && reac[4 * r + b2] == s) { free_ctx(c); return BDFB_ILL_INPUT; }
          w |= (uint32_t)s << (8 * a);
          if (s != 255) incoff[yoff[cc] + s + 1]++;
          if (p != 255) incoff[yoff[cc] + p + 1]++;
        }
        reac32[r] = w;
      }
    }
    for (int64_t i = 0; i < c->ny; ++i) incoff[i + 1] += incoff[i];
    if (incoff[c->ny] < 0 || (int64_t)incoff[c->ny] > (int64_t)0x7fffffff) { free_ctx(c); return BDFB_ILL_INPUT; }
    std::vector<uint16_t> inc(std::max<int64_t>(1, incoff[c->ny]));
    std::vector<int32_t> fill(incoff.begin(), incoff.end() - 1);
    for (int64_t cc = 0; cc < C; ++cc)
      for (int64_t r = roff[cc]; r < roff[cc + 1]; ++r) {
        const uint16_t rl = (uint16_t)(r - roff[cc]);
        for (int a = 0; a < 4; ++a) {
          const uint8_t s = reac[4 * r + a];
          if (s != 255) inc[fill[yoff[cc] + s]++] = (uint16_t)(rl << 1);
        }
        for (int a = 0; a < 4; ++a) {
          const uint8_t p = prod[4 * r + a];
          if (p != 255) inc[fill[yoff[cc] + p]++] = (uint16_t)((rl << 1) | 1u);
        }
      }
    TRY(dev_alloc_copy(&c->d_n, n.data(), n.size()));
    TRY(dev_alloc_copy(&c->d_yoff, yoff.data(), yoff.size()));
    TRY(dev_alloc_copy(&c->d_rxnoff, roff.data(), roff.size()));
    TRY(dev_alloc_copy(&c->d_reac, reac32.data(), reac32.size()));
    TRY(dev_alloc_copy(&c->d_incoff, incoff.data(), incoff.size()));
    TRY(dev_alloc_copy(&c->d_inc, inc.data(), inc.size()));
    // gather schedules of the cells of more than 32 species (one warp per
    // cell): entries y_off .. y_off + 31 of a per-species array hold lane l's
    // species, up to four bytes (255 = none).  Species in decreasing order of
    // cost (4-entry trips of the gather loop, plus one for the switch), ties
    // by index, each to the lane with the least cost so far (ties: lowest
    // lane) that has a free byte.
    bool any_big = false;
    for (int64_t cc = 0; cc < C; ++cc) any_big = any_big || n[cc] > 32;
    if (any_big) {
      std::vector<uint32_t> gs(c->ny, 0xffffffffu);
      std::vector<int> ord;
      for (int64_t cc = 0; cc < C; ++cc) {
        const int nn = n[cc];
        if (nn <= 32) continue;
        auto cost = [&](int sp) {
          const int len = incoff[yoff[cc] + sp + 1] - incoff[yoff[cc] + sp];
          return (len + 3) / 4 + 1;
        };
        ord.resize(nn);
        for (int sp = 0; sp < nn; ++sp) ord[sp] = sp;
        std::stable_sort(ord.begin(), ord.end(), [&](int a2, int b2) { return cost(a2) > cost(b2); });
        int load[32] = {0}, cnt[32] = {0};
        for (int sp : ord) {
          int best = -1;
          for (int l = 0; l < 32; ++l)
            if (cnt[l] < 4 && (best < 0 || load[l] < load[best])) best = l;
          if (best < 0) { free_ctx(c); return BDFB_ILL_INPUT; }   // n > 128: not a one-warp cell
          uint32_t& w = gs[yoff[cc] + best];
          w = (w & ~(0xffu << (8 * cnt[best]))) | ((uint32_t)sp << (8 * cnt[best]));
          cnt[best]++;
          load[best] += cost(sp);
        }
      }
      TRY(dev_alloc_copy(&c->d_gsched, gs.data(), gs.size()));
    }
  }
  TRY(dev_alloc_copy(&c->d_k, k.data(), k.size()));
  // schedules: [0] tiles by size class, largest class first; [1] one cell
  // per warp in input order (all on the NMAX 56 variant; launched on the
  // NMAX 16 one-warp kernel when every cell fits it)
  c->h_cls.assign(C, 0);
  for (int64_t i = 0; i < C; ++i) c->h_cls[i] = (int8_t)cls[i];
  {
    std::vector<int32_t> all(C);
    for (int64_t i = 0; i < C; ++i) all[i] = (int32_t)i;
    TRY(upload_sched(c, 0, launch_order(c->h_cls, n, all), c->h_cls, false));
    std::vector<int8_t> v4(C, 4);
    TRY(upload_sched(c, 1, all, v4, true));
  }
  TRY(dev_alloc_copy<CellState>(&c->d_state, nullptr, C));
  TRY(dev_alloc_copy<double>(&c->d_z, nullptr, 6 * std::max<int64_t>(c->ny, 1)));
  TRY(dev_alloc_copy<double>(&c->d_acorp, nullptr, c->ny));
  TRY(dev_alloc_copy<unsigned>(&c->d_counter, nullptr, NVAR + 1));
  TRY(dev_alloc_copy<int32_t>(&c->d_status, nullptr, C));
  TRY(setup_launch(c));
  *out = c;
  return BDFB_SUCCESS;
}

extern "C" void bdfb_destroy(bdfb_ctx* ctx) { free_ctx(ctx); }

extern "C" int bdfb_set_stream(bdfb_ctx* ctx, void* stream) {
  if (!ctx) return BDFB_ILL_INPUT;
  ctx->stream = as_stream(stream);
  if (ctx->grid) grid_set_stream(ctx->grid, ctx->stream);
  if (ctx->shared) shared_set_stream(ctx->shared, ctx->stream);
  if (ctx->ark) ark_set_stream(ctx->ark, ctx->stream);
  return BDFB_SUCCESS;
}

extern "C" int bdfb_set_tolerances(bdfb_ctx* ctx, double rtol, double atol) {
  if (!ctx || !(rtol >= 0.0) || !(atol > 0.0) || !std::isfinite(rtol) || !std::isfinite(atol))
    return BDFB_ILL_INPUT;
  ctx->rtol = rtol;
  ctx->atol = atol;
  if (ctx->grid) grid_set_tolerances(ctx->grid, rtol, atol);
  if (ctx->shared) shared_set_tolerances(ctx->shared, rtol, atol);
  if (ctx->ark) ark_set_tolerances(ctx->ark, rtol, atol);
  return BDFB_SUCCESS;
}

extern "C" int bdfb_set_option(bdfb_ctx* ctx, const char* key, int64_t v) {
  if (!ctx || !key) return BDFB_ILL_INPUT;
  // the grids solve by GMRES, shared networks by their sparse LU: only the
  // default linear solver
  if ((ctx->grid || ctx->shared) && !std::strcmp(key, "lsolver")) return v == 0 ? BDFB_SUCCESS : BDFB_ILL_INPUT;
  if (ctx->shared) return shared_set_option(ctx->shared, key, v);
  if (ctx->grid && ctx->kind == BDFB_BRUSSELATOR1D && !std::strcmp(key, "imex")) {
    if (v != 0 && v != 1) return BDFB_ILL_INPUT;
    if (v == 1 && !ctx->ark) {
      const double* p = ctx->line_par;
      int r = ark_create((int64_t)p[5], p[0], p[1], p[2], p[3], p[4], &ctx->ark);
      if (r) return r;
      ark_set_stream(ctx->ark, ctx->stream);
      ark_set_tolerances(ctx->ark, ctx->rtol, ctx->atol);
      r = ark_set_mxstep(ctx->ark, ctx->mxstep);
      if (!r) r = ark_set_precision(ctx->ark, ctx->line_prec);
      if (!r && ctx->line_dloop != -1) r = ark_set_device_loop(ctx->ark, ctx->line_dloop);
      if (r) return r;
    }
    ctx->imex = (int)v;
    return BDFB_SUCCESS;
  }
  if (ctx->grid && ctx->kind == BDFB_BRUSSELATOR1D && !std::strcmp(key, "device_loop")) {
    if (v < -1 || v > 1) return BDFB_ILL_INPUT;
    if (ctx->ark) {
      const int r = ark_set_device_loop(ctx->ark, (int)v);
      if (r) return r;
    }
    ctx->line_dloop = (int)v;
    return BDFB_SUCCESS;
  }
  if (ctx->grid && ctx->kind == BDFB_BRUSSELATOR1D && !std::strcmp(key, "precision")) {
    if (v != 0 && v != 1) return BDFB_ILL_INPUT;
    ctx->line_prec = (int)v;
    const int r = grid_set_option(ctx->grid, "precision", v);   // the BDF / GMRES path
    if (r) return r;
    return ctx->ark ? ark_set_precision(ctx->ark, (int)v) : BDFB_SUCCESS;
  }
  if (ctx->grid) {
    if (!std::strcmp(key, "mxstep") && v >= 1) {
      ctx->mxstep = v;
      if (ctx->ark) ark_set_mxstep(ctx->ark, v);
    }
    return grid_set_option(ctx->grid, key, v);
  }
  if (!std::strcmp(key, "mxstep")) {
    if (v < 1 || v > 1000000000) return BDFB_ILL_INPUT;
    ctx->mxstep = v;
  } else if (!std::strcmp(key, "mapping")) {
    if (v != 0 && v != 32) return BDFB_ILL_INPUT;
    ctx->mapping = (int)v;
  } else if (!std::strcmp(key, "precision")) {
    if (v != 0 && v != 1) return BDFB_ILL_INPUT;
    if (v == 1 && ctx->kind != BDFB_MASSACTION) return BDFB_ILL_INPUT;  // residual needs reaction data
    if (v == 1 && (ctx->predictor || ctx->rec_x)) return BDFB_ILL_INPUT;
    ctx->precision = (int)v;
  } else if (!std::strcmp(key, "mixed_small")) {
    if (v != 0 && v != 1) return BDFB_ILL_INPUT;
    if (v == 1 && ctx->kind != BDFB_MASSACTION) return BDFB_ILL_INPUT;
    ctx->mixed_small = (int)v;
  } else if (!std::strcmp(key, "graph")) {
    if (v != 0 && v != 1) return BDFB_ILL_INPUT;
    ctx->graph = (int)v;
  } else if (!std::strcmp(key, "autotune")) {
    if (v != 0 && v != 1) return BDFB_ILL_INPUT;
    ctx->autotune = (int)v;
    ctx->tuned_prec = -1;     // tune again on the next integrate
  } else if (!std::strcmp(key, "qmax")) {
    if (v < 1 || v > QMAX) return BDFB_ILL_INPUT;
    ctx->qmax = (int)v;
  } else if (!std::strcmp(key, "predictor")) {
    if (v != 0 && v != 1) return BDFB_ILL_INPUT;
    if (v == 1 && (ctx->maxn > MLP_NO || !ctx->fits_w16 || ctx->precision != 0 || ctx->lsolver))
      return BDFB_ILL_INPUT;
    ctx->predictor = (int)v;
  } else if (!std::strcmp(key, "lsolver")) {
    if (v != 0 && v != 1) return BDFB_ILL_INPUT;
    if (v == 1 && (ctx->predictor || ctx->rec_x)) return BDFB_ILL_INPUT;
    ctx->lsolver = (int)v;
  } else if (!std::strcmp(key, "interp")) {
    if (v != 0 && v != 1) return BDFB_ILL_INPUT;
    if (v == 1 && !ctx->d_yout && ctx->ny > 0) {
      if (cudaMalloc(&ctx->d_yout, ctx->ny * sizeof(double)) != cudaSuccess) {
        ctx->d_yout = nullptr;
        return BDFB_MEM_FAIL;
      }
    }
    ctx->interp = (int)v;
  } else if (!std::strcmp(key, "grouped")) {
    if (v != 0 && v != 1) return BDFB_ILL_INPUT;
    ctx->grouped = (int)v;
    ctx->gfresh = true;       // the next integrate starts from the state of bdfb_init
  } else {
    return BDFB_ILL_INPUT;
  }
  return BDFB_SUCCESS;
}

extern "C" int bdfb_init(bdfb_ctx* ctx, double t0, const double* y0, int32_t mem) {
  if (!ctx || !std::isfinite(t0) || (ctx->ny > 0 && !y0)) return BDFB_ILL_INPUT;
  if (mem != BDFB_MEM_HOST && mem != BDFB_MEM_DEVICE) return BDFB_ILL_INPUT;
  if (ctx->shared) {
    const int r = shared_init(ctx->shared, t0, y0, mem);
    ctx->initialized = r == 0;
    return r;
  }
  if (ctx->grid) {
    int r = grid_init(ctx->grid, t0, y0, mem);
    if (!r && ctx->ark) r = ark_init(ctx->ark, t0, y0, mem);
    ctx->initialized = r == 0;
    return r;
  }
  std::vector<CellState> st(std::max<int64_t>(ctx->ncell, 1));
  std::memset(st.data(), 0, st.size() * sizeof(CellState));
  for (auto& s : st) { s.t = t0; s.q = 1; s.crate = 1.0; }
  cudaStream_t s = ctx->stream;
  if (ctx->ncell > 0)
    BDFB_CUDA(cudaMemcpyAsync(ctx->d_state, st.data(), ctx->ncell * sizeof(CellState),
                              cudaMemcpyHostToDevice, s));
  BDFB_CUDA(cudaMemsetAsync(ctx->d_z, 0, 6 * std::max<int64_t>(ctx->ny, 1) * sizeof(double), s));
  BDFB_CUDA(cudaMemsetAsync(ctx->d_acorp, 0, std::max<int64_t>(ctx->ny, 1) * sizeof(double), s));
  if (ctx->ny > 0)
    BDFB_CUDA(cudaMemcpyAsync(ctx->d_z, y0, ctx->ny * sizeof(double),
                              mem == BDFB_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  BDFB_CUDA(cudaStreamSynchronize(s));   // the host staging vector goes out of scope
  ctx->t0 = t0;
  ctx->gfresh = true;
  ctx->initialized = true;
  return BDFB_SUCCESS;
}

// kernel row of the factorisation options: FP32 LU with refinement
// (precision 1), FP64 Gauss-Jordan inverse (lsolver 1) or FP64 LU
// Kernel row (0 FP64 LU, 1 FP32 LU with FP64 refinement, 2 FP64
// Gauss-Jordan inverse) of variant v.  Precision 1 factors in FP32 the cells
// of more than 32 species (the NMAX 56 kernels), where the n^3 factorisation
// dominates a step; smaller cells keep FP64 factors unless mixed_small is set:
// on B300 two FP64 refinement residuals per solve cost more there than the
// FP64 factorisations they replace (measured per size class on its own
// tiling: n = 54 1.11x faster in FP32, n = 32 1.10x, n = 10 1.48x and n = 3
// 1.56x slower; n = 32 on one warp per cell 1.04x faster, n = 10 1.32x
// slower -- a row is chosen per kernel, and the one-warp 32-species kernel
// also takes the small cells of mapping 32).
constexpr int MIXED_NMAX = 56;
static int row_of(const bdfb_ctx* ctx, int v) {
  if (ctx->precision == 1 && (ctx->mixed_small || VAR_NMAX[v] >= MIXED_NMAX)) return 1;
  return ctx->lsolver ? 2 : 0;
}
// the configuration the kernel rows follow (a tuned schedule or a captured
// graph is valid for one value)
static int rows_key(const bdfb_ctx* ctx) { return ctx->precision + 2 * ctx->lsolver + 4 * ctx->mixed_small; }

// The one-warp-per-cell kernel of mapping 32 (and of the learned guess): the
// smallest shared-memory layout every cell fits
static int one_warp_variant(const bdfb_ctx* ctx, bool learn) {
  if (learn || (ctx->fits_w16 && row_of(ctx, VAR_W16) == 0)) return VAR_W16;
  if (ctx->fits_w32) return VAR_W32;
  return 4;
}

// Params of an integrate call (schedule fields filled by the caller)
static Params base_params(bdfb_ctx* ctx, double tout) {
  Params P;
  std::memset(&P, 0, sizeof P);   // padding too: Params are compared bytewise
  P.kind = ctx->kind;
  P.qmax = ctx->qmax;
  P.ny = ctx->ny;
  P.n = ctx->d_n;
  P.y_off = ctx->d_yoff;
  P.rxn_off = ctx->d_rxnoff;
  P.reac = ctx->d_reac;
  P.k = ctx->d_k;
  P.inc_off = ctx->d_incoff;
  P.inc = ctx->d_inc;
  P.gsched = ctx->d_gsched;
  P.tile_counter = ctx->d_counter;
  P.worst = reinterpret_cast<int*>(ctx->d_counter + NVAR);
  P.st = ctx->d_state;
  P.z = ctx->d_z;
  P.acorp = ctx->d_acorp;
  P.status = ctx->d_status;
  P.tout = tout;
  P.rtol = ctx->rtol;
  P.atol = ctx->atol;
  P.mxstep = (int32_t)std::min<int64_t>(ctx->mxstep, 0x7fffffff);
  static const Consts K = make_consts();
  P.K = K;
  P.mlp = ctx->predictor ? ctx->mlp : nullptr;
  P.rec_x = ctx->rec_x;
  P.rec_t = ctx->rec_t;
  P.rec_cap = ctx->rec_cap;
  P.rec_count = ctx->rec_count;
  P.interp = ctx->interp;
  P.yout = ctx->interp ? ctx->d_yout : nullptr;
  return P;
}

// global workspace of a kernel variant (workspace_doubles_per_warp): one
// slice per resident warp, allocated on first use
static int ensure_fbws(bdfb_ctx* ctx, int pr, int v) {
  const int64_t per = workspace_doubles_per_warp(v, pr);
  if (per == 0 || ctx->d_fbws[pr][v]) return 0;
  const size_t bytes = (size_t)ctx->pgrid[pr][v] * per * sizeof(double);
  if (cudaMalloc(&ctx->d_fbws[pr][v], bytes) != cudaSuccess) {
    ctx->d_fbws[pr][v] = nullptr;
    return BDFB_MEM_FAIL;
  }
  return 0;
}

// The launch sequence of one integrate call on stream s: clear the tile
// counters, then fork one persistent launch per variant of the schedule,
// largest cells first, each on its own stream so that smaller cells fill
// the SMs the larger ones release, and join.  `single`: the variant the
// one-cell tiles of the one-warp-per-cell schedule (variant 4's range) run on.
static int launch_all(bdfb_ctx* ctx, const Params& P, const Sched& S, int single, cudaStream_t s) {
  BDFB_CUDA(cudaMemsetAsync(ctx->d_counter, 0, (NVAR + 1) * sizeof(unsigned), s));
  BDFB_CUDA(cudaEventRecord(ctx->evfork, s));
  for (int k = 0; k < NVAR; ++k) {
    const int v = VAR_ORDER[k];
    const int t0 = S.vbeg[v], t1 = S.vend[v];
    if (t1 <= t0) continue;
    const int kv = v == 4 ? single : v;
    const int pr = row_of(ctx, kv);
    const cells_kernel_t kf = var_kernel(pr, kv);
    if (!kf) return BDFB_ILL_INPUT;
    // mixed precision: the launched variant's FP64 fallback workspace must exist
    if (workspace_doubles_per_warp(kv, pr) && !ctx->d_fbws[pr][kv]) return BDFB_MEM_FAIL;
    cudaStream_t cs = ctx->cstream[v];
    BDFB_CUDA(cudaStreamWaitEvent(cs, ctx->evfork, 0));
    const int grid = std::min(ctx->pgrid[pr][kv], t1 - t0);
    kf<<<grid, 32, var_smem(pr, kv), cs>>>(P, t0, t1, ctx->d_counter + v, ctx->d_fbws[pr][kv]);
    BDFB_CUDA(cudaGetLastError());
    BDFB_CUDA(cudaEventRecord(ctx->evjoin[v], cs));
    BDFB_CUDA(cudaStreamWaitEvent(s, ctx->evjoin[v], 0));
  }
  return 0;
}

// Option "graph": the launch sequence is captured once into a CUDA graph
// and replayed; a later call with the same parameters but another tout
// patches tout into the kernel nodes; anything else recaptures.
static int launch_graph(bdfb_ctx* ctx, const Params& P, int m, int single, cudaStream_t s) {
  Params key = P;
  key.tout = 0.0;
  const bool same = ctx->gexec && ctx->gkey_gen == ctx->sched_gen && ctx->gkey_m == m &&
                    ctx->gkey_single == single && ctx->gkey_rows == rows_key(ctx) &&
                    !std::memcmp(&key, &ctx->gkey, sizeof key);
  if (!same) {
    if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; }
    if (ctx->cgraph) { cudaGraphDestroy(ctx->cgraph); ctx->cgraph = nullptr; }
    // captured on a stream of the context (the legacy default stream cannot
    // be captured); the graph is launched on s
    BDFB_CUDA(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int r = launch_all(ctx, P, ctx->sched[m], single, ctx->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
    if (r || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return r ? r : BDFB_CUDA_FAIL;
    }
    ctx->cgraph = g;
    BDFB_CUDA(cudaGraphInstantiate(&ctx->gexec, g, 0));
    ctx->gkey = key;
    ctx->gkey_gen = ctx->sched_gen;
    ctx->gkey_m = m;
    ctx->gkey_single = single;
    ctx->gkey_rows = rows_key(ctx);
    ctx->graph_captures++;
  } else {
    size_t nn = 0;
    BDFB_CUDA(cudaGraphGetNodes(ctx->cgraph, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    BDFB_CUDA(cudaGraphGetNodes(ctx->cgraph, nodes.data(), &nn));
    for (size_t i = 0; i < nn; ++i) {
      cudaGraphNodeType ty;
      BDFB_CUDA(cudaGraphNodeGetType(nodes[i], &ty));
      if (ty != cudaGraphNodeTypeKernel) continue;
      cudaKernelNodeParams kp;
      BDFB_CUDA(cudaGraphKernelNodeGetParams(nodes[i], &kp));
      Params pn = *static_cast<Params*>(kp.kernelParams[0]);
      pn.tout = P.tout;
      int t0 = *static_cast<int*>(kp.kernelParams[1]);
      int t1 = *static_cast<int*>(kp.kernelParams[2]);
      unsigned* cnt = *static_cast<unsigned**>(kp.kernelParams[3]);
      double* fb = *static_cast<double**>(kp.kernelParams[4]);
      void* args[5] = {&pn, &t0, &t1, &cnt, &fb};
      kp.kernelParams = args;
      kp.extra = nullptr;
      BDFB_CUDA(cudaGraphExecKernelNodeSetParams(ctx->gexec, nodes[i], &kp));
    }
  }
  BDFB_CUDA(cudaGraphLaunch(ctx->gexec, s));
  ctx->graph_launches++;
  return 0;
}

// Autotuner: for every size class with more than one variant that can run
// its cells (its own tiling, the next larger one, and for cells of at most
// 16 species the one-warp NMAX 16 kernel), integrate a sample of the class
// (its first 16384 cells) from the current state to tout once per variant
// on scratch copies of the state, time each launch with events, and keep
// the fastest (another variant must beat the class's own by 3%).  The
// context's state is not touched.  Builds schedule 2.
static int run_autotune(bdfb_ctx* ctx, const Params& P0, cudaStream_t s) {
  const int64_t C = ctx->ncell;
  constexpr int64_t SAMPLE = 16384;
  std::vector<std::vector<int32_t>> members(NCLASS);
  for (int64_t i = 0; i < C; ++i)
    if ((int64_t)members[ctx->h_cls[i]].size() < SAMPLE) members[ctx->h_cls[i]].push_back((int32_t)i);
  CellState* st2 = nullptr;
  double *z2 = nullptr, *acorp2 = nullptr;
  TileDesc* tiles2 = nullptr;
  int32_t* tcells2 = nullptr;
  unsigned* cnt2 = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = 0;
  auto fail = [&](int r) { if (!rc) rc = r; };
  const size_t zbytes = 6 * (size_t)std::max<int64_t>(ctx->ny, 1) * sizeof(double);
  if (cudaMalloc(&st2, C * sizeof(CellState)) != cudaSuccess || cudaMalloc(&z2, zbytes) != cudaSuccess ||
      cudaMalloc(&acorp2, std::max<int64_t>(ctx->ny, 1) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&tiles2, SAMPLE * sizeof(TileDesc)) != cudaSuccess ||
      cudaMalloc(&tcells2, SAMPLE * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&cnt2, (NVAR + 1) * sizeof(unsigned)) != cudaSuccess)
    fail(BDFB_MEM_FAIL);
  if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) fail(BDFB_CUDA_FAIL);
  std::vector<int8_t> var(C, 0);
  for (int cl = 0; cl < NCLASS && !rc; ++cl) {
    ctx->tuned_var[cl] = cl;
    for (int v = 0; v < NVAR; ++v) ctx->tune_ms[cl][v] = 0.f;
    if (members[cl].empty()) continue;
    // the class's own tiling first, then every other variant whose NMAX
    // covers the class (small workloads can favour more lanes per cell:
    // more warps in flight); nothing to time when there is no alternative
    std::vector<int> cand = {cl};
    for (int v = 0; v < NVAR; ++v)
      if (v != cl && var_kernel(row_of(ctx, v), v) && VAR_NMAX[v] >= CLS_NMAX[cl]) cand.push_back(v);
    if (cand.size() == 1) continue;
    float best = 0.f;
    for (int v : cand) {
      const int pr = row_of(ctx, v);
      if (ensure_fbws(ctx, pr, v)) { fail(BDFB_MEM_FAIL); break; }
      for (int32_t c : members[cl]) var[c] = (int8_t)v;
      std::vector<TileDesc> tiles;
      std::vector<int32_t> tcells;
      int vb[NVAR], ve[NVAR];
      make_tiles(launch_order(var, ctx->h_n, members[cl]), var, false, tiles, tcells, vb, ve);
      const int nt = (int)tiles.size();
      Params Pt = P0;
      Pt.st = st2;
      Pt.z = z2;
      Pt.acorp = acorp2;
      Pt.tiles = tiles2;
      Pt.tile_cells = tcells2;
      Pt.ntiles = nt;
      Pt.tile_counter = cnt2;
      Pt.worst = reinterpret_cast<int*>(cnt2 + NVAR);
      Pt.yout = nullptr;                // trials leave the output alone
      Pt.status = nullptr;
      Pt.rec_x = nullptr;
      Pt.mlp = nullptr;
      if (cudaMemcpyAsync(tiles2, tiles.data(), nt * sizeof(TileDesc), cudaMemcpyHostToDevice, s) ||
          cudaMemcpyAsync(tcells2, tcells.data(), tcells.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s)) {
        fail(BDFB_CUDA_FAIL);
        break;
      }
      const cells_kernel_t kf = var_kernel(pr, v);
      // short trials (small classes) are repeated and the fastest kept
      float ms = 0.f;
      for (int rep = 0; rep < 3 && !rc; ++rep) {
        if (cudaMemcpyAsync(st2, ctx->d_state, C * sizeof(CellState), cudaMemcpyDeviceToDevice, s) ||
            cudaMemcpyAsync(z2, ctx->d_z, zbytes, cudaMemcpyDeviceToDevice, s) ||
            cudaMemcpyAsync(acorp2, ctx->d_acorp, std::max<int64_t>(ctx->ny, 1) * sizeof(double),
                            cudaMemcpyDeviceToDevice, s) ||
            cudaMemsetAsync(cnt2, 0, (NVAR + 1) * sizeof(unsigned), s)) {
          fail(BDFB_CUDA_FAIL);
          break;
        }
        cudaEventRecord(e0, s);
        kf<<<std::min(ctx->pgrid[pr][v], nt), 32, var_smem(pr, v), s>>>(
            Pt, 0, nt, cnt2, ctx->d_fbws[pr][v]);
        cudaEventRecord(e1, s);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
          fail(BDFB_CUDA_FAIL);
          break;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        ms = rep == 0 ? t : std::min(ms, t);
        if (ms >= 20.f) break;
      }
      if (rc) break;
      ctx->tune_ms[cl][v] = ms;
      if (v == cl) best = ms;
      else if (ms < 0.97f * best) { best = ms; ctx->tuned_var[cl] = v; }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(st2); cudaFree(z2); cudaFree(acorp2); cudaFree(tiles2); cudaFree(tcells2); cudaFree(cnt2);
  if (rc) return rc;
  std::vector<int32_t> all(C);
  for (int64_t i = 0; i < C; ++i) {
    all[i] = (int32_t)i;
    var[i] = (int8_t)ctx->tuned_var[ctx->h_cls[i]];
  }
  const int r = upload_sched(ctx, 2, launch_order(var, ctx->h_n, all), var, false);
  if (r) return r;
  ctx->tuned_prec = rows_key(ctx);
  return 0;
}

// ---- grouped task-local Newton mode (option "grouped")
static int group_launch(bdfb_ctx* ctx, const GroupParams& GP, cudaStream_t s) {
  const Sched& S = ctx->sched[0];
  BDFB_CUDA(cudaMemsetAsync(ctx->d_counter, 0, (NVAR + 1) * sizeof(unsigned), s));
  for (int cl = NCLASS - 1; cl >= 0; --cl) {
    const int t0 = S.vbeg[cl], t1 = S.vend[cl];
    if (t1 <= t0) continue;
    GROUP_KERNELS[cl]<<<std::min(ctx->gpgrid[cl], t1 - t0), 32, CELLS_SMEM[0][cl], s>>>(GP, t0, t1,
                                                                                         ctx->d_counter + cl);
    BDFB_CUDA(cudaGetLastError());
  }
  return 0;
}

static GroupParams group_params(bdfb_ctx* ctx) {
  GroupParams GP;
  std::memset(&GP, 0, sizeof GP);
  GP.P = base_params(ctx, 0.0);
  GP.P.tiles = ctx->sched[0].d_tiles;
  GP.P.tile_cells = ctx->sched[0].d_tcells;
  GP.P.ntiles = ctx->sched[0].ntiles;
  GP.lu = ctx->d_glu;
  GP.lu_off = ctx->d_gluoff;
  GP.dinv = ctx->d_gdinv;
  GP.perm = ctx->d_gperm;
  GP.crate = ctx->d_gcrate;
  GP.failed = ctx->d_gflag;
  GP.iters = ctx->d_giters;
  return GP;
}

static int group_rhs(void* user, const double* y, double* f, cudaStream_t s) {
  bdfb_ctx* ctx = static_cast<bdfb_ctx*>(user);
  GroupParams GP = group_params(ctx);
  GP.mode = 1;
  GP.zp0 = y;
  GP.out = f;
  return group_launch(ctx, GP, s);
}

static int group_solve(void* user, const double* zp0, const double* zp1, const double* ewt, double gamma,
                       double gammap, double rl1, double Eq, int setup, double* acor, int* failed,
                       int64_t* iters, int64_t* sweeps, cudaStream_t s) {
  bdfb_ctx* ctx = static_cast<bdfb_ctx*>(user);
  GroupParams GP = group_params(ctx);
  GP.mode = 0;
  GP.setup = setup;
  GP.gamma = gamma;
  GP.gammap = gammap;
  GP.rl1 = rl1;
  GP.Eq = Eq;
  GP.zp0 = zp0;
  GP.zp1 = zp1;
  GP.ewt = ewt;
  GP.out = acor;
  BDFB_CUDA(cudaMemsetAsync(ctx->d_gflag, 0, sizeof(int), s));
  BDFB_CUDA(cudaMemsetAsync(ctx->d_giters, 0, 2 * sizeof(unsigned long long), s));
  const int r = group_launch(ctx, GP, s);
  if (r) return r;
  int fl = 0;
  unsigned long long it[2] = {0, 0};
  BDFB_CUDA(cudaMemcpyAsync(&fl, ctx->d_gflag, sizeof(int), cudaMemcpyDeviceToHost, s));
  BDFB_CUDA(cudaMemcpyAsync(it, ctx->d_giters, sizeof it, cudaMemcpyDeviceToHost, s));
  BDFB_CUDA(cudaStreamSynchronize(s));
  *failed = fl;
  *iters = (int64_t)it[0];
  *sweeps = (int64_t)it[1];
  return 0;
}

static int grouped_integrate(bdfb_ctx* ctx, double tout, double* y, int32_t* status, int32_t mem) {
  if (ctx->precision != 0 || ctx->lsolver || ctx->predictor || ctx->rec_x) return BDFB_ILL_INPUT;
  cudaStream_t s = ctx->stream;
  if (!ctx->gg) {
    const int64_t C = ctx->ncell;
    std::vector<int64_t> off(C);
    int64_t tot = 0;
    for (int64_t i = 0; i < C; ++i) { off[i] = tot; tot += (int64_t)ctx->h_n[i] * ctx->h_n[i]; }
    int r = dev_alloc_copy(&ctx->d_gluoff, off.data(), C);
    if (!r) r = dev_alloc_copy<double>(&ctx->d_glu, nullptr, tot);
    if (!r) r = dev_alloc_copy<double>(&ctx->d_gdinv, nullptr, ctx->ny);
    if (!r) r = dev_alloc_copy<int16_t>(&ctx->d_gperm, nullptr, ctx->ny);
    if (!r) r = dev_alloc_copy<double>(&ctx->d_gcrate, nullptr, C);
    if (!r) r = dev_alloc_copy<int>(&ctx->d_gflag, nullptr, 1);
    if (!r) r = dev_alloc_copy<unsigned long long>(&ctx->d_giters, nullptr, 2);
    for (int cl = 0; cl < NCLASS && !r; ++cl) {
      int per_sm = 0;
      if (cudaFuncSetAttribute(GROUP_KERNELS[cl], cudaFuncAttributeMaxDynamicSharedMemorySize,
                               CELLS_SMEM[0][cl]) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, GROUP_KERNELS[cl], 32, CELLS_SMEM[0][cl]) !=
              cudaSuccess)
        r = BDFB_CUDA_FAIL;
      ctx->gpgrid[cl] = std::max(1, per_sm) * sm_count();
    }
    GridExternal ext;
    ext.user = ctx;
    ext.rhs = group_rhs;
    ext.solve = group_solve;
    if (!r) r = grid_create_external(ctx->ny, ext, &ctx->gg);
    if (r) return r;
  }
  grid_set_stream(ctx->gg, s);
  grid_set_tolerances(ctx->gg, ctx->rtol, ctx->atol);
  {
    int r = grid_set_option(ctx->gg, "mxstep", ctx->mxstep);
    if (!r) r = grid_set_option(ctx->gg, "qmax", ctx->qmax);
    if (!r) r = grid_set_option(ctx->gg, "interp", ctx->interp);
    if (r) return r;
  }
  if (ctx->gfresh) {
    const int r = grid_init(ctx->gg, ctx->t0, ctx->d_z, BDFB_MEM_DEVICE);
    if (r) return r;
    ctx->gfresh = false;
  }
  const int r = grid_integrate(ctx->gg, tout, y, mem);
  if (status) {
    std::vector<int32_t> sv(ctx->ncell, r);
    if (mem == BDFB_MEM_HOST) std::memcpy(status, sv.data(), ctx->ncell * sizeof(int32_t));
    else BDFB_CUDA(cudaMemcpy(status, sv.data(), ctx->ncell * sizeof(int32_t), cudaMemcpyHostToDevice));
  }
  return r;
}

extern "C" int bdfb_integrate(bdfb_ctx* ctx, double tout, double* y, int32_t* status, int32_t mem) {
  if (!ctx || !ctx->initialized || !std::isfinite(tout)) return BDFB_ILL_INPUT;
  if (mem != BDFB_MEM_HOST && mem != BDFB_MEM_DEVICE) return BDFB_ILL_INPUT;
  if (ctx->shared && shared_percell(ctx->shared)) return shared_integrate_cells(ctx->shared, tout, y, status, mem);
  if (ctx->shared) {
    const int r = shared_integrate(ctx->shared, tout, y, mem);
    if (status && ctx->ncell > 0) {
      std::vector<int32_t> sv(ctx->ncell, r);
      if (mem == BDFB_MEM_HOST) std::memcpy(status, sv.data(), ctx->ncell * sizeof(int32_t));
      else BDFB_CUDA(cudaMemcpy(status, sv.data(), ctx->ncell * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    return r;
  }
  if (ctx->grid) {
    const int r = ctx->imex ? ark_integrate(ctx->ark, tout, y, mem) : grid_integrate(ctx->grid, tout, y, mem);
    if (status) {
      const int32_t sv = r;
      if (mem == BDFB_MEM_HOST) *status = sv;
      else BDFB_CUDA(cudaMemcpy(status, &sv, sizeof sv, cudaMemcpyHostToDevice));
    }
    return r;
  }
  if (ctx->ncell == 0) return BDFB_SUCCESS;
  if (ctx->grouped) return grouped_integrate(ctx, tout, y, status, mem);
  if (ctx->predictor && !ctx->mlp) return BDFB_ILL_INPUT;
  cudaStream_t s = ctx->stream;
  const bool learn = ctx->predictor || ctx->rec_x;
  // one warp per cell: the NMAX 16 kernel when every cell fits it
  // one warp per cell: the smallest one-warp kernel every cell fits
  const int single = one_warp_variant(ctx, learn);
  int m = (ctx->mapping == 32 || learn) ? 1 : 0;
  Params P = base_params(ctx, tout);
  if (m == 0 && ctx->autotune) {
    if (ctx->tuned_prec != rows_key(ctx)) {
      P.tiles = ctx->sched[0].d_tiles;
      P.tile_cells = ctx->sched[0].d_tcells;
      P.ntiles = ctx->sched[0].ntiles;
      int r = run_autotune(ctx, P, s);
      if (r) return r;
    }
    m = 2;
  }
  const Sched& S = ctx->sched[m];
  P.tiles = S.d_tiles;
  P.tile_cells = S.d_tcells;
  P.ntiles = S.ntiles;
  // the workspace of the variant each range is launched on (variant 4's
  // range runs on `single` under the one-warp-per-cell schedule)
  for (int v = 0; v < NVAR; ++v)
    if (S.vend[v] > S.vbeg[v]) {
      const int kv = v == 4 ? single : v;
      const int r = ensure_fbws(ctx, row_of(ctx, kv), kv);
      if (r) return r;
    }
  BDFB_CUDA(cudaEventRecord(ctx->ev0, s));
  if (ctx->graph) {
    const int r = launch_graph(ctx, P, m, single, s);
    if (r) return r;
  } else {
    const int r = launch_all(ctx, P, S, single, s);
    if (r) return r;
  }
  BDFB_CUDA(cudaEventRecord(ctx->ev1, s));
  if (y) {
    BDFB_CUDA(cudaMemcpyAsync(y, ctx->interp ? ctx->d_yout : ctx->d_z, ctx->ny * sizeof(double),
                              mem == BDFB_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
  }
  if (status) {
    BDFB_CUDA(cudaMemcpyAsync(status, ctx->d_status, ctx->ncell * sizeof(int32_t),
                              mem == BDFB_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
  }
  int worst = 0;
  BDFB_CUDA(cudaMemcpyAsync(&worst, ctx->d_counter + NVAR, sizeof(int), cudaMemcpyDeviceToHost, s));
  BDFB_CUDA(cudaStreamSynchronize(s));
  cudaEventElapsedTime(&ctx->last_ms, ctx->ev0, ctx->ev1);
  return worst;
}

static int fetch_states(bdfb_ctx* ctx, std::vector<CellState>& st) {
  st.resize(std::max<int64_t>(ctx->ncell, 1));
  if (ctx->ncell > 0) {
    BDFB_CUDA(cudaStreamSynchronize(ctx->stream));
    BDFB_CUDA(cudaMemcpy(st.data(), ctx->d_state, ctx->ncell * sizeof(CellState), cudaMemcpyDeviceToHost));
  }
  return 0;
}

extern "C" int bdfb_get_op_profile(bdfb_ctx* ctx, double* out, int32_t nkinds) {
  if (!ctx || !out || !ctx->grid || nkinds < GOP_N) return BDFB_ILL_INPUT;
  grid_profile(ctx->grid, out);
  return GOP_N;
}

extern "C" int bdfb_phase_cycles(uint64_t* out, int nphase, int reset) {
#ifdef BDFB_PHASES
  if (!out || nphase < bdfb::NPHASE) return BDFB_ILL_INPUT;
  static unsigned long long h[256][bdfb::NPHASE];
  BDFB_CUDA(cudaDeviceSynchronize());
  BDFB_CUDA(cudaMemcpyFromSymbol(h, bdfb::g_phase_cycles, sizeof h));
  for (int k = 0; k < bdfb::NPHASE; ++k) {
    out[k] = 0;
    for (int r = 0; r < 256; ++r) out[k] += h[r][k];
  }
  if (reset) {
    std::memset(h, 0, sizeof h);
    BDFB_CUDA(cudaMemcpyToSymbol(bdfb::g_phase_cycles, h, sizeof h));
  }
  return bdfb::NPHASE;
#else
  (void)out; (void)nphase; (void)reset;
  return BDFB_ILL_INPUT;
#endif
}

extern "C" int bdfb_get_stats(bdfb_ctx* ctx, bdfb_stats* out) {
  if (!ctx || !out) return BDFB_ILL_INPUT;
  if (ctx->grouped && ctx->gg) {    // every cell takes every grouped step
    int64_t g[8];
    double ms = 0.0;
    grid_stats(ctx->gg, g, &ms);
    std::memset(out, 0, sizeof *out);
    out->ncell = ctx->ncell;
    const int64_t C = ctx->ncell;
    out->nsteps = g[0] * C; out->nfevals = g[1] * C; out->nlinsetups = g[2] * C;
    out->nniters = g[3]; out->nncfails = g[4] * C; out->netfails = g[5] * C;
    out->max_steps = out->min_steps = g[0];
    out->last_kernel_ms = ms;
    return BDFB_SUCCESS;
  }
  if (ctx->shared && shared_percell(ctx->shared)) {   // sums over the cells' own counters
    std::vector<int64_t> rows;
    double ms = 0.0;
    const int r = shared_cell_stats(ctx->shared, rows, &ms);
    if (r) return r;
    std::memset(out, 0, sizeof *out);
    const int64_t C = ctx->ncell;
    out->ncell = C;
    out->min_steps = C ? INT64_MAX : 0;
    for (int64_t c = 0; c < C; ++c) {
      const int64_t* o = rows.data() + 8 * c;
      out->nsteps += o[0]; out->nfevals += o[1]; out->nlinsetups += o[2]; out->nniters += o[3];
      out->nncfails += o[4]; out->netfails += o[5];
      out->max_steps = std::max(out->max_steps, o[0]);
      out->min_steps = std::min(out->min_steps, o[0]);
    }
    out->last_kernel_ms = ms;
    return BDFB_SUCCESS;
  }
  if (ctx->shared) {               // every cell takes every grouped step
    int64_t g[8];
    double ms = 0.0, h = 0.0;
    int q = 0;
    shared_stats(ctx->shared, g, &ms, &q, &h);
    std::memset(out, 0, sizeof *out);
    const int64_t C = ctx->ncell;
    out->ncell = C;
    out->nsteps = g[0] * C; out->nfevals = g[1] * C; out->nlinsetups = g[2] * C;
    out->nniters = g[3]; out->nncfails = g[4] * C; out->netfails = g[5] * C;
    out->max_steps = out->min_steps = g[0];
    out->last_kernel_ms = ms;
    return BDFB_SUCCESS;
  }
  if (ctx->grid && ctx->imex) {    // IMEX ARK: blocks are formed at every Newton iteration
    int64_t g[8];
    double ms = 0.0;
    ark_stats(ctx->ark, g, &ms);
    std::memset(out, 0, sizeof *out);
    out->ncell = ctx->ncell;
    out->nsteps = g[0]; out->nfevals = g[2]; out->nlinsetups = g[3]; out->nniters = g[3];
    out->nncfails = g[4]; out->netfails = g[5];
    out->max_steps = out->min_steps = g[0];
    out->last_kernel_ms = ms;
    return BDFB_SUCCESS;
  }
  if (ctx->grid) {
    int64_t g[8];
    double ms = 0.0;
    grid_stats(ctx->grid, g, &ms);
    std::memset(out, 0, sizeof *out);
    out->ncell = ctx->ncell;
    out->nsteps = g[0]; out->nfevals = g[1]; out->nlinsetups = g[2]; out->nniters = g[3];
    out->nncfails = g[4]; out->netfails = g[5];
    out->max_steps = out->min_steps = g[0];
    out->last_kernel_ms = ms;
    return BDFB_SUCCESS;
  }
  std::vector<CellState> st;
  int r = fetch_states(ctx, st);
  if (r) return r;
  std::memset(out, 0, sizeof *out);
  out->ncell = ctx->ncell;
  out->min_steps = ctx->ncell ? INT64_MAX : 0;
  for (int64_t i = 0; i < ctx->ncell; ++i) {
    const CellState& s = st[i];
    out->nsteps += s.nst;
    out->nfevals += s.nfe;
    out->nlinsetups += s.nsetups;
    out->nniters += s.nni;
    out->nncfails += s.ncfn;
    out->netfails += s.netf;
    out->max_steps = std::max<int64_t>(out->max_steps, s.nst);
    out->min_steps = std::min<int64_t>(out->min_steps, s.nst);
    out->ncells_failed += s.status != 0;
    out->nrefine += s.nrefine;
    out->nrefine_fallback += s.nrefine_fb;
    out->nguess += s.nguess;
    out->nguess_fallback += s.nguess_fb;
  }
  out->graph_captures = ctx->graph_captures;
  out->graph_launches = ctx->graph_launches;
  out->last_kernel_ms = ctx->last_ms;
  return BDFB_SUCCESS;
}

extern "C" int bdfb_get_cell_stats(bdfb_ctx* ctx, int64_t* out, int32_t mem) {
  if (!ctx || (!out && ctx->ncell > 0)) return BDFB_ILL_INPUT;
  if (mem != BDFB_MEM_HOST && mem != BDFB_MEM_DEVICE) return BDFB_ILL_INPUT;
  if (ctx->shared && shared_percell(ctx->shared)) {
    std::vector<int64_t> rows;
    double ms = 0.0;
    const int r = shared_cell_stats(ctx->shared, rows, &ms);
    if (r) return r;
    if (ctx->ncell == 0) return BDFB_SUCCESS;
    if (mem == BDFB_MEM_HOST) std::memcpy(out, rows.data(), rows.size() * sizeof(int64_t));
    else BDFB_CUDA(cudaMemcpy(out, rows.data(), rows.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    return BDFB_SUCCESS;
  }
  if (ctx->shared) {
    int64_t g[8];
    double ms = 0.0, h = 0.0;
    int q = 0;
    shared_stats(ctx->shared, g, &ms, &q, &h);
    if (mem == BDFB_MEM_HOST) std::memcpy(out, g, sizeof g);
    else BDFB_CUDA(cudaMemcpy(out, g, sizeof g, cudaMemcpyHostToDevice));
    return BDFB_SUCCESS;
  }
  if (ctx->grid) {
    int64_t g[8];
    double ms = 0.0;
    if (ctx->imex) ark_stats(ctx->ark, g, &ms);
    else grid_stats(ctx->grid, g, &ms);
    if (mem == BDFB_MEM_HOST) std::memcpy(out, g, sizeof g);
    else BDFB_CUDA(cudaMemcpy(out, g, sizeof g, cudaMemcpyHostToDevice));
    return BDFB_SUCCESS;
  }
  if (ctx->grouped && ctx->gg) {   // the shared counters in every row
    int64_t g[8];
    double ms = 0.0, h = 0.0;
    int q = 0;
    grid_stats(ctx->gg, g, &ms);
    grid_next_step(ctx->gg, &q, &h);
    int64_t hb;
    std::memcpy(&hb, &h, sizeof hb);
    const int64_t row[8] = {g[0], g[1], g[2], g[3] / std::max<int64_t>(ctx->ncell, 1), g[4], g[5], q, hb};
    std::vector<int64_t> v(8 * ctx->ncell);
    for (int64_t i = 0; i < ctx->ncell; ++i) std::memcpy(v.data() + 8 * i, row, sizeof row);
    if (ctx->ncell == 0) return BDFB_SUCCESS;
    if (mem == BDFB_MEM_HOST) std::memcpy(out, v.data(), v.size() * sizeof(int64_t));
    else BDFB_CUDA(cudaMemcpy(out, v.data(), v.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    return BDFB_SUCCESS;
  }
  std::vector<CellState> st;
  int r = fetch_states(ctx, st);
  if (r) return r;
  std::vector<int64_t> v(8 * std::max<int64_t>(ctx->ncell, 1));
  for (int64_t i = 0; i < ctx->ncell; ++i) {
    const CellState& s = st[i];
    int64_t hb;
    std::memcpy(&hb, &s.hlast, sizeof hb);
    int64_t* o = v.data() + 8 * i;
    o[0] = s.nst; o[1] = s.nfe; o[2] = s.nsetups; o[3] = s.nni;
    o[4] = s.ncfn; o[5] = s.netf; o[6] = s.qlast; o[7] = hb;
  }
  if (ctx->ncell == 0) return BDFB_SUCCESS;
  if (mem == BDFB_MEM_HOST) std::memcpy(out, v.data(), 8 * ctx->ncell * sizeof(int64_t));
  else BDFB_CUDA(cudaMemcpy(out, v.data(), 8 * ctx->ncell * sizeof(int64_t), cudaMemcpyHostToDevice));
  return BDFB_SUCCESS;
}

extern "C" int bdfb_get_mapping(bdfb_ctx* ctx, int32_t* out, float* trial_ms) {
  if (!ctx || !out) return BDFB_ILL_INPUT;
  std::memset(out, 0, 3 * NCLASS * sizeof(int32_t));
  if (trial_ms) std::memset(trial_ms, 0, NCLASS * NVAR * sizeof(float));
  if (ctx->grid || ctx->shared) return BDFB_SUCCESS;
  const bool learn = ctx->predictor || ctx->rec_x;
  for (int64_t i = 0; i < ctx->ncell; ++i) out[3 * ctx->h_cls[i] + 2]++;
  for (int cl = 0; cl < NCLASS; ++cl) {
    if (!out[3 * cl + 2]) continue;
    int v = cl;
    if (learn || ctx->mapping == 32) v = one_warp_variant(ctx, learn);
    else if (ctx->autotune && ctx->tuned_prec == rows_key(ctx)) v = ctx->tuned_var[cl];
    out[3 * cl] = VAR_G[v];
    out[3 * cl + 1] = VAR_NMAX[v];
    if (trial_ms && ctx->autotune && ctx->tuned_prec >= 0)
      for (int k = 0; k < NVAR; ++k) trial_ms[cl * NVAR + k] = ctx->tune_ms[cl][k];
  }
  return BDFB_SUCCESS;
}

extern "C" int bdfb_load_mlp(bdfb_ctx* ctx, const void* packed, int64_t bytes) {
  if (!ctx || ctx->grid || ctx->shared || (packed && bytes != PACKED_BYTES)) return BDFB_ILL_INPUT;
  if (packed && (reinterpret_cast<uintptr_t>(packed) & 15u)) return BDFB_ILL_INPUT;
  ctx->mlp = packed;
  return BDFB_SUCCESS;
}

extern "C" int bdfb_set_record(bdfb_ctx* ctx, float* x, float* t, int64_t cap, unsigned long long* count) {
  if (!ctx || ctx->grid || ctx->shared) return BDFB_ILL_INPUT;
  if (!x) {
    ctx->rec_x = nullptr; ctx->rec_t = nullptr; ctx->rec_cap = 0; ctx->rec_count = nullptr;
    return BDFB_SUCCESS;
  }
  if (!t || !count || cap < 0 || ctx->maxn > MLP_NO || !ctx->fits_w16 || ctx->precision != 0 ||
      ctx->lsolver)
    return BDFB_ILL_INPUT;
  ctx->rec_x = x; ctx->rec_t = t; ctx->rec_cap = cap; ctx->rec_count = count;
  return BDFB_SUCCESS;
}

// ------------------------------------------------------ batched LU entries
extern "C" int bdfb_batched_lu_factor(int64_t nb, int n, double* a, int32_t* piv, int32_t* info,
                                      void* stream) {
  if (nb < 0 || n < 1 || n > LU_NMAX || (nb > 0 && (!a || !piv || !info))) return BDFB_ILL_INPUT;
  if (nb == 0) return BDFB_SUCCESS;
  const int smem = (int)sizeof(CellSmem<LU_NMAX>) + LU_NMAX * (int)sizeof(int16_t);
  BDFB_CUDA(cudaFuncSetAttribute(k_lu_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int64_t grid = std::min<int64_t>(nb, (int64_t)sm_count() * 6);
  k_lu_factor<<<(int)grid, 32, smem, as_stream(stream)>>>(nb, n, a, piv, info);
  BDFB_CUDA(cudaGetLastError());
  return BDFB_SUCCESS;
}

extern "C" int bdfb_batched_solve_mixed(int64_t nb, int n, const double* a, const double* b,
                                        double* x, int32_t* sweeps, void* stream) {
  if (nb < 0 || n < 1 || n > LU_NMAX || (nb > 0 && (!a || !b || !x || !sweeps))) return BDFB_ILL_INPUT;
  if (nb == 0) return BDFB_SUCCESS;
  const int smem = (int)sizeof(CellSmem<LU_NMAX, 1>) + LU_NMAX * (LU_NMAX + 1) * (int)sizeof(double);
  BDFB_CUDA(cudaFuncSetAttribute(k_solve_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int64_t grid = std::min<int64_t>(nb, (int64_t)sm_count() * 4);
  k_solve_mixed<<<(int)grid, 32, smem, as_stream(stream)>>>(nb, n, a, b, x, sweeps);
  BDFB_CUDA(cudaGetLastError());
  return BDFB_SUCCESS;
}

extern "C" int bdfb_batched_lu_solve(int64_t nb, int n, const double* lu, const int32_t* piv,
                                     double* b, void* stream) {
  if (nb < 0 || n < 1 || n > LU_NMAX || (nb > 0 && (!lu || !piv || !b))) return BDFB_ILL_INPUT;
  if (nb == 0) return BDFB_SUCCESS;
  const int smem = (int)sizeof(CellSmem<LU_NMAX>);
  BDFB_CUDA(cudaFuncSetAttribute(k_lu_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int64_t grid = std::min<int64_t>(nb, (int64_t)sm_count() * 6);
  k_lu_solve<<<(int)grid, 32, smem, as_stream(stream)>>>(nb, n, lu, piv, b);
  BDFB_CUDA(cudaGetLastError());
  return BDFB_SUCCESS;
}
