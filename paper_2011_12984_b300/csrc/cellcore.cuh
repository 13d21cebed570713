// cellcore.cuh - per-cell device building blocks of the batched BDF step.
//
// A cell (one small independent ODE system, the paper's "submodel" case of
// Sec. 2; one diagonal block of the block-diagonal Jacobian of Fig. 1) is
// owned by a group of G lanes of one warp (G = 1, 4, 8, 16 or 32).  Lane
// `rank` of a group owns the vector elements i = rank + G s, s < NPL, which
// live in registers; the cell's matrix M = I - gamma J, the gathered state and
// the reaction rates live in the group's slice of shared memory.  Group-wide
// reductions are xor-butterflies, so every lane of a group holds bitwise the
// same scalars and all control flow is uniform inside a group.
#pragma once

#include <cstring>
#include <type_traits>

#include "common.cuh"

namespace bdfb {

// ------------------------------------------------------------- phase timers
// Builds with -DBDFB_PHASES only (a plain build compiles the marks away):
// lane 0 of each one-warp block charges the SM clock cycles between marks to
// the phase it leaves, in one of 256 rows of counters (rows by block, so the
// fire-and-forget atomic adds do not contend); the clock and the current
// phase live in the block's shared memory, so any device function can mark.
// Cycles a warp waits for a pipe that its neighbours keep busy count in the
// phase it waits in: the shares show where a step's time goes.  Only the
// per-cell step kernels start the clock.
enum {
  PH_CTRL, PH_PRED, PH_JAC, PH_LU_PIV, PH_LU_UPD, PH_RATES, PH_GATHER, PH_TRI, PH_RES, PH_NORM,
  PH_NEWT, PH_ACCEPT, PH_FAIL, PH_TILE, NPHASE
};
#ifdef BDFB_PHASES
__device__ unsigned long long g_phase_cycles[256][NPHASE];
__device__ __forceinline__ long long& ph_clock() {
  __shared__ long long t;
  return t;
}
__device__ __forceinline__ int& ph_current() {
  __shared__ int k;
  return k;
}
__device__ __forceinline__ void ph_start(int k) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) { ph_clock() = clock64(); ph_current() = k; }
  __syncwarp();
}
// Kernels that never start the clock (the grouped and standalone solvers
// reach these marks through shared helpers) hold no valid phase: the index is
// checked before any counter is touched.
__device__ __forceinline__ void ph_mark(int k) {
  if ((threadIdx.x & 31) == 0) {
    const long long now = clock64();
    const unsigned cur = (unsigned)ph_current();
    if (cur < (unsigned)NPHASE)
      atomicAdd(&g_phase_cycles[blockIdx.x & 255][cur], (unsigned long long)(now - ph_clock()));
    ph_clock() = now;
    ph_current() = k;
  }
}
#else
__device__ __forceinline__ void ph_start(int) {}
__device__ __forceinline__ void ph_mark(int) {}
#endif

// ------------------------------------------------------------------ groups
template <int G>
struct Grp {
  unsigned mask;
  int rank;
  __device__ __forceinline__ Grp() {
    const int l = threadIdx.x & 31;
    rank = l % G;
    mask = (G == 32) ? FULL_MASK : (((1u << G) - 1u) << (l - rank));
  }
  __device__ __forceinline__ void sync() const {
    if (G > 1) __syncwarp(mask);
  }
  __device__ __forceinline__ double sum(double v) const {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
    return v;
  }
  // The same sum when only ranks [0, nl) can hold nonzero values: a
  // butterfly over the smallest power-of-two span of ranks holding them,
  // then rank 0's total to every lane.  FP64 adds are charged per warp
  // instruction however few lanes use them, so a 3-species cell on 32 lanes
  // adds in 2 levels instead of 5 (the broadcast is an integer shuffle).
  // nl >= G gives sum(v) unchanged, bit for bit.
  __device__ __forceinline__ double sum_first(double v, int nl) const {
    if (G == 1) return v;
    int span = G;
    while (span > 1 && (span >> 1) >= nl) span >>= 1;
    if (span == G) return sum(v);
    for (int o = span >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
    return __shfl_sync(mask, v, 0, G);
  }
  __device__ __forceinline__ bool any(bool p) const {
    if (G == 1) return p;
    return (__ballot_sync(mask, p) & mask) != 0u;
  }
  __device__ __forceinline__ double bcast(double v, int src) const {
    return G > 1 ? __shfl_sync(mask, v, src, G) : v;
  }
  __device__ __forceinline__ int bcast(int v, int src) const {
    return G > 1 ? __shfl_sync(mask, v, src, G) : v;
  }
  __device__ __forceinline__ float bcast(float v, int src) const {
    return G > 1 ? __shfl_sync(mask, v, src, G) : v;
  }
};

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// |a| as an integer key (the bit patterns of non-negative IEEE values order
// like the values; a NaN's key exceeds infinity's), and infinity's key
__device__ __forceinline__ long long abs_key_t(double a) {
  return __double_as_longlong(a) & 0x7fffffffffffffffLL;
}
__device__ __forceinline__ long long abs_key_t(float a) {
  return (long long)(__float_as_uint(a) & 0x7fffffffu);
}
template <typename T>
__host__ __device__ constexpr long long inf_key() {
  return sizeof(T) == 8 ? 0x7ff0000000000000LL : 0x7f800000LL;
}

// lane grid for 2-D work on a group's matrix: R rows x C columns of lanes
template <int G>
struct LaneGrid {
  static constexpr int R = G >= 16 ? 4 : (G >= 4 ? 2 : 1);
  static constexpr int C = G / R;
};

constexpr int ZCOLS = 6;      // Nordsieck columns z_0 .. z_5 (orders <= 5)

// ------------------------------------------------------- BDF coefficients
constexpr int QMAX = 5;

// constant-step Nordsieck coefficients and error constants of orders 1..QMAX
struct Consts {
  double l[QMAX + 1][QMAX + 1];  // l[q][j], coefficients of prod_{i<=q} (1 + x/i)
  double rl1[QMAX + 1];          // 1 / l[q][1]
  double E[QMAX + 1][3];         // E_q, E_{q-1}, E_{q+1}
  double E2[QMAX + 1][3];        // their squares
  double qfact[QMAX + 2];        // q!
};

// the tables above, built on the host once
inline Consts make_consts() {
  Consts K;
  std::memset(&K, 0, sizeof K);
  for (int q = 1; q <= QMAX; ++q) {
    double l[QMAX + 2] = {0};
    l[0] = 1.0;
    for (int i = 1; i <= q; ++i)
      for (int j = i; j >= 1; --j) l[j] += l[j - 1] / (double)i;
    for (int j = 0; j <= q; ++j) K.l[q][j] = l[j];
  }
  K.qfact[0] = 1.0;
  for (int q = 1; q <= QMAX + 1; ++q) K.qfact[q] = K.qfact[q - 1] * q;
  for (int q = 1; q <= QMAX; ++q) {
    K.rl1[q] = 1.0 / K.l[q][1];
    K.E[q][0] = 1.0 / ((q + 1) * K.l[q][1]);
    K.E[q][1] = q > 1 ? K.qfact[q - 1] / K.l[q - 1][1] : 0.0;
    if (q < QMAX) {
      // l_1 of order q+1
      double l1 = 0.0;
      for (int i = 1; i <= q + 1; ++i) l1 += 1.0 / (double)i;
      K.E[q][2] = 1.0 / ((q + 2) * l1);
    }
    for (int k = 0; k < 3; ++k) K.E2[q][k] = K.E[q][k] * K.E[q][k];
  }
  return K;
}


// reaction rates (RHS scratch) and dr[a][r] = d rate_r / d y_(reactant a) at
// the setup point (mass action).  FP64 path: the rates live only inside a RHS call and
// the derivatives only inside a setup, so they share storage; the mixed path
// keeps the derivatives for the refinement residual of every Newton step.
template <int NMAX, bool SHARE, bool DR>
struct RateBufs {
  double rates[2 * NMAX];
  double dr[4][DR ? 2 * NMAX : 1];   // [reactant slot][reaction]: lanes over reactions hit distinct banks
};
template <int NMAX>
struct RateBufs<NMAX, true, true> {
  union {
    double rates[2 * NMAX];
    double dr[4][2 * NMAX];
  };
};

// the per-reaction derivatives pay off from 16 species up (below, a tile
// holds many small cells and the shared memory goes to residency)
template <int NMAX, int PREC>
struct UsesDr {
  static constexpr bool value = PREC == 1 || NMAX >= 16;
};
// the largest FP64 cells keep those derivatives (touched only at a setup) in a
// per-warp global workspace instead: their shared memory bounds residency,
// and 8 rather than 7 warps per SM fit without them
template <int NMAX, int PREC>
struct DrGlobal {
  static constexpr bool value = PREC != 1 && NMAX >= 56;
};

// where the history saved before a step attempt lives: 0 the group's shared
// memory, 1 registers (the FP64 kernels of the largest cells), 2 the warp's
// global workspace beside the FP64 fallback matrix (the mixed-precision
// kernels of the largest cells, whose registers are taken: leaving shared
// memory lets 12 warps per SM fit instead of 10).  It is written once per
// attempt and read back only when the attempt fails.
template <int NMAX, int PREC>
struct ZHome {
  static constexpr int value = NMAX >= 56 ? (PREC == 1 ? 2 : 1) : 0;
};
template <bool AWAY, int NMAX>
struct ZsBuf {
  double zs[ZCOLS][NMAX];
};
template <int NMAX>
struct ZsBuf<true, NMAX> {};

// per-cell shared memory.  PREC = 0: M and its LU factors in FP64.  PREC = 1
// (mixed precision): M and its LU factors in FP32 (pivot reciprocals in the
// float view of dinv).  PREC = 2: M and its Gauss-Jordan inverse in FP64.
// All keep the
// FP64 reaction derivatives of the last setup (computed once per reaction, then
// gathered into the rows of J; mixed precision reuses them in the refinement
// residual).
template <int NMAX, int PREC = 0>
struct CellSmem : RateBufs<NMAX, PREC != 1, UsesDr<NMAX, PREC>::value && !DrGlobal<NMAX, PREC>::value>,
                  ZsBuf<ZHome<NMAX, PREC>::value != 0, NMAX> {
  static constexpr bool DR = UsesDr<NMAX, PREC>::value;
  static constexpr bool DRG = DrGlobal<NMAX, PREC>::value;   // derivatives in global memory
  typename std::conditional<PREC == 1, float, double>::type M[NMAX][NMAX + 1];
  // history saved before a step attempt (zs, the base); the FP64 kernel of
  // the largest cells keeps it in registers instead
  static constexpr bool ZREG = ZHome<NMAX, PREC>::value == 1;
  static constexpr bool ZGLOB = ZHome<NMAX, PREC>::value == 2;
  double dinv[NMAX];          // 1 / U_kk
  double ybuf[NMAX];          // gathered state / right-hand side
  int16_t perm[NMAX];         // row i of P M is row perm[i] of M
};

template <int NPL, typename T>
__device__ __forceinline__ T pick(const T (&x)[NPL], int slot) {
  T v = x[0];
#pragma unroll
  for (int s = 1; s < NPL; ++s)
    if (slot == s) v = x[s];
  return v;
}
template <int NPL, typename T>
__device__ __forceinline__ void place(T (&x)[NPL], int slot, T v) {
#pragma unroll
  for (int s = 0; s < NPL; ++s)
    if (slot == s) x[s] = v;
}

// description of one cell's problem data (global memory)
struct CellDesc {
  int n, nr, kind;
  const double* k;          // mass action: rate per reaction; Robertson: (k1, k2, k3)
  const uint32_t* reac;     // 4 reactant species packed in bytes (255 = none)
  const int32_t* inc_off;   // species i of this cell: entries inc_off[i] .. inc_off[i+1)
  const uint16_t* inc;      // (reaction << 1) | (1 if produced, 0 if consumed)
  // one-warp cells of more than 32 species: the species whose sums lane l
  // forms (gs[l], up to four species bytes, low byte first, 255 = none), or
  // null; see gather_species_bal
  const uint32_t* gs;
};

// sqrt(sum (x_i w_i)^2 / n) over the group's elements
template <int G, int NPL>
__device__ __forceinline__ double wrms(const Grp<G>& g, int n, const double (&x)[NPL],
                                       const double (&w)[NPL]) {
  double s = 0.0;
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    if (i < n) {
      const double v = x[p] * w[p];
      s = fma(v, v, s);
    }
  }
  return sqrt(g.sum_first(s, n) / (double)n);
}

// squared WRMS norm, sum (x_i w_i)^2 / n, in FP64 (rn = 1/n).  The step loop
// compares squared norms, which keeps its tests in FP64 without a square root.
template <int G, int NPL>
__device__ __forceinline__ double wrms2(const Grp<G>& g, int n, double rn, const double (&x)[NPL],
                                        const double (&w)[NPL]) {
  double s = 0.0;
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    if (i < n) {
      const double v = x[p] * w[p];
      s = fma(v, v, s);
    }
  }
  return g.sum_first(s, n) * rn;
}

// step-size ratio 1 / ((safety^2 d2)^(e) + 1e-6) from a squared error norm d2,
// in FP32 (about 7 significant digits): the seed of eta64 and the value the
// step/order choice is made on when no two candidates are near a tie
__device__ __forceinline__ double eta_from(double d2, float safety2, float e) {
  const float x = fmaxf((float)fmin(d2 * safety2, 1.0e30), 1.0e-37f);
  return (double)(1.0f / (exp2f(e * __log2f(x)) + 1.0e-6f));
}

// the same ratio from FP32 work only: the squared norm converted on the
// integer pipe (to_f32), clamped to [1e-37, 1e30] (NaN to the upper end), so
// no FP64 instruction is issued -- the seed of the step/order choice
__device__ __forceinline__ float eta_f(double d2, float safety2, float e) {
  float x = to_f32(d2) * safety2;
  if (!(x <= 1.0e30f)) x = 1.0e30f;
  if (x < 1.0e-37f) x = 1.0e-37f;
  return 1.0f / (exp2f(e * __log2f(x)) + 1.0e-6f);
}

// 2^n as a double for -1022 <= n <= 1023 (built from the exponent bits)
__device__ __forceinline__ double pow2i(int n) {
  return __longlong_as_double((long long)(n + 1023) << 52);
}

// 1 / a for a > 0 normal: the FP32 reciprocal refined by one Newton step,
// y <- y (2 - a y), in FP64 (relative error about 2^-47)
__device__ __forceinline__ double recip64(double a) {
  const double y = (double)__frcp_rn((float)a);
  return y * fma(-a, y, 2.0);
}

// x^(1/k) for an even k in [2, 14] and x >= 0, to about 1e-13 relative: the
// argument is reduced by an exact power of two 2^(jk) (root scaled by 2^j),
// an FP32 root of the reduced argument seeds one Newton step for r^k = x,
// r <- r + r (x / r^k - 1) / k, in FP64.
__device__ __forceinline__ double root_k(double x, int k, double rk) {
  if (!(x > 0.0)) return 0.0;
  if (!(x < 1.0e308)) return x;
  const int e = (int)((__double_as_longlong(x) >> 52) & 0x7ff) - 1023;
  const int j = e / k;
  const double xs = x * pow2i(-j * k);          // |log2 xs| < k + 1: inside the FP32 range
  const double r = (double)exp2f(__log2f((float)xs) / (float)k);
  const double s = r * r;
  double p = s;                                 // r^k = s^(k/2)
  for (int i = 2; i < k; i += 2) p *= s;
  const double t = fma(xs, recip64(p), -1.0);   // x / r^k - 1, about 1e-7
  return fma(r * t, rk, r) * pow2i(j);
}

// 1 / k for an even k in [2, 14] without an FP64 division
__device__ __forceinline__ double inv_even(int k) {
  switch (k) {
    case 2: return 1.0 / 2.0;
    case 4: return 1.0 / 4.0;
    case 6: return 1.0 / 6.0;
    case 8: return 1.0 / 8.0;
    case 10: return 1.0 / 10.0;
    case 12: return 1.0 / 12.0;
    default: return 1.0 / 14.0;
  }
}

// the FP64 counterpart of eta_from: 1 / ((safety^2 d2)^(1/k) + 1e-6), k even
__device__ __forceinline__ double eta64(double d2, double safety2, int k) {
  return recip64(root_k(d2 * safety2, k, inv_even(k)) + 1.0e-6);
}

// finiteness on the integer pipe: an IEEE double is inf or NaN exactly when
// its exponent bits are all ones
__device__ __forceinline__ bool finite_bits(double x) {
  return (__double_as_longlong(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}

// a + b for a produced species (plus = 1), a - b for a consumed one: one FP64
// add of b with its sign bit set from the flag on the integer pipe (a - b is
// a + (-b) exactly), where a select between the two sums would issue both
__device__ __forceinline__ double add_signed(double a, double b, uint32_t plus) {
  return a + __longlong_as_double(__double_as_longlong(b) ^ ((long long)(~plus & 1u) << 63));
}
__device__ __forceinline__ float add_signed(float a, float b, uint32_t plus) {
  return a + __uint_as_float(__float_as_uint(b) ^ ((~plus & 1u) << 31));
}

// 1 / a for a finite nonzero a: recip_nr of |a| with a's sign put back on
// the integer pipe (four FP64 FMAs where a division issues many more)
__device__ __forceinline__ double recip_signed(double a) {
  const long long sgn = __double_as_longlong(a) & (long long)0x8000000000000000ULL;
  const double r = recip_nr(__longlong_as_double(__double_as_longlong(a) ^ sgn));
  return __longlong_as_double(__double_as_longlong(r) ^ sgn);
}
__device__ __forceinline__ float recip_t(float a) { return 1.0f / a; }
__device__ __forceinline__ double recip_t(double a) { return recip_signed(a); }

template <int G, int NPL>
__device__ __forceinline__ bool all_finite(const Grp<G>& g, int n, const double (&x)[NPL]) {
  bool bad = false;
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    if (i < n && !finite_bits(x[p])) bad = true;
  }
  return !g.any(bad);
}

template <int G, int NPL, int NMAX, int PREC>
__device__ __forceinline__ void scatter_y(const Grp<G>& g, CellSmem<NMAX, PREC>& S, int n,
                                          const double (&y)[NPL]) {
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    if (i < n) S.ybuf[i] = y[p];
  }
  g.sync();
}

// out_i = sum of +vals[r] over the reactions r producing species i and -vals[r]
// over those consuming it, in incidence-list (reaction) order.  One pass over
// the lane's species' lists back to back (a running sum flushed at each
// species), so that the group waits for the longest total, not for the
// longest list of every slot.
template <int G, int NPL>
__device__ __forceinline__ void gather_species(const Grp<G>& g, const CellDesc& c, const double* vals,
                                               double (&out)[NPL]) {
#pragma unroll
  for (int p = 0; p < NPL; ++p) out[p] = 0.0;
  int p = 0, e = 0, e1 = 0;
  double acc = 0.0;
  if (g.rank < c.n) { e = __ldg(c.inc_off + g.rank); e1 = __ldg(c.inc_off + g.rank + 1); }
  else p = NPL;
  while (p < NPL) {
    if (e < e1) {
      // four entries per trip: their index and value loads are in flight
      // together, the adds stay in list order
      const int m = min(4, e1 - e);
      uint32_t v[4];
      double r[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = u < m ? __ldg(c.inc + e + u) : 0u;
#pragma unroll
      for (int u = 0; u < 4; ++u) r[u] = vals[v[u] >> 1];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (u < m) acc = add_signed(acc, r[u], v[u]);
      e += m;
    } else {
      place(out, p, acc);
      acc = 0.0;
      ++p;
      const int i = g.rank + G * p;
      if (p < NPL && i < c.n) { e = __ldg(c.inc_off + i); e1 = __ldg(c.inc_off + i + 1); }
      else p = NPL;
    }
  }
}

// The same sums for a one-warp cell of more than 32 species, with the
// species spread over the lanes by a schedule built when the problem is
// created (longest lists first, each to the lane with the least work), so that
// the warp waits for about the mean of the lanes' list lengths instead of the
// longest pair of lists.  Every species is still summed alone, from zero, in
// incidence-list order, so the sums equal gather_species's bit for bit; they
// go through `sums` (n doubles of shared memory, free while the gather runs)
// to the lanes that own the species.
template <int G, int NPL>
__device__ __forceinline__ void gather_species_bal(const Grp<G>& g, const CellDesc& c, const double* vals,
                                                   double* sums, double (&out)[NPL]) {
  uint32_t sl = __ldg(c.gs + g.rank);
  int sp = (int)(sl & 255u);
  int e = 0, e1 = 0;
  double acc = 0.0;
  if (sp != 255) { e = __ldg(c.inc_off + sp); e1 = __ldg(c.inc_off + sp + 1); }
  while (sp != 255) {
    if (e < e1) {
      const int m = min(4, e1 - e);
      uint32_t v[4];
      double r[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = u < m ? __ldg(c.inc + e + u) : 0u;
#pragma unroll
      for (int u = 0; u < 4; ++u) r[u] = vals[v[u] >> 1];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (u < m) acc = add_signed(acc, r[u], v[u]);
      e += m;
    } else {
      sums[sp] = acc;
      acc = 0.0;
      sl = (sl >> 8) | 0xff000000u;
      sp = (int)(sl & 255u);
      if (sp != 255) { e = __ldg(c.inc_off + sp); e1 = __ldg(c.inc_off + sp + 1); }
    }
  }
  g.sync();
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    out[p] = i < c.n ? sums[i] : 0.0;
  }
}

// ------------------------------------------------------------ right-hand side
// f = f(y).  Mass action: rate_r = k_r prod_{s in R(r)} y_s, then each species
// sums -rate over reactions consuming it and +rate over reactions producing
// it, in reaction order (the incidence lists are built in that order).
template <int G, int NPL, int NMAX, int PREC>
__device__ __forceinline__ void rhs(const Grp<G>& g, const CellDesc& c, CellSmem<NMAX, PREC>& S, const double (&y)[NPL],
                    double (&f)[NPL]) {
  ph_mark(PH_RATES);
  scatter_y<G, NPL, NMAX>(g, S, c.n, y);
  if (c.kind == BDFB_ROBERTSON) {
    const double* k = c.k;
    const double y0 = S.ybuf[0], y1 = S.ybuf[1], y2 = S.ybuf[2];
    // every lane forms the three rows and keeps its own: FP64 instructions
    // cost a warp issue slot whatever the active lanes, so per-row branches
    // would issue each row's arithmetic separately
    const double b = k[2] * y1 * y2, c2 = k[1] * y1 * y1;
    const double f0 = fma(-k[0], y0, b), f1 = fma(k[0], y0, -b) - c2;
#pragma unroll
    for (int p = 0; p < NPL; ++p) {
      const int i = g.rank + G * p;
      f[p] = i == 0 ? f0 : (i == 1 ? f1 : (i == 2 ? c2 : 0.0));
    }
  } else {
    for (int r = g.rank; r < c.nr; r += G) {
      const uint32_t rc = __ldg(c.reac + r);
      double rate = __ldg(c.k + r);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const uint32_t s = (rc >> (8 * a)) & 255u;
        if (s != 255u) rate *= S.ybuf[s];
      }
      S.rates[r] = rate;
    }
    g.sync();
    ph_mark(PH_GATHER);
    if (G == 32 && NPL > 1 && c.gs) gather_species_bal<G, NPL>(g, c, S.rates, S.ybuf, f);
    else gather_species<G, NPL>(g, c, S.rates, f);
  }
  g.sync();
}

// M = I - gamma J(y) into shared memory (rows owned by lanes).  J entries are
// accumulated in reaction order as in the definition; M is formed without a
// fused multiply-add so it equals the textbook rounding of 1 - gamma J.
template <int G, int NPL, int NMAX, int PREC>
__device__ __forceinline__ void form_M(const Grp<G>& g, const CellDesc& c, CellSmem<NMAX, PREC>& S,
                       const double (&y)[NPL], double gamma) {
  scatter_y<G, NPL, NMAX>(g, S, c.n, y);
  const int n = c.n;
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    if (i >= n) continue;
    double* row = S.M[i];
    for (int j = 0; j < n; ++j) row[j] = 0.0;
    if (c.kind == BDFB_ROBERTSON) {
      // the entries once for every lane, each lane keeping its row (no
      // divergent per-row FP64 branches)
      const double* k = c.k;
      const double y1 = S.ybuf[1], y2 = S.ybuf[2];
      const double a = k[2] * y2, b = k[2] * y1, d = 2.0 * k[1] * y1;
      const double m11 = -a - d;
      row[0] = i == 0 ? -k[0] : (i == 1 ? k[0] : 0.0);
      row[1] = i == 0 ? a : (i == 1 ? m11 : d);
      row[2] = i == 0 ? b : (i == 1 ? -b : 0.0);
    } else {
      const int e1 = __ldg(c.inc_off + i + 1);
      for (int e = __ldg(c.inc_off + i); e < e1; ++e) {
        const uint32_t v = __ldg(c.inc + e);
        const int r = (int)(v >> 1);
        const uint32_t rc = __ldg(c.reac + r);
        const double kr = __ldg(c.k + r);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const uint32_t s = (rc >> (8 * a)) & 255u;
          if (s == 255u) continue;
          double d = kr;
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const uint32_t sb = (rc >> (8 * b)) & 255u;
            if (b != a && sb != 255u) d *= S.ybuf[sb];
          }
          row[s] = add_signed(row[s], d, v);
        }
      }
    }
    for (int j = 0; j < n; ++j) row[j] = __dsub_rn(i == j ? 1.0 : 0.0, __dmul_rn(gamma, row[j]));
  }
  g.sync();
}

// ---------------------------------------------------------------- dense LU
// Partial pivoting's row choice at column k: the row i in [k, n) of largest
// |M[i][k]| (ties to the lowest row) and its key (the bit pattern of |M[i][k]|,
// which orders like the value; a NaN's key exceeds infinity's), -1 when the
// group holds no row.  Each lane scans its rows, then warp reductions on the
// integer pipe (redux.sync) combine the lanes: an FP32 key in one maximum, an
// FP64 key by its high word and then its low word, then the lowest row that
// holds the maximum -- three dependent reductions where a shuffle butterfly
// takes log2(G) rounds of three shuffles each.
template <int G, int NMAX, typename T>
__device__ __forceinline__ int pivot_search(const Grp<G>& g, const T (*M)[NMAX + 1], int n, int k,
                                            long long& key) {
  long long best = -1;
  int p = n;
  for (int i = k + g.rank; i < n; i += G) {
    const long long v = abs_key_t(M[i][k]);
    if (v > best) { best = v; p = i; }
  }
  if constexpr (G == 1) {
    key = best;
    return p;
  } else if constexpr (sizeof(T) == 4) {
    const unsigned u = (unsigned)(best + 1);          // keys < 2^31; 0: no row
    const unsigned m = __reduce_max_sync(g.mask, u);
    const unsigned r = __reduce_min_sync(g.mask, (m != 0u && u == m) ? (unsigned)p : 0xffffffffu);
    key = (long long)m - 1;
    return m ? (int)r : n;
  } else {
    const unsigned hi = best >= 0 ? (unsigned)(best >> 32) + 1u : 0u;   // 0: no row
    const unsigned mh = __reduce_max_sync(g.mask, hi);
    const bool top = mh != 0u && hi == mh;
    const unsigned ml = __reduce_max_sync(g.mask, top ? (unsigned)best : 0u);
    const unsigned r = __reduce_min_sync(g.mask, (top && (unsigned)best == ml) ? (unsigned)p : 0xffffffffu);
    key = mh ? (((long long)(mh - 1u) << 32) | (long long)ml) : -1;
    return mh ? (int)r : n;
  }
}

// Right-looking LU with partial pivoting of the n x n matrix in S.M (ties in
// |pivot| go to the lowest row).  Returns 0 or k + 1 when pivot k is zero (or
// no finite pivot exists).  pivk (optional) records the pivot row of each step.
// One pivot at a time (the small groups, where the lanes form no grid).
// UNITU: the strictly upper part is stored divided by its row's pivot (P M =
// L D U' with U' unit upper, D = diag(1 / dinv)), so that a solve needs one
// vector scaling by dinv instead of a multiply per back-substitution column.
template <int G, int NMAX, typename T, bool UNITU = false>
__device__ __forceinline__ int lu_factor1(const Grp<G>& g, T (*M)[NMAX + 1], T* dinv, int16_t* perm, int n,
                          int16_t* pivk = nullptr) {
  for (int i = g.rank; i < n; i += G) perm[i] = (int16_t)i;
  g.sync();
  for (int k = 0; k < n; ++k) {
    // pivot search on integer keys (a NaN key exceeds every finite one and
    // is rejected below)
    long long best;
    const int p = pivot_search<G, NMAX, T>(g, M, n, k, best);
    if (p >= n || best <= 0 || best >= inf_key<T>()) return k + 1;
    if (pivk && g.rank == 0) pivk[k] = (int16_t)p;
    if (p != k) {
      for (int j = g.rank; j < n; j += G) {
        const T a = M[k][j];
        M[k][j] = M[p][j];
        M[p][j] = a;
      }
      if (g.rank == 0) {
        const int16_t a = perm[k];
        perm[k] = perm[p];
        perm[p] = a;
      }
    }
    g.sync();
    const T rinv = recip_t(M[k][k]);
    if (g.rank == 0) dinv[k] = rinv;
    for (int i = k + 1 + g.rank; i < n; i += G) M[i][k] *= rinv;
    g.sync();
    // rank-1 update of the trailing block, lanes on an R x C grid
    {
      constexpr int R = LaneGrid<G>::R, C = LaneGrid<G>::C;
      constexpr int NJ = (NMAX + C - 1) / C;
      const int li = g.rank / C, lj = g.rank % C;
      // column slots that still hold trailing columns (the same for the
      // whole group): slots past it would issue predicated-off FP64 work
      const int nbu = (n - k - 1 + C - 1) / C;
      T u[NJ];
#pragma unroll
      for (int b = 0; b < NJ; ++b) {
        if (b >= nbu) break;
        const int j = k + 1 + lj + C * b;
        u[b] = j < n ? M[k][j] : (T)0;
      }
      for (int i = k + 1 + li; i < n; i += R) {
        const T lik = M[i][k];
#pragma unroll
        for (int b = 0; b < NJ; ++b) {
          if (b >= nbu) break;
          const int j = k + 1 + lj + C * b;
          if (j < n) M[i][j] = fma_t(-lik, u[b], M[i][j]);
        }
      }
      if constexpr (UNITU) {
        g.sync();                     // every lane has read row k
        for (int j = k + 1 + g.rank; j < n; j += G) M[k][j] *= rinv;
      }
    }
    g.sync();
  }
  return 0;
}

// Partial pivoting at column k (rows k..n-1): the largest |M[i][k]|, ties to
// the lowest row, found on integer keys (the bit patterns of non-negative
// IEEE doubles order like their values; a NaN key exceeds every finite one and
// is rejected), then rows k and p swapped across all columns.  Returns false
// when the pivot is zero or not finite.
template <int G, int NMAX, typename T>
__device__ __forceinline__ bool pivot_swap(const Grp<G>& g, T (*M)[NMAX + 1], int16_t* perm, int n, int k,
                                           int16_t* pivk) {
  long long best;
  const int p = pivot_search<G, NMAX, T>(g, M, n, k, best);
  if (p >= n || best <= 0 || best >= inf_key<T>()) return false;
  if (pivk && g.rank == 0) pivk[k] = (int16_t)p;
  if (p != k) {
    for (int j = g.rank; j < n; j += G) {
      const T a = M[k][j];
      M[k][j] = M[p][j];
      M[p][j] = a;
    }
    if (g.rank == 0) {
      const int16_t a = perm[k];
      perm[k] = perm[p];
      perm[p] = a;
    }
  }
  g.sync();
  return true;
}

// LU with partial pivoting, P M = L U, in place (L unit lower below the
// diagonal, U on and above; dinv[k] = 1 / U_kk; perm: row i of P M is row
// perm[i] of M; pivk[k], if given, the row swapped with k at step k).  Returns
// 0, or k + 1 when pivot k is zero or not finite.
// Pivots are taken two at a time: column k is pivoted and scaled, column k+1
// receives step k's update and is pivoted and scaled, row k+1 receives step
// k's update, and the trailing block takes both rank-1 updates in one pass
// (each element read and written once per two pivots, the two fused
// multiply-adds in the order of two single steps, so the factors are those
// of the one-pivot-at-a-time elimination bit for bit).
// UNITU: the strictly upper part is stored divided by its row's pivot (P M =
// L D U' with U' unit upper, D = diag(1 / dinv)), so that a solve needs one
// vector scaling by dinv instead of a multiply per back-substitution column.
template <int G, int NMAX, typename T, bool UNITU = false>
__device__ __forceinline__ int lu_factor(const Grp<G>& g, T (*M)[NMAX + 1], T* dinv, int16_t* perm, int n,
                         int16_t* pivk = nullptr) {
  if constexpr (G < 8) {
    return lu_factor1<G, NMAX, T, UNITU>(g, M, dinv, perm, n, pivk);
  } else {
  for (int i = g.rank; i < n; i += G) perm[i] = (int16_t)i;
  g.sync();
  constexpr int R = LaneGrid<G>::R, C = LaneGrid<G>::C;
  constexpr int NJ = (NMAX + C - 1) / C;
  const int li = g.rank / C, lj = g.rank % C;
  int k = 0;
  for (; k + 1 < n; k += 2) {
    const int k1 = k + 1, k2 = k + 2;
    ph_mark(PH_LU_PIV);
    // ---- column k
    if (!pivot_swap<G, NMAX, T>(g, M, perm, n, k, pivk)) return k + 1;
    const T r0 = recip_t(M[k][k]);
    if (g.rank == 0) dinv[k] = r0;
    for (int i = k1 + g.rank; i < n; i += G) {
      const T l = M[i][k] * r0;
      M[i][k] = l;
      M[i][k1] = fma_t(-l, M[k][k1], M[i][k1]);     // column k+1 gets step k's update
    }
    g.sync();
    // ---- column k+1
    if (!pivot_swap<G, NMAX, T>(g, M, perm, n, k1, pivk)) return k1 + 1;
    const T r1 = recip_t(M[k1][k1]);
    if (g.rank == 0) dinv[k1] = r1;
    for (int i = k2 + g.rank; i < n; i += G) M[i][k1] *= r1;
    {
      const T l = M[k1][k];                        // row k+1 gets step k's update
      for (int j = k2 + g.rank; j < n; j += G) M[k1][j] = fma_t(-l, M[k][j], M[k1][j]);
    }
    g.sync();
    // ---- both updates of the trailing block, lanes on an R x C grid; column
    // slots past the trailing width would issue predicated-off FP64 work
    ph_mark(PH_LU_UPD);
    {
      const int nbu = (n - k2 + C - 1) / C;
      T u0[NJ], u1[NJ];
#pragma unroll
      for (int b = 0; b < NJ; ++b) {
        if (b >= nbu) break;
        const int j = k2 + lj + C * b;
        u0[b] = j < n ? M[k][j] : (T)0;
        u1[b] = j < n ? M[k1][j] : (T)0;
      }
      for (int i = k2 + li; i < n; i += R) {
        const T a0 = M[i][k], a1 = M[i][k1];
#pragma unroll
        for (int b = 0; b < NJ; ++b) {
          if (b >= nbu) break;
          const int j = k2 + lj + C * b;
          if (j < n) M[i][j] = fma_t(-a1, u1[b], fma_t(-a0, u0[b], M[i][j]));
        }
      }
      if constexpr (UNITU) {
        g.sync();                     // every lane has read rows k and k+1
        for (int j = k1 + g.rank; j < n; j += G) M[k][j] *= r0;
        for (int j = k2 + g.rank; j < n; j += G) M[k1][j] *= r1;
      }
    }
    g.sync();
  }
  if (k < n) {                        // the last pivot of an odd order
    if (!pivot_swap<G, NMAX, T>(g, M, perm, n, k, pivk)) return k + 1;
    if (g.rank == 0) dinv[k] = recip_t(M[k][k]);
    g.sync();
  }
  return 0;
  }
}

// x <- (P M)^{-1} P x with the factors above; x distributed over the group,
// held and updated in type V (FP64, or FP32 with FP32 factors)
template <int G, int NPL, int NMAX, typename T, bool UNITU = false, typename V = double>
__device__ __forceinline__ void lu_solve(const Grp<G>& g, const T (*M)[NMAX + 1], const T* dinv,
                         const int16_t* perm, V* buf, int n, V (&x)[NPL]) {
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    if (i < n) buf[i] = x[p];
  }
  g.sync();
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    if (i < n) x[p] = buf[perm[i]];
  }
  g.sync();
  // L y = P b (unit lower).  Columns j in [G s - 1, G (s + 1) - 1) have rows
  // below them only in slots s.. NPL-1: the slots are split at compile time,
  // since a predicated-off FP64 instruction costs an issue like a live one
  // (the column loops are kept rolled: unrolled by 2 or 4 they ran 1-7 %
  // slower, FP64 and FP32 alike)
  int j = 0;
#pragma unroll
  for (int s = 0; s < NPL; ++s) {
    const int jend = min(n - 1, G * (s + 1) - 1);
#pragma unroll 1
    for (; j < jend; ++j) {
      const V xj = g.bcast(pick(x, j / G), j % G);
#pragma unroll
      for (int p = s; p < NPL; ++p) {
        const int i = g.rank + G * p;
        if (i > j && i < n) x[p] = fma_t(-(V)M[i][j], xj, x[p]);
      }
    }
  }
  if constexpr (UNITU) {                         // y <- D^{-1} y
#pragma unroll
    for (int p = 0; p < NPL; ++p) {
      const int i = g.rank + G * p;
      if (i < n) x[p] *= (V)dinv[i];
    }
  }
  // U x = y (U' x = y when UNITU).  Columns j in (G s, G (s + 1)] have rows
  // above them only in slots 0..s
  j = n - 1;
#pragma unroll
  for (int s = NPL - 1; s >= 0; --s) {
    const int jlo = (s == 0 && !UNITU) ? -1 : G * s;   // column 0 scales its own entry
#pragma unroll 1
    for (; j > jlo; --j) {
      const int owner = j % G, slot = j / G;
      V xj = g.bcast(pick(x, slot), owner);
      if constexpr (!UNITU) {
        xj *= (V)dinv[j];
        if (g.rank == owner) place(x, slot, xj);
      }
#pragma unroll
      for (int p = 0; p <= s; ++p) {
        const int i = g.rank + G * p;
        if (i < j) x[p] = fma_t(-(V)M[i][j], xj, x[p]);
      }
    }
  }
}

}  // namespace bdfb
