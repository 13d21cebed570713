// mixed.cuh - FP32 factorisation of M = I - gamma J with FP64 iterative
// refinement, per cell (mass-action cells).
//
// B300 runs FP32 FMAs 64x faster than FP64 ones, so the block is factored in
// FP32 (LU with partial pivoting, the FP64 path's elimination in FP32; each
// correction is an FP32 forward and back substitution) and only the
// refinement residual r = b - M x is FP64.  An explicit FP32 Gauss-Jordan
// inverse (parallel matrix-vector corrections) issued three times the
// setup's instructions and was slower on B300.
// The residual does not store the FP64 matrix: M x = x - gamma J x with J x
// assembled from the reaction derivatives d rate_r / d y_s kept (FP64) from
// the setup point, reaction by reaction and species by species in the same
// incidence order as the right-hand side.  A solve is accepted at normwise
// backward error |r|_inf / (|M|_inf |x|_inf + |b|_inf) <= 1e-12; after
// MAXREF sweeps without that, the cell falls back to an FP64 LU of the same
// M (in a global-memory workspace) until its next setup.
#pragma once

#include "cellcore.cuh"

namespace bdfb {

constexpr int MAXREF = 5;
constexpr double BERR_TOL = 1e-12;

template <int G>
__device__ __forceinline__ double gmaxd(const Grp<G>& g, double v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(g.mask, v, o, G));
  return v;
}

// max |v| over the group on the integer pipe: the bit patterns of
// non-negative doubles order like their values (a NaN's key lies above
// infinity's, so a NaN wins and fails every later <= test); the maximum of
// the keys' high words, then of the low words of the keys that hold it (two
// redux.sync reductions)
__device__ __forceinline__ long long abs_key(double v) {
  return __double_as_longlong(v) & 0x7fffffffffffffffLL;
}
template <int G>
__device__ __forceinline__ double gmax_key(const Grp<G>& g, long long k) {
  if constexpr (G == 1) {
    return __longlong_as_double(k);
  } else {
    const unsigned hi = (unsigned)(k >> 32), lo = (unsigned)k;
    const unsigned mh = __reduce_max_sync(g.mask, hi);
    const unsigned ml = __reduce_max_sync(g.mask, hi == mh ? lo : 0u);
    return __longlong_as_double((long long)(((unsigned long long)mh << 32) | ml));
  }
}

template <int G>
__device__ __forceinline__ float bcastf(const Grp<G>& g, float v, int src) {
  return G > 1 ? __shfl_sync(g.mask, v, src, G) : v;
}

// scale * d rate_r / d y_{s_a} for every reaction r and reactant slot a at y
// (FP64), into S.dr (or drg, the per-warp global workspace of the cells whose
// shared memory holds no derivatives); lanes over reactions.  scale = 1: the derivatives
// themselves (kept by mixed precision for its residual); scale = -gamma:
// their contributions to M = I - gamma J (form_M64_scaled).
template <int G, int NPL, int NMAX, int PREC>
__device__ __forceinline__ void reaction_derivs(const Grp<G>& g, const CellDesc& c,
                                                CellSmem<NMAX, PREC>& S, const double (&y)[NPL],
                                                double scale = 1.0, double (*drg)[2 * NMAX] = nullptr) {
  double (*dr)[2 * NMAX];
  if constexpr (CellSmem<NMAX, PREC>::DRG) dr = drg;      // the per-warp global workspace
  else dr = S.dr;
  scatter_y<G, NPL, NMAX>(g, S, c.n, y);
  for (int r = g.rank; r < c.nr; r += G) {
    const uint32_t rc = __ldg(c.reac + r);
    const double kr = __ldg(c.k + r) * scale;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      double d = 0.0;
      if (((rc >> (8 * a)) & 255u) != 255u) {
        d = kr;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const uint32_t sb = (rc >> (8 * b)) & 255u;
          if (b != a && sb != 255u) d *= S.ybuf[sb];
        }
      }
      dr[a][r] = d;
    }
  }
  g.sync();
}

// FP32 copy of M = I - gamma J from S.dr (rows owned by lanes) into the
// packed float view of S.M; returns |M|_inf (group-uniform).
template <int G, int NPL, int NMAX>
__device__ __forceinline__ double form_M32(const Grp<G>& g, const CellDesc& c, CellSmem<NMAX, 1>& S,
                                           double gamma) {
  float (*M)[NMAX + 1] = reinterpret_cast<float (*)[NMAX + 1]>(&S.M[0][0]);
  const int n = c.n;
  const float gf = (float)gamma;
  double mnorm = 0.0;
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    if (i >= n) continue;
    float* row = M[i];
    for (int j = 0; j < n; ++j) row[j] = 0.0f;
    const int e1 = __ldg(c.inc_off + i + 1);
    for (int e = __ldg(c.inc_off + i); e < e1; ++e) {
      const uint32_t v = __ldg(c.inc + e);
      const int r = (int)(v >> 1);
      const uint32_t rc = __ldg(c.reac + r);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const uint32_t s = (rc >> (8 * a)) & 255u;
        if (s == 255u) continue;
        const float d = (float)S.dr[a][r];
        row[s] = add_signed(row[s], d, v);
      }
    }
    float rs = 0.0f;
    for (int j = 0; j < n; ++j) {
      const float m = (i == j ? 1.0f : 0.0f) - gf * row[j];
      row[j] = m;
      rs += fabsf(m);
    }
    mnorm = fmax(mnorm, (double)rs);
  }
  g.sync();
  return gmaxd(g, mnorm);
}

// FP64 M = I - gamma J from S.dr into Mg: the FP64 path's M in shared
// memory, or the mixed path's fallback matrix in the cell's global-memory
// workspace.  Rows are summed in the order of the direct definition (the
// incidence lists' reaction order), so M equals the entry-by-entry formation.
template <int G, int NPL, int NMAX, int PREC>
__device__ __forceinline__ void form_M64_from_dr(const Grp<G>& g, const CellDesc& c,
                                                 CellSmem<NMAX, PREC>& S, double gamma,
                                                 double (*Mg)[NMAX + 1]) {
  const int n = c.n;
  g.sync();
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    if (i >= n) continue;
    double* row = Mg[i];
    for (int j = 0; j < n; ++j) row[j] = 0.0;
    const int e1 = __ldg(c.inc_off + i + 1);
    for (int e = __ldg(c.inc_off + i); e < e1; ++e) {
      const uint32_t v = __ldg(c.inc + e);
      const int r = (int)(v >> 1);
      const uint32_t rc = __ldg(c.reac + r);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const uint32_t s = (rc >> (8 * a)) & 255u;
        if (s == 255u) continue;
        const double d = S.dr[a][r];
        row[s] = add_signed(row[s], d, v);
      }
    }
    for (int j = 0; j < n; ++j) row[j] = __dsub_rn(i == j ? 1.0 : 0.0, __dmul_rn(gamma, row[j]));
  }
  g.sync();
}

// M = I - gamma J into Mg from derivatives scaled by -gamma (reaction_derivs
// with scale = -gamma): row i accumulates, in reaction order, +d for the
// reactions producing species i and -d for those consuming it, then 1 on the
// diagonal -- no separate pass forming 1 - gamma J
template <int G, int NPL, int NMAX, int PREC>
__device__ __forceinline__ void form_M64_scaled(const Grp<G>& g, const CellDesc& c, CellSmem<NMAX, PREC>& S,
                                                double (*Mg)[NMAX + 1], const double (*drg)[2 * NMAX] = nullptr) {
  const double (*dr)[2 * NMAX];
  if constexpr (CellSmem<NMAX, PREC>::DRG) dr = drg;
  else dr = S.dr;
  const int n = c.n;
  g.sync();
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    if (i >= n) continue;
    double* row = Mg[i];
    for (int j = 0; j < n; ++j) row[j] = 0.0;
    const int e1 = __ldg(c.inc_off + i + 1);
    for (int e = __ldg(c.inc_off + i); e < e1; ++e) {
      const uint32_t v = __ldg(c.inc + e);
      const int r = (int)(v >> 1);
      const uint32_t rc = __ldg(c.reac + r);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const uint32_t s = (rc >> (8 * a)) & 255u;
        if (s == 255u) continue;
        const double d = dr[a][r];
        row[s] = add_signed(row[s], d, v);
      }
    }
    row[i] += 1.0;
  }
  g.sync();
}

// jx = J x (FP64) from the stored reaction derivatives
template <int G, int NPL, int NMAX>
__device__ __forceinline__ void jac_vec(const Grp<G>& g, const CellDesc& c, CellSmem<NMAX, 1>& S,
                                        const double (&x)[NPL], double (&jx)[NPL]) {
  scatter_y<G, NPL, NMAX>(g, S, c.n, x);
  for (int r = g.rank; r < c.nr; r += G) {
    const uint32_t rc = __ldg(c.reac + r);
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const uint32_t sp = (rc >> (8 * a)) & 255u;
      if (sp != 255u) s = fma(S.dr[a][r], S.ybuf[sp], s);
    }
    S.rates[r] = s;
  }
  g.sync();
  if (G == 32 && NPL > 1 && c.gs) gather_species_bal<G, NPL>(g, c, S.rates, S.ybuf, jx);
  else gather_species<G, NPL>(g, c, S.rates, jx);
  g.sync();
}


// In-place Gauss-Jordan inverse with partial pivoting (ties to the lowest
// row) of the n x n matrix A (FP32 or FP64); the block inverse the paper
// applies to its 3x3 reaction blocks (Sec. 7), here for any block size.
// Returns 0 or k + 1 when no nonzero pivot exists in column k.  piv (n
// entries) and colk (n values): scratch.
template <int G, int NMAX, typename T>
__device__ __forceinline__ int gj_inverse(const Grp<G>& g, T (*A)[NMAX + 1], int16_t* piv,
                                          T* colk, int n) {
  constexpr int R = LaneGrid<G>::R, C = LaneGrid<G>::C;
  constexpr int NJ = (NMAX + C - 1) / C;
  const int li = g.rank / C, lj = g.rank % C;
  for (int k = 0; k < n; ++k) {
    T best = T(-1);
    int p = n;
    for (int i = k + g.rank; i < n; i += G) {
      const T v = A[i][k] < T(0) ? -A[i][k] : A[i][k];
      if (v > best) { best = v; p = i; }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(g.mask, best, o, G);
      const int op = __shfl_xor_sync(g.mask, p, o, G);
      if (ob > best || (ob == best && op < p)) { best = ob; p = op; }
    }
    if (!(best > T(0)) || p >= n) return k + 1;
    if (g.rank == 0) piv[k] = (int16_t)p;
    if (p != k)
      for (int j = g.rank; j < n; j += G) {
        const T t = A[k][j];
        A[k][j] = A[p][j];
        A[p][j] = t;
      }
    g.sync();
    const T pinv = T(1) / A[k][k];
    g.sync();
    // row k <- row k / pivot, with the pivot slot becoming 1 / pivot; keep
    // column k (the elimination factors) before it is overwritten
    for (int j = g.rank; j < n; j += G) A[k][j] = (j == k) ? pinv : A[k][j] * pinv;
    for (int i = g.rank; i < n; i += G) colk[i] = A[i][k];
    g.sync();
    // eliminate column k from every other row (lanes on an R x C grid)
    T u[NJ];
#pragma unroll
    for (int b = 0; b < NJ; ++b) {
      const int j = lj + C * b;
      u[b] = j < n ? A[k][j] : T(0);
    }
    for (int i = li; i < n; i += R) {
      if (i == k) continue;
      const T f = colk[i];
#pragma unroll
      for (int b = 0; b < NJ; ++b) {
        const int j = lj + C * b;
        if (j < n) A[i][j] = (j == k) ? -f * u[b] : fma_t(-f, u[b], A[i][j]);
      }
    }
    g.sync();
  }
  // undo the row exchanges as column exchanges, last first
  for (int k = n - 1; k >= 0; --k) {
    const int p = piv[k];
    if (p != k)
      for (int i = g.rank; i < n; i += G) {
        const T t = A[i][k];
        A[i][k] = A[i][p];
        A[i][p] = t;
      }
    g.sync();
  }
  return 0;
}

// x = Ainv r (lanes own rows; r gathered through shared memory); x may
// alias r
template <int G, int NPL, int NMAX, typename T>
__device__ __forceinline__ void apply_inverse(const Grp<G>& g, const T (*Ainv)[NMAX + 1], T* buf,
                                              int n, const T (&r)[NPL], T (&x)[NPL]) {
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    if (i < n) buf[i] = r[p];
  }
  g.sync();
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    T s = T(0);
    if (i < n) {
      const T* row = Ainv[i];
      for (int j = 0; j < n; ++j) s = fma_t(row[j], buf[j], s);
    }
    x[p] = s;
  }
  g.sync();
}

// Solve M x = b (M = I - gammap J at the setup point) to backward error
// <= 1e-12 by corrections with the FP32 inverse in S.M and FP64 residuals;
// b is replaced by x.  Returns the number of sweeps, or -1 when the tolerance
// was not reached (b then holds the last iterate).
template <int G, int NPL, int NMAX>
__device__ __forceinline__ int refined_solve(const Grp<G>& g, const CellDesc& c, CellSmem<NMAX, 1>& S,
                                             double gammap, double mnorm, double (&b)[NPL]) {
  float* buf = reinterpret_cast<float*>(S.ybuf);
  const int n = c.n;
  double x[NPL], r[NPL], jx[NPL];
  // norms as integer keys and FP32 <-> FP64 conversions on the integer pipe
  // (to_f32 flushes magnitudes below 2^-126: a residual that small in every
  // entry ends the sweeps unconverged and takes the FP64 fallback)
  long long bk = 0;
  ph_mark(PH_NORM);
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    x[p] = 0.0;
    r[p] = b[p];
    if (g.rank + G * p < n) bk = max(bk, abs_key(b[p]));
  }
  const double bn = gmax_key(g, bk);
  int sweeps = -1;
  for (int it = 1; it <= MAXREF; ++it) {
    float c32[NPL];
#pragma unroll
    for (int p = 0; p < NPL; ++p) c32[p] = to_f32(r[p]);
    ph_mark(PH_TRI);
    lu_solve<G, NPL, NMAX, float, true, float>(g, S.M, reinterpret_cast<const float*>(S.dinv), S.perm, buf, n, c32);
    ph_mark(PH_RES);
#pragma unroll
    for (int p = 0; p < NPL; ++p) x[p] += to_f64(c32[p]);
    jac_vec<G, NPL, NMAX>(g, c, S, x, jx);
    ph_mark(PH_NORM);
    long long rk = 0, xk = 0;
#pragma unroll
    for (int p = 0; p < NPL; ++p) {
      r[p] = b[p] - fma(-gammap, jx[p], x[p]);
      if (g.rank + G * p < n) {
        rk = max(rk, abs_key(r[p]));
        xk = max(xk, abs_key(x[p]));
      }
    }
    const double rn = gmax_key(g, rk), xn = gmax_key(g, xk);
    if (rn <= BERR_TOL * (mnorm * xn + bn)) { sweeps = it; break; }
  }
#pragma unroll
  for (int p = 0; p < NPL; ++p) b[p] = x[p];
  return sweeps;
}

}  // namespace bdfb
