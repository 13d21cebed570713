// mixed.cuh - FP32 factorisation of M = I - gamma J with FP64 iterative
// refinement, per cell (mass-action cells).
//
// B300 runs FP32 FMAs 64x faster than FP64 ones, so the block LU and the
// triangular solves run in FP32 and only the refinement residual r = b - M x
// is FP64.  The residual does not store the FP64 matrix: M x = x - gamma J x
// with J x assembled from the reaction derivatives d rate_r / d y_s kept
// (FP64) from the setup point, reaction by reaction and species by species
// in the same incidence order as the right-hand side.  A solve is accepted at
// normwise backward error |r|_inf / (|M|_inf |x|_inf + |b|_inf) <= 1e-12;
// after MAXREF sweeps without that, the cell falls back to an FP64 LU of the
// same M until its next setup.
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

template <int G>
__device__ __forceinline__ float bcastf(const Grp<G>& g, float v, int src) {
  return G > 1 ? __shfl_sync(g.mask, v, src, G) : v;
}

// d rate_r / d y_{s_a} for every reaction r and reactant slot a at y (FP64),
// into S.dr; lanes over reactions.
template <int G, int NPL, int NMAX>
__device__ __forceinline__ void reaction_derivs(const Grp<G>& g, const CellDesc& c,
                                                CellSmem<NMAX, 1>& S, const double (&y)[NPL]) {
  scatter_y<G, NPL, NMAX>(g, S, c.n, y);
  for (int r = g.rank; r < c.nr; r += G) {
    const uint32_t rc = __ldg(c.reac + r);
    const double kr = __ldg(c.k + r);
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
      S.dr[r][a] = d;
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
        const float d = (float)S.dr[r][a];
        row[s] = (v & 1u) ? row[s] + d : row[s] - d;
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

// FP64 M = I - gamma J from S.dr into S.M (the fallback factorisation)
template <int G, int NPL, int NMAX>
__device__ __forceinline__ void form_M64_from_dr(const Grp<G>& g, const CellDesc& c,
                                                 CellSmem<NMAX, 1>& S, double gamma) {
  const int n = c.n;
  g.sync();
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    if (i >= n) continue;
    double* row = S.M[i];
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
        const double d = S.dr[r][a];
        row[s] = (v & 1u) ? row[s] + d : row[s] - d;
      }
    }
    for (int j = 0; j < n; ++j) row[j] = __dsub_rn(i == j ? 1.0 : 0.0, __dmul_rn(gamma, row[j]));
  }
  g.sync();
}

// x <- (P M32)^{-1} P x in FP32 (factors in the packed float view of S.M)
template <int G, int NPL, int NMAX>
__device__ __forceinline__ void lu_solve32(const Grp<G>& g, CellSmem<NMAX, 1>& S, int n,
                                           float (&x)[NPL]) {
  const float (*M)[NMAX + 1] = reinterpret_cast<const float (*)[NMAX + 1]>(&S.M[0][0]);
  const float* dinv = reinterpret_cast<const float*>(S.dinv);
  float* buf = reinterpret_cast<float*>(S.ybuf);
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    if (i < n) buf[i] = x[p];
  }
  g.sync();
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    if (i < n) x[p] = buf[S.perm[i]];
  }
  g.sync();
  for (int j = 0; j < n; ++j) {
    const float xj = bcastf(g, pick(x, j / G), j % G);
#pragma unroll
    for (int p = 0; p < NPL; ++p) {
      const int i = g.rank + G * p;
      if (i > j && i < n) x[p] = fmaf(-M[i][j], xj, x[p]);
    }
  }
  for (int j = n - 1; j >= 0; --j) {
    const int owner = j % G, slot = j / G;
    const float xj = bcastf(g, pick(x, slot), owner) * dinv[j];
    if (g.rank == owner) place(x, slot, xj);
#pragma unroll
    for (int p = 0; p < NPL; ++p) {
      const int i = g.rank + G * p;
      if (i < j) x[p] = fmaf(-M[i][j], xj, x[p]);
    }
  }
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
      if (sp != 255u) s = fma(S.dr[r][a], S.ybuf[sp], s);
    }
    S.rates[r] = s;
  }
  g.sync();
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const int i = g.rank + G * p;
    double acc = 0.0;
    if (i < c.n) {
      const int e1 = __ldg(c.inc_off + i + 1);
      for (int e = __ldg(c.inc_off + i); e < e1; ++e) {
        const uint32_t v = __ldg(c.inc + e);
        const double rt = S.rates[v >> 1];
        acc = (v & 1u) ? acc + rt : acc - rt;
      }
    }
    jx[p] = acc;
  }
  g.sync();
}

// Solve M x = b (M = I - gammap J at the setup point) to backward error
// <= 1e-12 by FP32 LU solves and FP64 residuals; b is replaced by x.
// Returns the number of sweeps, or -1 when the tolerance was not reached
// (b then holds the last iterate).
template <int G, int NPL, int NMAX>
__device__ __forceinline__ int refined_solve(const Grp<G>& g, const CellDesc& c, CellSmem<NMAX, 1>& S,
                                             double gammap, double mnorm, double (&b)[NPL]) {
  const int n = c.n;
  double x[NPL], r[NPL], jx[NPL];
  double bn = 0.0;
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    x[p] = 0.0;
    r[p] = b[p];
    if (g.rank + G * p < n) bn = fmax(bn, fabs(b[p]));
  }
  bn = gmaxd(g, bn);
  int sweeps = -1;
  for (int it = 1; it <= MAXREF; ++it) {
    float c32[NPL];
#pragma unroll
    for (int p = 0; p < NPL; ++p) c32[p] = (float)r[p];
    lu_solve32<G, NPL, NMAX>(g, S, n, c32);
#pragma unroll
    for (int p = 0; p < NPL; ++p) x[p] += (double)c32[p];
    jac_vec<G, NPL, NMAX>(g, c, S, x, jx);
    double rn = 0.0, xn = 0.0;
#pragma unroll
    for (int p = 0; p < NPL; ++p) {
      r[p] = b[p] - fma(-gammap, jx[p], x[p]);
      if (g.rank + G * p < n) {
        rn = fmax(rn, fabs(r[p]));
        xn = fmax(xn, fabs(x[p]));
      }
    }
    rn = gmaxd(g, rn);
    xn = gmaxd(g, xn);
    if (rn <= BERR_TOL * (mnorm * xn + bn)) { sweeps = it; break; }
  }
#pragma unroll
  for (int p = 0; p < NPL; ++p) b[p] = x[p];
  return sweeps;
}

}  // namespace bdfb
