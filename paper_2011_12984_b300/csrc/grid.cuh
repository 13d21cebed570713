// grid.cuh - internal interface of the grouped (one coupled system) integrator
// for the Brusselator reaction-diffusion grid.
#pragma once

#include "common.cuh"

namespace bdfb {

struct GridBDF;

// kinds of timed operations of the profile option (bdfb_get_op_profile)
enum GridOp {
  GOP_WRMS, GOP_DOTS, GOP_LINCOMB, GOP_LINSUM, GOP_PREDICT, GOP_ACCEPT, GOP_RESCALE, GOP_EWT,
  GOP_NEWTON, GOP_MUL, GOP_RHS, GOP_APPLY, GOP_PSETUP, GOP_PSCALE, GOP_N
};

int grid_create(int nx, double A, double B, double eps, double D, GridBDF** out);
// dim 3: the nx^3 reaction-diffusion grid (D); dim 1: the advection-reaction
// line of nx points over [0, len) with speed c (first-order upwind)
int grid_create_line_or_cube(int dim, int64_t nx, double A, double B, double eps, double D, double c,
                             double len, GridBDF** out);
// A system whose right-hand side and Newton solve are supplied from outside
// (the grouped "task-local Newton" mode of the per-cell problems): the grid
// integrator's control (prediction, global error test, step and order
// selection) drives them.  rhs: f = f(y).  solve: given the predicted z0, z1,
// the error weights and gamma (gammap: gamma of the last setup; setup = 1
// asks for fresh Jacobians at z0 first), run the Newton iterations and
// leave the converged correction in acor; *failed = 1 when any part of the
// system did not converge; *iters = Newton iterations it took (summed over
// the parts), *sweeps = right-hand-side evaluations of the whole system they
// amount to.  Both return 0 or a negative code.
struct GridExternal {
  void* user;
  int (*rhs)(void* user, const double* y, double* f, cudaStream_t s);
  int (*solve)(void* user, const double* zp0, const double* zp1, const double* ewt, double gamma,
               double gammap, double rl1, double Eq, int setup, double* acor, int* failed, int64_t* iters,
               int64_t* sweeps, cudaStream_t s);
};
int grid_create_external(int64_t N, GridExternal ext, GridBDF** out);
void grid_destroy(GridBDF* g);
void grid_set_stream(GridBDF* g, cudaStream_t s);
void grid_set_tolerances(GridBDF* g, double rtol, double atol);
int grid_set_option(GridBDF* g, const char* key, int64_t v);
int grid_init(GridBDF* g, double t0, const double* y0, int mem);
int grid_integrate(GridBDF* g, double tout, double* y, int mem);
// stats: nst, nfe, nsetups, nni, ncfn, netf, nli (GMRES iterations), nlfail
void grid_stats(GridBDF* g, int64_t out[8], double* last_ms);
// order and step size the next step will try
void grid_next_step(GridBDF* g, int* q, double* h);
// option "profile": per GridOp kind, out[3k..3k+2] = launches, summed event
// milliseconds, summed algorithmic GB since the option was set
void grid_profile(GridBDF* g, double* out);

}  // namespace bdfb
