// grid.cuh - internal interface of the grouped (one coupled system) integrator
// for the Brusselator reaction-diffusion grid.
#pragma once

#include "common.cuh"

namespace bdfb {

struct GridBDF;

int grid_create(int nx, double A, double B, double eps, double D, GridBDF** out);
// dim 3: the nx^3 reaction-diffusion grid (D); dim 1: the advection-reaction
// line of nx points over [0, len) with speed c (first-order upwind)
int grid_create_line_or_cube(int dim, int64_t nx, double A, double B, double eps, double D, double c,
                             double len, GridBDF** out);
void grid_destroy(GridBDF* g);
void grid_set_stream(GridBDF* g, cudaStream_t s);
void grid_set_tolerances(GridBDF* g, double rtol, double atol);
int grid_set_option(GridBDF* g, const char* key, int64_t v);
int grid_init(GridBDF* g, double t0, const double* y0, int mem);
int grid_integrate(GridBDF* g, double tout, double* y, int mem);
// stats: nst, nfe, nsetups, nni, ncfn, netf, nli (GMRES iterations), nlfail
void grid_stats(GridBDF* g, int64_t out[8], double* last_ms);

}  // namespace bdfb
