// sparse.cuh - block-diagonal matrices whose blocks share one sparsity
// pattern (Sec. 5: one copy of the CSR index arrays for all blocks), their
// batched LU factorisation and solve, and the integrator of many cells that
// share one (larger, sparse) mass-action network.
#pragma once

#include <vector>

#include "common.cuh"

namespace bdfb {

struct SharedInt;

// BDFB_MASSACTION_SHARED: cells [0, ncell) sharing the network of the
// problem; states species-major (y[s ncell + c]).  Integrated as one grouped
// system (grid integrator control) with task-local Newton solves per cell on
// the shared sparse pattern.
int shared_create(const bdfb_problem* prob, SharedInt** out);
void shared_destroy(SharedInt* S);
void shared_set_stream(SharedInt* S, cudaStream_t s);
void shared_set_tolerances(SharedInt* S, double rtol, double atol);
int shared_set_option(SharedInt* S, const char* key, int64_t v);
int shared_init(SharedInt* S, double t0, const double* y0, int mem);
int shared_integrate(SharedInt* S, double tout, double* y, int mem);
// option "grouped" 0: every cell with its own step size and order, one
// thread per cell on the shared sparse pattern (set before shared_init)
bool shared_percell(const SharedInt* S);
int shared_integrate_cells(SharedInt* S, double tout, double* y, int32_t* status, int mem);
// per-cell mode: rows of nst, nfe, nsetups, nni, ncfn, netf, qlast, hlast bits
int shared_cell_stats(SharedInt* S, std::vector<int64_t>& rows, double* last_ms);
// nst, nfe, nsetups, nni (summed over cells), ncfn, netf, LU entries of the
// shared pattern (with fill), entries of M's pattern; *q, *h of the next step
void shared_stats(SharedInt* S, int64_t out[8], double* last_ms, int* q, double* h);

}  // namespace bdfb
