// ark.cuh - IMEX additive Runge-Kutta integrator for the 1-D demonstration
// problem (Sec. 7): first-order upwind advection explicit, Brusselator
// reactions implicit, each implicit stage solved by Newton with the 3x3
// point blocks of the reaction Jacobian (one task per GPU).
#pragma once

#include "common.cuh"

namespace bdfb {

struct ArkLine;

// nx points on the periodic line [0, len), speed c, reactions A, B, eps
int ark_create(int64_t nx, double A, double B, double eps, double c, double len, ArkLine** out);
void ark_destroy(ArkLine* g);
void ark_set_stream(ArkLine* g, cudaStream_t s);
void ark_set_tolerances(ArkLine* g, double rtol, double atol);
int ark_set_mxstep(ArkLine* g, int64_t v);
// 0: FP64 throughout; 1: FP32 3x3 Newton blocks and norm weights, FP64 state,
// stage sums and Newton residual
int ark_set_precision(ArkLine* g, int prec);
// 1 (default where cooperative launches exist): the step loop to tout runs
// in one cooperative launch with grid-wide barriers instead of host round
// trips; 0: host-driven, one launch and one readback per reduction
int ark_set_device_loop(ArkLine* g, int on);
int ark_init(ArkLine* g, double t0, const double* y0, int mem);
// advance to tout (last step clamped onto tout); y (3 nx, species-major) out
int ark_integrate(ArkLine* g, double tout, double* y, int mem);
// nst, nfe (advection evaluations), nfi (reaction evaluations), nni, ncfn, netf, 0, 0
void ark_stats(ArkLine* g, int64_t out[8], double* last_ms);

}  // namespace bdfb
