// Launchers of the topology-optimisation kernels (ddel_topopt.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ddel_launch.h"

namespace ddel {

int filter_radius_cells(double r_min);
// Hat density filter (transpose = 0) or its transpose (the chain rule, transpose = 1).
void launch_filter(const DevTables& t, double r_min, const double* in, double* out, int transpose,
                   cudaStream_t st);
// dc/drho~ per element from the displacement.
void launch_sensitivity(const DevTables& t, double E, double p, const double* rho_f, const double* u,
                        double* dcf, cudaStream_t st);
// out = a . b (deterministic two-level sum).
void launch_dot(const double* a, const double* b, int64_t n, double* partials, unsigned* ticket,
                double* out, cudaStream_t st);
void launch_fill(double* x, int64_t n, double v, cudaStream_t st);
// OC update in place; out[0] = lambda, out[1] = dv . rho_new, out[2] = max |change|.
cudaError_t launch_oc(double* rho, const double* dc, const double* dv, int64_t n, double target,
                      double rho_min, double move, double* partials, double* out, cudaStream_t st);

}  // namespace ddel
