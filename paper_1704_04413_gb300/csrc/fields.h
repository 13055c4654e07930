// Launchers of the per-cell field kernels (fields.cu), used by the C ABI.
#pragma once
#include <cuda_runtime.h>

#include "step.cuh"

namespace lbm {
struct InitParams {
  int neq;       // highest order of f^(0)
  int thermal;   // theta field used
  double tau;    // relaxation time of the a1^(2) of the initial f^(1)
  double rho0;   // shifted storage reference
  double s;      // shifted storage scale
};
}  // namespace lbm

long long lbm_partials_count(const lbm::StepGeom& g);
cudaError_t lbm_launch_init(int lat, int prec, const double* rho, const double* ux, const double* uy,
                            const double* th, const double* grad, void* f, const lbm::StepGeom& g,
                            const lbm::InitParams& ip, cudaStream_t st);
cudaError_t lbm_launch_moments(int lat, int prec, const void* f, const lbm::StepGeom& g, double rho0, double inv_s,
                               int thermal, double* rho, double* ux, double* uy, double* th, cudaStream_t st);
cudaError_t lbm_launch_get_plane(int lat, int prec, const void* f, const lbm::StepGeom& g, int i, double rho0,
                                 double inv_s, double* out, cudaStream_t st);
cudaError_t lbm_launch_set_plane(int lat, int prec, void* f, const lbm::StepGeom& g, int i, double rho0, double s,
                                 const double* in, cudaStream_t st);
cudaError_t lbm_launch_conservation(int lat, int prec, const void* f, const lbm::StepGeom& g, double rho0,
                                    double inv_s, double* partials, double* out4, cudaStream_t st);
cudaError_t lbm_launch_diagnostics(const double* ux, const double* uy, const lbm::StepGeom& g, double* partials,
                                   double* out4, cudaStream_t st);
