// Stream-and-collide kernels of the D2V37 lattice, thermal (theta from the energy moment).
#include "step.cuh"

cudaError_t lbm_launch_step_d2v37_thermal(int coll, int prec, const void* fin, void* fout, const lbm::StepGeom& g,
                                          const lbm::CollParamsD& pd, cudaStream_t st) {
  return lbm::launch_step_lattice<lbm::D2V37, true>(coll, prec, fin, fout, g, pd, st);
}
