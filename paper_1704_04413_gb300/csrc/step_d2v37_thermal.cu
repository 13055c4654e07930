// Stream-and-collide kernels of the D2V37 lattice, thermal (theta from the energy moment).
#include "step.cuh"

cudaError_t lbm_launch_step_d2v37_thermal(LBM_STEP_LAUNCHER_ARGS) {
  return lbm::launch_step_lattice<lbm::D2V37, true>(coll, prec, fin, fout, g, pd, fd_mom, st, ctl);
}
