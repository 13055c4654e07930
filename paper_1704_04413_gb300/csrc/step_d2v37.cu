// Stream-and-collide kernels of the D2V37 lattice (isothermal).
#include "step.cuh"

cudaError_t lbm_launch_step_d2v37(LBM_STEP_LAUNCHER_ARGS) {
  return lbm::launch_step_lattice<lbm::D2V37, false>(coll, prec, fin, fout, g, pd, fd_mom, st, ctl);
}
