// Stream-and-collide kernels of the D2Q9 lattice (isothermal).
#include "step.cuh"

cudaError_t lbm_launch_step_d2q9(LBM_STEP_LAUNCHER_ARGS) {
  return lbm::launch_step_lattice<lbm::D2Q9, false>(coll, prec, fin, fout, g, pd, fd_mom, st, ctl);
}
