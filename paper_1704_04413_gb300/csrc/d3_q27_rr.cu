// D3Q27 (Tab. II) step kernels with the RR collision.
#include "d3.cuh"

LBM3_STEP_SIG(lbm3_step_d3q27_rr) {
  return lbm::launch_step3_prec<lbm::D3Q27, lbm::COLL_RR>(prec, fin, fout, g, pd, st);
}
