// D3V39 (Tab. II) step kernels with the PR collision.
#include "d3.cuh"

LBM3_STEP_SIG(lbm3_step_d3v39_pr) {
  return lbm::launch_step3_prec<lbm::D3V39, lbm::COLL_PR>(prec, fin, fout, g, pd, st);
}
