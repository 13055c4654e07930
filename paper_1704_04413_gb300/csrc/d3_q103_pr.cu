// D3Q103 (Tab. II) step kernels with the PR collision, FP64 and FP32 storage.
#include "d3.cuh"

LBM3_STEP_SIG(lbm3_step_d3q103_pr) {
  return lbm::launch_step3_prec_wide<lbm::D3Q103, lbm::COLL_PR>(prec, fin, fout, g, pd, st);
}
