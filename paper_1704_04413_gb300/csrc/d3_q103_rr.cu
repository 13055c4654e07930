// D3Q103 (Tab. II) step kernels with the RR collision, FP64 and FP32 storage.
#include "d3.cuh"

LBM3_STEP_SIG(lbm3_step_d3q103_rr) {
  return lbm::launch_step3_prec_wide<lbm::D3Q103, lbm::COLL_RR>(prec, fin, fout, g, pd, st);
}
