// D3Q103 (Tab. II) step kernels with the BGK collision, FP64 and FP32 storage.
#include "d3.cuh"

LBM3_STEP_SIG(lbm3_step_d3q103_bgk) {
  return lbm::launch_step3_prec_wide<lbm::D3Q103, lbm::COLL_BGK>(prec, fin, fout, g, pd, st);
}
