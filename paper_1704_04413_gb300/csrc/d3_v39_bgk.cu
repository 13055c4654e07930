// D3V39 (Tab. II) step kernels with the BGK collision.
#include "d3.cuh"

LBM3_STEP_SIG(lbm3_step_d3v39_bgk) {
  return lbm::launch_step3_prec<lbm::D3V39, lbm::COLL_BGK>(prec, fin, fout, g, pd, st);
}
