// D3Q103 (Tab. II) step kernels with the RR collision and shifted 16-bit storage (binary16, bfloat16, fixed
// point), in a translation unit of their own so that they compile in parallel with the wide formats'.
#include "d3.cuh"

LBM3_STEP_SIG(lbm3_step_d3q103_rr16) {
  return lbm::launch_step3_prec_16<lbm::D3Q103, lbm::COLL_RR>(prec, fin, fout, g, pd, st);
}
