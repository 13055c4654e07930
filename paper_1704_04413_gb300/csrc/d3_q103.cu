// D3Q103 (Tab. II): initial state, moments, planes and conservation sums, and the dispatch table of the
// lattice (the step kernels are in d3_q103_<collision>.cu for FP64 / FP32 storage and
// d3_q103_<collision>16.cu for the 16-bit formats).
#include "d3.cuh"

LBM3_STEP_SIG(lbm3_step_d3q103_bgk);
LBM3_STEP_SIG(lbm3_step_d3q103_pr);
LBM3_STEP_SIG(lbm3_step_d3q103_rr);
LBM3_STEP_SIG(lbm3_step_d3q103_bgk16);
LBM3_STEP_SIG(lbm3_step_d3q103_pr16);
LBM3_STEP_SIG(lbm3_step_d3q103_rr16);

static cudaError_t step_d3q103(int coll, int prec, const void* fin, void* fout, const lbm::Geom3& g,
                            const lbm::CollParamsD& pd, cudaStream_t st) {
  const bool wide = prec == lbm::PREC_F64 || prec == lbm::PREC_F32;
  switch (coll) {
    case lbm::COLL_BGK: return (wide ? lbm3_step_d3q103_bgk : lbm3_step_d3q103_bgk16)(prec, fin, fout, g, pd, st);
    case lbm::COLL_PR: return (wide ? lbm3_step_d3q103_pr : lbm3_step_d3q103_pr16)(prec, fin, fout, g, pd, st);
    case lbm::COLL_RR: return (wide ? lbm3_step_d3q103_rr : lbm3_step_d3q103_rr16)(prec, fin, fout, g, pd, st);
  }
  return cudaErrorInvalidValue;
}

extern const lbm::Lat3Ops lbm3_ops_d3q103 = lbm::Ops3<lbm::D3Q103>::table(step_d3q103);
