// D3Q27 (Tab. II): initial state, moments, planes and conservation sums, and the dispatch table of the
// lattice (the step kernels are in d3_q27_bgk.cu, d3_q27_pr.cu, d3_q27_rr.cu).
#include "d3.cuh"

LBM3_STEP_SIG(lbm3_step_d3q27_bgk);
LBM3_STEP_SIG(lbm3_step_d3q27_pr);
LBM3_STEP_SIG(lbm3_step_d3q27_rr);

static cudaError_t step_d3q27(int coll, int prec, const void* fin, void* fout, const lbm::Geom3& g,
                            const lbm::CollParamsD& pd, cudaStream_t st) {
  switch (coll) {
    case lbm::COLL_BGK: return lbm3_step_d3q27_bgk(prec, fin, fout, g, pd, st);
    case lbm::COLL_PR: return lbm3_step_d3q27_pr(prec, fin, fout, g, pd, st);
    case lbm::COLL_RR: return lbm3_step_d3q27_rr(prec, fin, fout, g, pd, st);
  }
  return cudaErrorInvalidValue;
}

extern const lbm::Lat3Ops lbm3_ops_d3q27 = lbm::Ops3<lbm::D3Q27>::table(step_d3q27);
