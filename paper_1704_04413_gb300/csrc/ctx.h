// Internal state of a context (opaque to C ABI users), shared by the translation units that implement
// the ABI (api.cu, batch.cu).
#pragma once
#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "step.cuh"

struct lbm_ctx {
  lbm_params p;
  int V = 0;
  int nmax = 0;
  int prec = 0;   // PREC_*
  int neq = 0, nreg = 0;
  double cs2 = 0, tau = 0, rho0 = 1, s = 1;
  double tau3 = 0, tau4 = 0;  // relaxation times of orders 3 and 4 of f^(1) (= tau unless set)
  size_t elem = 0;  // bytes per stored value
  lbm::StepGeom g{};
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;
  double* scratch = nullptr;  // 8 * ncells doubles, for host transfers and diagnostics
  double* partials = nullptr;
  double* out4 = nullptr;     // device: 4 sums, then the error word
  double* host4 = nullptr;    // pinned host copy of the same
  void* closure_buf = nullptr;  // features and outputs of the learned closure (lazily allocated)
  void* fd_mom = nullptr;       // rho, ux, uy, theta [4][ny][nx] of the finite-difference variant
  int* dev_err = nullptr;     // device error word (bounded device waits record LBM_ETIMEOUT there)
  lbm::StageCtl ctl{};        // what the staged step kernels get: dev_err, wait limit, test fault hook
  long long steps = 0;
  cudaStream_t st = nullptr;
  int device = 0;
  char err[256] = {0};
};

// Collision parameters of a context: relaxation factors, orders, storage shift and scale (api.cu).
lbm::CollParamsD lbm_ctx_coll_params(const lbm_ctx* c);

// Launch one time step of a context from `fin` to `fout` (api.cu).
cudaError_t lbm_ctx_launch_step(lbm_ctx* c, const void* fin, void* fout);
