// Fused stream-and-collide kernel: one thread per cell pulls its V
// populations from the neighbours x - xi_i (Sec. III.A; periodic wrap or
// zero-gradient clamp), collides them (collide.cuh) and stores them in the
// other buffer.  Populations are SoA, f[i][y][x] with a padded row pitch, so
// each warp reads 32 consecutive x of one plane (coalesced; the x shift only
// moves the 128-byte window) and writes 32 aligned consecutive x.  Pull
// streaming is a permutation: every stored value is read once per step, so the
// kernel moves 2 V sizeof(storage) bytes per cell and is bound by HBM.
#pragma once
#include <cuda_runtime.h>

#include "collide.cuh"

namespace lbm {

enum { BC_PERIODIC = 0, BC_ZERO_GRADIENT = 1 };
enum { PREC_F64 = 0, PREC_F32 = 1, PREC_F16 = 2, PREC_BF16 = 3 };

struct StepGeom {
  long long plane;  // elements per population plane (ny * pitch)
  int pitch;        // elements per row
  int nx, ny;
  int bcx, bcy;
};

struct CollParamsD {
  double omega, om1;
  int neq, nreg;
  double rho0, s, inv_s;
};

template <class Real>
__host__ __device__ inline CollParams<Real> cast_params(const CollParamsD& d) {
  CollParams<Real> p;
  p.omega = (Real)d.omega;
  p.om1 = (Real)d.om1;
  p.neq = d.neq;
  p.nreg = d.nreg;
  p.rho0 = (Real)d.rho0;
  p.s = (Real)d.s;
  p.inv_s = (Real)d.inv_s;
  return p;
}

__device__ __forceinline__ int src_coord(int x, int c, int n, int bc) {
  int s = x - c;
  if (bc == BC_PERIODIC) {
    if (s < 0) s += n;
    if (s >= n) s -= n;
    // |c| <= 3 < n is not required: fold again for tiny grids
    if (s < 0 || s >= n) s = ((s % n) + n) % n;
  } else {
    s = s < 0 ? 0 : (s > n - 1 ? n - 1 : s);
  }
  return s;
}

constexpr int STEP_BX = 128;

template <class L, int COLL, bool THERMAL, class Real, class S>
__global__ void __launch_bounds__(STEP_BX) k_step(const S* __restrict__ fin, S* __restrict__ fout, StepGeom g,
                                                  CollParams<Real> P) {
  const int x = blockIdx.x * STEP_BX + threadIdx.x;
  if (x >= g.nx) return;
  for (int y = blockIdx.y; y < g.ny; y += gridDim.y) {
  Real q[L::Q];
  sfor<0, L::Q>([&](auto I) {
    constexpr int i = LBM_CI(I);
    const int xs = src_coord(x, L::CX[i], g.nx, g.bcx);
    const int ys = src_coord(y, L::CY[i], g.ny, g.bcy);
    q[i] = (Real)Store<S>::ld(fin + (long long)i * g.plane + (long long)ys * g.pitch + xs);
  });
  collide<L, COLL, THERMAL, Store<S>::SHIFTED>(q, P);
  const long long o = (long long)y * g.pitch + x;
  sfor<0, L::Q>([&](auto I) {
    constexpr int i = LBM_CI(I);
    Store<S>::st(fout + (long long)i * g.plane + o, q[i]);
  });
  }
}

template <class L, int COLL, bool THERMAL, class Real, class S>
inline cudaError_t launch_step_t(const void* fin, void* fout, const StepGeom& g, const CollParamsD& pd,
                                 cudaStream_t st) {
  dim3 grid((g.nx + STEP_BX - 1) / STEP_BX, g.ny < 65535 ? g.ny : 65535);
  k_step<L, COLL, THERMAL, Real, S>
      <<<grid, STEP_BX, 0, st>>>((const S*)fin, (S*)fout, g, cast_params<Real>(pd));
  return cudaGetLastError();
}

template <class L, int COLL, bool THERMAL>
inline cudaError_t launch_step_prec(int prec, const void* fin, void* fout, const StepGeom& g,
                                    const CollParamsD& pd, cudaStream_t st) {
  switch (prec) {
    case PREC_F64: return launch_step_t<L, COLL, THERMAL, double, double>(fin, fout, g, pd, st);
    case PREC_F32: return launch_step_t<L, COLL, THERMAL, float, float>(fin, fout, g, pd, st);
    case PREC_F16: return launch_step_t<L, COLL, THERMAL, float, __half>(fin, fout, g, pd, st);
    case PREC_BF16: return launch_step_t<L, COLL, THERMAL, float, __nv_bfloat16>(fin, fout, g, pd, st);
  }
  return cudaErrorInvalidValue;
}

template <class L, bool THERMAL>
inline cudaError_t launch_step_lattice(int coll, int prec, const void* fin, void* fout, const StepGeom& g,
                                       const CollParamsD& pd, cudaStream_t st) {
  switch (coll) {
    case COLL_BGK: return launch_step_prec<L, COLL_BGK, THERMAL>(prec, fin, fout, g, pd, st);
    case COLL_PR: return launch_step_prec<L, COLL_PR, THERMAL>(prec, fin, fout, g, pd, st);
    case COLL_RR: return launch_step_prec<L, COLL_RR, THERMAL>(prec, fin, fout, g, pd, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbm

// One translation unit per lattice instantiates its kernels behind these.
cudaError_t lbm_launch_step_d2q9(int coll, int prec, const void* fin, void* fout, const lbm::StepGeom& g,
                                 const lbm::CollParamsD& pd, cudaStream_t st);
cudaError_t lbm_launch_step_d2v17(int coll, int prec, const void* fin, void* fout, const lbm::StepGeom& g,
                                  const lbm::CollParamsD& pd, cudaStream_t st);
cudaError_t lbm_launch_step_d2v37(int coll, int prec, const void* fin, void* fout, const lbm::StepGeom& g,
                                  const lbm::CollParamsD& pd, cudaStream_t st);
cudaError_t lbm_launch_step_d2v37_thermal(int coll, int prec, const void* fin, void* fout, const lbm::StepGeom& g,
                                          const lbm::CollParamsD& pd, cudaStream_t st);
