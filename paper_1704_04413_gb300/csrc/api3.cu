// C ABI of the 3D lattices (include/lbm3.h): contexts, parameter validation, buffers and the calls that
// launch the kernels of d3.cuh through each lattice's Lat3Ops table.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <initializer_list>
#include <new>

#include "../../include/lbm3.h"
#include "d3.cuh"

extern const lbm::Lat3Ops lbm3_ops_d3q19;
extern const lbm::Lat3Ops lbm3_ops_d3q27;
extern const lbm::Lat3Ops lbm3_ops_d3v39;
extern const lbm::Lat3Ops lbm3_ops_d3q103;

namespace {

const lbm::Lat3Ops* ops_of(int lattice) {
  switch (lattice) {
    case LBM_D3Q19: return &lbm3_ops_d3q19;
    case LBM_D3Q27: return &lbm3_ops_d3q27;
    case LBM_D3V39: return &lbm3_ops_d3v39;
    case LBM_D3Q103: return &lbm3_ops_d3q103;
  }
  return nullptr;
}

bool is_pow2(double s) {
  if (!(s > 0) || !std::isfinite(s)) return false;
  int e = 0;
  return std::frexp(s, &e) == 0.5;
}

constexpr int kPartials = 1024;  // blocks of the conservation reduction

}  // namespace

struct lbm3_ctx {
  lbm3_params p;
  const lbm::Lat3Ops* ops = nullptr;
  int prec = 0, neq = 0, nreg = 0;
  double tau = 0, rho0 = 1, s = 1;
  size_t elem = 0;
  lbm::Geom3 g{};
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;
  double* scratch = nullptr;   // 13 doubles per cell: host transfers of rho, u, grad and planes
  double* partials = nullptr;  // 4 x kPartials
  double* out4 = nullptr;
  double* host4 = nullptr;     // pinned
  cudaStream_t st = nullptr;
  int device = 0;
};

static long long cells(const lbm3_ctx* c) { return (long long)c->p.nx * c->p.ny * c->p.nz; }

static lbm::CollParamsD coll_params(const lbm3_ctx* c) {
  lbm::CollParamsD pd{};
  pd.omega = 1.0 / c->tau;
  pd.om1 = 1.0 - 1.0 / c->tau;
  pd.om1_3 = pd.om1;
  pd.om1_4 = pd.om1;
  pd.tau = c->tau;
  pd.tau3 = c->tau;
  pd.neq = c->neq;
  pd.nreg = c->nreg;
  pd.rho0 = c->rho0;
  pd.s = c->s;
  pd.inv_s = 1.0 / c->s;
  return pd;
}

static int ensure_scratch(lbm3_ctx* c) {
  if (c->scratch) return LBM_OK;
  if (cudaMalloc(&c->scratch, sizeof(double) * 13 * (size_t)cells(c)) != cudaSuccess) {
    cudaGetLastError();
    c->scratch = nullptr;
    return LBM_ENOMEM;
  }
  return LBM_OK;
}

#define LBM3_CK(expr)            \
  do {                           \
    if ((expr) != cudaSuccess) { \
      cudaGetLastError();        \
      return LBM_ECUDA;          \
    }                            \
  } while (0)

extern "C" {

int lbm3_lattice_info(int lattice, int* V, int* cx, int* cy, int* cz, double* w, double* cs2) {
  const lbm::Lat3Ops* o = ops_of(lattice);
  if (!o) return LBM_EINVAL;
  if (V) *V = o->V;
  for (int i = 0; i < o->V; ++i) {
    if (cx) cx[i] = o->cx[i];
    if (cy) cy[i] = o->cy[i];
    if (cz) cz[i] = o->cz[i];
    if (w) w[i] = o->w[i];
  }
  if (cs2) *cs2 = o->cs2;
  return LBM_OK;
}

void lbm3_destroy(lbm3_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->st) cudaStreamSynchronize(c->st);
  cudaFree(c->buf[0]);
  cudaFree(c->buf[1]);
  cudaFree(c->scratch);
  cudaFree(c->partials);
  cudaFree(c->out4);
  cudaFreeHost(c->host4);
  delete c;
}

int lbm3_create(const lbm3_params* p, lbm3_ctx** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (!p) return LBM_EINVAL;
  const lbm::Lat3Ops* o = ops_of(p->lattice);
  if (!o) return LBM_EINVAL;
  if (p->hermite_order < 1 || p->hermite_order > o->nmax) return LBM_EINVAL;
  if (p->reg_order != 0 && (p->reg_order < 2 || p->reg_order > o->nmax)) return LBM_EINVAL;
  if (p->collision < LBM_BGK || p->collision > LBM_RR) return LBM_EINVAL;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return LBM_EINVAL;
  for (int b : {p->bc_x, p->bc_y, p->bc_z})
    if (b != LBM_PERIODIC && b != LBM_ZERO_GRADIENT) return LBM_EINVAL;
  int prec;
  if (p->compute == LBM_F64 && p->storage == LBM_F64)
    prec = lbm::PREC_F64;
  else if (p->compute == LBM_F32 && p->storage == LBM_F32)
    prec = lbm::PREC_F32;
  else if (p->compute == LBM_F32 && p->storage == LBM_F16_SHIFT)
    prec = lbm::PREC_F16;
  else if (p->compute == LBM_F32 && p->storage == LBM_BF16_SHIFT)
    prec = lbm::PREC_BF16;
  else if (p->compute == LBM_F32 && p->storage == LBM_I16_SHIFT)
    prec = lbm::PREC_I16;
  else
    return LBM_EINVAL;
  if (prec != lbm::PREC_F64 && prec != lbm::PREC_F32 && !o->sixteen_bit) return LBM_EINVAL;
  double tau = p->tau;
  if (!(tau > 0)) {
    if (!(p->nu > 0) || !std::isfinite(p->nu)) return LBM_EINVAL;
    tau = p->nu / o->cs2 + 0.5;  // nu = cs^2 (tau - 1/2)
  }
  if (!(tau > 0.5) || !std::isfinite(tau)) return LBM_EINVAL;
  const double rho0 = p->rho0 == 0 ? 1.0 : p->rho0;
  const double s = p->store_scale == 0 ? 1.0 : p->store_scale;
  if (!(rho0 > 0) || !std::isfinite(rho0) || !is_pow2(s)) return LBM_EINVAL;

  lbm3_ctx* c = new (std::nothrow) lbm3_ctx();
  if (!c) return LBM_ENOMEM;
  c->p = *p;
  c->ops = o;
  cudaGetDevice(&c->device);
  c->prec = prec;
  c->neq = p->hermite_order;
  c->nreg = p->reg_order == 0 ? o->nmax : p->reg_order;
  c->tau = tau;
  c->rho0 = rho0;
  c->s = s;
  c->elem = prec == lbm::PREC_F64 ? 8 : prec == lbm::PREC_F32 ? 4 : 2;
  c->st = (cudaStream_t)p->stream;
  const size_t row_bytes = ((size_t)p->nx * c->elem + 127) / 128 * 128;
  c->g.pitch = (int)(row_bytes / c->elem);
  c->g.plane = (long long)c->g.pitch * p->ny;
  c->g.pstride = c->g.plane * p->nz;
  c->g.nx = p->nx;
  c->g.ny = p->ny;
  c->g.nz = p->nz;
  c->g.bc[0] = p->bc_x;
  c->g.bc[1] = p->bc_y;
  c->g.bc[2] = p->bc_z;
  const size_t bytes = (size_t)o->V * (size_t)c->g.pstride * c->elem;
  cudaError_t e;
  if ((e = cudaMalloc(&c->buf[0], bytes)) != cudaSuccess || (e = cudaMalloc(&c->buf[1], bytes)) != cudaSuccess ||
      (e = cudaMalloc(&c->partials, sizeof(double) * 4 * kPartials)) != cudaSuccess ||
      (e = cudaMalloc(&c->out4, 5 * sizeof(double))) != cudaSuccess ||
      (e = cudaMallocHost(&c->host4, 5 * sizeof(double))) != cudaSuccess) {
    const int rc = e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
    cudaGetLastError();
    lbm3_destroy(c);
    return rc;
  }
  // out4[4] holds the status word of the staged step kernels (0 = every copy wait completed)
  c->g.status = reinterpret_cast<int*>(c->out4 + 4);
  c->g.wait_ns = lbm::kBulkWaitNs;
  c->g.fault_block = -1;
  // padding columns are never read by a kernel; clear them once so transfers are deterministic
  if (cudaMemsetAsync(c->buf[0], 0, bytes, c->st) != cudaSuccess ||
      cudaMemsetAsync(c->buf[1], 0, bytes, c->st) != cudaSuccess ||
      cudaMemsetAsync(c->out4, 0, 5 * sizeof(double), c->st) != cudaSuccess) {
    cudaGetLastError();
    lbm3_destroy(c);
    return LBM_ECUDA;
  }
  *out = c;
  return LBM_OK;
}

}  // extern "C"

extern "C" {

double lbm3_tau(const lbm3_ctx* c) { return c ? c->tau : 0.0; }

int lbm3_test_inject_copy_fault(lbm3_ctx* c, int block, double wait_seconds) {
  if (!c || block < -1 || !(wait_seconds > 0) || wait_seconds > 10.0) return LBM_EINVAL;
  c->g.fault_block = block;
  c->g.wait_ns = (unsigned long long)(wait_seconds * 1e9);
  return LBM_OK;
}

int lbm3_init(lbm3_ctx* c, const double* rho, const double* u, const double* grad, int on_device) {
  if (!c || !rho || !u) return LBM_EINVAL;
  LBM3_CK(cudaSetDevice(c->device));
  const long long n = cells(c);
  const double *dr = rho, *du = u, *dg = grad;
  if (!on_device) {
    const int rc = ensure_scratch(c);
    if (rc) return rc;
    double* s = c->scratch;
    LBM3_CK(cudaMemcpyAsync(s, rho, sizeof(double) * n, cudaMemcpyHostToDevice, c->st));
    LBM3_CK(cudaMemcpyAsync(s + n, u, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->st));
    if (grad) LBM3_CK(cudaMemcpyAsync(s + 4 * n, grad, sizeof(double) * 9 * n, cudaMemcpyHostToDevice, c->st));
    dr = s;
    du = s + n;
    dg = grad ? s + 4 * n : nullptr;
  }
  const lbm::Init3Params ip{c->neq, c->tau, c->rho0, c->s};
  LBM3_CK(c->ops->init(c->prec, dr, du, dg, c->buf[0], c->g, ip, c->st));
  c->cur = 0;
  if (!on_device) LBM3_CK(cudaStreamSynchronize(c->st));  // host arrays may be released on return
  return LBM_OK;
}

int lbm3_step(lbm3_ctx* c, int n) {
  if (!c || n < 0) return LBM_EINVAL;
  LBM3_CK(cudaSetDevice(c->device));
  const lbm::CollParamsD pd = coll_params(c);
  for (int k = 0; k < n; ++k) {
    LBM3_CK(c->ops->step(c->p.collision, c->prec, c->buf[c->cur], c->buf[c->cur ^ 1], c->g, pd, c->st));
    c->cur ^= 1;
  }
  return LBM_OK;
}

int lbm3_moments(lbm3_ctx* c, double* rho, double* u, int on_device) {
  if (!c) return LBM_EINVAL;
  LBM3_CK(cudaSetDevice(c->device));
  const long long n = cells(c);
  if (on_device) {
    LBM3_CK(c->ops->moments(c->prec, c->buf[c->cur], c->g, c->rho0, 1.0 / c->s, rho, u, c->st));
    return LBM_OK;
  }
  const int rc = ensure_scratch(c);
  if (rc) return rc;
  double* s = c->scratch;
  LBM3_CK(c->ops->moments(c->prec, c->buf[c->cur], c->g, c->rho0, 1.0 / c->s, rho ? s : nullptr,
                          u ? s + n : nullptr, c->st));
  if (rho) LBM3_CK(cudaMemcpyAsync(rho, s, sizeof(double) * n, cudaMemcpyDeviceToHost, c->st));
  if (u) LBM3_CK(cudaMemcpyAsync(u, s + n, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->st));
  LBM3_CK(cudaStreamSynchronize(c->st));
  return LBM_OK;
}

int lbm3_conservation(lbm3_ctx* c, double out[4]) {
  if (!c || !out) return LBM_EINVAL;
  LBM3_CK(cudaSetDevice(c->device));
  LBM3_CK(c->ops->conservation(c->prec, c->buf[c->cur], c->g, c->rho0, 1.0 / c->s, c->partials, kPartials,
                               c->out4, c->st));
  LBM3_CK(cudaMemcpyAsync(c->host4, c->out4, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  LBM3_CK(cudaStreamSynchronize(c->st));
  if (*reinterpret_cast<const int*>(c->host4 + 4) != 0) return LBM_ETIMEOUT;
  bool finite = true;
  for (int k = 0; k < 4; ++k) {
    out[k] = c->host4[k];
    finite = finite && std::isfinite(out[k]);
  }
  return finite ? LBM_OK : LBM_EUNSTABLE;
}

int lbm3_get_populations(lbm3_ctx* c, double* f, int on_device) {
  if (!c || !f) return LBM_EINVAL;
  LBM3_CK(cudaSetDevice(c->device));
  const long long n = cells(c);
  if (!on_device) {
    const int rc = ensure_scratch(c);
    if (rc) return rc;
  }
  for (int i = 0; i < c->ops->V; ++i) {
    double* dst = on_device ? f + (long long)i * n : c->scratch;
    LBM3_CK(c->ops->get_plane(c->prec, c->buf[c->cur], c->g, i, c->rho0, 1.0 / c->s, dst, c->st));
    if (!on_device) {
      LBM3_CK(cudaMemcpyAsync(f + (long long)i * n, c->scratch, sizeof(double) * n, cudaMemcpyDeviceToHost,
                              c->st));
      LBM3_CK(cudaStreamSynchronize(c->st));
    }
  }
  LBM3_CK(cudaMemcpyAsync(c->host4 + 4, c->out4 + 4, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  LBM3_CK(cudaStreamSynchronize(c->st));
  return *reinterpret_cast<const int*>(c->host4 + 4) != 0 ? LBM_ETIMEOUT : LBM_OK;
}

int lbm3_set_populations(lbm3_ctx* c, const double* f, int on_device) {
  if (!c || !f) return LBM_EINVAL;
  LBM3_CK(cudaSetDevice(c->device));
  const long long n = cells(c);
  if (!on_device) {
    const int rc = ensure_scratch(c);
    if (rc) return rc;
  }
  for (int i = 0; i < c->ops->V; ++i) {
    const double* src = on_device ? f + (long long)i * n : c->scratch;
    if (!on_device)
      LBM3_CK(cudaMemcpyAsync(c->scratch, f + (long long)i * n, sizeof(double) * n, cudaMemcpyHostToDevice,
                              c->st));
    LBM3_CK(c->ops->set_plane(c->prec, c->buf[c->cur], c->g, i, c->rho0, c->s, src, c->st));
    if (!on_device) LBM3_CK(cudaStreamSynchronize(c->st));
  }
  return LBM_OK;
}

}  // extern "C"
