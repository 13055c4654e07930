// C ABI of liblbm (include/lbm.h): context management, host/device transfer,
// time stepping and diagnostics.  Every computation is a kernel of this
// library; this file only validates, allocates, copies and launches.
#include <cuda_runtime.h>

#include <cmath>
#include <initializer_list>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/lbm.h"
#include "ctx.h"
#include "fields.h"
#include "step.cuh"


using namespace lbm;


namespace {

const char* kMsgs[] = {"ok", "invalid argument", "out of device memory", "CUDA error", "unstable (non-finite state)",
                       "device wait timed out", "file I/O error"};

int fail(lbm_ctx* c, int code, const char* what) {
  if (c) snprintf(c->err, sizeof(c->err), "%s", what);
  return code;
}

int cuda_fail(lbm_ctx* c, cudaError_t e, const char* where) {
  if (c) snprintf(c->err, sizeof(c->err), "%s: %s", where, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
}

#define LBM_CK(c, call)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
  } while (0)

long long ncells(const lbm_ctx* c) { return (long long)c->p.nx * c->p.ny; }

template <class L>
void lattice_copy(int* V, int* cx, int* cy, double* w, double* cs2) {
  if (V) *V = L::Q;
  for (int i = 0; i < L::Q; ++i) {
    if (cx) cx[i] = L::CX[i];
    if (cy) cy[i] = L::CY[i];
    if (w) w[i] = L::W[i];
  }
  if (cs2) *cs2 = L::CS2;
}

int lattice_nmax(int lat) { return lat == LBM_D2V17 ? 3 : 4; }

}  // namespace

CollParamsD lbm_ctx_coll_params(const lbm_ctx* c) {
  CollParamsD pd;
  pd.omega = 1.0 / c->tau;
  pd.om1 = 1.0 - 1.0 / c->tau;
  pd.om1_3 = 1.0 - 1.0 / c->tau3;
  pd.om1_4 = 1.0 - 1.0 / c->tau4;
  pd.tau = c->tau;
  pd.tau3 = c->tau3;
  pd.neq = c->neq;
  pd.nreg = c->nreg;
  pd.rho0 = c->rho0;
  pd.s = c->s;
  pd.inv_s = 1.0 / c->s;
  return pd;
}

cudaError_t lbm_ctx_launch_step(lbm_ctx* c, const void* fin, void* fout) {
  const CollParamsD pd = lbm_ctx_coll_params(c);
  const int coll = c->p.collision;
  switch (c->p.lattice) {
    case LBM_D2Q9: return lbm_launch_step_d2q9(coll, c->prec, fin, fout, c->g, pd, c->fd_mom, &c->ctl, c->st);
    case LBM_D2V17:
      return lbm_launch_step_d2v17(coll, c->prec, fin, fout, c->g, pd, c->fd_mom, &c->ctl, c->st);
    case LBM_D2V37:
      return c->p.thermal
                 ? lbm_launch_step_d2v37_thermal(coll, c->prec, fin, fout, c->g, pd, c->fd_mom, &c->ctl, c->st)
                 : lbm_launch_step_d2v37(coll, c->prec, fin, fout, c->g, pd, c->fd_mom, &c->ctl, c->st);
  }
  return cudaErrorInvalidValue;
}

namespace {

int ensure_scratch(lbm_ctx* c) {
  if (c->scratch) return LBM_OK;
  LBM_CK(c, cudaMalloc(&c->scratch, sizeof(double) * 8 * (size_t)ncells(c)));
  return LBM_OK;
}

bool is_pow2(double s) {
  if (!(s > 0) || !std::isfinite(s)) return false;
  int e;
  return std::frexp(s, &e) == 0.5;
}

}  // namespace

extern "C" {

const char* lbm_strerror(int code) {
  int k = -code;
  if (k < 0 || k >= (int)(sizeof(kMsgs) / sizeof(kMsgs[0]))) return "unknown status";
  return kMsgs[k];
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err : "no context"; }

int lbm_lattice_info(int lattice, int* V, int* cx, int* cy, double* w, double* cs2) {
  switch (lattice) {
    case LBM_D2Q9: lattice_copy<D2Q9>(V, cx, cy, w, cs2); return LBM_OK;
    case LBM_D2V17: lattice_copy<D2V17>(V, cx, cy, w, cs2); return LBM_OK;
    case LBM_D2V37: lattice_copy<D2V37>(V, cx, cy, w, cs2); return LBM_OK;
  }
  return LBM_EINVAL;
}

void lbm_destroy(lbm_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->st) cudaStreamSynchronize(c->st);
  cudaFree(c->buf[0]);
  cudaFree(c->buf[1]);
  cudaFree(c->scratch);
  cudaFree(c->partials);
  cudaFree(c->out4);
  cudaFree(c->dev_err);
  cudaFree(c->closure_buf);
  cudaFree(c->fd_mom);
  cudaFreeHost(c->host4);
  delete c;
}

int lbm_create(const lbm_params* p, lbm_ctx** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (!p) return LBM_EINVAL;
  if (p->lattice < LBM_D2Q9 || p->lattice > LBM_D2V37) return LBM_EINVAL;
  const int nmax = lattice_nmax(p->lattice);
  if (p->hermite_order < 2 || p->hermite_order > nmax) return LBM_EINVAL;
  if (p->reg_order != 0 && (p->reg_order < 2 || p->reg_order > nmax)) return LBM_EINVAL;
  if (p->collision < LBM_BGK || p->collision > LBM_RR) return LBM_EINVAL;
  if (p->thermal != 0 && p->thermal != 1) return LBM_EINVAL;
  if (p->thermal && p->lattice != LBM_D2V37) return LBM_EINVAL;
  if (p->nx < 1 || p->ny < 1) return LBM_EINVAL;
  if (p->bc_x < 0 || p->bc_x > 1 || p->bc_y < 0 || p->bc_y > 1) return LBM_EINVAL;
  int prec;
  if (p->compute == LBM_F64 && p->storage == LBM_F64)
    prec = PREC_F64;
  else if (p->compute == LBM_F32 && p->storage == LBM_F32)
    prec = PREC_F32;
  else if (p->compute == LBM_F32 && p->storage == LBM_F16_SHIFT)
    prec = PREC_F16;
  else if (p->compute == LBM_F32 && p->storage == LBM_BF16_SHIFT)
    prec = PREC_BF16;
  else if (p->compute == LBM_F32 && p->storage == LBM_I16_SHIFT)
    prec = PREC_I16;
  else
    return LBM_EINVAL;
  double cs2 = 0;
  lbm_lattice_info(p->lattice, nullptr, nullptr, nullptr, nullptr, &cs2);
  double tau = p->tau;
  if (!(tau > 0)) {
    if (!(p->nu > 0) || !std::isfinite(p->nu)) return LBM_EINVAL;
    tau = p->nu / cs2 + 0.5;  // nu = cs^2 (tau - 1/2), Sec. II.B / III.A
  }
  if (!(tau > 0.5) || !std::isfinite(tau)) return LBM_EINVAL;
  // one relaxation time per order of f^(1) (Eq. GenRegCollision): unset = tau, PR / RR only
  for (double tn : {p->tau3, p->tau4})
    if (tn != 0 && (!(tn > 0.5) || !std::isfinite(tn))) return LBM_EINVAL;
  if (p->collision == LBM_BGK && (p->tau3 != 0 || p->tau4 != 0)) return LBM_EINVAL;
  if (p->a1_source != LBM_A1_PROJECTION &&
      (p->a1_source != LBM_A1_FINITE_DIFFERENCE || p->collision != LBM_RR))
    return LBM_EINVAL;
  const double rho0 = p->rho0 == 0 ? 1.0 : p->rho0;
  const double s = p->store_scale == 0 ? 1.0 : p->store_scale;
  if (!(rho0 > 0) || !std::isfinite(rho0) || !is_pow2(s)) return LBM_EINVAL;

  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_ENOMEM;
  c->p = *p;
  cudaGetDevice(&c->device);
  c->V = 0;
  lbm_lattice_info(p->lattice, &c->V, nullptr, nullptr, nullptr, nullptr);
  c->nmax = nmax;
  c->prec = prec;
  c->neq = p->hermite_order;
  c->nreg = p->reg_order == 0 ? nmax : p->reg_order;
  c->cs2 = cs2;
  c->tau = tau;
  c->tau3 = p->tau3 != 0 ? p->tau3 : tau;
  c->tau4 = p->tau4 != 0 ? p->tau4 : tau;
  c->rho0 = rho0;
  c->s = s;
  c->elem = prec == PREC_F64 ? 8 : prec == PREC_F32 ? 4 : 2;  // the three 16-bit formats
  c->st = (cudaStream_t)p->stream;
  const size_t row_bytes = ((size_t)p->nx * c->elem + 127) / 128 * 128; // rows start on 128-byte lines
  c->g.pitch = (int)(row_bytes / c->elem);
  c->g.plane = (long long)c->g.pitch * p->ny;
  c->g.nx = p->nx;
  c->g.ny = p->ny;
  c->g.bcx = p->bc_x;
  c->g.bcy = p->bc_y;
  c->g.nsm = 1;
  cudaDeviceGetAttribute(&c->g.nsm, cudaDevAttrMultiProcessorCount, c->device);
  const size_t bytes = (size_t)c->V * (size_t)c->g.plane * c->elem;
  int rc = LBM_OK;
  cudaError_t e;
  if ((e = cudaMalloc(&c->buf[0], bytes)) != cudaSuccess || (e = cudaMalloc(&c->buf[1], bytes)) != cudaSuccess ||
      (e = cudaMalloc(&c->partials, sizeof(double) * (size_t)lbm_partials_count(c->g))) != cudaSuccess ||
      (e = cudaMalloc(&c->out4, 5 * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&c->dev_err, sizeof(int))) != cudaSuccess ||
      (e = cudaMallocHost(&c->host4, 5 * sizeof(double))) != cudaSuccess ||
      (p->a1_source == LBM_A1_FINITE_DIFFERENCE &&
       (e = cudaMalloc(&c->fd_mom, 4 * (size_t)p->nx * (size_t)p->ny * (prec == PREC_F64 ? 8 : 4))) != cudaSuccess)) {
    rc = e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
    cudaGetLastError();
    lbm_destroy(c);
    return rc;
  }
  // padding columns are never read by a kernel; clear them once for deterministic checkpoints
  if ((e = cudaMemsetAsync(c->buf[0], 0, bytes, c->st)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->buf[1], 0, bytes, c->st)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->st)) != cudaSuccess) {
    lbm_destroy(c);
    return LBM_ECUDA;
  }
  c->ctl.status = c->dev_err;
  c->ctl.wait_ns = lbm::kBulkWaitNs;
  c->ctl.fault_block = -1;
  *out = c;
  return LBM_OK;
}

int lbm_test_inject_copy_fault(lbm_ctx* c, int block, double wait_seconds) {
  if (!c || block < -1 || !(wait_seconds > 0) || wait_seconds > 10.0) return LBM_EINVAL;
  c->ctl.fault_block = block;
  c->ctl.wait_ns = (unsigned long long)(wait_seconds * 1e9);
  return LBM_OK;
}

long long lbm_step_count(const lbm_ctx* c) { return c ? c->steps : -1; }
double lbm_tau(const lbm_ctx* c) { return c ? c->tau : 0.0; }

int lbm_init(lbm_ctx* c, const double* rho, const double* ux, const double* uy, const double* theta,
             const double* grad_u, int on_device) {
  if (!c || !rho || !ux || !uy) return fail(c, LBM_EINVAL, "lbm_init: rho, ux, uy are required");
  LBM_CK(c, cudaSetDevice(c->device));
  const long long n = ncells(c);
  const double *dr = rho, *du = ux, *dv = uy, *dt = c->p.thermal ? theta : nullptr, *dg = grad_u;
  if (!on_device) {
    int rc = ensure_scratch(c);
    if (rc) return rc;
    const size_t b = sizeof(double) * (size_t)n;
    double* s = c->scratch;
    LBM_CK(c, cudaMemcpyAsync(s, rho, b, cudaMemcpyHostToDevice, c->st));
    LBM_CK(c, cudaMemcpyAsync(s + n, ux, b, cudaMemcpyHostToDevice, c->st));
    LBM_CK(c, cudaMemcpyAsync(s + 2 * n, uy, b, cudaMemcpyHostToDevice, c->st));
    dr = s;
    du = s + n;
    dv = s + 2 * n;
    if (dt) {
      LBM_CK(c, cudaMemcpyAsync(s + 3 * n, theta, b, cudaMemcpyHostToDevice, c->st));
      dt = s + 3 * n;
    }
    if (dg) {
      LBM_CK(c, cudaMemcpyAsync(s + 4 * n, grad_u, 4 * b, cudaMemcpyHostToDevice, c->st));
      dg = s + 4 * n;
    }
  }
  InitParams ip{c->neq, c->p.thermal, c->tau, c->rho0, c->s};
  c->cur = 0;
  LBM_CK(c, lbm_launch_init(c->p.lattice, c->prec, dr, du, dv, dt, dg, c->buf[0], c->g, ip, c->st));
  if (!on_device) LBM_CK(c, cudaStreamSynchronize(c->st));
  c->steps = 0;
  return LBM_OK;
}

int lbm_step(lbm_ctx* c, int n) {
  if (!c || n < 0) return fail(c, LBM_EINVAL, "lbm_step: n must be >= 0");
  LBM_CK(c, cudaSetDevice(c->device));
  for (int k = 0; k < n; ++k) {
    LBM_CK(c, lbm_ctx_launch_step(c, c->buf[c->cur], c->buf[c->cur ^ 1]));
    c->cur ^= 1;
  }
  c->steps += n;
  return LBM_OK;
}

int lbm_moments(lbm_ctx* c, double* rho, double* ux, double* uy, double* theta, int on_device) {
  if (!c) return LBM_EINVAL;
  LBM_CK(c, cudaSetDevice(c->device));
  const long long n = ncells(c);
  if (on_device) {
    LBM_CK(c, lbm_launch_moments(c->p.lattice, c->prec, c->buf[c->cur], c->g, c->rho0, 1.0 / c->s, c->p.thermal,
                                 rho, ux, uy, theta, c->st));
    return LBM_OK;
  }
  int rc = ensure_scratch(c);
  if (rc) return rc;
  double* s = c->scratch;
  LBM_CK(c, lbm_launch_moments(c->p.lattice, c->prec, c->buf[c->cur], c->g, c->rho0, 1.0 / c->s, c->p.thermal,
                               rho ? s : nullptr, ux ? s + n : nullptr, uy ? s + 2 * n : nullptr,
                               theta ? s + 3 * n : nullptr, c->st));
  const size_t b = sizeof(double) * (size_t)n;
  if (rho) LBM_CK(c, cudaMemcpyAsync(rho, s, b, cudaMemcpyDeviceToHost, c->st));
  if (ux) LBM_CK(c, cudaMemcpyAsync(ux, s + n, b, cudaMemcpyDeviceToHost, c->st));
  if (uy) LBM_CK(c, cudaMemcpyAsync(uy, s + 2 * n, b, cudaMemcpyDeviceToHost, c->st));
  if (theta) LBM_CK(c, cudaMemcpyAsync(theta, s + 3 * n, b, cudaMemcpyDeviceToHost, c->st));
  LBM_CK(c, cudaStreamSynchronize(c->st));
  return LBM_OK;
}

int lbm_conservation(lbm_ctx* c, double out[4]) {
  if (!c || !out) return LBM_EINVAL;
  LBM_CK(c, cudaSetDevice(c->device));
  LBM_CK(c, lbm_launch_conservation(c->p.lattice, c->prec, c->buf[c->cur], c->g, c->rho0, 1.0 / c->s, c->partials,
                                    c->out4, c->st));
  LBM_CK(c, cudaMemcpyAsync(c->host4, c->out4, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  LBM_CK(c, cudaMemcpyAsync(c->host4 + 4, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  LBM_CK(c, cudaStreamSynchronize(c->st));
  if (*reinterpret_cast<int*>(c->host4 + 4) != 0) return fail(c, LBM_ETIMEOUT, "a step kernel's bounded wait ran out");
  bool finite = true;
  for (int k = 0; k < 4; ++k) {
    out[k] = c->host4[k];
    finite = finite && std::isfinite(out[k]);
  }
  return finite ? LBM_OK : fail(c, LBM_EUNSTABLE, "lbm_conservation: non-finite state");
}

int lbm_diagnostics(lbm_ctx* c, double out[4]) {
  if (!c || !out) return LBM_EINVAL;
  LBM_CK(c, cudaSetDevice(c->device));
  int rc = ensure_scratch(c);
  if (rc) return rc;
  const long long n = ncells(c);
  double* ux = c->scratch;
  double* uy = c->scratch + n;
  LBM_CK(c, lbm_launch_moments(c->p.lattice, c->prec, c->buf[c->cur], c->g, c->rho0, 1.0 / c->s, 0, nullptr, ux, uy,
                               nullptr, c->st));
  LBM_CK(c, lbm_launch_diagnostics(ux, uy, c->g, c->partials, c->out4, c->st));
  LBM_CK(c, cudaMemcpyAsync(c->host4, c->out4, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  LBM_CK(c, cudaMemcpyAsync(c->host4 + 4, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  LBM_CK(c, cudaStreamSynchronize(c->st));
  if (*reinterpret_cast<int*>(c->host4 + 4) != 0) return fail(c, LBM_ETIMEOUT, "a step kernel's bounded wait ran out");
  const double inv = 1.0 / (double)n;
  const double m0 = c->host4[0] * inv, m1 = c->host4[2] * inv;
  const double v0 = c->host4[1] * inv - m0 * m0, v1 = c->host4[3] * inv - m1 * m1;
  out[0] = m0;
  out[1] = std::sqrt(v0 > 0 ? v0 : 0.0);
  out[2] = m1;
  out[3] = std::sqrt(v1 > 0 ? v1 : 0.0);
  bool finite = true;
  for (int k = 0; k < 4; ++k) finite = finite && std::isfinite(c->host4[k]);
  return finite ? LBM_OK : fail(c, LBM_EUNSTABLE, "lbm_diagnostics: non-finite state");
}

int lbm_get_populations(lbm_ctx* c, double* f, int on_device) {
  if (!c || !f) return LBM_EINVAL;
  LBM_CK(c, cudaSetDevice(c->device));
  const long long n = ncells(c);
  if (!on_device) {
    int rc = ensure_scratch(c);
    if (rc) return rc;
  }
  for (int i = 0; i < c->V; ++i) {
    double* dst = on_device ? f + (long long)i * n : c->scratch;
    LBM_CK(c, lbm_launch_get_plane(c->p.lattice, c->prec, c->buf[c->cur], c->g, i, c->rho0, 1.0 / c->s, dst, c->st));
    if (!on_device)
      LBM_CK(c, cudaMemcpyAsync(f + (long long)i * n, dst, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, c->st));
  }
  if (!on_device) LBM_CK(c, cudaStreamSynchronize(c->st));
  return LBM_OK;
}

int lbm_set_populations(lbm_ctx* c, const double* f, int on_device) {
  if (!c || !f) return LBM_EINVAL;
  LBM_CK(c, cudaSetDevice(c->device));
  const long long n = ncells(c);
  if (!on_device) {
    int rc = ensure_scratch(c);
    if (rc) return rc;
  }
  for (int i = 0; i < c->V; ++i) {
    const double* src = f + (long long)i * n;
    if (!on_device) {
      // two halves of the scratch alternate so a copy never overwrites a plane still being encoded
      double* dst = c->scratch + (i & 1) * n;
      LBM_CK(c, cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, c->st));
      src = dst;
    }
    LBM_CK(c, lbm_launch_set_plane(c->p.lattice, c->prec, c->buf[c->cur], c->g, i, c->rho0, c->s, src, c->st));
  }
  if (!on_device) LBM_CK(c, cudaStreamSynchronize(c->st));
  c->steps = 0;
  return LBM_OK;
}

// ---------------------------------------------------------------------------
// Checkpoints
// ---------------------------------------------------------------------------
namespace {
struct CkptHeader {
  char tag[8];  // "LBMCKPT1"
  int32_t lattice, hermite_order, reg_order, collision, thermal, nx, ny, bc_x, bc_y, prec, pitch, V;
  double tau, rho0, s;
  int64_t steps;
};
}  // namespace

int lbm_save(lbm_ctx* c, const char* path) {
  if (!c || !path) return LBM_EINVAL;
  LBM_CK(c, cudaSetDevice(c->device));
  const size_t bytes = (size_t)c->V * (size_t)c->g.plane * c->elem;
  char* host = new (std::nothrow) char[bytes];
  if (!host) return fail(c, LBM_ENOMEM, "lbm_save: host buffer");
  cudaError_t e = cudaMemcpyAsync(host, c->buf[c->cur], bytes, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) {
    delete[] host;
    return cuda_fail(c, e, "lbm_save: copy");
  }
  CkptHeader h{};
  memcpy(h.tag, "LBMCKPT1", 8);
  h.lattice = c->p.lattice;
  h.hermite_order = c->neq;
  h.reg_order = c->nreg;
  h.collision = c->p.collision;
  h.thermal = c->p.thermal;
  h.nx = c->p.nx;
  h.ny = c->p.ny;
  h.bc_x = c->p.bc_x;
  h.bc_y = c->p.bc_y;
  h.prec = c->prec;
  h.pitch = c->g.pitch;
  h.V = c->V;
  h.tau = c->tau;
  h.rho0 = c->rho0;
  h.s = c->s;
  h.steps = c->steps;
  FILE* fp = fopen(path, "wb");
  bool ok = fp && fwrite(&h, sizeof(h), 1, fp) == 1 && fwrite(host, 1, bytes, fp) == bytes;
  if (fp) ok = (fclose(fp) == 0) && ok;
  delete[] host;
  return ok ? LBM_OK : fail(c, LBM_EIO, "lbm_save: write failed");
}

int lbm_load(lbm_ctx* c, const char* path) {
  if (!c || !path) return LBM_EINVAL;
  LBM_CK(c, cudaSetDevice(c->device));
  FILE* fp = fopen(path, "rb");
  if (!fp) return fail(c, LBM_EIO, "lbm_load: cannot open");
  CkptHeader h{};
  if (fread(&h, sizeof(h), 1, fp) != 1 || memcmp(h.tag, "LBMCKPT1", 8) != 0) {
    fclose(fp);
    return fail(c, LBM_EIO, "lbm_load: not a checkpoint");
  }
  if (h.lattice != c->p.lattice || h.hermite_order != c->neq || h.reg_order != c->nreg ||
      h.collision != c->p.collision || h.thermal != c->p.thermal || h.nx != c->p.nx || h.ny != c->p.ny ||
      h.bc_x != c->p.bc_x || h.bc_y != c->p.bc_y || h.prec != c->prec || h.pitch != c->g.pitch || h.V != c->V ||
      h.tau != c->tau || h.rho0 != c->rho0 || h.s != c->s) {
    fclose(fp);
    return fail(c, LBM_EINVAL, "lbm_load: checkpoint parameters differ from the context");
  }
  const size_t bytes = (size_t)c->V * (size_t)c->g.plane * c->elem;
  char* host = new (std::nothrow) char[bytes];
  if (!host) {
    fclose(fp);
    return fail(c, LBM_ENOMEM, "lbm_load: host buffer");
  }
  const bool ok = fread(host, 1, bytes, fp) == bytes;
  fclose(fp);
  if (!ok) {
    delete[] host;
    return fail(c, LBM_EIO, "lbm_load: truncated file");
  }
  c->cur = 0;
  cudaError_t e = cudaMemcpyAsync(c->buf[0], host, bytes, cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  delete[] host;
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_load: copy");
  c->steps = h.steps;
  return LBM_OK;
}

}  // extern "C"
