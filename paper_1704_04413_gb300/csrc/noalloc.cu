// Allocation-free conservation sums (lbm_conservation_noalloc in lbm.h).
//
// Some callers cannot call cudaMalloc at the point where they need the sums:
// code running inside a memory budget owned by another allocator (a framework
// memory pool that holds all device memory), real-time loops that forbid
// allocation after start-up, or plug-in hosts that hand out device buffers but
// no allocation rights.  For them this entry point takes the populations and
// the 4-double output as caller-owned device memory and keeps its only scratch
// (the per-block partial sums of the two-pass reduction) in the file-scope
// device array below, which every GPU that loads the library holds until the
// process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lbm.h"
#include "fields.h"

namespace {

constexpr int kPartialsPerBlock = 4;  // mass, x-momentum, y-momentum, energy
constexpr int kCellsPerBlock = 256;   // cells one reduction block covers (fields.cu)
constexpr long long kMaxBlocks = LBM_NOALLOC_MAX_CELLS / kCellsPerBlock;

// Partial sums of the reduction.  Shared by every call on a device; each call's blocks overwrite
// the slots they use before the final pass reads them, so nothing has to start at zero.
static __device__ __align__(256) double g_noalloc_partials[kMaxBlocks * kPartialsPerBlock];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_partials_ptr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_partials on the current device, looked up once per device.
int partials_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ECUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_partials_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return LBM_ECUDA;
    g_partials_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_ptr[dev];
  return LBM_OK;
}

// True when p is memory a kernel on the current device may read and write: device or managed memory.
// Host memory (pageable or pinned) is refused, so that a host address passed by mistake returns
// LBM_EINVAL instead of reaching the kernel.
bool device_accessible(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the error the failed query recorded
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool is_pow2(double s) {
  if (!(s > 0)) return false;
  int e = 0;
  return frexp(s, &e) == 0.5;
}

}  // namespace

extern "C" int lbm_conservation_noalloc(int lattice, int storage, const void* f, int nx, int ny, int pitch,
                                        double rho0, double store_scale, double* out4, void* stream) {
  if (lattice < LBM_D2Q9 || lattice > LBM_D2V37 || !f || !out4) return LBM_EINVAL;
  if (nx < 1 || ny < 1 || pitch < nx) return LBM_EINVAL;
  if ((long long)nx * ny > LBM_NOALLOC_MAX_CELLS) return LBM_EINVAL;  // beyond the static scratch
  int prec;
  switch (storage) {
    case LBM_F64: prec = lbm::PREC_F64; break;
    case LBM_F32: prec = lbm::PREC_F32; break;
    case LBM_F16_SHIFT: prec = lbm::PREC_F16; break;
    case LBM_BF16_SHIFT: prec = lbm::PREC_BF16; break;
    case LBM_I16_SHIFT: prec = lbm::PREC_I16; break;
    default: return LBM_EINVAL;
  }
  const double r0 = rho0 == 0 ? 1.0 : rho0;
  const double s = store_scale == 0 ? 1.0 : store_scale;
  if (!(r0 > 0) || !is_pow2(s)) return LBM_EINVAL;
  if (!device_accessible(f) || !device_accessible(out4)) return LBM_EINVAL;
  double* partials = nullptr;
  const int rc = partials_for_current_device(&partials);
  if (rc != LBM_OK) return rc;
  lbm::StepGeom g{};
  g.pitch = pitch;
  g.plane = (long long)pitch * ny;
  g.nx = nx;
  g.ny = ny;
  const cudaError_t e = lbm_launch_conservation(lattice, prec, f, g, r0, 1.0 / s, partials, out4,
                                                static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
