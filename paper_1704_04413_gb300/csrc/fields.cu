// Per-cell kernels around the step: initial state (Sec. III.B), macroscopic
// fields (Sec. II.A), population transfer, FP64 conservation sums and the
// flow diagnostics of Sec. III.B.  All of them work in double precision; none
// is on the time-stepping path.
#include <cuda_runtime.h>

#include "fields.h"

namespace lbm {

constexpr int FB = 256;  // threads per block of the per-cell kernels

template <class L, class S, int i>
__device__ __forceinline__ double decode(const S* f, long long off, double rho0, double inv_s) {
  const double q = (double)Store<S>::ld(f + off);
  if constexpr (Store<S>::SHIFTED) {
    constexpr double w = L::W[i];
    return w * (rho0 + q * inv_s);
  } else {
    return q;
  }
}

// ---------------------------------------------------------------------------
// Initial state: f = f^(0),N + f^(1) (Sec. III.B), f^(1) from the
// Chapman-Enskog a1^(2) of the velocity gradients (App. A) and the recursions
// (App. C) up to the lattice's highest order.
// ---------------------------------------------------------------------------
template <class L, class S, bool THERMAL>
__global__ void k_init(const double* __restrict__ rho, const double* __restrict__ ux, const double* __restrict__ uy,
                       const double* __restrict__ theta, const double* __restrict__ grad, S* __restrict__ f,
                       StepGeom g, InitParams ip) {
  const long long c = (long long)blockIdx.x * FB + threadIdx.x;
  const long long n = (long long)g.nx * g.ny;
  if (c >= n) return;
  const int x = (int)(c % g.nx), y = (int)(c / g.nx);
  // FP64 arithmetic for FP64 storage, FP32 otherwise (the state is stored in 32 bits or fewer)
  using Real = typename std::conditional<std::is_same<S, double>::value, double, float>::type;
  constexpr double c2 = L::CS2;
  const Real r = (Real)rho[c], u = (Real)ux[c], v = (Real)uy[c];
  const Real th = (THERMAL && theta) ? (Real)theta[c] : Real(1);
  const Real e = Real(c2) * (th - Real(1));
  Real A[5][5], B[5][5] = {}, C[5][5];
  equilibrium_coefficients<L, THERMAL>(r, u, v, e, A);
  const bool neq_part = grad != nullptr;
  if (neq_part) {
    // d[a][b] = d_b u_a
    const Real d[2][2] = {{(Real)grad[c], (Real)grad[n + c]}, {(Real)grad[2 * n + c], (Real)grad[3 * n + c]}};
    const Real div = d[0][0] + d[1][1];
    const Real pre = -(Real)ip.tau * r * Real(c2) * th;
    Real sxx = Real(2) * d[0][0], syy = Real(2) * d[1][1];
    if (THERMAL) {  // traceless part, D = 2
      sxx -= div;
      syy -= div;
    }
    B[2][0] = pre * sxx;
    B[0][2] = pre * syy;
    B[1][1] = pre * (d[0][1] + d[1][0]);
    a1_third_from_second<L, THERMAL>(u, v, B);
    a1_fourth<L, THERMAL>(u, v, e, B);
  }
  sfor<0, L::NMAX + 1>([&](auto N) {
    constexpr int nn = LBM_CI(N);
    sfor<0, nn + 1>([&](auto Aa) {
      constexpr int a = LBM_CI(Aa);
      constexpr int b = nn - a;
      if constexpr (L::keep(a, b)) {
        constexpr double sc = 1.0 / (factorial(a) * factorial(b) * ipow(c2, a + b));
        Real val = (nn <= ip.neq) ? A[a][b] : Real(0);
        if constexpr (nn >= 2) val += B[a][b];
        if constexpr (Store<S>::SHIFTED) val *= (Real)ip.s;
        C[a][b] = val * Real(sc);
      }
    });
  });
  const long long o = (long long)y * g.pitch + x;
  const Real shift = Store<S>::SHIFTED ? (Real)(-ip.s * ip.rho0) : Real(0);
  rebuild<L, Store<S>::SHIFTED>(C, [&](auto I, Real acc) {
    constexpr int i = LBM_CI(I);
    Store<S>::st(f + (long long)i * g.plane + o, acc + shift);
  });
}

// Macroscopic fields of the stored state (Sec. II.A).
// Compensated FP32 sum (Knuth's two-sum of every term, the rounding errors summed alongside): s + c keeps about
// twice the FP32 precision.  add_scaled takes k x for a small integer k exactly: a power of two scales exactly,
// another k adds the product's rounding error (fmaf) to c.
struct CSum32 {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    const float z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
  }
  template <int k>
  __device__ __forceinline__ void add_scaled(float x) {
    constexpr int a = k < 0 ? -k : k;
    if constexpr ((a & (a - 1)) == 0) {
      add((float)k * x);
    } else {
      const float p = (float)k * x;
      c += fmaf((float)k, x, -p);
      add(p);
    }
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// One block row of FB columns of one grid row (blockIdx.y, then every gridDim.y-th row): no 64-bit division of
// the cell index.  The FP64 sums skip the terms whose velocity factor is zero, the energy sum is made only
// where theta is asked for on a thermal lattice (E2), and u = j * (1 / rho): GB300's FP64 rate makes these
// the kernel's cost (65536 D2Q9 cells: 12.3 us before).  FP32 storage sums in compensated FP32 (CSum32).
template <class L, class S, bool E2>
__global__ void k_moments(const S* __restrict__ f, StepGeom g, double rho0, double inv_s, int thermal,
                          double* __restrict__ rho, double* __restrict__ ux, double* __restrict__ uy,
                          double* __restrict__ theta) {
  const int x = (int)blockIdx.x * FB + (int)threadIdx.x;
  if (x >= g.nx) return;
  for (int y = blockIdx.y; y < g.ny; y += gridDim.y) {
    const long long c = (long long)y * g.nx + x;
    const long long o = (long long)y * g.pitch + x;
    double r = 0, jx = 0, jy = 0, e2 = 0;
    if constexpr (std::is_same<S, float>::value && !E2) {
      // FP32 populations summed exactly enough in compensated FP32 (about 1e-14 relative): FP32 work instead of
      // FP64, whose rate on GB300 made these sums the pass's cost
      CSum32 sr, sx, sy;
      sfor<0, L::Q>([&](auto I) {
        constexpr int i = LBM_CI(I);
        constexpr int cx = L::CX[i], cy = L::CY[i];
        const float fi = __ldg(f + (long long)i * g.plane + o);
        sr.add(fi);
        if constexpr (cx != 0) sx.add_scaled<cx>(fi);
        if constexpr (cy != 0) sy.add_scaled<cy>(fi);
      });
      r = sr.value();
      jx = sx.value();
      jy = sy.value();
    } else {
      sfor<0, L::Q>([&](auto I) {
        constexpr int i = LBM_CI(I);
        constexpr double cx = L::CX[i], cy = L::CY[i];
        const double fi = decode<L, S, i>(f, (long long)i * g.plane + o, rho0, inv_s);
        r += fi;
        if constexpr (cx != 0.0) jx += cx * fi;
        if constexpr (cy != 0.0) jy += cy * fi;
        if constexpr (E2 && cx * cx + cy * cy != 0.0) e2 += (cx * cx + cy * cy) * fi;
      });
    }
    const double ir = 1.0 / r;
    const double u = jx * ir, v = jy * ir;
    if (rho) rho[c] = r;
    if (ux) ux[c] = u;
    if (uy) uy[c] = v;
    if (theta) theta[c] = E2 ? (e2 * ir - u * u - v * v) / (2.0 * L::CS2) : 1.0;
  }
}

// Population transfer between the stored (padded, encoded) layout and dense doubles, one plane.
template <class L, class S>
__global__ void k_get_plane(const S* __restrict__ f, StepGeom g, int i, double rho0, double inv_s,
                            double* __restrict__ out) {
  const long long c = (long long)blockIdx.x * FB + threadIdx.x;
  const long long n = (long long)g.nx * g.ny;
  if (c >= n) return;
  const int x = (int)(c % g.nx), y = (int)(c / g.nx);
  const double q = (double)Store<S>::ld(f + (long long)i * g.plane + (long long)y * g.pitch + x);
  double w = 0.0;
  sfor<0, L::Q>([&](auto I) {
    constexpr int k = LBM_CI(I);
    constexpr double wk = L::W[k];
    if (k == i) w = wk;
  });
  out[c] = Store<S>::SHIFTED ? w * (rho0 + q * inv_s) : q;
}

template <class L, class S>
__global__ void k_set_plane(S* __restrict__ f, StepGeom g, int i, double rho0, double s,
                            const double* __restrict__ in) {
  const long long c = (long long)blockIdx.x * FB + threadIdx.x;
  const long long n = (long long)g.nx * g.ny;
  if (c >= n) return;
  const int x = (int)(c % g.nx), y = (int)(c / g.nx);
  double w = 1.0;
  sfor<0, L::Q>([&](auto I) {
    constexpr int k = LBM_CI(I);
    constexpr double wk = L::W[k];
    if (k == i) w = wk;
  });
  const double v = Store<S>::SHIFTED ? (in[c] / w - rho0) * s : in[c];
  Store<S>::st(f + (long long)i * g.plane + (long long)y * g.pitch + x, v);
}

// ---------------------------------------------------------------------------
// Deterministic reductions: a fixed per-thread order, a warp-shuffle tree and
// a fixed-order block tree give per-block partials; one block then adds the
// partials in an order fixed by their count (k_sum_partials).
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* partial_out) {
  __shared__ double sh[FB / 32][K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double a = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    v[k] = a;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[wid][k] = v[k];
  __syncthreads();
  if (threadIdx.x < K) {
    double a = 0.0;
    for (int w = 0; w < FB / 32; ++w) a += sh[w][threadIdx.x];
    partial_out[threadIdx.x] = a;
  }
}

template <class L, class S>
__global__ void k_conservation_partials(const S* __restrict__ f, StepGeom g, double rho0, double inv_s,
                                        double* __restrict__ partials) {
  const long long c = (long long)blockIdx.x * FB + threadIdx.x;
  const long long n = (long long)g.nx * g.ny;
  double v[4] = {0, 0, 0, 0};
  if (c < n) {
    const int x = (int)(c % g.nx), y = (int)(c / g.nx);
    const long long o = (long long)y * g.pitch + x;
    sfor<0, L::Q>([&](auto I) {
      constexpr int i = LBM_CI(I);
      constexpr double cx = L::CX[i], cy = L::CY[i];
      const double fi = decode<L, S, i>(f, (long long)i * g.plane + o, rho0, inv_s);
      v[0] += fi;
      v[1] += cx * fi;
      v[2] += cy * fi;
      v[3] += 0.5 * (cx * cx + cy * cy) * fi;
    });
  }
  block_sum<4>(v, partials + 4LL * blockIdx.x);
}

// Second pass of the two-pass sums: one block of SUM_T threads.  Thread t adds the partials t, t + SUM_T,
// t + 2 SUM_T, ... (coalesced), then the threads' sums are combined by a warp shuffle tree and the warps'
// sums in warp order.  The order of every addition is fixed by nblocks alone, so the result is the same
// bits on every run.
constexpr int SUM_T = 256;
__global__ void __launch_bounds__(SUM_T) k_sum_partials(const double* __restrict__ partials, int nblocks, int k_per,
                                                       double* __restrict__ out) {
  __shared__ double sh[SUM_T / 32][4];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = t; b < nblocks; b += SUM_T)
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < k_per) a[k] += partials[(long long)b * k_per + k];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_down_sync(0xffffffffu, a[k], o);
    if (lane == 0) sh[wid][k] = a[k];
  }
  __syncthreads();
  if (t < k_per) {
    double r = 0.0;
    for (int w = 0; w < SUM_T / 32; ++w) r += sh[w][t];
    out[t] = r;
  }
}

// u^2 and enstrophy density omega^2 / 2 with fourth-order centred differences (Sec. III.B)
__device__ __forceinline__ int nb(int x, int d, int n, int bc) {
  int s = x + d;
  if (bc == BC_PERIODIC) {
    s = ((s % n) + n) % n;
  } else {
    s = s < 0 ? 0 : (s > n - 1 ? n - 1 : s);
  }
  return s;
}

__global__ void k_diag_partials(const double* __restrict__ ux, const double* __restrict__ uy, StepGeom g,
                                double* __restrict__ partials) {
  const long long c = (long long)blockIdx.x * FB + threadIdx.x;
  const long long n = (long long)g.nx * g.ny;
  double v[4] = {0, 0, 0, 0};
  if (c < n) {
    const int x = (int)(c % g.nx), y = (int)(c / g.nx);
    auto at = [&](const double* a, int xx, int yy) { return a[(long long)yy * g.nx + xx]; };
    const double dvdx = (-at(uy, nb(x, 2, g.nx, g.bcx), y) + 8.0 * at(uy, nb(x, 1, g.nx, g.bcx), y) -
                         8.0 * at(uy, nb(x, -1, g.nx, g.bcx), y) + at(uy, nb(x, -2, g.nx, g.bcx), y)) / 12.0;
    const double dudy = (-at(ux, x, nb(y, 2, g.ny, g.bcy)) + 8.0 * at(ux, x, nb(y, 1, g.ny, g.bcy)) -
                         8.0 * at(ux, x, nb(y, -1, g.ny, g.bcy)) + at(ux, x, nb(y, -2, g.ny, g.bcy))) / 12.0;
    const double w = dvdx - dudy;
    const double u2 = ux[c] * ux[c] + uy[c] * uy[c];
    const double ens = 0.5 * w * w;
    v[0] = u2;
    v[1] = u2 * u2;
    v[2] = ens;
    v[3] = ens * ens;
  }
  block_sum<4>(v, partials + 4LL * blockIdx.x);
}

// ---------------------------------------------------------------------------
// Dispatch
// ---------------------------------------------------------------------------
static inline unsigned nblk(const StepGeom& g) { return (unsigned)(((long long)g.nx * g.ny + FB - 1) / FB); }

template <class L, class S>
static cudaError_t init_t(const double* rho, const double* ux, const double* uy, const double* th, const double* grad,
                          void* f, const StepGeom& g, const InitParams& ip, cudaStream_t st) {
  if (ip.thermal)
    k_init<L, S, true><<<nblk(g), FB, 0, st>>>(rho, ux, uy, th, grad, (S*)f, g, ip);
  else
    k_init<L, S, false><<<nblk(g), FB, 0, st>>>(rho, ux, uy, th, grad, (S*)f, g, ip);
  return cudaGetLastError();
}

template <class L>
static cudaError_t init_l(int prec, const double* rho, const double* ux, const double* uy, const double* th,
                          const double* grad, void* f, const StepGeom& g, const InitParams& ip, cudaStream_t st) {
  switch (prec) {
    case PREC_F64: return init_t<L, double>(rho, ux, uy, th, grad, f, g, ip, st);
    case PREC_F32: return init_t<L, float>(rho, ux, uy, th, grad, f, g, ip, st);
    case PREC_F16: return init_t<L, __half>(rho, ux, uy, th, grad, f, g, ip, st);
    case PREC_BF16: return init_t<L, __nv_bfloat16>(rho, ux, uy, th, grad, f, g, ip, st);
    case PREC_I16: return init_t<L, short>(rho, ux, uy, th, grad, f, g, ip, st);
  }
  return cudaErrorInvalidValue;
}

#define LBM_DISPATCH_LATTICE(lat, FN, ...)                  \
  switch (lat) {                                            \
    case 0: return FN<D2Q9>(__VA_ARGS__);                   \
    case 1: return FN<D2V17>(__VA_ARGS__);                  \
    case 2: return FN<D2V37>(__VA_ARGS__);                  \
  }                                                         \
  return cudaErrorInvalidValue;

#define LBM_DISPATCH_PREC(prec, FN, L, ...)                    \
  switch (prec) {                                              \
    case PREC_F64: return FN<L, double>(__VA_ARGS__);          \
    case PREC_F32: return FN<L, float>(__VA_ARGS__);           \
    case PREC_F16: return FN<L, __half>(__VA_ARGS__);          \
    case PREC_BF16: return FN<L, __nv_bfloat16>(__VA_ARGS__);  \
    case PREC_I16: return FN<L, short>(__VA_ARGS__);           \
  }                                                            \
  return cudaErrorInvalidValue;

template <class L, class S>
static cudaError_t moments_t(const void* f, const StepGeom& g, double rho0, double inv_s, int thermal, double* rho,
                             double* ux, double* uy, double* th, cudaStream_t st) {
  const dim3 grid((unsigned)((g.nx + FB - 1) / FB), (unsigned)(g.ny < 65535 ? g.ny : 65535));
  if (th && thermal)
    k_moments<L, S, true><<<grid, FB, 0, st>>>((const S*)f, g, rho0, inv_s, thermal, rho, ux, uy, th);
  else
    k_moments<L, S, false><<<grid, FB, 0, st>>>((const S*)f, g, rho0, inv_s, thermal, rho, ux, uy, th);
  return cudaGetLastError();
}
template <class L>
static cudaError_t moments_l(int prec, const void* f, const StepGeom& g, double rho0, double inv_s, int thermal,
                             double* rho, double* ux, double* uy, double* th, cudaStream_t st) {
  LBM_DISPATCH_PREC(prec, moments_t, L, f, g, rho0, inv_s, thermal, rho, ux, uy, th, st)
}

template <class L, class S>
static cudaError_t getp_t(const void* f, const StepGeom& g, int i, double rho0, double inv_s, double* out,
                          cudaStream_t st) {
  k_get_plane<L, S><<<nblk(g), FB, 0, st>>>((const S*)f, g, i, rho0, inv_s, out);
  return cudaGetLastError();
}
template <class L>
static cudaError_t getp_l(int prec, const void* f, const StepGeom& g, int i, double rho0, double inv_s, double* out,
                          cudaStream_t st) {
  LBM_DISPATCH_PREC(prec, getp_t, L, f, g, i, rho0, inv_s, out, st)
}

template <class L, class S>
static cudaError_t setp_t(void* f, const StepGeom& g, int i, double rho0, double s, const double* in,
                          cudaStream_t st) {
  k_set_plane<L, S><<<nblk(g), FB, 0, st>>>((S*)f, g, i, rho0, s, in);
  return cudaGetLastError();
}
template <class L>
static cudaError_t setp_l(int prec, void* f, const StepGeom& g, int i, double rho0, double s, const double* in,
                          cudaStream_t st) {
  LBM_DISPATCH_PREC(prec, setp_t, L, f, g, i, rho0, s, in, st)
}

template <class L, class S>
static cudaError_t cons_t(const void* f, const StepGeom& g, double rho0, double inv_s, double* partials,
                          double* out4, cudaStream_t st) {
  const unsigned nb_ = nblk(g);
  k_conservation_partials<L, S><<<nb_, FB, 0, st>>>((const S*)f, g, rho0, inv_s, partials);
  k_sum_partials<<<1, SUM_T, 0, st>>>(partials, (int)nb_, 4, out4);
  return cudaGetLastError();
}
template <class L>
static cudaError_t cons_l(int prec, const void* f, const StepGeom& g, double rho0, double inv_s, double* partials,
                          double* out4, cudaStream_t st) {
  LBM_DISPATCH_PREC(prec, cons_t, L, f, g, rho0, inv_s, partials, out4, st)
}

}  // namespace lbm

using namespace lbm;

long long lbm_partials_count(const StepGeom& g) { return 4LL * nblk(g); }

cudaError_t lbm_launch_init(int lat, int prec, const double* rho, const double* ux, const double* uy,
                            const double* th, const double* grad, void* f, const StepGeom& g, const InitParams& ip,
                            cudaStream_t st) {
  LBM_DISPATCH_LATTICE(lat, init_l, prec, rho, ux, uy, th, grad, f, g, ip, st)
}

cudaError_t lbm_launch_moments(int lat, int prec, const void* f, const StepGeom& g, double rho0, double inv_s,
                               int thermal, double* rho, double* ux, double* uy, double* th, cudaStream_t st) {
  LBM_DISPATCH_LATTICE(lat, moments_l, prec, f, g, rho0, inv_s, thermal, rho, ux, uy, th, st)
}

cudaError_t lbm_launch_get_plane(int lat, int prec, const void* f, const StepGeom& g, int i, double rho0,
                                 double inv_s, double* out, cudaStream_t st) {
  LBM_DISPATCH_LATTICE(lat, getp_l, prec, f, g, i, rho0, inv_s, out, st)
}

cudaError_t lbm_launch_set_plane(int lat, int prec, void* f, const StepGeom& g, int i, double rho0, double s,
                                 const double* in, cudaStream_t st) {
  LBM_DISPATCH_LATTICE(lat, setp_l, prec, f, g, i, rho0, s, in, st)
}

cudaError_t lbm_launch_conservation(int lat, int prec, const void* f, const StepGeom& g, double rho0, double inv_s,
                                    double* partials, double* out4, cudaStream_t st) {
  LBM_DISPATCH_LATTICE(lat, cons_l, prec, f, g, rho0, inv_s, partials, out4, st)
}

cudaError_t lbm_launch_diagnostics(const double* ux, const double* uy, const StepGeom& g, double* partials,
                                   double* out4, cudaStream_t st) {
  const unsigned nb_ = nblk(g);
  k_diag_partials<<<nb_, FB, 0, st>>>(ux, uy, g, partials);
  k_sum_partials<<<1, SUM_T, 0, st>>>(partials, (int)nb_, 4, out4);
  return cudaGetLastError();
}
