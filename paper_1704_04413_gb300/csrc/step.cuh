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

#include <type_traits>

#include "bulk.cuh"
#include "collide.cuh"
#include "lbm.h"

namespace lbm {

enum { BC_PERIODIC = 0, BC_ZERO_GRADIENT = 1 };
enum { PREC_F64 = 0, PREC_F32 = 1, PREC_F16 = 2, PREC_BF16 = 3, PREC_I16 = 4 };

struct StepGeom {
  long long plane;  // elements per population plane (ny * pitch)
  int pitch;        // elements per row
  int nx, ny;
  int bcx, bcy;
  int nsm;          // SMs of the device (persistent grids)
};

struct CollParamsD {
  double omega, om1;  // 1 / tau, 1 - 1 / tau (order 2 of f^(1); BGK)
  double om1_3, om1_4;  // 1 - 1 / tau_n of the order-3 and order-4 coefficients of f^(1)
  double tau, tau3;     // tau_2, tau_3 (finite-difference a1)
  int neq, nreg;
  double rho0, s, inv_s;
};

template <class Real>
__host__ __device__ inline CollParams<Real> cast_params(const CollParamsD& d) {
  using Sc = typename Scalar<Real>::type;
  CollParams<Real> p;
  p.omega = Real((Sc)d.omega);
  p.om1 = Real((Sc)d.om1);
  p.om1_3 = Real((Sc)d.om1_3);
  p.om1_4 = Real((Sc)d.om1_4);
  p.tau = Real((Sc)d.tau);
  p.tau3 = Real((Sc)d.tau3);
  p.neq = d.neq;
  p.nreg = d.nreg;
  p.rho0 = Real((Sc)d.rho0);
  p.s = Real((Sc)d.s);
  p.inv_s = Real((Sc)d.inv_s);
  return p;
}

// Parameters of a 2D collision on lattice L with storage S (coll: COLL_*), with the per-coefficient factors
// of the rebuild (plain storage has no scale).
template <class L, class Real, class S>
inline CollParams<Real> coll_params_2d(const CollParamsD& d, int coll) {
  CollParams<Real> p = cast_params<Real>(d);
  set_coef_factors<L>(p, coll, d.neq, d.nreg, d.omega, d.om1, d.om1_3, d.om1_4, Store<S>::SHIFTED ? d.s : 1.0);
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

#ifndef LBM_STEP_BX
#define LBM_STEP_BX 128
#endif
#ifndef LBM_STEP_MINB_LARGE
#define LBM_STEP_MINB_LARGE 5
#endif
#ifndef LBM_STEP_MINB_LARGE_ISO32
#define LBM_STEP_MINB_LARGE_ISO32 7
#endif
constexpr int STEP_BX = LBM_STEP_BX;  // cells (threads) per block

// Byte offsets of the pulled source of population i relative to the cell's address in plane 0,
// (i * plane - cy_i * pitch - cx_i) * sizeof(S) (interior cells, no wrap), and of its store,
// i * plane * sizeof(S).  Kernel parameters: they enter the address adds as constant-bank operands.
template <int Q>
struct PullOffsets {
  long long src[Q];
  long long dst[Q];
  int cy[Q];  // y-velocity components, indexed at run time by the staged kernel's copy-issuing lanes
};

// Offsets of the pulled source / the store of population i as template accessors: from the kernel
// parameters (single-grid launches) or recomputed from the grid geometry (batched launches).
template <int Q>
struct ParamOffsets {
  const PullOffsets<Q>& o;
  template <int i>
  __device__ __forceinline__ long long src() const { return o.src[i]; }
  template <int i>
  __device__ __forceinline__ long long dst() const { return o.dst[i]; }
};
template <class L, class S>
struct GeomOffsets {
  long long plane_b, pitch_b;  // bytes
  template <int i>
  __device__ __forceinline__ long long src() const {
    constexpr int cx = L::CX[i], cy = L::CY[i];
    return i * plane_b - cy * pitch_b - cx * (long long)sizeof(S);
  }
  template <int i>
  __device__ __forceinline__ long long dst() const { return i * plane_b; }
};

// Raw loads issued in program order (volatile asm keeps them ahead of the arithmetic that consumes
// them, so all V loads of a cell are in flight together).
template <class S>
__device__ __forceinline__ auto ld_raw(const char* p);
template <>
__device__ __forceinline__ auto ld_raw<double>(const char* p) {
  double v;
  asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
template <>
__device__ __forceinline__ auto ld_raw<float>(const char* p) {
  float v;
  asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
template <>
__device__ __forceinline__ auto ld_raw<__half>(const char* p) {
  unsigned short u;
  asm volatile("ld.global.nc.b16 %0, [%1];" : "=h"(u) : "l"(p));
  return __half2float(__ushort_as_half(u));
}
template <>
__device__ __forceinline__ auto ld_raw<__nv_bfloat16>(const char* p) {
  unsigned short u;
  asm volatile("ld.global.nc.b16 %0, [%1];" : "=h"(u) : "l"(p));
  return __bfloat162float(__ushort_as_bfloat16(u));
}
template <>
__device__ __forceinline__ auto ld_raw<short>(const char* p) {
  short u;
  asm volatile("ld.global.nc.s16 %0, [%1];" : "=h"(u) : "l"(p));
  return (float)u * (1.0f / kFix16);
}

// Registers: the D2V37 kernels are capped so that at least LBM_STEP_MINB_LARGE blocks fit on an SM; the
// isothermal ones with FP32 arithmetic fit 72 registers without spills, seven blocks (28 warps) a SM:
// measured on the 1024^2 shear layer, 18.3 -> 18.9 GLUPS alone and 0.748 -> 0.776 of the measured copy
// in the benchmark; FP64 and thermal kernels would spill at that cap.
template <class L, bool THERMAL, class Real>
struct StepBlocks {
  static constexpr int MIN =
      L::Q > 20 ? ((!THERMAL && sizeof(Real) == 4) ? LBM_STEP_MINB_LARGE_ISO32 : LBM_STEP_MINB_LARGE) : 1;
};

// One block = STEP_BX consecutive cells of one row; the grid is 1D over (row, column block).
// FD: a1 from central differences of the moments field mom[4][ny][nx] (rho, ux, uy, theta after streaming;
// the pass k_stream_moments writes it); neighbours follow the streaming rule (periodic wrap, or the
// clamped edge cell on a zero-gradient axis).
template <class L, int COLL, bool THERMAL, class Real, class S, bool FD, class OFF>
__device__ __forceinline__ void step_cell(const S* __restrict__ fin, S* __restrict__ fout, const StepGeom& g,
                                          const CollParams<Real>& P, const OFF& off,
                                          const Real* __restrict__ mom, int x, int y) {
  const long long cen = (long long)y * g.pitch + x;
  Real q[L::Q];
  // Rows at least VMAX away from the y edges (a block-uniform test): one load sequence for every
  // column.  The x wrap (or clamp) enters as a per-thread base pointer for each x-velocity, moved
  // by a whole row only where x - c_x leaves [0, nx); one fold suffices because nx >= VMAX.
  // Keeping a single copy of the V loads matters: a second unrolled copy for edge columns,
  // executed by a few warps per row, evicted the hot code from the instruction cache.
  if (y >= L::VMAX && y + L::VMAX < g.ny && g.nx >= L::VMAX) {
    const char* c = reinterpret_cast<const char*>(fin + cen);
    const char* cb[2 * L::VMAX + 1];
    sfor<0, 2 * L::VMAX + 1>([&](auto J) {
      constexpr int cx = LBM_CI(J) - L::VMAX;
      if constexpr (cx == 0) {
        cb[LBM_CI(J)] = c;
      } else {
        const int xs = x - cx;
        int fix;
        if (g.bcx == BC_PERIODIC)
          fix = (xs < 0 ? g.nx : 0) - (xs >= g.nx ? g.nx : 0);
        else
          fix = (xs < 0 ? -xs : 0) - (xs >= g.nx ? xs - g.nx + 1 : 0);
        cb[LBM_CI(J)] = c + (long long)fix * (long long)sizeof(S);
      }
    });
    sfor<0, L::Q>([&](auto I) {
      constexpr int i = LBM_CI(I);
      q[i] = (Real)ld_raw<S>(cb[L::CX[i] + L::VMAX] + off.template src<i>());
    });
  } else {
    const char* b = reinterpret_cast<const char*>(fin);
    sfor<0, L::Q>([&](auto I) {
      constexpr int i = LBM_CI(I);
      const int xs = src_coord(x, L::CX[i], g.nx, g.bcx);
      const int ys = src_coord(y, L::CY[i], g.ny, g.bcy);
      q[i] = (Real)ld_raw<S>(b + off.template dst<i>() + ((long long)ys * g.pitch + xs) * (long long)sizeof(S));
    });
  }
  Real grad[6];
  if constexpr (FD) {
    const long long n = (long long)g.nx * g.ny;
    const long long ce = (long long)y * g.nx + src_coord(x, -1, g.nx, g.bcx);
    const long long cw = (long long)y * g.nx + src_coord(x, 1, g.nx, g.bcx);
    const long long cn = (long long)src_coord(y, -1, g.ny, g.bcy) * g.nx + x;
    const long long cs = (long long)src_coord(y, 1, g.ny, g.bcy) * g.nx + x;
    const Real *mu = mom + n, *mv = mom + 2 * n, *mt = mom + 3 * n;
    grad[0] = Real(0.5) * (mu[ce] - mu[cw]);
    grad[1] = Real(0.5) * (mu[cn] - mu[cs]);
    grad[2] = Real(0.5) * (mv[ce] - mv[cw]);
    grad[3] = Real(0.5) * (mv[cn] - mv[cs]);
    grad[4] = Real(0.5) * (mt[ce] - mt[cw]);
    grad[5] = Real(0.5) * (mt[cn] - mt[cs]);
  }
  collide<L, COLL, THERMAL, Store<S>::SHIFTED, Real, false, FD>(q, P, nullptr, grad);
  char* o = reinterpret_cast<char*>(fout + cen);
  sfor<0, L::Q>([&](auto I) {
    constexpr int i = LBM_CI(I);
    Store<S>::st(reinterpret_cast<S*>(o + off.template dst<i>()), q[i]);
  });
}

// One block = STEP_BX consecutive cells of one row; the grid is 1D over (row, column block).  (A persistent
// grid sized so that every block walks the same number of row tiles measured 30 % slower on GB300 at both
// 1024^2 and 4096^2 than one block per tile, whose blocks the hardware schedules as others finish.)
template <class L, int COLL, bool THERMAL, class Real, class S, bool FD = false>
__global__ void __launch_bounds__(STEP_BX, StepBlocks<L, THERMAL, Real>::MIN)
    k_step(const S* __restrict__ fin, S* __restrict__ fout, StepGeom g, int nbx, CollParams<Real> P,
           const __grid_constant__ PullOffsets<L::Q> off, const Real* __restrict__ mom = nullptr) {
  const int y = blockIdx.x / nbx;
  const int bx = blockIdx.x - y * nbx;
  const int x = bx * STEP_BX + threadIdx.x;
  if (x >= g.nx) return;
  step_cell<L, COLL, THERMAL, Real, S, FD>(fin, fout, g, P, ParamOffsets<L::Q>{off}, mom, x, y);
}

// ---------------------------------------------------------------------------
// Two cells per thread.  Thread t of a block handles columns x = 2t, 2t + 1 of its row; the
// arithmetic runs on both at once in packed FP32x2 (vec2.cuh).  A population whose x-velocity
// is even is pulled with one 8-byte (FP32) or 4-byte (FP16/BF16) aligned load for both cells,
// an odd one with two scalar loads; every store is one aligned pair.
// ---------------------------------------------------------------------------
#ifndef LBM_STEP_PAIRS
#define LBM_STEP_PAIRS 1
#endif
#ifndef LBM_STEP2_MINB_LARGE
#define LBM_STEP2_MINB_LARGE 2
#endif
#ifndef LBM_STEP_STAGED
#define LBM_STEP_STAGED 1
#endif
#ifndef LBM_STEP2_MINB_LARGE_F16
#define LBM_STEP2_MINB_LARGE_F16 4
#endif
#ifndef LBM_STEP_PAIRS_LARGE_16
#define LBM_STEP_PAIRS_LARGE_16 1
#endif
#ifndef LBM_STEP_PAIRS_LARGE_16_MIN
#define LBM_STEP_PAIRS_LARGE_16_MIN (1LL << 21)
#endif

template <class S>
__device__ __forceinline__ F2 ld_pair(const char* p);
template <>
__device__ __forceinline__ F2 ld_pair<float>(const char* p) {
  float a, b;
  asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(a), "=f"(b) : "l"(p));
  return F2(a, b);
}
template <>
__device__ __forceinline__ F2 ld_pair<__half>(const char* p) {
  unsigned u;
  asm volatile("ld.global.nc.b32 %0, [%1];" : "=r"(u) : "l"(p));
  __half2 h = *reinterpret_cast<__half2*>(&u);
  return F2(__half22float2(h));
}
template <>
__device__ __forceinline__ F2 ld_pair<short>(const char* p) {
  unsigned u;
  asm volatile("ld.global.nc.b32 %0, [%1];" : "=r"(u) : "l"(p));
  const float a = (float)(short)(u & 0xffffu), b = (float)(short)(u >> 16);
  return F2(a, b) * F2(1.0f / kFix16);
}
template <>
__device__ __forceinline__ F2 ld_pair<__nv_bfloat16>(const char* p) {
  unsigned u;
  asm volatile("ld.global.nc.b32 %0, [%1];" : "=r"(u) : "l"(p));
  __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&u);
  return F2(__bfloat1622float2(h));
}

template <class S>
__device__ __forceinline__ void st_pair(S* p, F2 v);
template <>
__device__ __forceinline__ void st_pair<float>(float* p, F2 v) {
  *reinterpret_cast<float2*>(p) = v.v;
}
template <>
__device__ __forceinline__ void st_pair<__half>(__half* p, F2 v) {
  *reinterpret_cast<__half2*>(p) = __floats2half2_rn(v.v.x, v.v.y);
}
template <>
__device__ __forceinline__ void st_pair<short>(short* p, F2 v) {
  const unsigned lo = (unsigned short)fix16_encode(v.v.x), hi = (unsigned short)fix16_encode(v.v.y);
  *reinterpret_cast<unsigned*>(p) = lo | (hi << 16);
}
template <>
__device__ __forceinline__ void st_pair<__nv_bfloat16>(__nv_bfloat16* p, F2 v) {
  *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(v.v.x, v.v.y);
}

// Blocks per SM of the pair kernel.  D2V37 with binary16 storage is held to four blocks (128 registers; it
// takes 122): at five (96 registers) its 44 B of spills cost 35.7 -> 30.6 GLUPS at 4096^2.  The others keep
// their unbounded allocation (bfloat16 D2V37: 126 registers).
template <class L, class S>
struct Step2Blocks {
  static constexpr int MIN =
      L::Q > 20 ? (std::is_same<S, __half>::value ? LBM_STEP2_MINB_LARGE_F16 : LBM_STEP2_MINB_LARGE) : 1;
};

// Two neighbouring cells (x, x+1) of row y: pull, collide, store.  xw is the first column of the
// thread's warp (the interior test is uniform across the warp).
// EARLY: store each population as soon as the collision rebuilds it (one row pair at a time, so fewer values
// stay live), else after the whole collision.  Measured on GB300: early stores take the batched three-lattice
// step from 93.8 to 90.5 us, and cost the single-grid kernels 2-4 % (D2Q9 FP32 1024^2, binary16 D2Q9 and
// D2V37 at 4096^2), which keep the late stores.
template <class L, int COLL, class S, class OFF, bool EARLY = false>
__device__ __forceinline__ void step2_cells(const S* __restrict__ fin, S* __restrict__ fout, const StepGeom& g,
                                            const CollParams<F2>& P, const OFF& off, int x, int y, int xw) {
  const bool two = x + 1 < g.nx;
  const long long cen = (long long)y * g.pitch + x;
  F2 q[L::Q];
  // One load sequence for all rows VMAX away from the y edges, when either the warp's 64 columns
  // need no x wrap or the x wrap is periodic on an even nx.  In the latter case both cells of a
  // pair wrap together for an even c_x (x - c_x is even, so the 8-byte pair load stays aligned),
  // and each cell gets its own base pointer for an odd c_x.  Base pointers move by a whole row only
  // where x - c_x leaves [0, nx) (one fold: nx >= VMAX).
  const bool x_inner = xw >= L::VMAX && xw + 63 + L::VMAX < g.nx;
  const bool x_wrap_ok = g.bcx == BC_PERIODIC && (g.nx & 1) == 0 && g.nx >= L::VMAX;
  if (y >= L::VMAX && y + L::VMAX < g.ny && (x_inner || x_wrap_ok)) {
    const char* c = reinterpret_cast<const char*>(fin + cen);
    const char* cb0[2 * L::VMAX + 1];
    const char* cb1[2 * L::VMAX + 1];
    auto fold = [&](int xs) { return (xs < 0 ? g.nx : 0) - (xs >= g.nx ? g.nx : 0); };
    sfor<0, 2 * L::VMAX + 1>([&](auto J) {
      constexpr int j = LBM_CI(J);
      constexpr int cx = j - L::VMAX;
      if constexpr (cx == 0) {
        cb0[j] = c;
        cb1[j] = c;
      } else {
        cb0[j] = c + (long long)fold(x - cx) * (long long)sizeof(S);
        cb1[j] = (cx % 2 == 0) ? cb0[j] : c + (long long)fold(x + 1 - cx) * (long long)sizeof(S);
      }
    });
    sfor<0, L::Q>([&](auto I) {
      constexpr int i = LBM_CI(I);
      constexpr int j = L::CX[i] + L::VMAX;
      const long long so = off.template src<i>();
      if constexpr (L::CX[i] % 2 == 0) {
        q[i] = ld_pair<S>(cb0[j] + so);
      } else {
        const float a = ld_raw<S>(cb0[j] + so);
        const float b = ld_raw<S>(cb1[j] + so + (long long)sizeof(S));
        q[i] = F2(a, b);
      }
    });
  } else {
    const char* b = reinterpret_cast<const char*>(fin);
    const int x1 = two ? x + 1 : x;  // a missing second cell repeats the first; it is not stored
    sfor<0, L::Q>([&](auto I) {
      constexpr int i = LBM_CI(I);
      constexpr int cx = L::CX[i], cy = L::CY[i];
      const int ys = src_coord(y, cy, g.ny, g.bcy);
      const int xs0 = src_coord(x, cx, g.nx, g.bcx);
      const int xs1 = src_coord(x1, cx, g.nx, g.bcx);
      const long long row = (long long)ys * g.pitch;
      const float a = ld_raw<S>(b + off.template dst<i>() + (row + xs0) * (long long)sizeof(S));
      const float c = ld_raw<S>(b + off.template dst<i>() + (row + xs1) * (long long)sizeof(S));
      q[i] = F2(a, c);
    });
  }
  char* o = reinterpret_cast<char*>(fout + cen);
  if constexpr (EARLY) {
    collide<L, COLL, false, Store<S>::SHIFTED, F2>(q, P, nullptr, nullptr, [&](auto I, F2 v) {
      constexpr int i = LBM_CI(I);
      if (two)
        st_pair<S>(reinterpret_cast<S*>(o + off.template dst<i>()), v);
      else
        Store<S>::st(reinterpret_cast<S*>(o + off.template dst<i>()), v.v.x);
    });
  } else {
    collide<L, COLL, false, Store<S>::SHIFTED>(q, P);
    if (two) {
      sfor<0, L::Q>([&](auto I) {
        constexpr int i = LBM_CI(I);
        st_pair<S>(reinterpret_cast<S*>(o + off.template dst<i>()), q[i]);
      });
    } else {
      sfor<0, L::Q>([&](auto I) {
        constexpr int i = LBM_CI(I);
        Store<S>::st(reinterpret_cast<S*>(o + off.template dst<i>()), q[i].v.x);
      });
    }
  }
}

template <class L, int COLL, class S>
__global__ void __launch_bounds__(STEP_BX, Step2Blocks<L, S>::MIN)
    k_step2(const S* __restrict__ fin, S* __restrict__ fout, StepGeom g, int nbx, CollParams<F2> P,
            const __grid_constant__ PullOffsets<L::Q> off) {
  const int y = blockIdx.x / nbx;
  const int bx = blockIdx.x - y * nbx;
  const int x = 2 * (bx * STEP_BX + threadIdx.x);
  if (x >= g.nx) return;
  const int xw = 2 * (bx * STEP_BX + (threadIdx.x & ~31));  // first column of the warp's 64
  step2_cells<L, COLL, S>(fin, fout, g, P, ParamOffsets<L::Q>{off}, x, y, xw);
}


// ---------------------------------------------------------------------------
// Staged pair kernel for x-periodic grids whose rows are whole 16-byte units (the same collision as
// k_step2).  A persistent block walks a contiguous run of row tiles of BXT = 512 cells.  Its producer warp
// copies each population's pulled source row segment (row y - c_y) with one cp.async.bulk into a ring of
// shared-memory stages (full barrier: the copied bytes; empty barrier: one arrival per compute warp); a row
// that fits a tile is copied whole and wrapped by index, longer rows carry PAD cells of margin and their
// edge tiles copy the wrapped columns.  4 compute warps take two cell pairs a thread per tile.  The copies
// run ahead of the compute, so the bytes in flight no longer depend on the warps the registers allow.
// ---------------------------------------------------------------------------
template <class S>
__device__ __forceinline__ float sm_decode(S v);
template <>
__device__ __forceinline__ float sm_decode<float>(float v) { return v; }
template <>
__device__ __forceinline__ float sm_decode<__half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float sm_decode<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float sm_decode<short>(short v) { return (float)v * (1.0f / kFix16); }
__device__ __forceinline__ double sm_decode_d(double v) { return v; }

// Two neighbouring staged cells (p even: one aligned vector read).
template <class S>
__device__ __forceinline__ F2 sm_pair(const S* p);
template <>
__device__ __forceinline__ F2 sm_pair<float>(const float* p) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  return F2(v.x, v.y);
}
template <>
__device__ __forceinline__ F2 sm_pair<__half>(const __half* p) {
  const float2 v = __half22float2(*reinterpret_cast<const __half2*>(p));
  return F2(v.x, v.y);
}
template <>
__device__ __forceinline__ F2 sm_pair<__nv_bfloat16>(const __nv_bfloat16* p) {
  const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
  return F2(v.x, v.y);
}
template <>
__device__ __forceinline__ F2 sm_pair<short>(const short* p) {
  const short2 v = *reinterpret_cast<const short2*>(p);
  return F2((float)v.x * (1.0f / kFix16), (float)v.y * (1.0f / kFix16));
}

template <class L, class S>
struct Stage2 {
  static constexpr int UNIT = 16 / (int)sizeof(S);                           // cells per 16 bytes
  static constexpr int PAD = (L::VMAX + UNIT - 1) / UNIT * UNIT;              // stencil margin, whole units
  static constexpr int BXT = 512;                                             // cells per tile
  static constexpr int W = BXT + 2 * PAD;                                     // cells per staged row
  static constexpr int ROW_BYTES = W * (int)sizeof(S);
  static constexpr int STAGE_BYTES = L::Q * ROW_BYTES;
  static constexpr int STAGES_FIT = 64 * 1024 / STAGE_BYTES;
  static constexpr int STAGES = STAGES_FIT < 2 ? 2 : (STAGES_FIT > 4 ? 4 : STAGES_FIT);
  static constexpr int SMEM = STAGES * STAGE_BYTES + 128;
  static constexpr int CW = 4;                                                // compute warps
  static constexpr int THREADS = 32 * CW + 32;                                // + the producer warp
  static constexpr int PAIRS = BXT / (2 * 32 * CW);                           // cell pairs a thread per tile
  // binary16 and bfloat16 storage of D2Q9 and D2V17 (measured at 4096^2: D2Q9 FP16 121 -> 131, D2V17
  // 80.8 -> 83.5 GLUPS); FP32 stays on k_step2, which already reaches the HBM roofline there (staged: 95
  // -> 78), as does the fixed-point format (staged: D2Q9 119.7 -> 110.4), and D2V37 takes 226-250
  // registers here (one block a SM)
  static constexpr bool ENABLED =
      L::Q <= 20 && (std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value);
  static constexpr int MIN_BLOCKS = L::Q <= 9 ? 5 : 4;
};

// ROWS: how the staged rows hold the x wrap.  ROWS_WHOLE: every row fits one tile (nbt == 1) and the wrap is
// an index inside the staged row.  ROWS_MARGIN: the staged rows carry PAD cells of margin (edge tiles copy
// the wrapped columns), so the staged source of population i for cell x sits at a compile-time offset -c_x
// from the cell's own slot.  ROWS_ANY: decided at run time from nbt, one staged position per x-velocity
// (the form D2V17 runs fastest in: 83.4 GLUPS at 4096^2 with binary16, against 80.9 with the two
// compile-time forms; D2Q9 takes those: 131 -> 139).
enum { ROWS_ANY = 0, ROWS_WHOLE = 1, ROWS_MARGIN = 2 };
template <class L, int COLL, class S, int ROWS>
__global__ void __launch_bounds__(Stage2<L, S>::THREADS, Stage2<L, S>::MIN_BLOCKS)
    k_step2_staged(const S* __restrict__ fin, S* __restrict__ fout, StepGeom g, int nbt, long long ntiles,
                   CollParams<F2> P, const __grid_constant__ PullOffsets<L::Q> off, StageCtl ctl) {
  using St = Stage2<L, S>;
  constexpr int NS = St::STAGES;
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t full[NS], empty[NS];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], St::CW);
    }
    mbar_init_fence();
  }
  __syncthreads();
  const bool whole_rows = ROWS == ROWS_ANY ? nbt == 1 : ROWS == ROWS_WHOLE;
  const long long t_begin = blockIdx.x * ntiles / gridDim.x;
  const int n_mine = (int)((blockIdx.x + 1LL) * ntiles / gridDim.x - t_begin);
  const int y_begin = (int)(t_begin / nbt), bx_begin = (int)(t_begin - (long long)y_begin * nbt);

  if (warp == St::CW) {
    // producer: tile k of this block goes to stage k % NS once the compute warps released its previous use
    int k = 0, bx = bx_begin, y = y_begin;
    bool ok = true;
    for (; k < n_mine; ++k) {
      const int s = k % NS;
      if (k >= NS) ok = mbar_wait(&empty[s], (uint32_t)(((k / NS) + 1) & 1), ctl.wait_ns);
      if (!__all_sync(0xffffffffu, ok)) break;
      // test hook: the last tile's copies are announced but not issued (its stage is never written, and
      // every earlier stage has been consumed, so no copy is in flight when the block ends)
      const bool skip = (int)blockIdx.x == ctl.fault_block && k == n_mine - 1;
      const int x0 = bx * St::BXT;
      const int xa = max(x0 - St::PAD, 0), xb = min(x0 + St::BXT + St::PAD, g.nx);
      const int left = (!whole_rows && x0 - St::PAD < 0) ? St::PAD : 0;
      const int right =
          (!whole_rows && x0 + St::BXT + St::PAD > g.nx) ? min(x0 + St::BXT + St::PAD - g.nx, St::PAD) : 0;
      const uint32_t per_row = (uint32_t)(xb - xa + left + right) * (uint32_t)sizeof(S);
      if (lane == 0) mbar_arrive_expect_tx(&full[s], per_row * (uint32_t)L::Q);
      __syncwarp();
      unsigned char* st = sm + (size_t)s * St::STAGE_BYTES;
      const char* base = reinterpret_cast<const char*>(fin);
      for (int i = lane; i < L::Q && !skip; i += 32) {  // one population per lane
        const int ys = src_coord(y, off.cy[i], g.ny, g.bcy);
        const char* src = base + off.dst[i] + (long long)ys * g.pitch * (long long)sizeof(S);
        unsigned char* dst = st + i * St::ROW_BYTES;
        bulk_g2s(dst + (xa - x0 + St::PAD) * (int)sizeof(S), src + (long long)xa * sizeof(S),
                 (uint32_t)(xb - xa) * (uint32_t)sizeof(S), &full[s]);
        if (left)
          bulk_g2s(dst, src + (long long)(g.nx - St::PAD) * sizeof(S), (uint32_t)St::PAD * (uint32_t)sizeof(S),
                   &full[s]);
        if (right)
          bulk_g2s(dst + (g.nx - x0 + St::PAD) * (int)sizeof(S), src, (uint32_t)right * (uint32_t)sizeof(S),
                   &full[s]);
      }
      if (++bx == nbt) {
        bx = 0;
        ++y;
      }
    }
    if (!ok && lane == 0) {
      // a compute warp stopped releasing stages: flag it, and wait (bounded) for the copies that may still
      // be in flight, the last use of every stage, before the block's shared memory is released
      atomicExch(ctl.status, LBM_ETIMEOUT);
      for (int j = 1; j <= NS; ++j)
        if (k - j >= 0) mbar_wait(&full[(k - j) % NS], (uint32_t)(((k - j) / NS) & 1), ctl.wait_ns);
    }
    return;
  }

  // compute warps
  int bx = bx_begin, y = y_begin;
  for (int k = 0; k < n_mine; ++k) {
    const int s = k % NS;
    if (!__all_sync(0xffffffffu, mbar_wait(&full[s], (uint32_t)((k / NS) & 1), ctl.wait_ns))) {
      if (lane == 0) atomicExch(ctl.status, LBM_ETIMEOUT);
      return;
    }
    const int x0 = bx * St::BXT;
    const S* sp = reinterpret_cast<const S*>(sm + (size_t)s * St::STAGE_BYTES);
    sfor<0, St::PAIRS>([&](auto Pp) {
      constexpr int pr = LBM_CI(Pp);
      const int x = x0 + pr * (64 * St::CW) + 2 * tid;
      const bool active = x < g.nx;
      const bool two = x + 1 < g.nx;
      F2 q[L::Q];
      if (active) {
        // staged positions of the pulled sources x - cx and x + 1 - cx; an even cx moves both cells of the
        // pair together (x is even), so it is one aligned vector read
        const S* row0 = sp + (x - x0 + St::PAD);
        if constexpr (ROWS == ROWS_MARGIN) {
          // margins hold the wrapped columns: population i's source is row0 + i W - c_x (immediates)
          sfor<0, L::Q>([&](auto I) {
            constexpr int i = LBM_CI(I);
            constexpr int o = i * St::W - L::CX[i];
            if constexpr (L::CX[i] % 2 == 0) {
              q[i] = sm_pair<S>(row0 + o);
            } else {
              q[i] = F2(sm_decode<S>(row0[o]), sm_decode<S>(row0[o + 1]));
            }
          });
        } else {
          // one staged position per x-velocity, the wrap by index when the row is staged whole
          int pos0[2 * L::VMAX + 1], pos1[2 * L::VMAX + 1];
          sfor<0, 2 * L::VMAX + 1>([&](auto J) {
            constexpr int j = LBM_CI(J);
            int xs0 = x - (j - L::VMAX), xs1 = x + 1 - (j - L::VMAX);
            if (whole_rows) {
              xs0 += (xs0 < 0 ? g.nx : 0) - (xs0 >= g.nx ? g.nx : 0);
              xs1 += (xs1 < 0 ? g.nx : 0) - (xs1 >= g.nx ? g.nx : 0);
            }
            pos0[j] = xs0 - x0 + St::PAD;
            pos1[j] = xs1 - x0 + St::PAD;
          });
          sfor<0, L::Q>([&](auto I) {
            constexpr int i = LBM_CI(I);
            constexpr int j = L::CX[i] + L::VMAX;
            const S* row = sp + i * St::W;
            if constexpr (L::CX[i] % 2 == 0) {
              q[i] = sm_pair<S>(row + pos0[j]);
            } else {
              q[i] = F2(sm_decode<S>(row[pos0[j]]), sm_decode<S>(row[pos1[j]]));
            }
          });
        }
      }
      if constexpr (pr == St::PAIRS - 1) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);  // this warp has read the stage: the producer may refill it
      }
      if (active) {
        collide<L, COLL, false, Store<S>::SHIFTED>(q, P);
        char* o = reinterpret_cast<char*>(fout + ((long long)y * g.pitch + x));
        if (two) {
          sfor<0, L::Q>([&](auto I) {
            constexpr int i = LBM_CI(I);
            st_pair<S>(reinterpret_cast<S*>(o + off.dst[i]), q[i]);
          });
        } else {
          sfor<0, L::Q>([&](auto I) {
            constexpr int i = LBM_CI(I);
            Store<S>::st(reinterpret_cast<S*>(o + off.dst[i]), q[i].v.x);
          });
        }
      }
    });
    if (++bx == nbt) {
      bx = 0;
      ++y;
    }
  }
}

// Blocks of the staged pair kernel resident per SM, times the SM count (per device, taken once).
template <class L, int COLL, class S, int ROWS>
inline int staged2_grid(int* out) {
  static int dev_cached = -1, grid_cached = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if (dev != dev_cached) {
    auto k = k_step2_staged<L, COLL, S, ROWS>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Stage2<L, S>::SMEM);
    if (e != cudaSuccess) return (int)e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, Stage2<L, S>::THREADS, Stage2<L, S>::SMEM);
    if (e != cudaSuccess) return (int)e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
    grid_cached = per_sm * sms;
    dev_cached = dev;
  }
  *out = grid_cached;
  return 0;
}

template <class L, int COLL, class S>
inline cudaError_t launch_step2_t(const void* fin, void* fout, const StepGeom& g, const CollParamsD& pd,
                                  cudaStream_t st, const StageCtl* ctl = nullptr) {
  PullOffsets<L::Q> off;
  for (int i = 0; i < L::Q; ++i) {
    off.dst[i] = (long long)i * g.plane * (long long)sizeof(S);
    off.src[i] = off.dst[i] - ((long long)L::CY[i] * g.pitch + L::CX[i]) * (long long)sizeof(S);
    off.cy[i] = L::CY[i];
  }
  using St = Stage2<L, S>;
  if constexpr (St::ENABLED) {
    if (LBM_STEP_STAGED && ctl != nullptr && g.bcx == BC_PERIODIC && g.nx % St::UNIT == 0 && g.nx >= St::PAD) {
    const int nbt = (g.nx + St::BXT - 1) / St::BXT;
    const long long ntiles = (long long)nbt * g.ny;
    int grid = 0;
    if constexpr (L::Q <= 9) {
      const int e = nbt == 1 ? staged2_grid<L, COLL, S, ROWS_WHOLE>(&grid) : staged2_grid<L, COLL, S, ROWS_MARGIN>(&grid);
      if (e) return (cudaError_t)e;
      const long long nb = ntiles < grid ? ntiles : grid;
      if (nbt == 1)
        k_step2_staged<L, COLL, S, ROWS_WHOLE><<<(unsigned)nb, St::THREADS, St::SMEM, st>>>(
            (const S*)fin, (S*)fout, g, nbt, ntiles, coll_params_2d<L, F2, S>(pd, COLL), off, *ctl);
      else
        k_step2_staged<L, COLL, S, ROWS_MARGIN><<<(unsigned)nb, St::THREADS, St::SMEM, st>>>(
            (const S*)fin, (S*)fout, g, nbt, ntiles, coll_params_2d<L, F2, S>(pd, COLL), off, *ctl);
    } else {
      const int e = staged2_grid<L, COLL, S, ROWS_ANY>(&grid);
      if (e) return (cudaError_t)e;
      const long long nb = ntiles < grid ? ntiles : grid;
      k_step2_staged<L, COLL, S, ROWS_ANY><<<(unsigned)nb, St::THREADS, St::SMEM, st>>>(
          (const S*)fin, (S*)fout, g, nbt, ntiles, coll_params_2d<L, F2, S>(pd, COLL), off, *ctl);
    }
    return cudaGetLastError();
    }
  }
  const int nbx = (g.nx + 2 * STEP_BX - 1) / (2 * STEP_BX);
  const long long nblocks = (long long)nbx * g.ny;
  if (nblocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_step2<L, COLL, S><<<(unsigned)nblocks, STEP_BX, 0, st>>>((const S*)fin, (S*)fout, g, nbx,
                                                                 coll_params_2d<L, F2, S>(pd, COLL), off);
  return cudaGetLastError();
}

template <class L, int COLL, bool THERMAL, class Real, class S>
inline cudaError_t launch_step_t(const void* fin, void* fout, const StepGeom& g, const CollParamsD& pd,
                                 cudaStream_t st) {
  PullOffsets<L::Q> off;
  for (int i = 0; i < L::Q; ++i) {
    off.dst[i] = (long long)i * g.plane * (long long)sizeof(S);
    off.src[i] = off.dst[i] - ((long long)L::CY[i] * g.pitch + L::CX[i]) * (long long)sizeof(S);
  }
  const int nbx = (g.nx + STEP_BX - 1) / STEP_BX;
  const long long nblocks = (long long)nbx * g.ny;
  if (nblocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_step<L, COLL, THERMAL, Real, S>
      <<<(unsigned)nblocks, STEP_BX, 0, st>>>((const S*)fin, (S*)fout, g, nbx, coll_params_2d<L, Real, S>(pd, COLL),
                                              off);
  return cudaGetLastError();
}

// Moments pass of the finite-difference variant: rho, ux, uy, theta of every cell after pull streaming,
// into mom[4][ny][nx].
template <class L, bool THERMAL, class Real, class S>
__global__ void __launch_bounds__(128) k_stream_moments(const S* __restrict__ fin, StepGeom g, CollParams<Real> P,
                                                        Real* __restrict__ mom) {
  const long long n = (long long)g.nx * g.ny;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int x = (int)(c % g.nx), y = (int)(c / g.nx);
  Real q[L::Q];
  sfor<0, L::Q>([&](auto I) {
    constexpr int i = LBM_CI(I);
    const int xs = src_coord(x, L::CX[i], g.nx, g.bcx);
    const int ys = src_coord(y, L::CY[i], g.ny, g.bcy);
    q[i] = (Real)Store<S>::ld(fin + (long long)i * g.plane + (long long)ys * g.pitch + xs);
  });
  Real rho, ux, uy, th;
  cell_macro<L, THERMAL, Store<S>::SHIFTED>(q, P, rho, ux, uy, th);
  mom[c] = rho;
  mom[n + c] = ux;
  mom[2 * n + c] = uy;
  mom[3 * n + c] = th;
}

// One RR step with a1 from finite differences: the moments pass, then the step kernel reading them.
template <class L, bool THERMAL, class Real, class S>
inline cudaError_t launch_step_fd_t(const void* fin, void* fout, const StepGeom& g, const CollParamsD& pd,
                                    void* mom, cudaStream_t st) {
  const long long n = (long long)g.nx * g.ny;
  const CollParams<Real> P = coll_params_2d<L, Real, S>(pd, COLL_RR);
  k_stream_moments<L, THERMAL, Real, S><<<(unsigned)((n + 127) / 128), 128, 0, st>>>((const S*)fin, g, P,
                                                                                     (Real*)mom);
  PullOffsets<L::Q> off;
  for (int i = 0; i < L::Q; ++i) {
    off.dst[i] = (long long)i * g.plane * (long long)sizeof(S);
    off.src[i] = off.dst[i] - ((long long)L::CY[i] * g.pitch + L::CX[i]) * (long long)sizeof(S);
  }
  const int nbx = (g.nx + STEP_BX - 1) / STEP_BX;
  const long long nblocks = (long long)nbx * g.ny;
  if (nblocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_step<L, COLL_RR, THERMAL, Real, S, true><<<(unsigned)nblocks, STEP_BX, 0, st>>>(
      (const S*)fin, (S*)fout, g, nbx, P, off, (const Real*)mom);
  return cudaGetLastError();
}

template <class L, bool THERMAL>
inline cudaError_t launch_step_fd(int prec, const void* fin, void* fout, const StepGeom& g, const CollParamsD& pd,
                                  void* mom, cudaStream_t st) {
  switch (prec) {
    case PREC_F64: return launch_step_fd_t<L, THERMAL, double, double>(fin, fout, g, pd, mom, st);
    case PREC_F32: return launch_step_fd_t<L, THERMAL, float, float>(fin, fout, g, pd, mom, st);
    case PREC_F16: return launch_step_fd_t<L, THERMAL, float, __half>(fin, fout, g, pd, mom, st);
    case PREC_BF16: return launch_step_fd_t<L, THERMAL, float, __nv_bfloat16>(fin, fout, g, pd, mom, st);
    case PREC_I16: return launch_step_fd_t<L, THERMAL, float, short>(fin, fout, g, pd, mom, st);
  }
  return cudaErrorInvalidValue;
}

template <class L, int COLL, bool THERMAL>
inline cudaError_t launch_step_prec(int prec, const void* fin, void* fout, const StepGeom& g,
                                    const CollParamsD& pd, cudaStream_t st, const StageCtl* ctl) {
  // Two cells per thread pay off while the pair's registers stay low (D2Q9, D2V17).  D2V37 keeps one
  // cell per thread in FP32 and FP64 (HBM-bound: its 28 resident warps per SM in FP32, 20 in FP64, keep
  // more bytes in flight than the pair kernel's 16-20), but with 16-bit storage, which is issue-bound, the
  // packed FP32x2 arithmetic wins from LBM_STEP_PAIRS_LARGE_16_MIN cells up (measured on GB300 at 4096^2:
  // BF16 27.4 -> 36.6 GLUPS, FP16 27.4 -> 35.4, fixed point 26.1 -> 30.7); below that the grid is a few
  // waves and the scalar kernel's shorter blocks are as fast or faster.
  if constexpr (!THERMAL && LBM_STEP_PAIRS_LARGE_16 && L::Q > 20) {
    if ((long long)g.nx * g.ny >= LBM_STEP_PAIRS_LARGE_16_MIN) switch (prec) {
      case PREC_F16: return launch_step2_t<L, COLL, __half>(fin, fout, g, pd, st, ctl);
      case PREC_BF16: return launch_step2_t<L, COLL, __nv_bfloat16>(fin, fout, g, pd, st, ctl);
      case PREC_I16: return launch_step2_t<L, COLL, short>(fin, fout, g, pd, st, ctl);
      default: break;
    }
  }
  if constexpr (!THERMAL && LBM_STEP_PAIRS && L::Q <= 20) {
    switch (prec) {
      case PREC_F64: return launch_step_t<L, COLL, THERMAL, double, double>(fin, fout, g, pd, st);
      case PREC_F32: return launch_step2_t<L, COLL, float>(fin, fout, g, pd, st, ctl);
      case PREC_F16: return launch_step2_t<L, COLL, __half>(fin, fout, g, pd, st, ctl);
      case PREC_BF16: return launch_step2_t<L, COLL, __nv_bfloat16>(fin, fout, g, pd, st, ctl);
      case PREC_I16: return launch_step2_t<L, COLL, short>(fin, fout, g, pd, st, ctl);
    }
  } else {
    switch (prec) {
      case PREC_F64: return launch_step_t<L, COLL, THERMAL, double, double>(fin, fout, g, pd, st);
      case PREC_F32: return launch_step_t<L, COLL, THERMAL, float, float>(fin, fout, g, pd, st);
      case PREC_F16: return launch_step_t<L, COLL, THERMAL, float, __half>(fin, fout, g, pd, st);
      case PREC_BF16: return launch_step_t<L, COLL, THERMAL, float, __nv_bfloat16>(fin, fout, g, pd, st);
      case PREC_I16: return launch_step_t<L, COLL, THERMAL, float, short>(fin, fout, g, pd, st);
    }
  }
  return cudaErrorInvalidValue;
}

// fd_mom: moments buffer of the finite-difference variant (RR only), nullptr = a1 by projection.
template <class L, bool THERMAL>
inline cudaError_t launch_step_lattice(int coll, int prec, const void* fin, void* fout, const StepGeom& g,
                                       const CollParamsD& pd, void* fd_mom, cudaStream_t st, const StageCtl* ctl) {
  if (fd_mom) return coll == COLL_RR ? launch_step_fd<L, THERMAL>(prec, fin, fout, g, pd, fd_mom, st)
                                     : cudaErrorInvalidValue;
  switch (coll) {
    case COLL_BGK: return launch_step_prec<L, COLL_BGK, THERMAL>(prec, fin, fout, g, pd, st, ctl);
    case COLL_PR: return launch_step_prec<L, COLL_PR, THERMAL>(prec, fin, fout, g, pd, st, ctl);
    case COLL_RR: return launch_step_prec<L, COLL_RR, THERMAL>(prec, fin, fout, g, pd, st, ctl);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbm

// One translation unit per lattice instantiates its kernels behind these.  `ctl` carries the context's
// device error word and wait limit (nullptr: the staged kernels are not used).
#define LBM_STEP_LAUNCHER_ARGS                                                                      \
  int coll, int prec, const void *fin, void *fout, const lbm::StepGeom &g, const lbm::CollParamsD &pd, \
      void *fd_mom, const lbm::StageCtl *ctl, cudaStream_t st
cudaError_t lbm_launch_step_d2q9(LBM_STEP_LAUNCHER_ARGS);
cudaError_t lbm_launch_step_d2v17(LBM_STEP_LAUNCHER_ARGS);
cudaError_t lbm_launch_step_d2v37(LBM_STEP_LAUNCHER_ARGS);
cudaError_t lbm_launch_step_d2v37_thermal(LBM_STEP_LAUNCHER_ARGS);
