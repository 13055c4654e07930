// Stream-and-collide with the pulled populations staged in shared memory by
// the Tensor Memory Accelerator.
//
// Persistent CTAs walk a static list of tiles (BY rows x BX columns).  One
// producer warp issues, for every population i of an interior tile, one
// 3-D TMA box load of plane i, rows y0 - cy_i .. y0 - cy_i + BY - 1, columns
// x0 - HX .. x0 + BX + HX - 1 (HX >= the largest |cx|, rounded so the box
// starts on a 16-byte boundary) into a stage of a ring of shared-memory
// buffers, completing on the stage's "full" mbarrier.  Consumer warps (one
// per tile row) wait on it, read each population at its streamed offset
// (column + HX - cx_i) from shared memory, release the stage on its "empty"
// mbarrier, collide and store.  The loads of the next stages stay in flight
// while the consumers compute, independently of the consumers' registers.
// Tiles whose boxes would cross the domain edge (periodic wrap, clamping,
// ragged tiles) are pulled directly from global memory by the consumers.
//
// Every mbarrier wait is bounded; a wait that runs out records LBM_ETIMEOUT
// in the context's error word and the CTA drains its copies and returns.
#pragma once
#include <cuda.h>

#include "step.cuh"

namespace lbm {

constexpr int kTimeoutCode = 5;          // written to the error word (host maps it to LBM_ETIMEOUT)
constexpr long kWaitLimit = 1L << 22;    // bounded mbarrier polling

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  for (long it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

// Tile geometry of one kernel instantiation.
template <class L, class S, bool PAIR>
struct TmaCfg {
  static constexpr int CPT = PAIR ? 2 : 1;                  // cells per consumer thread
  static constexpr int BX = 32 * CPT;                       // tile columns: one warp per row
#ifndef LBM_TMA_BY
#define LBM_TMA_BY 8
#endif
#ifndef LBM_TMA_STAGES_LARGE
#define LBM_TMA_STAGES_LARGE 2
#endif
#ifndef LBM_TMA_STAGES_SMALL
#define LBM_TMA_STAGES_SMALL 3
#endif
  static constexpr int BY = LBM_TMA_BY;                     // tile rows = consumer warps
  static constexpr int ALIGN = 16 / (int)sizeof(S) > 0 ? 16 / (int)sizeof(S) : 1;
  static constexpr int HX = ((L::VMAX + ALIGN - 1) / ALIGN) * ALIGN;  // halo columns, 16-byte multiple
  static constexpr int BOXW = BX + 2 * HX;                  // box columns
  static constexpr int BOX_BYTES = BY * BOXW * (int)sizeof(S);
  static constexpr int SLOT = (BOX_BYTES + 127) / 128 * 128;  // bytes of one population in a stage
  static constexpr int STAGE = L::Q * SLOT;
  static constexpr int STAGES = L::Q > 9 ? LBM_TMA_STAGES_LARGE : LBM_TMA_STAGES_SMALL;
  static constexpr int THREADS = 32 * (BY + 1);             // consumers + one producer warp
  static constexpr int SMEM = STAGES * STAGE + 2 * STAGES * 8;
  static constexpr int MINB = L::Q > 20 ? (BY > 8 ? 1 : 2) : 1;
};

// A tile is served by TMA when its boxes stay inside the domain (no wrap, no clamp, no ragged edge).
__device__ __forceinline__ bool tma_tile(int x0, int y0, int bx, int by, int hx, int vmax, const StepGeom& g) {
  return x0 - hx >= 0 && x0 + bx + hx <= g.nx && y0 - vmax >= 0 && y0 + by + vmax <= g.ny;
}

template <class S>
__device__ __forceinline__ float lds_val(const S* p) {
  return (float)*p;
}
template <>
__device__ __forceinline__ float lds_val<__half>(const __half* p) {
  return __half2float(*p);
}
template <>
__device__ __forceinline__ float lds_val<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}
template <>
__device__ __forceinline__ float lds_val<short>(const short* p) {
  return (float)*p * (1.0f / kFix16);
}
template <class S>
__device__ __forceinline__ F2 lds_pair(const S* p);  // 2 consecutive, aligned to 2 elements
template <>
__device__ __forceinline__ F2 lds_pair<float>(const float* p) {
  return F2(*reinterpret_cast<const float2*>(p));
}
template <>
__device__ __forceinline__ F2 lds_pair<__half>(const __half* p) {
  return F2(__half22float2(*reinterpret_cast<const __half2*>(p)));
}
template <>
__device__ __forceinline__ F2 lds_pair<__nv_bfloat16>(const __nv_bfloat16* p) {
  return F2(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p)));
}
template <>
__device__ __forceinline__ F2 lds_pair<short>(const short* p) {
  const unsigned u = *reinterpret_cast<const unsigned*>(p);
  return F2((float)(short)(u & 0xffffu), (float)(short)(u >> 16)) * F2(1.0f / kFix16);
}

template <class L, int COLL, class S, bool PAIR>
__global__ void __launch_bounds__(TmaCfg<L, S, PAIR>::THREADS, TmaCfg<L, S, PAIR>::MINB)
    k_step_tma(const S* __restrict__ fin, S* __restrict__ fout, StepGeom g, int ntx, int ntiles,
               CollParams<typename std::conditional<PAIR, F2, float>::type> P,
               const __grid_constant__ PullOffsets<L::Q> off, const __grid_constant__ CUtensorMap tmap,
               int* __restrict__ err) {
  using C = TmaCfg<L, S, PAIR>;
  using Real = typename std::conditional<PAIR, F2, float>::type;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE);
  uint64_t* empty = full + C::STAGES;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], C::BY);
    }
    mbar_fence_init();
  }
  __syncthreads();

  if (warp == C::BY) {  // ---------------- producer ----------------
    if (lane != 0) return;
    long k = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int ty = t / ntx, tx = t - ty * ntx;
      const int x0 = tx * C::BX, y0 = ty * C::BY;
      if (!tma_tile(x0, y0, C::BX, C::BY, C::HX, L::VMAX, g)) continue;
      const int s = (int)(k % C::STAGES);
      if (!mbar_wait_bounded(&empty[s], (unsigned)(((k / C::STAGES) & 1) ^ 1))) {
        atomicExch(err, kTimeoutCode);
        ok = false;
        break;
      }
      mbar_arrive_expect_tx(&full[s], (unsigned)(L::Q * C::BOX_BYTES));
      unsigned char* dst = smem + s * C::STAGE;
      sfor<0, L::Q>([&](auto I) {
        constexpr int i = LBM_CI(I);
        constexpr int cy = L::CY[i];
        tma_load_3d(dst + i * C::SLOT, &tmap, x0 - C::HX, y0 - cy, i, &full[s]);
      });
      ++k;
    }
    if (!ok) {  // let the copies already issued land before the CTA's shared memory goes away
      for (long j = k - C::STAGES > 0 ? k - C::STAGES : 0; j < k; ++j)
        mbar_wait_bounded(&full[j % C::STAGES], (unsigned)((j / C::STAGES) & 1));
    }
    return;
  }

  // ---------------- consumers: warp = row of the tile ----------------
  long k = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int ty = t / ntx, tx = t - ty * ntx;
    const int x0 = tx * C::BX, y0 = ty * C::BY;
    const int y = y0 + warp;
    const int x = x0 + C::CPT * lane;
    Real q[L::Q];
    if (tma_tile(x0, y0, C::BX, C::BY, C::HX, L::VMAX, g)) {
      const int s = (int)(k % C::STAGES);
      if (!mbar_wait_bounded(&full[s], (unsigned)((k / C::STAGES) & 1))) {
        atomicExch(err, kTimeoutCode);
        return;
      }
      const S* base = reinterpret_cast<const S*>(smem + s * C::STAGE) + warp * C::BOXW + C::CPT * lane + C::HX;
      sfor<0, L::Q>([&](auto I) {
        constexpr int i = LBM_CI(I);
        constexpr int cx = L::CX[i];
        const S* p = base + (i * (C::SLOT / (int)sizeof(S)) - cx);
        if constexpr (PAIR) {
          if constexpr (cx % 2 == 0)
            q[i] = lds_pair<S>(p);
          else
            q[i] = F2(lds_val<S>(p), lds_val<S>(p + 1));
        } else {
          q[i] = lds_val<S>(p);
        }
      });
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
      ++k;
      collide<L, COLL, false, Store<S>::SHIFTED>(q, P);
      char* o = reinterpret_cast<char*>(fout + (long long)y * g.pitch + x);
      sfor<0, L::Q>([&](auto I) {
        constexpr int i = LBM_CI(I);
        if constexpr (PAIR)
          st_pair<S>(reinterpret_cast<S*>(o + off.dst[i]), q[i]);
        else
          Store<S>::st(reinterpret_cast<S*>(o + off.dst[i]), q[i]);
      });
    } else {
      // edge or ragged tile: pull straight from global memory with the boundary rule
      if (y >= g.ny || x >= g.nx) continue;
      const bool two = PAIR && x + 1 < g.nx;
      const int x1 = two ? x + 1 : x;
      const char* b = reinterpret_cast<const char*>(fin);
      sfor<0, L::Q>([&](auto I) {
        constexpr int i = LBM_CI(I);
        constexpr int cx = L::CX[i], cy = L::CY[i];
        const int ys = src_coord(y, cy, g.ny, g.bcy);
        const long long row = (long long)ys * g.pitch;
        const int xs0 = src_coord(x, cx, g.nx, g.bcx);
        const float a = ld_raw<S>(b + off.dst[i] + (row + xs0) * (long long)sizeof(S));
        if constexpr (PAIR) {
          const int xs1 = src_coord(x1, cx, g.nx, g.bcx);
          const float c = ld_raw<S>(b + off.dst[i] + (row + xs1) * (long long)sizeof(S));
          q[i] = F2(a, c);
        } else {
          q[i] = a;
        }
      });
      collide<L, COLL, false, Store<S>::SHIFTED>(q, P);
      char* o = reinterpret_cast<char*>(fout + (long long)y * g.pitch + x);
      sfor<0, L::Q>([&](auto I) {
        constexpr int i = LBM_CI(I);
        S* d = reinterpret_cast<S*>(o + off.dst[i]);
        if constexpr (PAIR) {
          if (two)
            st_pair<S>(d, q[i]);
          else
            Store<S>::st(d, q[i].v.x);
        } else {
          Store<S>::st(d, q[i]);
        }
      });
    }
  }
}

template <class L, int COLL, class S, bool PAIR>
inline cudaError_t launch_step_tma_t(const void* fin, void* fout, const StepGeom& g, const CollParamsD& pd,
                                     const CUtensorMap* tmap, int* err, cudaStream_t st) {
  using C = TmaCfg<L, S, PAIR>;
  using Real = typename std::conditional<PAIR, F2, float>::type;
  auto kern = k_step_tma<L, COLL, S, PAIR>;
  static int blocks_per_sm = 0;  // per instantiation, first launch
  if (blocks_per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, C::THREADS, C::SMEM);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm < 1) return cudaErrorInvalidConfiguration;
  }
  PullOffsets<L::Q> off;
  for (int i = 0; i < L::Q; ++i) {
    off.dst[i] = (long long)i * g.plane * (long long)sizeof(S);
    off.src[i] = off.dst[i] - ((long long)L::CY[i] * g.pitch + L::CX[i]) * (long long)sizeof(S);
  }
  const int ntx = (g.nx + C::BX - 1) / C::BX, nty = (g.ny + C::BY - 1) / C::BY;
  const long long ntiles = (long long)ntx * nty;
  if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  const long long slots = (long long)blocks_per_sm * g.nsm;
  const unsigned grid = (unsigned)(ntiles < slots ? ntiles : slots);
  kern<<<grid, C::THREADS, C::SMEM, st>>>((const S*)fin, (S*)fout, g, ntx, (int)ntiles, cast_params<Real>(pd), off,
                                          *tmap, err);
  return cudaGetLastError();
}

template <class L, int COLL>
inline cudaError_t launch_step_tma_prec(int prec, const void* fin, void* fout, const StepGeom& g,
                                        const CollParamsD& pd, const CUtensorMap* tmap, int* err, cudaStream_t st) {
  constexpr bool PAIR = L::Q <= 20;  // two cells per thread pay off while registers stay low (D2Q9, D2V17)
  switch (prec) {
    case PREC_F32: return launch_step_tma_t<L, COLL, float, PAIR>(fin, fout, g, pd, tmap, err, st);
    case PREC_F16: return launch_step_tma_t<L, COLL, __half, PAIR>(fin, fout, g, pd, tmap, err, st);
    case PREC_BF16: return launch_step_tma_t<L, COLL, __nv_bfloat16, PAIR>(fin, fout, g, pd, tmap, err, st);
    case PREC_I16: return launch_step_tma_t<L, COLL, short, PAIR>(fin, fout, g, pd, tmap, err, st);
  }
  return cudaErrorInvalidValue;
}

// Isothermal FP32 / 16-bit steps go through the TMA kernel when a tensor map is given, else (and for
// FP64 and thermal runs) through the register-pull kernels of step.cuh.
template <class L, bool THERMAL>
inline cudaError_t launch_step_any(int coll, int prec, const void* fin, void* fout, const StepGeom& g,
                                   const CollParamsD& pd, const void* tmap, int* err, cudaStream_t st) {
  if constexpr (!THERMAL) {
    if (tmap && prec != PREC_F64) {
      const CUtensorMap* m = static_cast<const CUtensorMap*>(tmap);
      switch (coll) {
        case COLL_BGK: return launch_step_tma_prec<L, COLL_BGK>(prec, fin, fout, g, pd, m, err, st);
        case COLL_PR: return launch_step_tma_prec<L, COLL_PR>(prec, fin, fout, g, pd, m, err, st);
        case COLL_RR: return launch_step_tma_prec<L, COLL_RR>(prec, fin, fout, g, pd, m, err, st);
      }
      return cudaErrorInvalidValue;
    }
  }
  return launch_step_lattice<L, THERMAL>(coll, prec, fin, fout, g, pd, st);
}

}  // namespace lbm
