// Learned a1^(2) closure for coarse grids: a per-cell MLP
//   features (27 used of 32) -> 64 -> 64 -> 64 -> 3 (of 8), GELU on the hidden layers,
// predicting the subgrid stress <rho u_a u_b> - rho_bar u_bar_a u_bar_b that box filtering of a
// fine run leaves out of the coarse equilibrium, which the coarse RR step adds to its a1^(2).
//
// Every matrix product runs on the tensor cores, BF16 x BF16 -> FP32.  Inference (lbm_closure_forward and
// the fused closure step) runs on the 5th-generation tensor core: per 128-row tile each layer is a chain of
// tcgen05 MMAs into a TMEM accumulator (tc.cuh), whose rows the block's threads read back, activate, round
// to BF16 and store as the next layer's shared-memory operand.  Training uses warp MMAs
// (mma.sync m16n8k16): it keeps each layer's activations in shared memory and forms the weight gradients
// (activation^T x upstream gradient) and the input gradients (upstream gradient x weights) with
// the same MMA, accumulating per-block partial gradients into FP32 with atomics; Adam updates
// FP32 master weights and refreshes their BF16 copies.
//
// Parameters (flat FP32, the layout of lbm_closure_set_weights): W1[64][32] b1[64] W2[64][64]
// b2[64] W3[64][64] b3[64] W4[8][64] b4[8]; row n of W holds the weights of output n.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstddef>
#include <cstring>
#include <new>

#include "../../include/lbm.h"
#include "ctx.h"
#include "fields.h"
#include "tc.cuh"
#include "vec2.cuh"

namespace {

constexpr int NI = LBM_CLOSURE_IN;    // 32
constexpr int NH = LBM_CLOSURE_HID;   // 64
constexpr int NO = LBM_CLOSURE_OUT;   // 8
constexpr int NUSED_OUT = 3;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NI;
constexpr int OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH * NH;
constexpr int OFF_W4 = OFF_B3 + NH, OFF_B4 = OFF_W4 + NO * NH;
constexpr int NPARAM = OFF_B4 + NO;
static_assert(NPARAM == LBM_CLOSURE_NPARAM, "parameter count");

// ---------------------------------------------------------------------------
// GELU, tanh form (Hendrycks & Gimpel): 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))).  tanh is the
// hardware approximation (tanh.approx.f32, relative error about 2^-11): its error is below the BF16
// rounding every activation gets next, and it keeps the layer chain short.  Training and inference use
// the same function.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float tanh_hw(float u) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
  return t;
}
__device__ __forceinline__ float gelu(float z) {
  const float k = 0.7978845608028654f;
  const float u = k * (z + 0.044715f * z * z * z);
  return 0.5f * z * (1.0f + tanh_hw(u));
}
__device__ __forceinline__ float gelu_grad(float z) {
  const float k = 0.7978845608028654f;
  const float u = k * (z + 0.044715f * z * z * z);
  const float t = tanh_hw(u);
  return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * k * (1.0f + 3.0f * 0.044715f * z * z);
}

// GELU of two values in packed FP32x2 (the same tanh form; per lane the operations of gelu() written out as
// z^2, 1 + c z^2, (k z)(...), then 0.5 z + 0.5 z tanh), for the tensor-core epilogue.
__device__ __forceinline__ float2 gelu2(float2 z) {
  const float2 z2 = __fmul2_rn(z, z);
  const float2 t = __ffma2_rn(make_float2(0.044715f, 0.044715f), z2, make_float2(1.0f, 1.0f));
  const float2 u = __fmul2_rn(__fmul2_rn(make_float2(0.7978845608028654f, 0.7978845608028654f), z), t);
  const float2 th = make_float2(tanh_hw(u.x), tanh_hw(u.y));
  const float2 hz = __fmul2_rn(make_float2(0.5f, 0.5f), z);
  return __ffma2_rn(hz, th, hz);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t pack_raw(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  const uint32_t a = __bfloat16_as_ushort(lo), b = __bfloat16_as_ushort(hi);
  return a | (b << 16);
}

// D = A(16x16, row) x B(16x8, col) + D, BF16 inputs, FP32 accumulate.
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One 16x8 output tile of C = A(M x K) B(K x N) at (m0, n0), A and B read through accessors that
// return BF16 elements (any layout / transpose).  Fragment ownership: lane = 4 g + t.
template <class FA, class FB>
__device__ __forceinline__ void mma_tile(float (&acc)[4], int m0, int n0, int K, FA a, FB b) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t ra[4], rb[2];
    ra[0] = pack_raw(a(m0 + g, k0 + 2 * t), a(m0 + g, k0 + 2 * t + 1));
    ra[1] = pack_raw(a(m0 + g + 8, k0 + 2 * t), a(m0 + g + 8, k0 + 2 * t + 1));
    ra[2] = pack_raw(a(m0 + g, k0 + 2 * t + 8), a(m0 + g, k0 + 2 * t + 9));
    ra[3] = pack_raw(a(m0 + g + 8, k0 + 2 * t + 8), a(m0 + g + 8, k0 + 2 * t + 9));
    rb[0] = pack_raw(b(k0 + 2 * t, n0 + g), b(k0 + 2 * t + 1, n0 + g));
    rb[1] = pack_raw(b(k0 + 2 * t + 8, n0 + g), b(k0 + 2 * t + 9, n0 + g));
    mma16816(acc, ra, rb);
  }
}

// BF16 weights in shared memory, [out][in] rows as in the parameter layout.
struct __align__(16) SmemWeights {
  __nv_bfloat16 w1[NH * NI], w2[NH * NH], w3[NH * NH], w4[NO * NH];
  float b1[NH], b2[NH], b3[NH], b4[NO];
};
static_assert(sizeof(SmemWeights) % 16 == 0, "whole 16-byte vectors");
static_assert((OFF_W1 * 2) % 16 == 0 && (OFF_W2 * 2) % 16 == 0 && (OFF_W3 * 2) % 16 == 0 && (OFF_W4 * 2) % 16 == 0,
              "BF16 weight blocks start on 16-byte boundaries");
static_assert((OFF_B1 * 4) % 16 == 0 && (OFF_B2 * 4) % 16 == 0 && (OFF_B3 * 4) % 16 == 0 && (OFF_B4 * 4) % 16 == 0,
              "FP32 bias blocks start on 16-byte boundaries");

// Source of the j-th 16-byte vector of SmemWeights: the four BF16 weight blocks of the BF16 copy, then
// the four FP32 bias blocks of the master weights (all 16-byte aligned: separate cudaMalloc buffers).
__device__ __forceinline__ const uint4* weight_vec(int j, const __nv_bfloat16* wb, const float* wf) {
  constexpr int E1 = NH * NI * 2 / 16, E2 = E1 + NH * NH * 2 / 16, E3 = E2 + NH * NH * 2 / 16,
                E4 = E3 + NO * NH * 2 / 16, F1 = E4 + NH * 4 / 16, F2 = F1 + NH * 4 / 16, F3 = F2 + NH * 4 / 16;
  const char* b = reinterpret_cast<const char*>(wb);
  const char* f = reinterpret_cast<const char*>(wf);
  if (j < E1) return reinterpret_cast<const uint4*>(b + OFF_W1 * 2) + j;
  if (j < E2) return reinterpret_cast<const uint4*>(b + OFF_W2 * 2) + (j - E1);
  if (j < E3) return reinterpret_cast<const uint4*>(b + OFF_W3 * 2) + (j - E2);
  if (j < E4) return reinterpret_cast<const uint4*>(b + OFF_W4 * 2) + (j - E3);
  if (j < F1) return reinterpret_cast<const uint4*>(f + OFF_B1 * 4) + (j - E4);
  if (j < F2) return reinterpret_cast<const uint4*>(f + OFF_B2 * 4) + (j - F1);
  if (j < F3) return reinterpret_cast<const uint4*>(f + OFF_B3 * 4) + (j - F2);
  return reinterpret_cast<const uint4*>(f + OFF_B4 * 4) + (j - F3);
}

// Copy of the network into shared memory (the caller synchronizes the block afterwards).  Every thread
// issues all its 16-byte loads before its first store, so the copy costs about one L2 round trip
// instead of one per element.
__device__ void load_weights(SmemWeights& s, const __nv_bfloat16* wb, const float* wf) {
  constexpr int N16 = (int)(sizeof(SmemWeights) / 16);
  constexpr int R = (N16 + 127) / 128;
  uint4* dst = reinterpret_cast<uint4*>(&s);
  for (int j0 = 0; j0 < N16; j0 += R * (int)blockDim.x) {
    uint4 r[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int j = j0 + (int)threadIdx.x + k * (int)blockDim.x;
      if (j < N16) r[k] = __ldg(weight_vec(j, wb, wf));
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int j = j0 + (int)threadIdx.x + k * (int)blockDim.x;
      if (j < N16) dst[j] = r[k];
    }
  }
}

// ---------------------------------------------------------------------------
// Inference on the 5th-generation tensor core.  A block runs two independent groups of 128 threads (TC_G), each
// taking 128 rows at a time with its own operand buffer, TMEM accumulator and mbarrier, so that one group's
// MMAs run while the other applies its activations; the weights in shared memory serve both.  Each layer is a
// chain of tcgen05 MMAs (M = 128 rows, N = 64 outputs, or 16 for the output layer, K = 16 a step) issued by one
// thread of the group into its TMEM accumulator, completing on its mbarrier.  Each thread then loads its row
// of the accumulator from TMEM, adds the bias, applies GELU, rounds to BF16 and writes the row into the
// group's shared operand of the next layer.  Operands are in the canonical no-swizzle K-major layout: core
// matrix (row group g, K chunk c) of 8 rows x 8 BF16 at element ((g * KCH + c) * 64), KCH = K / 8.
// ---------------------------------------------------------------------------
constexpr int TC_M = 128;  // rows of a group's tile, threads of a group
constexpr int TC_G = 2;    // groups a block
constexpr int TC_NO = 16;  // output layer padded to the smallest N of an M = 128 MMA
constexpr int TC_COLS = 128;  // TMEM columns a block: 64 a group

struct __align__(128) SmemTc {
  __nv_bfloat16 w1[NH * NI];        // 4 KB
  __nv_bfloat16 w2[NH * NH];        // 8 KB
  __nv_bfloat16 w3[NH * NH];        // 8 KB
  __nv_bfloat16 w4[TC_NO * NH];     // 2 KB, rows NO..15 zero
  __nv_bfloat16 a[TC_G][TC_M * NH]; // 16 KB a group: the current layer's input rows
  float b1[NH], b2[NH], b3[NH], b4[NO];
  uint64_t bar[TC_G];
  uint32_t tmem;
};
static_assert(offsetof(SmemTc, a) % 128 == 0 && offsetof(SmemTc, w4) % 128 == 0, "128-byte core matrices");

// Element offset of (row r, column k) in the canonical layout of a matrix with K columns.
__device__ __forceinline__ int canon(int r, int k, int K) {
  return ((r >> 3) * (K >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

// Barrier of one group (named barrier 1 + g, its 128 threads), and the same with a logical AND of `pred`.
// (Immediate barrier numbers: a register operand makes the compiler reserve all sixteen.)
__device__ __forceinline__ void group_sync(int g) {
  static_assert(TC_G == 2 && TC_M == 128, "barriers 1 and 2 of 128 threads");
  if (g == 0)
    asm volatile("bar.sync 1, 128;" ::: "memory");
  else
    asm volatile("bar.sync 2, 128;" ::: "memory");
}
__device__ __forceinline__ bool group_sync_and(int g, bool pred) {
  uint32_t out;
  if (g == 0)
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, 128, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(out)
        : "r"((uint32_t)pred)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 2, 128, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(out)
        : "r"((uint32_t)pred)
        : "memory");
  return out != 0;
}

// Bias, GELU and BF16 rounding of this thread's accumulator row (64 TMEM columns from trow), written as row m
// of the group's next-layer input a.
__device__ __forceinline__ void tc_hidden_epilogue(__nv_bfloat16* a, uint32_t trow, const float* bias, int m) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t r[16];
    lbm::tc::ld_32x32b_x16(trow + 16 * q, r);
    lbm::tc::wait_ld();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint4 v;
      uint32_t* pv = reinterpret_cast<uint32_t*>(&v);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = 16 * q + 8 * h + 2 * e;
        const float2 z = __fadd2_rn(make_float2(__uint_as_float(r[8 * h + 2 * e]), __uint_as_float(r[8 * h + 2 * e + 1])),
                                    *reinterpret_cast<const float2*>(bias + k));
        const float2 a2 = gelu2(z);
        pv[e] = pack_bf16(a2.x, a2.y);
      }
      *reinterpret_cast<uint4*>(a + canon(m, 16 * q + 8 * h, NH)) = v;
    }
  }
}

// Group g issues one layer (K / 16 MMA steps into its 64 TMEM columns) and waits for it; false (for the whole
// group) if the wait ran out.
__device__ __forceinline__ bool tc_layer(SmemTc& s, int g, const __nv_bfloat16* w, int K, int N, uint32_t& phase) {
  lbm::tc::fence_async_smem();
  lbm::tc::fence_before_sync();
  group_sync(g);
  lbm::tc::fence_after_sync();
  if ((threadIdx.x & (TC_M - 1)) == 0) {
    const uint32_t sbo = (uint32_t)(K / 8) * 128u;
    const uint32_t a0 = lbm::smem_addr(s.a[g]), b0 = lbm::smem_addr(w);
    for (int k = 0; k < K / 16; ++k)
      lbm::tc::mma_bf16(s.tmem + 64u * g, lbm::tc::smem_desc(a0 + 256u * k, 128u, sbo),
                        lbm::tc::smem_desc(b0 + 256u * k, 128u, sbo), lbm::tc::idesc_bf16_f32(TC_M, N), k > 0);
    lbm::tc::commit(&s.bar[g]);
  }
  const bool ok = group_sync_and(g, lbm::mbar_wait(&s.bar[g], phase));  // every thread of the group waited
  phase ^= 1u;
  lbm::tc::fence_after_sync();
  return ok;
}

// Block set-up of the tensor-core network: weights and biases into shared memory, the groups' mbarriers and
// TMEM_COLS columns of tensor memory (64 a group; at most four such blocks fit a SM's shared memory, 512
// columns).
__device__ void tc_setup(SmemTc& s, const __nv_bfloat16* wb, const float* wf) {
  const int t = threadIdx.x;
  // the four weight matrices as 16-byte vectors (W1 256, W2 and W3 512 each, W4 128 with its padding rows),
  // every load of a thread issued before its first store: one L2 round trip rather than one per vector
  constexpr int V1 = NH * NI / 8, V2 = V1 + NH * NH / 8, V3 = V2 + NH * NH / 8, V4 = V3 + TC_NO * NH / 8;
  constexpr int R = (V4 + TC_G * TC_M - 1) / (TC_G * TC_M);
  uint4 v[R];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int j = t + k * TC_G * TC_M;
    v[k] = make_uint4(0u, 0u, 0u, 0u);
    if (j < V1) v[k] = __ldg(reinterpret_cast<const uint4*>(wb + OFF_W1) + j);
    else if (j < V2) v[k] = __ldg(reinterpret_cast<const uint4*>(wb + OFF_W2) + (j - V1));
    else if (j < V3) v[k] = __ldg(reinterpret_cast<const uint4*>(wb + OFF_W3) + (j - V2));
    else if (j < V3 + NO * NH / 8) v[k] = __ldg(reinterpret_cast<const uint4*>(wb + OFF_W4) + (j - V3));
  }
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int j = t + k * TC_G * TC_M;
    if (j < V1) *reinterpret_cast<uint4*>(s.w1 + canon(j / (NI / 8), 8 * (j % (NI / 8)), NI)) = v[k];
    else if (j < V2) *reinterpret_cast<uint4*>(s.w2 + canon((j - V1) / 8, 8 * ((j - V1) % 8), NH)) = v[k];
    else if (j < V3) *reinterpret_cast<uint4*>(s.w3 + canon((j - V2) / 8, 8 * ((j - V2) % 8), NH)) = v[k];
    else if (j < V4) *reinterpret_cast<uint4*>(s.w4 + canon((j - V3) / 8, 8 * ((j - V3) % 8), NH)) = v[k];
  }
  for (int k = t; k < NH; k += blockDim.x) {
    s.b1[k] = wf[OFF_B1 + k];
    s.b2[k] = wf[OFF_B2 + k];
    s.b3[k] = wf[OFF_B3 + k];
  }
  if (t < NO) s.b4[t] = wf[OFF_B4 + t];
  if (t == 0) {
    for (int g = 0; g < TC_G; ++g) lbm::mbar_init(&s.bar[g], 1);
    lbm::mbar_init_fence();
  }
  if ((t >> 5) == 0) {
    lbm::tc::tmem_alloc(&s.tmem, TC_COLS);
    // no further allocation by this block: give up the permit at once (held, it kept the SM from taking the
    // other blocks it has room for: ncu measured one resident block a SM, 8 warps, against 32 possible)
    lbm::tc::tmem_relinquish();
  }
  lbm::tc::fence_before_sync();
  __syncthreads();
  lbm::tc::fence_after_sync();
}

// Whole block, after both groups' last use of tensor memory.
__device__ void tc_teardown(SmemTc& s) {
  lbm::tc::fence_before_sync();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    lbm::tc::fence_after_sync();
    lbm::tc::tmem_dealloc(s.tmem, TC_COLS);
  }
}

// Group g's four layers on the 128 rows it wrote into s.a[g] (layer-1 input, row m = this thread's); o
// receives this thread's NO outputs.  Returns false (for the whole group) if a wait on the tensor core ran
// out, o then NaN.
__device__ bool tc_network(SmemTc& s, int g, int m, uint32_t& phase, float (&o)[NO]) {
  // this warp's 32 TMEM lanes (warp w of the group reads lanes 32 w .. 32 w + 31) of the group's columns
  const uint32_t trow = s.tmem + 64u * g + ((uint32_t)(32 * (m >> 5)) << 16);
  bool ok = tc_layer(s, g, s.w1, NI, NH, phase);
  if (ok) tc_hidden_epilogue(s.a[g], trow, s.b1, m);
  ok = ok && tc_layer(s, g, s.w2, NH, NH, phase);
  if (ok) tc_hidden_epilogue(s.a[g], trow, s.b2, m);
  ok = ok && tc_layer(s, g, s.w3, NH, NH, phase);
  if (ok) tc_hidden_epilogue(s.a[g], trow, s.b3, m);
  ok = ok && tc_layer(s, g, s.w4, NH, TC_NO, phase);
  if (ok) {
    uint32_t r[16];
    lbm::tc::ld_32x32b_x16(trow, r);
    lbm::tc::wait_ld();
#pragma unroll
    for (int j = 0; j < NO; ++j) o[j] = __uint_as_float(r[j]) + s.b4[j];
  } else {
#pragma unroll
    for (int j = 0; j < NO; ++j) o[j] = __int_as_float(0x7fc00000);
  }
  return ok;
}

__global__ void __launch_bounds__(TC_G * TC_M, 4) k_mlp_forward_tc(const __nv_bfloat16* __restrict__ x, int n,
                                                                   const __nv_bfloat16* __restrict__ wb,
                                                                   const float* __restrict__ wf,
                                                                   float* __restrict__ y) {
  extern __shared__ __align__(128) unsigned char tc_smem[];
  SmemTc& s = *reinterpret_cast<SmemTc*>(tc_smem);
  const int g = threadIdx.x / TC_M, m = threadIdx.x % TC_M;
  tc_setup(s, wb, wf);
  uint32_t phase = 0;
  bool ok = true;
  for (long long r0 = ((long long)blockIdx.x * TC_G + g) * TC_M; r0 < n && ok;
       r0 += (long long)gridDim.x * TC_G * TC_M) {
    const long long row = r0 + m;
    // layer-1 input: this thread's row of x (32 BF16 = four 16-byte vectors)
#pragma unroll
    for (int c = 0; c < NI / 8; ++c) {
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (row < n) v = __ldg(reinterpret_cast<const uint4*>(x + row * NI + 8 * c));
      *reinterpret_cast<uint4*>(s.a[g] + canon(m, 8 * c, NI)) = v;
    }
    float o[NO];
    ok = tc_network(s, g, m, phase, o);
    if (row < n) {
      float4* yo = reinterpret_cast<float4*>(y + row * NO);
      yo[0] = make_float4(o[0], o[1], o[2], o[3]);
      yo[1] = make_float4(o[4], o[5], o[6], o[7]);
    }
  }
  tc_teardown(s);
}

// ---------------------------------------------------------------------------
// Training: one block = 64 samples (4 warps x 16 rows).  Loss = mean over samples of
// sum over the 3 used outputs of (y_pred - y)^2.
// ---------------------------------------------------------------------------
constexpr int TB = 64;  // samples per training block

struct SmemTrain {
  SmemWeights w;
  __nv_bfloat16 x[TB * NI];
  __nv_bfloat16 h[3][TB * NH];  // activations after GELU (BF16, the next layer's input)
  float z[3][TB * NH];          // pre-activations (FP32, for GELU')
  __nv_bfloat16 dz[TB * NH];    // upstream gradient of the current layer (BF16 MMA operand)
  __nv_bfloat16 dout[TB * 16];  // output gradient, 8 columns used + 8 zero columns (K padding)
  float loss[4];
};

__global__ void __launch_bounds__(128) k_mlp_train(const __nv_bfloat16* __restrict__ x, const float* __restrict__ yt,
                                                   int n, const __nv_bfloat16* __restrict__ wb,
                                                   const float* __restrict__ wf, float* __restrict__ grad,
                                                   float* __restrict__ loss_sum) {
  extern __shared__ __align__(16) unsigned char smraw[];
  SmemTrain& S = *reinterpret_cast<SmemTrain*>(smraw);
  load_weights(S.w, wb, wf);
  const long long s0 = (long long)blockIdx.x * TB;
  for (int i = threadIdx.x; i < TB * NI; i += blockDim.x) {
    const long long r = s0 + i / NI;
    S.x[i] = r < n ? x[s0 * NI + i] : __float2bfloat16(0.0f);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, warp = threadIdx.x >> 5;
  const int m0 = warp * 16;  // this warp's 16 samples
  const float inv_n = 1.0f / (float)n;

  // ---- forward, keeping z and h of every hidden layer ----
  const __nv_bfloat16* in = S.x;
  int in_dim = NI;
  const __nv_bfloat16* ws[3] = {S.w.w1, S.w.w2, S.w.w3};
  const float* bs[3] = {S.w.b1, S.w.b2, S.w.b3};
  for (int l = 0; l < 3; ++l) {
    for (int j = 0; j < 8; ++j) {
      float acc[4] = {bs[l][j * 8 + 2 * t], bs[l][j * 8 + 2 * t + 1], bs[l][j * 8 + 2 * t], bs[l][j * 8 + 2 * t + 1]};
      const __nv_bfloat16* A = in;
      const __nv_bfloat16* W = ws[l];
      const int K = in_dim;
      mma_tile(acc, m0, j * 8, K, [&](int r, int k) { return A[r * K + k]; }, [&](int k, int c) { return W[c * K + k]; });
      const int c0 = j * 8 + 2 * t;
      S.z[l][(m0 + g) * NH + c0] = acc[0];
      S.z[l][(m0 + g) * NH + c0 + 1] = acc[1];
      S.z[l][(m0 + g + 8) * NH + c0] = acc[2];
      S.z[l][(m0 + g + 8) * NH + c0 + 1] = acc[3];
      S.h[l][(m0 + g) * NH + c0] = __float2bfloat16(gelu(acc[0]));
      S.h[l][(m0 + g) * NH + c0 + 1] = __float2bfloat16(gelu(acc[1]));
      S.h[l][(m0 + g + 8) * NH + c0] = __float2bfloat16(gelu(acc[2]));
      S.h[l][(m0 + g + 8) * NH + c0 + 1] = __float2bfloat16(gelu(acc[3]));
    }
    __syncwarp();
    in = S.h[l];
    in_dim = NH;
  }
  // output layer, loss and its gradient (rows of this warp only)
  {
    float o[4] = {S.w.b4[2 * t], S.w.b4[2 * t + 1], S.w.b4[2 * t], S.w.b4[2 * t + 1]};
    const __nv_bfloat16* A = S.h[2];
    const __nv_bfloat16* W = S.w.w4;
    mma_tile(o, m0, 0, NH, [&](int r, int k) { return A[r * NH + k]; }, [&](int k, int c) { return W[c * NH + k]; });
    float lsum = 0.0f;
    for (int e = 0; e < 4; ++e) {
      const int r = m0 + g + (e >= 2 ? 8 : 0), c = 2 * t + (e & 1);
      const long long sr = s0 + r;
      float d = 0.0f;
      if (sr < n && c < NUSED_OUT) {
        const float diff = o[e] - yt[sr * NO + c];
        lsum += diff * diff;
        d = 2.0f * diff * inv_n;
      }
      S.dout[r * 16 + c] = __float2bfloat16(d);
      S.dout[r * 16 + c + 8] = __float2bfloat16(0.0f);
    }
    for (int o2 = 16; o2 > 0; o2 >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o2);
    if (lane == 0) S.loss[warp] = lsum;
  }
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(loss_sum, (S.loss[0] + S.loss[1] + S.loss[2] + S.loss[3]) * inv_n);

  // ---- backward ----
  // output layer: dW4[c][k] = sum_s dout[s][c] h3[s][k]; db4[c] = sum_s dout[s][c]; (warps split k in 16s)
  {
    float acc[4] = {0, 0, 0, 0};
    const __nv_bfloat16* D = S.dout;
    const __nv_bfloat16* H = S.h[2];
    // C[k][c] with M = hidden (warp's 16), N = 8 outputs, K = samples
    mma_tile(acc, m0, 0, TB, [&](int k, int s) { return H[s * NH + k]; }, [&](int s, int c) { return D[s * 16 + c]; });
    for (int e = 0; e < 4; ++e) {
      const int k = m0 + g + (e >= 2 ? 8 : 0), c = 2 * t + (e & 1);
      atomicAdd(&grad[OFF_W4 + c * NH + k], acc[e]);
    }
    if (warp == 0 && lane < NO) {
      float sb = 0.0f;
      for (int s = 0; s < TB; ++s) sb += __bfloat162float(S.dout[s * 16 + lane]);
      atomicAdd(&grad[OFF_B4 + lane], sb);
    }
  }
  // dh3[s][k] = sum_c dout[s][c] W4[c][k] (K = 16 with the zero padding), dz3 = dh3 * gelu'(z3)
  for (int j = 0; j < 8; ++j) {
    float acc[4] = {0, 0, 0, 0};
    const __nv_bfloat16* D = S.dout;
    const __nv_bfloat16* W = S.w.w4;
    mma_tile(acc, m0, j * 8, 16, [&](int s, int c) { return D[s * 16 + c]; },
             [&](int c, int k) { return c < NO ? W[c * NH + k] : __float2bfloat16(0.0f); });
    for (int e = 0; e < 4; ++e) {
      const int r = m0 + g + (e >= 2 ? 8 : 0), k = j * 8 + 2 * t + (e & 1);
      S.dz[r * NH + k] = __float2bfloat16(acc[e] * gelu_grad(S.z[2][r * NH + k]));
    }
  }
  __syncthreads();
  // hidden layers l = 2, 1, 0: grads of W_{l+1}, b_{l+1} from dz and the layer input; then dz of layer l-1
  const int offw[3] = {OFF_W1, OFF_W2, OFF_W3}, offb[3] = {OFF_B1, OFF_B2, OFF_B3};
  for (int l = 2; l >= 0; --l) {
    const __nv_bfloat16* X = l == 0 ? S.x : S.h[l - 1];
    const int K = l == 0 ? NI : NH;
    const __nv_bfloat16* DZ = S.dz;
    // dW[c][k] = sum_s dz[s][c] x[s][k]: C (M = 64 outputs c, N = K inputs), warps split M
    for (int j = 0; j < K / 8; ++j) {
      float acc[4] = {0, 0, 0, 0};
      mma_tile(acc, m0, j * 8, TB, [&](int c, int s) { return DZ[s * NH + c]; }, [&](int s, int k) { return X[s * K + k]; });
      for (int e = 0; e < 4; ++e) {
        const int c = m0 + g + (e >= 2 ? 8 : 0), k = j * 8 + 2 * t + (e & 1);
        atomicAdd(&grad[offw[l] + c * K + k], acc[e]);
      }
    }
    if (threadIdx.x < NH) {
      float sb = 0.0f;
      for (int s = 0; s < TB; ++s) sb += __bfloat162float(S.dz[s * NH + threadIdx.x]);
      atomicAdd(&grad[offb[l] + threadIdx.x], sb);
    }
    if (l == 0) break;
    // dh[s][k] = sum_c dz[s][c] W[c][k], dz_prev = dh * gelu'(z_{l-1}); computed into registers first
    float nd[8][4];
    const __nv_bfloat16* W = ws[l];
    for (int j = 0; j < 8; ++j) {
      nd[j][0] = nd[j][1] = nd[j][2] = nd[j][3] = 0.0f;
      mma_tile(nd[j], m0, j * 8, NH, [&](int s, int c) { return DZ[s * NH + c]; }, [&](int c, int k) { return W[c * NH + k]; });
    }
    __syncthreads();  // every warp has read dz (and, above, used it for dW) before it is overwritten
    for (int j = 0; j < 8; ++j)
      for (int e = 0; e < 4; ++e) {
        const int r = m0 + g + (e >= 2 ? 8 : 0), k = j * 8 + 2 * t + (e & 1);
        S.dz[r * NH + k] = __float2bfloat16(nd[j][e] * gelu_grad(S.z[l - 1][r * NH + k]));
      }
    __syncthreads();
  }
}

// Adam on the FP32 master weights, refresh of the BF16 copy, gradient reset.
__global__ void k_adam(float* __restrict__ w, __nv_bfloat16* __restrict__ wb, float* __restrict__ grad,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  const float gr = grad[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gr;
  const float vi = b2 * v[i] + (1.0f - b2) * gr * gr;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  w[i] = wi;
  wb[i] = __float2bfloat16(wi);
  grad[i] = 0.0f;
}

__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) wb[i] = __float2bfloat16(w[i]);
}

}  // namespace

// ---------------------------------------------------------------------------
// Features and filtered targets
// ---------------------------------------------------------------------------
namespace {

// Features of cell (x, y): (rho - 1, ux, uy) / u0 of the 3x3 stencil around it (periodic), row by row,
// then zeros up to LBM_CLOSURE_IN.
__global__ void k_features(const double* __restrict__ rho, const double* __restrict__ ux,
                           const double* __restrict__ uy, int nx, int ny, double inv_u0,
                           __nv_bfloat16* __restrict__ feat) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= (long long)nx * ny) return;
  const int x = (int)(c % nx), y = (int)(c / nx);
  __nv_bfloat16* f = feat + c * NI;
  int k = 0;
  for (int dy = -1; dy <= 1; ++dy)
    for (int dx = -1; dx <= 1; ++dx) {
      const int xs = (x + dx + nx) % nx, ys = (y + dy + ny) % ny;
      const long long s = (long long)ys * nx + xs;
      f[k++] = __float2bfloat16((float)((rho[s] - 1.0) * inv_u0));
      f[k++] = __float2bfloat16((float)(ux[s] * inv_u0));
      f[k++] = __float2bfloat16((float)(uy[s] * inv_u0));
    }
  for (; k < NI; ++k) f[k] = __float2bfloat16(0.0f);
}

// Box filter of a fine field set to the coarse grid (factor r): rho_bar, u_bar = <rho u> / rho_bar and
// the subgrid stress tau_ab = <rho u_a u_b> - rho_bar u_bar_a u_bar_b, scaled by 1/u0^2 into y.
__global__ void k_coarsen(const double* __restrict__ rho, const double* __restrict__ ux,
                          const double* __restrict__ uy, int nx, int ny, int r, double inv_u0,
                          double* __restrict__ rb, double* __restrict__ uxb, double* __restrict__ uyb,
                          float* __restrict__ y) {
  const int cx = nx / r, cy = ny / r;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= (long long)cx * cy) return;
  const int X = (int)(c % cx), Y = (int)(c / cx);
  double m = 0, jx = 0, jy = 0, pxx = 0, pxy = 0, pyy = 0;
  for (int j = 0; j < r; ++j)
    for (int i = 0; i < r; ++i) {
      const long long s = (long long)(Y * r + j) * nx + X * r + i;
      const double d = rho[s], u = ux[s], v = uy[s];
      m += d;
      jx += d * u;
      jy += d * v;
      pxx += d * u * u;
      pxy += d * u * v;
      pyy += d * v * v;
    }
  const double inv = 1.0 / (double)(r * r);
  m *= inv;
  jx *= inv;
  jy *= inv;
  pxx *= inv;
  pxy *= inv;
  pyy *= inv;
  const double u = jx / m, v = jy / m;
  rb[c] = m;
  uxb[c] = u;
  uyb[c] = v;
  const double s2 = inv_u0 * inv_u0;
  y[c * NO + 0] = (float)((pxx - m * u * u) * s2);
  y[c * NO + 1] = (float)((pxy - m * u * v) * s2);
  y[c * NO + 2] = (float)((pyy - m * v * v) * s2);
  for (int k = 3; k < NO; ++k) y[c * NO + k] = 0.0f;
}

}  // namespace

// D2Q9 RR step (FP32) with the closure's a1^(2) correction da = scale * y[cell][0..2].
__global__ void __launch_bounds__(128) k_step_closure(const float* __restrict__ fin, float* __restrict__ fout,
                                                      lbm::StepGeom g, lbm::CollParams<float> P,
                                                      const float* __restrict__ y, float scale) {
  using L = lbm::D2Q9;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= (long long)g.nx * g.ny) return;
  const int x = (int)(c % g.nx), yy = (int)(c / g.nx);
  float q[L::Q];
  lbm::sfor<0, L::Q>([&](auto I) {
    constexpr int i = LBM_CI(I);
    constexpr int cx = L::CX[i], cy = L::CY[i];
    const int xs = lbm::src_coord(x, cx, g.nx, g.bcx);
    const int ys = lbm::src_coord(yy, cy, g.ny, g.bcy);
    q[i] = fin[(long long)i * g.plane + (long long)ys * g.pitch + xs];
  });
  const float da[3] = {scale * y[c * NO + 0], scale * y[c * NO + 1], scale * y[c * NO + 2]};
  lbm::collide<L, lbm::COLL_RR, false, false, float, true>(q, P, da);
  lbm::sfor<0, L::Q>([&](auto I) {
    constexpr int i = LBM_CI(I);
    fout[(long long)i * g.plane + (long long)yy * g.pitch + x] = q[i];
  });
}

// ---------------------------------------------------------------------------
// Fused closure step: features, MLP and the corrected collision of a 32 x 4 tile of cells per block
// iteration of each of the block's two groups; thread 32 w + l of a group takes the cell in column l of row w
// of its tile, which is also its row of the network's 128-row tile.  The moments of the tile and its one-cell halo (periodic, as
// lbm_closure_features) are converted to BF16 features in shared memory once; each thread writes its
// cell's 27 features as its layer-1 input row, the block runs the tensor-core layer chain of
// lbm_closure_forward, and each thread pulls, collides and stores its cell as k_step_closure does with its
// own row of outputs.  Same arithmetic in the same order as features + forward + k_step_closure, so the
// result is bitwise the three-kernel path's.
// ---------------------------------------------------------------------------
constexpr int FT_X = 32, FT_Y = 4;
static_assert(FT_X * FT_Y == TC_M, "one network tile per cell tile");

struct SmemFused {
  SmemTc t;
  __nv_bfloat16 m[TC_G][FT_Y + 2][FT_X + 2][3];  // (rho - 1, ux, uy) / u0 of each group's tile and its halo
};

__global__ void __launch_bounds__(TC_G * TC_M, 3) k_step_closure_fused(const float* __restrict__ fin, float* __restrict__ fout,
                                                            lbm::StepGeom g, lbm::CollParams<float> P,
                                                            const double* __restrict__ rho,
                                                            const double* __restrict__ ux,
                                                            const double* __restrict__ uy, double inv_u0,
                                                            const __nv_bfloat16* __restrict__ wb,
                                                            const float* __restrict__ wf, float scale) {
  using L = lbm::D2Q9;
  extern __shared__ __align__(128) unsigned char tc_smem[];
  SmemFused& s = *reinterpret_cast<SmemFused*>(tc_smem);
  tc_setup(s.t, wb, wf);
  const int grp = threadIdx.x / TC_M, m = threadIdx.x % TC_M, lane = m & 31, warp = m >> 5;
  auto& hm = s.m[grp];
  const int tiles_x = (g.nx + FT_X - 1) / FT_X, tiles_y = (g.ny + FT_Y - 1) / FT_Y;
  uint32_t phase = 0;
  bool ok = true;
  for (long long tile = (long long)blockIdx.x * TC_G + grp; tile < (long long)tiles_x * tiles_y && ok;
       tile += (long long)gridDim.x * TC_G) {
    const int x0 = (int)(tile % tiles_x) * FT_X, y0 = (int)(tile / tiles_x) * FT_Y;
    group_sync(grp);  // previous tile's features are no longer read
    for (int k = m; k < (FT_Y + 2) * (FT_X + 2); k += TC_M) {
      const int hy = k / (FT_X + 2), hx = k - hy * (FT_X + 2);
      int xs = (x0 + hx - 1) % g.nx, ys = (y0 + hy - 1) % g.ny;
      if (xs < 0) xs += g.nx;
      if (ys < 0) ys += g.ny;
      const long long c = (long long)ys * g.nx + xs;
      hm[hy][hx][0] = __float2bfloat16((float)((rho[c] - 1.0) * inv_u0));
      hm[hy][hx][1] = __float2bfloat16((float)(ux[c] * inv_u0));
      hm[hy][hx][2] = __float2bfloat16((float)(uy[c] * inv_u0));
    }
    group_sync(grp);
    // feature k of this thread's cell: neighbour k / 3 (row-major over the 3 x 3 stencil), component k % 3;
    // zero beyond the 27 used inputs
#pragma unroll
    for (int c = 0; c < NI / 8; ++c) {
      uint4 v;
      uint32_t* pv = reinterpret_cast<uint32_t*>(&v);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        __nv_bfloat16 f2[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k = 8 * c + 2 * e + h;
          const int j = k / 3;
          f2[h] = k < 27 ? hm[warp + j / 3][lane + j % 3][k - 3 * j] : __float2bfloat16(0.0f);
        }
        pv[e] = pack_raw(f2[0], f2[1]);
      }
      *reinterpret_cast<uint4*>(s.t.a[grp] + canon(m, 8 * c, NI)) = v;
    }
    float o[NO];
    ok = tc_network(s.t, grp, m, phase, o);
    const int x = x0 + lane, yy = y0 + warp;
    if (ok && x < g.nx && yy < g.ny) {
      float q[L::Q];
      lbm::sfor<0, L::Q>([&](auto I) {
        constexpr int i = LBM_CI(I);
        constexpr int cx = L::CX[i], cy = L::CY[i];
        const int xs = lbm::src_coord(x, cx, g.nx, g.bcx);
        const int ys = lbm::src_coord(yy, cy, g.ny, g.bcy);
        q[i] = fin[(long long)i * g.plane + (long long)ys * g.pitch + xs];
      });
      const float da[3] = {scale * o[0], scale * o[1], scale * o[2]};
      lbm::collide<L, lbm::COLL_RR, false, false, float, true>(q, P, da);
      lbm::sfor<0, L::Q>([&](auto I) {
        constexpr int i = LBM_CI(I);
        fout[(long long)i * g.plane + (long long)yy * g.pitch + x] = q[i];
      });
    }
  }
  tc_teardown(s.t);
}

struct lbm_closure {
  float* w = nullptr;            // FP32 master weights
  __nv_bfloat16* wb = nullptr;   // BF16 copy
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* loss = nullptr;         // device accumulator
  float* loss_host = nullptr;    // pinned
  long long t = 0;               // Adam step count
  int device = 0;
};

extern "C" {

int lbm_closure_create(lbm_closure** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  lbm_closure* c = new (std::nothrow) lbm_closure();
  if (!c) return LBM_ENOMEM;
  cudaGetDevice(&c->device);
  const size_t fb = sizeof(float) * NPARAM;
  if (cudaMalloc(&c->w, fb) != cudaSuccess || cudaMalloc(&c->wb, sizeof(__nv_bfloat16) * NPARAM) != cudaSuccess ||
      cudaMalloc(&c->grad, fb) != cudaSuccess || cudaMalloc(&c->m, fb) != cudaSuccess ||
      cudaMalloc(&c->v, fb) != cudaSuccess || cudaMalloc(&c->loss, sizeof(float)) != cudaSuccess ||
      cudaMallocHost(&c->loss_host, sizeof(float)) != cudaSuccess) {
    lbm_closure_destroy(c);
    return LBM_ENOMEM;
  }
  cudaMemset(c->w, 0, fb);
  cudaMemset(c->wb, 0, sizeof(__nv_bfloat16) * NPARAM);
  cudaMemset(c->grad, 0, fb);
  cudaMemset(c->m, 0, fb);
  cudaMemset(c->v, 0, fb);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    lbm_closure_destroy(c);
    return LBM_ECUDA;
  }
  *out = c;
  return LBM_OK;
}

void lbm_closure_destroy(lbm_closure* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaFree(c->w);
  cudaFree(c->wb);
  cudaFree(c->grad);
  cudaFree(c->m);
  cudaFree(c->v);
  cudaFree(c->loss);
  cudaFreeHost(c->loss_host);
  delete c;
}

int lbm_closure_set_weights(lbm_closure* c, const float* w, int n) {
  if (!c || !w || n != NPARAM) return LBM_EINVAL;
  cudaSetDevice(c->device);
  if (cudaMemcpy(c->w, w, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess) return LBM_ECUDA;
  k_to_bf16<<<(NPARAM + 255) / 256, 256>>>(c->w, c->wb, NPARAM);
  cudaMemset(c->m, 0, sizeof(float) * NPARAM);
  cudaMemset(c->v, 0, sizeof(float) * NPARAM);
  cudaMemset(c->grad, 0, sizeof(float) * NPARAM);
  c->t = 0;
  return cudaDeviceSynchronize() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int lbm_closure_get_weights(lbm_closure* c, float* w, int n) {
  if (!c || !w || n != NPARAM) return LBM_EINVAL;
  cudaSetDevice(c->device);
  return cudaMemcpy(w, c->w, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

// Once per device (the current one): its SM count, the dynamic shared-memory limits and the largest shared-memory
// carveout of the two tensor-core kernels, and how many fused-step blocks a SM holds (by its shared memory, at most
// four: 128 TMEM columns a block).  The occupancy calculator gave one block a SM for the fused step, whose
// launches then ran two tile pairs a block in turn (ncu: 152 blocks, 8 warps a SM).
static int tc_device_setup(int* sms, int* fused_per_sm) {
  static int cached_dev = -1, cached_sms = 0, cached_fused = 1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ECUDA;
  if (dev != cached_dev) {
    int s = 0, smem_sm = 0, reserved = 0;
    if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SmemTc)) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
        cudaFuncSetAttribute(k_step_closure_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SmemFused)) != cudaSuccess ||
        cudaFuncSetAttribute(k_step_closure_fused, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess)
      return LBM_ECUDA;
    const int fit = smem_sm / ((int)sizeof(SmemFused) + reserved);
    cached_fused = fit < 1 ? 1 : (fit > 4 ? 4 : fit);
    cached_sms = s;
    cached_dev = dev;
  }
  *sms = cached_sms;
  if (fused_per_sm) *fused_per_sm = cached_fused;
  return LBM_OK;
}

int lbm_closure_forward(lbm_closure* c, const void* x, int n, float* y, void* stream) {
  if (!c || !x || !y || n < 0) return LBM_EINVAL;
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15u) return LBM_EINVAL;  // 16-byte rows
  if (n == 0) return LBM_OK;
  if (cudaSetDevice(c->device) != cudaSuccess) return LBM_ECUDA;
  int sms = 0;
  if (tc_device_setup(&sms, nullptr) != LBM_OK) return LBM_ECUDA;
  // two groups of 128 rows a block at a time, four blocks a SM (the shared memory and TMEM hold four)
  long long blocks = ((long long)n + TC_G * TC_M - 1) / (TC_G * TC_M);
  if (blocks > 4LL * sms) blocks = 4LL * sms;
  k_mlp_forward_tc<<<(unsigned)blocks, TC_G * TC_M, sizeof(SmemTc), (cudaStream_t)stream>>>(
      (const __nv_bfloat16*)x, n, c->wb, c->w, y);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

static int train_pass(lbm_closure* c, const void* x, const float* y, int n, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SmemTrain)) !=
        cudaSuccess)
      return LBM_ECUDA;
    attr = true;
  }
  cudaMemsetAsync(c->loss, 0, sizeof(float), st);
  const int blocks = (n + TB - 1) / TB;
  k_mlp_train<<<blocks, 128, sizeof(SmemTrain), st>>>((const __nv_bfloat16*)x, y, n, c->wb, c->w, c->grad, c->loss);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int lbm_closure_gradients(lbm_closure* c, const void* x, const float* y, int n, float* grad_host, float* loss) {
  if (!c || !x || !y || n < 1 || !grad_host) return LBM_EINVAL;
  cudaSetDevice(c->device);
  cudaMemset(c->grad, 0, sizeof(float) * NPARAM);
  int rc = train_pass(c, x, y, n, nullptr);
  if (rc != LBM_OK) return rc;
  if (cudaMemcpy(grad_host, c->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess) return LBM_ECUDA;
  if (loss && cudaMemcpy(loss, c->loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return LBM_ECUDA;
  cudaMemset(c->grad, 0, sizeof(float) * NPARAM);
  return LBM_OK;
}

int lbm_closure_train_step(lbm_closure* c, const void* x, const float* y, int n, float lr, float* loss,
                           void* stream) {
  if (!c || !x || !y || n < 1 || !(lr > 0)) return LBM_EINVAL;
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = train_pass(c, x, y, n, st);
  if (rc != LBM_OK) return rc;
  c->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f / (1.0f - powf(b1, (float)c->t)), c2 = 1.0f / (1.0f - powf(b2, (float)c->t));
  k_adam<<<(NPARAM + 255) / 256, 256, 0, st>>>(c->w, c->wb, c->grad, c->m, c->v, lr, b1, b2, 1e-8f, c1, c2);
  if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
  if (loss) {
    if (cudaMemcpyAsync(c->loss_host, c->loss, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return LBM_ECUDA;
    *loss = *c->loss_host;
  }
  return LBM_OK;
}

static bool closure_ctx_ok(const lbm_ctx* c) {
  return c->p.lattice == LBM_D2Q9 && c->p.collision == LBM_RR && c->prec == lbm::PREC_F32 && !c->p.thermal &&
         c->p.a1_source == LBM_A1_PROJECTION;
}

static lbm::CollParams<float> closure_coll_params(const lbm_ctx* c) {
  const lbm::CollParamsD pd = lbm_ctx_coll_params(c);
  lbm::CollParams<float> P = lbm::cast_params<float>(pd);
  lbm::set_coef_factors<lbm::D2Q9>(P, lbm::COLL_RR, pd.neq, pd.nreg, pd.omega, pd.om1, pd.om1_3, pd.om1_4, 1.0);
  return P;
}

int lbm_closure_apply(lbm_ctx* c, const float* y, double u0) {
  if (!c || !y || !(u0 > 0)) return LBM_EINVAL;
  if (!closure_ctx_ok(c)) return LBM_EINVAL;
  if (cudaSetDevice(c->device) != cudaSuccess) return LBM_ECUDA;
  const long long cells = (long long)c->p.nx * c->p.ny;
  // the correction Delta a1 enters the post-collision flux as (1 - 1/tau) Delta a1 = tau_sgs
  const float scale = (float)(u0 * u0 / (1.0 - 1.0 / c->tau));
  k_step_closure<<<(unsigned)((cells + 127) / 128), 128, 0, c->st>>>(
      static_cast<const float*>(c->buf[c->cur]), static_cast<float*>(c->buf[c->cur ^ 1]), c->g,
      closure_coll_params(c), y, scale);
  if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
  c->cur ^= 1;
  c->steps += 1;
  return LBM_OK;
}

int lbm_step_closure(lbm_ctx* c, lbm_closure* cl, double u0, int n) {
  if (!c || !cl || n < 0 || !(u0 > 0)) return LBM_EINVAL;
  if (!closure_ctx_ok(c)) return LBM_EINVAL;
  if (cudaSetDevice(c->device) != cudaSuccess) return LBM_ECUDA;
  const long long cells = (long long)c->p.nx * c->p.ny;
  if (!c->closure_buf) {
    // rho, ux, uy (double) | features (BF16) | outputs (FP32): the fused step uses the first part,
    // the rest serves callers composing the stages themselves
    const size_t bytes = cells * (3 * sizeof(double) + NI * sizeof(__nv_bfloat16) + NO * sizeof(float));
    if (cudaMalloc(&c->closure_buf, bytes) != cudaSuccess) return LBM_ENOMEM;
  }
  double* r = static_cast<double*>(c->closure_buf);
  double* u = r + cells;
  double* v = u + cells;
  const lbm::CollParams<float> P = closure_coll_params(c);
  const float scale = (float)(u0 * u0 / (1.0 - 1.0 / c->tau));
  const long long tiles = (long long)((c->p.nx + FT_X - 1) / FT_X) * ((c->p.ny + FT_Y - 1) / FT_Y);
  int sms = 0, per_sm = 1;
  if (tc_device_setup(&sms, &per_sm) != LBM_OK) return LBM_ECUDA;
  const long long grid = std::min<long long>((tiles + TC_G - 1) / TC_G, (long long)per_sm * sms);
  for (int k = 0; k < n; ++k) {
    if (lbm_moments(c, r, u, v, nullptr, 1) != LBM_OK) return LBM_ECUDA;
    k_step_closure_fused<<<(unsigned)grid, TC_G * TC_M, sizeof(SmemFused), c->st>>>(
        static_cast<const float*>(c->buf[c->cur]), static_cast<float*>(c->buf[c->cur ^ 1]), c->g, P, r, u, v,
        1.0 / u0, cl->wb, cl->w, scale);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    c->cur ^= 1;
    c->steps += 1;
  }
  return LBM_OK;
}

int lbm_closure_features(const double* rho, const double* ux, const double* uy, int nx, int ny, double u0,
                         void* feat, void* stream) {
  if (!rho || !ux || !uy || !feat || nx < 1 || ny < 1 || !(u0 > 0)) return LBM_EINVAL;
  const long long n = (long long)nx * ny;
  k_features<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(rho, ux, uy, nx, ny, 1.0 / u0,
                                                                          (__nv_bfloat16*)feat);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int lbm_closure_coarsen(const double* rho, const double* ux, const double* uy, int nx, int ny, int factor, double u0,
                        double* rho_c, double* ux_c, double* uy_c, float* y, void* stream) {
  if (!rho || !ux || !uy || !rho_c || !ux_c || !uy_c || !y || factor < 1 || nx % factor || ny % factor ||
      !(u0 > 0))
    return LBM_EINVAL;
  const long long n = (long long)(nx / factor) * (ny / factor);
  k_coarsen<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(rho, ux, uy, nx, ny, factor, 1.0 / u0,
                                                                          rho_c, ux_c, uy_c, y);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

}  // extern "C"
