// Learned a1^(2) closure for coarse grids: a per-cell MLP
//   features (27 used of 32) -> 64 -> 64 -> 64 -> 3 (of 8), GELU on the hidden layers,
// predicting the subgrid stress <rho u_a u_b> - rho_bar u_bar_a u_bar_b that box filtering of a
// fine run leaves out of the coarse equilibrium, which the coarse RR step adds to its a1^(2).
//
// Every matrix product runs on the tensor cores as BF16 x BF16 -> FP32 warp MMAs
// (mma.sync m16n8k16): inference chains the layers through registers (the FP32 accumulator
// fragment of one layer is, after bias + GELU and rounding to BF16, the A fragment of the next);
// training keeps each layer's activations in shared memory and forms the weight gradients
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
#include <cstring>
#include <new>

#include "../../include/lbm.h"
#include "ctx.h"
#include "fields.h"

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

// B fragments of a [out][in] weight matrix for the k-chunk k0 and output tile n0 (B[k][n] = W[n][k]).
__device__ __forceinline__ void wfrag(uint32_t (&rb)[2], const __nv_bfloat16* w, int in_dim, int k0, int n0) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const __nv_bfloat16* row = w + (n0 + g) * in_dim + k0 + 2 * t;
  rb[0] = *reinterpret_cast<const uint32_t*>(row);
  rb[1] = *reinterpret_cast<const uint32_t*>(row + 8);
}

// Hidden layer on register fragments of two independent 16-row tiles: in a[2][KC][4] (K = 16 KC), out
// GELU(a W^T + b) as the next layer's A fragments a_next[2][4][4] (K = 64).  Each weight fragment is read
// once for both tiles and the two MMA chains overlap.
template <int KC>
__device__ __forceinline__ void dense_gelu2(const uint32_t (&a)[2][KC][4], const __nv_bfloat16* w, const float* b,
                                            uint32_t (&a_next)[2][4][4]) {
  const int lane = threadIdx.x & 31, t = lane & 3;
  float acc[2][8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float b0 = b[j * 8 + 2 * t], b1 = b[j * 8 + 2 * t + 1];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      acc[h][j][0] = b0;
      acc[h][j][1] = b1;
      acc[h][j][2] = b0;
      acc[h][j][3] = b1;
    }
#pragma unroll
    for (int kc = 0; kc < KC; ++kc) {
      uint32_t rb[2];
      wfrag(rb, w, 16 * KC, kc * 16, j * 8);
      mma16816(acc[0][j], a[0][kc], rb);
      mma16816(acc[1][j], a[1][kc], rb);
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      a_next[h][kc][0] = pack_bf16(gelu(acc[h][2 * kc][0]), gelu(acc[h][2 * kc][1]));
      a_next[h][kc][1] = pack_bf16(gelu(acc[h][2 * kc][2]), gelu(acc[h][2 * kc][3]));
      a_next[h][kc][2] = pack_bf16(gelu(acc[h][2 * kc + 1][0]), gelu(acc[h][2 * kc + 1][1]));
      a_next[h][kc][3] = pack_bf16(gelu(acc[h][2 * kc + 1][2]), gelu(acc[h][2 * kc + 1][3]));
    }
}

// Output layer (8 columns, no activation) on two tiles: o[h] = b4 + h3[h] W4^T.
__device__ __forceinline__ void dense_out2(const uint32_t (&a)[2][4][4], const __nv_bfloat16* w, const float* b,
                                           float (&o)[2][4]) {
  const int t = threadIdx.x & 3;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    o[h][0] = b[2 * t];
    o[h][1] = b[2 * t + 1];
    o[h][2] = b[2 * t];
    o[h][3] = b[2 * t + 1];
  }
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    uint32_t rb[2];
    wfrag(rb, w, NH, kc * 16, 0);
    mma16816(o[0], a[0][kc], rb);
    mma16816(o[1], a[1][kc], rb);
  }
}

// Inference: y[n][NO] (FP32) for x[n][NI] (BF16); each warp takes 32 rows (two 16-row tiles) at a time.
__global__ void __launch_bounds__(128) k_mlp_forward(const __nv_bfloat16* __restrict__ x, int n,
                                                     const __nv_bfloat16* __restrict__ wb,
                                                     const float* __restrict__ wf, float* __restrict__ y) {
  __shared__ SmemWeights s;
  load_weights(s, wb, wf);
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (long long r0 = ((long long)blockIdx.x * nwarps + warp) * 32; r0 < n;
       r0 += (long long)gridDim.x * nwarps * 32) {
    uint32_t a0[2][2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long ra = r0 + 16 * h + g, rbr = ra + 8;
#pragma unroll
      for (int kc = 0; kc < 2; ++kc) {
        const int c = kc * 16 + 2 * t;
        a0[h][kc][0] = ra < n ? *reinterpret_cast<const uint32_t*>(x + ra * NI + c) : 0u;
        a0[h][kc][1] = rbr < n ? *reinterpret_cast<const uint32_t*>(x + rbr * NI + c) : 0u;
        a0[h][kc][2] = ra < n ? *reinterpret_cast<const uint32_t*>(x + ra * NI + c + 8) : 0u;
        a0[h][kc][3] = rbr < n ? *reinterpret_cast<const uint32_t*>(x + rbr * NI + c + 8) : 0u;
      }
    }
    uint32_t h1[2][4][4], h2[2][4][4], h3[2][4][4];
    dense_gelu2<2>(a0, s.w1, s.b1, h1);
    dense_gelu2<4>(h1, s.w2, s.b2, h2);
    dense_gelu2<4>(h2, s.w3, s.b3, h3);
    float o[2][4];
    dense_out2(h3, s.w4, s.b4, o);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long ra = r0 + 16 * h + g, rbr = ra + 8;
      if (ra < n) {
        y[ra * NO + 2 * t] = o[h][0];
        y[ra * NO + 2 * t + 1] = o[h][1];
      }
      if (rbr < n) {
        y[rbr * NO + 2 * t] = o[h][2];
        y[rbr * NO + 2 * t + 1] = o[h][3];
      }
    }
  }
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
// iteration (warp w takes row w of the tile, one cell per lane).  The moments of the tile and its
// one-cell halo (periodic, as lbm_closure_features) are converted to BF16 features in shared memory
// once; each warp builds its two 16-cell A fragments from them, runs the layer chain of
// k_mlp_forward, leaves the three used outputs of its 32 cells in shared memory and then pulls,
// collides and stores its cells as k_step_closure does.  Same arithmetic in the same order as
// features + forward + k_step_closure, so the result is bitwise the three-kernel path's.
// ---------------------------------------------------------------------------
constexpr int FT_X = 32, FT_Y = 4;

struct SmemFused {
  SmemWeights w;
  __nv_bfloat16 m[FT_Y + 2][FT_X + 2][3];  // (rho - 1, ux, uy) / u0 of the tile and its halo
  float y[FT_Y][FT_X][3];
};

__global__ void __launch_bounds__(128) k_step_closure_fused(const float* __restrict__ fin, float* __restrict__ fout,
                                                            lbm::StepGeom g, lbm::CollParams<float> P,
                                                            const double* __restrict__ rho,
                                                            const double* __restrict__ ux,
                                                            const double* __restrict__ uy, double inv_u0,
                                                            const __nv_bfloat16* __restrict__ wb,
                                                            const float* __restrict__ wf, float scale) {
  using L = lbm::D2Q9;
  __shared__ SmemFused s;
  load_weights(s.w, wb, wf);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, gq = lane >> 2, t = lane & 3;
  const int tiles_x = (g.nx + FT_X - 1) / FT_X, tiles_y = (g.ny + FT_Y - 1) / FT_Y;
  for (long long tile = blockIdx.x; tile < (long long)tiles_x * tiles_y; tile += gridDim.x) {
    const int x0 = (int)(tile % tiles_x) * FT_X, y0 = (int)(tile / tiles_x) * FT_Y;
    __syncthreads();  // previous tile's features and outputs are no longer read
    for (int k = threadIdx.x; k < (FT_Y + 2) * (FT_X + 2); k += blockDim.x) {
      const int hy = k / (FT_X + 2), hx = k - hy * (FT_X + 2);
      int xs = (x0 + hx - 1) % g.nx, ys = (y0 + hy - 1) % g.ny;
      if (xs < 0) xs += g.nx;
      if (ys < 0) ys += g.ny;
      const long long c = (long long)ys * g.nx + xs;
      s.m[hy][hx][0] = __float2bfloat16((float)((rho[c] - 1.0) * inv_u0));
      s.m[hy][hx][1] = __float2bfloat16((float)(ux[c] * inv_u0));
      s.m[hy][hx][2] = __float2bfloat16((float)(uy[c] * inv_u0));
    }
    __syncthreads();
    // feature k of the cell in column cx of this warp's row: neighbour k / 3 (row-major over the 3 x 3
    // stencil), component k % 3; zero beyond the 27 used inputs
    auto feat = [&](int cx, int k) -> __nv_bfloat16 {
      if (k >= 27) return __float2bfloat16(0.0f);
      const int j = k / 3;
      return s.m[warp + j / 3][cx + j % 3][k - 3 * j];
    };
    uint32_t a0[2][2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int ra = h * 16 + gq, rb = ra + 8;
#pragma unroll
      for (int kc = 0; kc < 2; ++kc) {
        const int c = kc * 16 + 2 * t;
        a0[h][kc][0] = pack_raw(feat(ra, c), feat(ra, c + 1));
        a0[h][kc][1] = pack_raw(feat(rb, c), feat(rb, c + 1));
        a0[h][kc][2] = pack_raw(feat(ra, c + 8), feat(ra, c + 9));
        a0[h][kc][3] = pack_raw(feat(rb, c + 8), feat(rb, c + 9));
      }
    }
    uint32_t h1[2][4][4], h2[2][4][4], h3[2][4][4];
    dense_gelu2<2>(a0, s.w.w1, s.w.b1, h1);
    dense_gelu2<4>(h1, s.w.w2, s.w.b2, h2);
    dense_gelu2<4>(h2, s.w.w3, s.w.b3, h3);
    float o[2][4];
    dense_out2(h3, s.w.w4, s.w.b4, o);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int ra = h * 16 + gq, rb = ra + 8;
      if (t == 0) {
        s.y[warp][ra][0] = o[h][0];
        s.y[warp][ra][1] = o[h][1];
        s.y[warp][rb][0] = o[h][2];
        s.y[warp][rb][1] = o[h][3];
      } else if (t == 1) {
        s.y[warp][ra][2] = o[h][0];
        s.y[warp][rb][2] = o[h][2];
      }
    }
    __syncwarp();
    const int x = x0 + lane, yy = y0 + warp;
    if (x < g.nx && yy < g.ny) {
      float q[L::Q];
      lbm::sfor<0, L::Q>([&](auto I) {
        constexpr int i = LBM_CI(I);
        constexpr int cx = L::CX[i], cy = L::CY[i];
        const int xs = lbm::src_coord(x, cx, g.nx, g.bcx);
        const int ys = lbm::src_coord(yy, cy, g.ny, g.bcy);
        q[i] = fin[(long long)i * g.plane + (long long)ys * g.pitch + xs];
      });
      const float da[3] = {scale * s.y[warp][lane][0], scale * s.y[warp][lane][1], scale * s.y[warp][lane][2]};
      lbm::collide<L, lbm::COLL_RR, false, false, float, true>(q, P, da);
      lbm::sfor<0, L::Q>([&](auto I) {
        constexpr int i = LBM_CI(I);
        fout[(long long)i * g.plane + (long long)yy * g.pitch + x] = q[i];
      });
    }
  }
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

int lbm_closure_forward(lbm_closure* c, const void* x, int n, float* y, void* stream) {
  if (!c || !x || !y || n < 0) return LBM_EINVAL;
  if (n == 0) return LBM_OK;
  cudaSetDevice(c->device);
  const long long pairs = ((long long)n + 31) / 32;  // 32 rows per warp iteration
  long long blocks = (pairs + 3) / 4;
  if (blocks > 4096) blocks = 4096;
  k_mlp_forward<<<(unsigned)blocks, 128, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)x, n, c->wb, c->w, y);
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
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_closure_fused, 128, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const long long grid = std::min<long long>(tiles, (long long)per_sm * c->g.nsm);
  for (int k = 0; k < n; ++k) {
    if (lbm_moments(c, r, u, v, nullptr, 1) != LBM_OK) return LBM_ECUDA;
    k_step_closure_fused<<<(unsigned)grid, 128, 0, c->st>>>(
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
