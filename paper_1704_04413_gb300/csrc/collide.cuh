// Per-cell arithmetic of the regularized lattice-Boltzmann step (Coreixas et
// al., arXiv 1704.04413): moments (Sec. II.A), equilibrium Hermite
// coefficients a0 (App. B, written out for 2D), off-equilibrium coefficients
// a1 by projection (Sec. II.E) or by recursion (Eqs. MalaspinasRecursiveRelation
// and RecursiveRelation_ThermalCase in the 2D form of App. C, Eq. a1Rec), the
// thermal a1^(3) filtering of App. C (Eq. TempGradLBM) and the rebuild of
// Eq. (GenRegCollision) with a single relaxation time.
//
// A 2D Hermite coefficient with a x-indices and b y-indices is kept as
// X[a][b]; its tensor multiplicity A^(n) of App. C is folded into the factor
// 1 / (a! b! cs^2(a+b)).  All lattice-dependent numbers are compile-time
// constants (lattice.cuh); loops over populations and orders are unrolled.
#pragma once
#include <type_traits>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lattice.cuh"
#include "vec2.cuh"

#define LBM_CI(X) decltype(X)::value

namespace lbm {

enum { COLL_BGK = 0, COLL_PR = 1, COLL_RR = 2 };

// Lane type of a compute type (F2 computes two cells in FP32 lanes).
template <class R>
struct Scalar {
  using type = R;
};
template <>
struct Scalar<F2> {
  using type = float;
};

// Slot of the 2D Hermite coefficient with a x-indices and b y-indices (order a + b <= 4) in the per-coefficient
// factor arrays below.
__host__ __device__ constexpr int coef_index(int a, int b) { return (a + b) * (a + b + 1) / 2 + a; }
constexpr int kCoefs = 15;

template <class Real>
struct CollParams {
  Real omega;  // 1 / tau
  Real om1;    // 1 - 1 / tau (order 2 of f^(1); BGK)
  Real om1_3;  // 1 - 1 / tau_3, 1 - 1 / tau_4: one relaxation time per order (Eq. GenRegCollision)
  Real om1_4;
  Real tau, tau3;  // tau_2 and tau_3 themselves (the finite-difference a1 of FD collisions)
  int neq;     // highest order of f^(0)
  int nreg;    // highest order of f^(1)
  Real rho0;   // shift of low-precision storage
  Real s;      // scale of low-precision storage
  Real inv_s;
  // 2D collisions (collide below): the rebuilt coefficient of order n = a + b >= 1 is
  //   C[a][b] = ka A[a][b] + kb B[a][b],   A = a0, B = s a1 (the projection in storage units),
  // ka = [n <= neq] s / (a! b! cs^2n) (times 1 / tau for BGK), kb = [2 <= n <= nreg] (1 - 1/tau_n) / (a! b! cs^2n),
  // so that the orders kept, the relaxation and the storage scale cost one multiply-add per coefficient, with
  // both factors as constant-bank operands; msn[n] = -s where f^(0) carries order n (n <= neq), else 0.
  Real ka[kCoefs], kb[kCoefs];
  Real msn[5];
};

// ---------------------------------------------------------------------------
// Storage formats.  Plain formats hold f_i.  Shifted low-precision formats
// hold g_i = (f_i / w_i - rho0) * s, i.e. the relative deviation from the
// reference equilibrium w_i rho0, times a power of two s.
// ---------------------------------------------------------------------------
template <class S>
struct Store;
template <>
struct Store<double> {
  static constexpr bool SHIFTED = false;
  __device__ static __forceinline__ double ld(const double* p) { return __ldg(p); }
  __device__ static __forceinline__ void st(double* p, double v) { *p = v; }
};
template <>
struct Store<float> {
  static constexpr bool SHIFTED = false;
  __device__ static __forceinline__ float ld(const float* p) { return __ldg(p); }
  __device__ static __forceinline__ void st(float* p, float v) { *p = v; }
};
template <>
struct Store<__half> {
  static constexpr bool SHIFTED = true;
  __device__ static __forceinline__ float ld(const __half* p) { return __half2float(__ldg(p)); }
  __device__ static __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
};
template <>
struct Store<__nv_bfloat16> {
  static constexpr bool SHIFTED = true;
  __device__ static __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
  __device__ static __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};
// 16-bit fixed point of the shifted deviation: n = round(2^15 g), g in [-1, 1) (saturating).  Uniform
// absolute resolution 2^-15 / s of f_i / w_i, where binary16 resolves only 2^-12 at |g| ~ 0.3.
constexpr float kFix16 = 32768.0f;
__device__ __forceinline__ short fix16_encode(float v) {
  int n = __float2int_rn(v * kFix16);
  n = n < -32768 ? -32768 : (n > 32767 ? 32767 : n);
  return (short)n;
}
template <>
struct Store<short> {
  static constexpr bool SHIFTED = true;
  __device__ static __forceinline__ float ld(const short* p) { return (float)__ldg(p) * (1.0f / kFix16); }
  __device__ static __forceinline__ void st(short* p, float v) { *p = fix16_encode(v); }
};

// ---------------------------------------------------------------------------
// Equilibrium coefficients a0 (App. B recursion specialised to 2D):
//   a0[a][b] = u_y a0[a][b-1] + (b-1) e a0[a][b-2]            (b > 0)
//   a0[a][0] = u_x a0[a-1][0] + (a-1) e a0[a-2][0]
// with e = cs^2 (theta - 1).
// ---------------------------------------------------------------------------
template <class L, bool THERMAL, class Real>
__device__ __forceinline__ void equilibrium_coefficients(Real rho, Real ux, Real uy, Real e, Real (&A)[5][5]) {
  A[0][0] = rho;
  sfor<1, L::NMAX + 1>([&](auto N) {
    constexpr int n = LBM_CI(N);
    sfor<0, n + 1>([&](auto Aa) {
      constexpr int a = LBM_CI(Aa);
      constexpr int b = n - a;
      if constexpr (L::keep(a, b)) {
        if constexpr (b > 0) {
          Real v = uy * A[a][b - 1];
          if constexpr (THERMAL && b >= 2) v += Real(b - 1) * e * A[a][b - 2];
          A[a][b] = v;
        } else {
          Real v = ux * A[a - 1][0];
          if constexpr (THERMAL && a >= 2) v += Real(a - 1) * e * A[a - 2][0];
          A[a][0] = v;
        }
      }
    });
  });
}

// Third-order a1 from a1^(2) (isothermal recursion, App. C Eq. a1Rec with no
// temperature gradient), then fourth order by App. C (theta-dependent form).
template <class L, bool THERMAL, class Real>
__device__ __forceinline__ void a1_third_from_second(Real ux, Real uy, Real (&B)[5][5]) {
  if constexpr (L::NMAX >= 3) {
    B[3][0] = Real(3) * ux * B[2][0];
    B[2][1] = Real(2) * ux * B[1][1] + uy * B[2][0];
    B[1][2] = Real(2) * uy * B[1][1] + ux * B[0][2];
    B[0][3] = Real(3) * uy * B[0][2];
  }
}
template <class L, bool THERMAL, class Real>
__device__ __forceinline__ void a1_fourth(Real ux, Real uy, Real e, Real (&B)[5][5]) {
  if constexpr (L::NMAX >= 4) {
    Real ex = -ux * ux, ey = -uy * uy;
    if constexpr (THERMAL) {
      ex += e;
      ey += e;
    }
    const Real uxy = ux * uy;
    B[4][0] = Real(4) * ux * B[3][0] + Real(6) * ex * B[2][0];
    B[3][1] = Real(3) * ux * B[2][1] + uy * B[3][0] + Real(3) * ex * B[1][1] - Real(3) * uxy * B[2][0];
    B[2][2] = Real(2) * (ux * B[1][2] + uy * B[2][1]) + ex * B[0][2] + ey * B[2][0] - Real(4) * uxy * B[1][1];
    B[1][3] = Real(3) * uy * B[1][2] + ux * B[0][3] + Real(3) * ey * B[1][1] - Real(3) * uxy * B[0][2];
    B[0][4] = Real(4) * uy * B[0][3] + Real(6) * ey * B[0][2];
  }
}

// ---------------------------------------------------------------------------
// Sums with compile-time coefficients.  The first term of a sum is written as a product (no addition of a
// zero), and a product by 1 is no instruction: add_term<FIRST>(acc, h, x) with h a constant.
// ---------------------------------------------------------------------------
template <bool FIRST, class Real>
__device__ __forceinline__ void add_term(Real& acc, double h, const Real& x) {
  if constexpr (FIRST)
    acc = (h == 1.0) ? x : Real(h) * x;
  else
    acc = madd(Real(h), x, acc);
}

// Reciprocal of a density (a value near 1).  Two cells: the hardware's approximate reciprocal refined by one
// Newton-Raphson step r' = r + r (1 - x r) in packed arithmetic, within about one unit in the last place.
// One cell (FP32, FP64): the division (with the approximate form, the 72-register one-cell D2V37 kernel of
// the batched sweep spilled 112 bytes).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float recip(float x) { return 1.0f / x; }
__device__ __forceinline__ F2 recip(F2 x) {
  const F2 r(rcp_approx(x.v.x), rcp_approx(x.v.y));
  const F2 e = __ffma2_rn(make_float2(-x.v.x, -x.v.y), r.v, make_float2(1.f, 1.f));
  return madd(r, e, r);
}
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// First b of parity par with a term in the row value g[a](v) of the rebuild (-1: none).
template <class L>
__host__ __device__ constexpr int rebuild_first_b(int a, int v, int par) {
  for (int b = par; b <= L::NMAX - a; b += 2)
    if (L::keep(a, b) && he(b, v, L::CS2) != 0.0) return b;
  return -1;
}
// First a with a term in population i's sum over the row values (-1: none).
template <class L>
__host__ __device__ constexpr int rebuild_first_a(int i) {
  for (int a = 0; a <= L::NMAX; ++a)
    if (L::keep(a, 0) && he(a, L::CX[i], L::CS2) != 0.0) return a;
  return -1;
}

// ---------------------------------------------------------------------------
// Rebuild: out_i = sum_{(a,b) kept} K_i He(a, cx_i) He(b, cy_i) C[a][b], with
// K_i = w_i for plain storage and 1 for shifted storage (whose C carry the
// factor s and whose w_i cancels).  Factorised by rows of equal cy:
//   g[a](v) = sum_b He(b, v) C[a][b],   out_i = sum_a K_i He(a, cx_i) g[a](cy_i),
// and g[a](+-v) = E +- O with E/O the even/odd-b parts.
// ---------------------------------------------------------------------------
// Row values g[a](v) and (v != 0) g[a](-v) of one row pair.
template <class L, int v, class Real>
__device__ __forceinline__ void rebuild_row_values(const Real (&C)[5][5], Real (&gp)[5], Real (&gm)[5]) {
  constexpr double c2 = L::CS2;
  sfor<0, L::NMAX + 1>([&](auto Aa) {
    constexpr int a = LBM_CI(Aa);
    if constexpr (L::keep(a, 0)) {
      constexpr int fe = rebuild_first_b<L>(a, v, 0), fo = rebuild_first_b<L>(a, v, 1);
      Real ev = Real(0), od = Real(0);
      sfor<0, L::NMAX + 1 - a>([&](auto Bb) {
        constexpr int b = LBM_CI(Bb);
        constexpr double h = he(b, v, c2);
        if constexpr (L::keep(a, b) && h != 0.0) {
          if constexpr (b % 2 == 0)
            add_term<b == fe>(ev, h, C[a][b]);
          else
            add_term<b == fo>(od, h, C[a][b]);
        }
      });
      if constexpr (fo < 0) {
        gp[a] = ev;
        if constexpr (v != 0) gm[a] = ev;
      } else {
        gp[a] = ev + od;
        if constexpr (v != 0) gm[a] = ev - od;
      }
    }
  });
}

// Population i from the row values g of its row.
template <class L, bool SHIFTED, int i, class Real>
__device__ __forceinline__ Real rebuild_pop(const Real (&g)[5]) {
  constexpr double c2 = L::CS2;
  constexpr int fa = rebuild_first_a<L>(i);
  Real acc = Real(0);
  sfor<0, L::NMAX + 1>([&](auto Aa) {
    constexpr int a = LBM_CI(Aa);
    constexpr double h = he(a, L::CX[i], c2) * (SHIFTED ? 1.0 : L::W[i]);
    if constexpr (h != 0.0 && L::keep(a, 0)) add_term<a == fa>(acc, h, g[a]);
  });
  return acc;
}

template <class L, bool SHIFTED, class Real, class F>
__device__ __forceinline__ void rebuild(const Real (&C)[5][5], F&& emit) {
  constexpr int V = L::VMAX;
  Real g[2 * V + 1][5];
  sfor<0, V + 1>([&](auto VV) {
    constexpr int v = LBM_CI(VV);
    if constexpr (has_row<L>(v) || has_row<L>(-v)) rebuild_row_values<L, v>(C, g[V + v], g[V - v]);
  });
  sfor<0, L::Q>([&](auto I) {
    constexpr int i = LBM_CI(I);
    constexpr int v = L::CY[i];
    emit(I, rebuild_pop<L, SHIFTED, i>(g[V + v]));
  });
}

template <class L, bool SHIFTED, class Real, class F>
__device__ __forceinline__ void rebuild_rows(const Real (&C)[5][5], F&& emit) {
  constexpr int V = L::VMAX;
  // rebuild() one row pair +-v at a time: its g[a](+-v) are made, its populations emitted, and the g die,
  // so that a caller storing each emitted population at once never holds more than one row pair's g
  sfor<0, V + 1>([&](auto VV) {
    constexpr int v = LBM_CI(VV);
    if constexpr (has_row<L>(v) || has_row<L>(-v)) {
      Real gp[5], gm[5];
      rebuild_row_values<L, v>(C, gp, gm);
      sfor<0, L::Q>([&](auto I) {
        constexpr int i = LBM_CI(I);
        if constexpr (L::CY[i] == v)
          emit(I, rebuild_pop<L, SHIFTED, i>(gp));
        else if constexpr (v != 0 && L::CY[i] == -v)
          emit(I, rebuild_pop<L, SHIFTED, i>(gm));
      });
    }
  });
}

// ---------------------------------------------------------------------------
// Reference state.  Moments are accumulated from the deviations
// d_i = f_i - w_i rho_ref of the populations from the rest equilibrium
// w_i rho_ref, whose Hermite moments are rho_ref for H^(0) and 0 for every
// other kept tensor (orthogonality, App. D).  So
//   M[a][b] = rho_ref [a=b=0] + kappa[a][b] + sum_i He(a,cx_i) He(b,cy_i) d_i,
// with no large constant left to cancel in a1 = M - a0.  For plain storage
// the reference is the rounded weight w^_i of the storage type (d_i = f_i - w^_i
// is then exact whenever f_i is within a factor 2 of w_i) and
// kappa[a][b] = sum_i He He (w^_i - w_i) restores the exact moments; shifted
// storage already holds s (f_i/w_i - rho0) and has kappa = 0.
// ---------------------------------------------------------------------------
template <class L, class Real>
__host__ __device__ constexpr double ref_weight(int i) {
  return (double)(Real)L::W[i];
}
template <class L, class Real>
__host__ __device__ constexpr double kappa(int a, int b) {
  double s = 0.0;
  for (int i = 0; i < L::Q; ++i) s += he(a, L::CX[i], L::CS2) * he(b, L::CY[i], L::CS2) * (ref_weight<L, Real>(i) - L::W[i]);
  return s;
}

// ---------------------------------------------------------------------------
// One collision.  PR/RR rebuild with one relaxation time per order of f^(1) (Eq. GenRegCollision with
// tau_{n,alpha} -> tau_n): f* = f^(0) + sum_n (1 - 1/tau_n) f^(1,n).  q holds the pulled populations in storage representation
// (converted to Real) and receives the post-collision ones.
// ---------------------------------------------------------------------------
// With CLOSURE, da[0..2] is added to the projected a1^(2) (xx, xy, yy) before the recursion (the
// learned coarse-grid closure; closure.cu).  With FD (RR only), a1^(2) and the thermal temperature-gradient
// terms come from the gradients grad[0..5] = d ux/dx, d ux/dy, d uy/dx, d uy/dy, d theta/dx, d theta/dy
// (Sec. II.E allows finite differences in place of the projection):
//   a1^(2)_ab = -tau rho cs^2 theta (d_a u_b + d_b u_a - delta_ab div u) (thermal, D = 2), -tau rho cs^2 S
//   (isothermal); mu cs^2 d_g theta = tau_3 rho cs^4 theta d_g theta in place of Eq. TempGradLBM.
// KeepInQ: the post-collision populations go back into q.  Any other Out is called as out(I, value) for each
// population as soon as it is rebuilt, one row pair at a time (rebuild_rows: a caller that stores it at once
// keeps fewer values live).
struct KeepInQ {};

// How the rebuilt coefficients take the orders kept, the relaxation times and the storage scale: from the
// per-coefficient factors ka, kb of CollParams (one multiply and one multiply-add a coefficient), or from the
// scalar parameters (a select, a multiply-add and the scale products).  Measured on GB300 at 4096^2 with 16-bit
// storage: the factors take D2Q9 from 140 to 151-156 GLUPS, while D2V17, whose staged kernel runs at its
// 96-register cap, keeps 83.5-84 GLUPS with the scalar form against 80.5-82.4 with the factors.
template <class L>
struct CoefFactors {
  static constexpr bool value = L::Q != 17;
};

// First population with a nonzero coefficient c_i in a sum over the populations (-1: none): the monomial
// moments (kind 0: cx^k cy^l) and the Hermite moments summed directly (kind 1: He_k(cx) He_l(cy)).
template <class L, bool SHIFTED>
__host__ __device__ constexpr int first_pop(int kind, int k, int l) {
  for (int i = 0; i < L::Q; ++i) {
    const double c = kind == 0 ? ipow(L::CX[i], k) * ipow(L::CY[i], l)
                               : he(k, L::CX[i], L::CS2) * he(l, L::CY[i], L::CS2);
    if (c != 0.0) return i;
  }
  return -1;
}
// First monomial moment D[k][l] (as 5 k + l) with a nonzero coefficient in the Hermite moment (a, b).
__host__ __device__ constexpr int first_mono(int a, int b, double c2) {
  for (int k = 0; k <= a; ++k)
    for (int l = 0; l <= b; ++l)
      if (he_coef(a, k, c2) * he_coef(b, l, c2) != 0.0) return 5 * k + l;
  return -1;
}

template <class L, int COLL, bool THERMAL, bool SHIFTED, class Real, bool CLOSURE = false, bool FD = false,
          class Out = KeepInQ>
__device__ __forceinline__ void collide(Real (&q)[L::Q], const CollParams<Real>& P, const Real* da = nullptr,
                                        const Real* grad = nullptr, Out&& out = Out{}) {
  using Sc = typename Scalar<Real>::type;
  static_assert(!(THERMAL && !__is_same(Sc, Real)), "the thermal path computes one cell per thread");
  constexpr double c2 = L::CS2;
  // highest monomial order of f the mode needs (PR takes its orders >= 3 directly, hmom_direct below)
  constexpr int PM = (COLL == COLL_PR) ? 2 : (COLL == COLL_RR ? (THERMAL ? 3 : 2) : 1);

  // Everything linear in the populations is kept in storage units: the deviations d_i (shifted storage
  // holds s (f_i / w_i - rho0), plain storage f_i - w^_i), their moments, a1 (B = s a1) and the rebuilt
  // coefficients C.  s is a power of two, so these are exactly s times the values in units of f; only rho
  // and u (and the equilibrium coefficients A = a0 made from them) are in units of f.
  Real d[L::Q];
  sfor<0, L::Q>([&](auto I) {
    constexpr int i = LBM_CI(I);
    if constexpr (SHIFTED)
      d[i] = q[i];
    else
      d[i] = q[i] - Real(ref_weight<L, Sc>(i));
  });

  // --- monomial moments of the deviations D[k][l] = sum_i d_i cx^k cy^l (w_i d_i shifted) (Sec. II.A) ---
  Real D[5][5];
  sfor<0, 5>([&](auto K) {
    constexpr int k = LBM_CI(K);
    sfor<0, 5 - k>([&](auto Lq) {
      constexpr int l = LBM_CI(Lq);
      if constexpr (L::keep(k, l) && k + l <= PM) {
        constexpr int fi = first_pop<L, SHIFTED>(0, k, l);
        Real acc = Real(0);
        sfor<0, L::Q>([&](auto I) {
          constexpr int i = LBM_CI(I);
          constexpr double c = ipow(L::CX[i], k) * ipow(L::CY[i], l) * (SHIFTED ? L::W[i] : 1.0);
          if constexpr (c != 0.0) add_term<i == fi>(acc, c, d[i]);
        });
        D[k][l] = acc;
      }
    });
  });

  // Hermite moments of f in storage units (see above), plus kappa for plain storage
  auto hmom = [&](auto Aa, auto Bb) -> Real {
    constexpr int a = LBM_CI(Aa);
    constexpr int b = LBM_CI(Bb);
    constexpr int fm = first_mono(a, b, c2);
    Real acc = Real(0);
    sfor<0, a + 1>([&](auto K) {
      constexpr int k = LBM_CI(K);
      sfor<0, b + 1>([&](auto Lq) {
        constexpr int l = LBM_CI(Lq);
        constexpr double h = he_coef(a, k, c2) * he_coef(b, l, c2);
        if constexpr (h != 0.0) add_term<5 * k + l == fm>(acc, h, D[k][l]);
      });
    });
    if constexpr (!SHIFTED) {
      constexpr double kp = kappa<L, Sc>(a, b);
      if constexpr (kp != 0.0) acc += Real(kp);
    }
    return acc;
  };

  // Hermite moment summed directly over the populations, sum_i He_a(cx_i) He_b(cy_i) d_i (+ kappa): the
  // projection of PR at orders >= 3.  Through the monomial moments, He_3 = c^3 - 3 cs^2 c would subtract
  // two sums of the slow populations' large deviations (each rounded) whose difference is small; summed
  // directly those populations enter with their small He values, which keeps the FP32 rounding of a1^(3)
  // (amplified by He_3 / (3! cs^6) in the fast populations' rebuild) several times smaller.
  auto hmom_direct = [&](auto Aa, auto Bb) -> Real {
    constexpr int a = LBM_CI(Aa);
    constexpr int b = LBM_CI(Bb);
    constexpr int fi = first_pop<L, SHIFTED>(1, a, b);
    Real acc = Real(0);
    sfor<0, L::Q>([&](auto I) {
      constexpr int i = LBM_CI(I);
      constexpr double c = he(a, L::CX[i], c2) * he(b, L::CY[i], c2) * (SHIFTED ? L::W[i] : 1.0);
      if constexpr (c != 0.0) add_term<i == fi>(acc, c, d[i]);
    });
    if constexpr (!SHIFTED) {
      constexpr double kp = kappa<L, Sc>(a, b);
      if constexpr (kp != 0.0) acc += Real(kp);
    }
    return acc;
  };

  const Real drho = hmom(IC<0>{}, IC<0>{});  // s (rho - rho_ref)
  Real rho, ux, uy, e = Real(0);
  if constexpr (THERMAL) {
    // FP64 recovery of rho, u and theta from the energy moment 2 rho E = sum f xi^2 (Sec. II.A)
    double r = 0.0, jx = 0.0, jy = 0.0, e2 = 0.0;
    sfor<0, L::Q>([&](auto I) {
      constexpr int i = LBM_CI(I);
      double fi;
      constexpr double wi = L::W[i];
      if constexpr (SHIFTED)
        fi = wi * ((double)P.rho0 + (double)q[i] * (double)P.inv_s);
      else
        fi = (double)q[i];
      constexpr double cx = L::CX[i], cy = L::CY[i], c_sq = cx * cx + cy * cy;
      r += fi;
      if constexpr (cx != 0.0) jx += cx * fi;
      if constexpr (cy != 0.0) jy += cy * fi;
      if constexpr (c_sq != 0.0) e2 += c_sq * fi;
    });
    const double uxd = jx / r, uyd = jy / r;
    const double theta = (e2 / r - uxd * uxd - uyd * uyd) / (2.0 * c2);
    rho = (Real)r;
    ux = (Real)uxd;
    uy = (Real)uyd;
    e = (Real)(c2 * (theta - 1.0));
  } else {
    Real irho;
    if constexpr (SHIFTED) {
      rho = madd(drho, P.inv_s, P.rho0);
      irho = recip(rho) * P.inv_s;  // also takes the momentum out of storage units
    } else {
      rho = Real(1) + drho;
      irho = recip(rho);
    }
    ux = hmom(IC<1>{}, IC<0>{}) * irho;
    uy = hmom(IC<0>{}, IC<1>{}) * irho;
  }

  Real A[5][5];
  equilibrium_coefficients<L, THERMAL>(rho, ux, uy, e, A);

  // B = s a1, from the moments in storage units minus s a0 where f^(0) carries the order
  Real B[5][5];
  if constexpr (COLL == COLL_PR) {
    // a1^(n) = sum_i H^(n)_i (f_i - f_i^(0)), n = 2..N (Sec. II.E); by orthogonality of the kept
    // basis, sum_i H_i f_i^(0) = a0 on the orders f^(0) carries and 0 above them.
    sfor<2, L::NMAX + 1>([&](auto N) {
      constexpr int n = LBM_CI(N);
      sfor<0, n + 1>([&](auto Aa) {
        constexpr int a = LBM_CI(Aa);
        constexpr int b = n - a;
        if constexpr (L::keep(a, b)) {
          Real v;
          if constexpr (n <= 2)
            v = hmom(IC<a>{}, IC<b>{});
          else
            v = hmom_direct(IC<a>{}, IC<b>{});
          B[a][b] = madd(A[a][b], P.msn[n], v);
        }
      });
    });
  } else if constexpr (COLL == COLL_RR && FD) {
    const Real th = THERMAL ? Real(1) + e * Real(1.0 / c2) : Real(1);
    Real pre = -P.tau * rho * Real(c2) * th;
    if constexpr (SHIFTED) pre = pre * P.s;
    const Real div = THERMAL ? grad[0] + grad[3] : Real(0);
    B[2][0] = pre * (Real(2) * grad[0] - div);
    B[1][1] = pre * (grad[1] + grad[2]);
    B[0][2] = pre * (Real(2) * grad[3] - div);
    a1_third_from_second<L, THERMAL>(ux, uy, B);
    if constexpr (THERMAL && L::NMAX >= 3) {
      Real mu_cs2 = P.tau3 * rho * Real(c2) * th * Real(c2);
      if constexpr (SHIFTED) mu_cs2 = mu_cs2 * P.s;
      const Real gx = mu_cs2 * grad[4], gy = mu_cs2 * grad[5];
      B[3][0] -= Real(3) * gx;
      B[2][1] -= gy;
      B[1][2] -= gx;
      B[0][3] -= Real(3) * gy;
    }
    a1_fourth<L, THERMAL>(ux, uy, e, B);
  } else if constexpr (COLL == COLL_RR) {
    B[2][0] = madd(A[2][0], P.msn[2], hmom(IC<2>{}, IC<0>{}));
    B[1][1] = madd(A[1][1], P.msn[2], hmom(IC<1>{}, IC<1>{}));
    B[0][2] = madd(A[0][2], P.msn[2], hmom(IC<0>{}, IC<2>{}));
    if constexpr (CLOSURE) {
      if constexpr (SHIFTED) {
        B[2][0] = madd(da[0], P.s, B[2][0]);
        B[1][1] = madd(da[1], P.s, B[1][1]);
        B[0][2] = madd(da[2], P.s, B[0][2]);
      } else {
        B[2][0] += da[0];
        B[1][1] += da[1];
        B[0][2] += da[2];
      }
    }
    a1_third_from_second<L, THERMAL>(ux, uy, B);
    if constexpr (THERMAL && L::NMAX >= 3) {
      // App. C steps 2-4: projected a1^(3), averaged temperature-gradient terms, rebuilt a1^(3)
      const Real p30 = madd(A[3][0], P.msn[3], hmom(IC<3>{}, IC<0>{}));
      const Real p21 = madd(A[2][1], P.msn[3], hmom(IC<2>{}, IC<1>{}));
      const Real p12 = madd(A[1][2], P.msn[3], hmom(IC<1>{}, IC<2>{}));
      const Real p03 = madd(A[0][3], P.msn[3], hmom(IC<0>{}, IC<3>{}));
      const Real third = Real(1) / Real(3);
      const Real gx = Real(0.5) * ((ux * B[2][0] - p30 * third) + (Real(2) * uy * B[1][1] + ux * B[0][2] - p12));
      const Real gy = Real(0.5) * ((uy * B[0][2] - p03 * third) + (Real(2) * ux * B[1][1] + uy * B[2][0] - p21));
      B[3][0] -= Real(3) * gx;
      B[2][1] -= gy;
      B[1][2] -= gx;
      B[0][3] -= Real(3) * gy;
    }
    a1_fourth<L, THERMAL>(ux, uy, e, B);
  }

  // --- coefficients of the rebuilt populations (Eq. GenRegCollision), minus the reference, in storage
  // units: C = ka a0 + kb s a1 (the factors hold the orders kept, the relaxation and 1 / (a! b! cs^2n)) ---
  Real C[5][5];
  sfor<0, L::NMAX + 1>([&](auto N) {
    constexpr int n = LBM_CI(N);
    sfor<0, n + 1>([&](auto Aa) {
      constexpr int a = LBM_CI(Aa);
      constexpr int b = n - a;
      if constexpr (L::keep(a, b)) {
        constexpr int k = coef_index(a, b);
        if constexpr (n == 0) {
          C[0][0] = (COLL == COLL_BGK) ? P.omega * drho : drho;  // s (a0^(0) - rho_ref)
        } else if constexpr (CoefFactors<L>::value) {
          if constexpr (COLL == COLL_BGK || n == 1)
            C[a][b] = P.ka[k] * A[a][b];
          else
            C[a][b] = madd(P.kb[k], B[a][b], P.ka[k] * A[a][b]);
        } else {
          constexpr double sc = 1.0 / (factorial(a) * factorial(b) * ipow(c2, n));
          Real v = (n <= P.neq) ? A[a][b] : Real(0);
          if constexpr (SHIFTED) v = v * P.s;
          if constexpr (COLL == COLL_BGK) {
            v = v * P.omega;
          } else if constexpr (n >= 2) {
            if (n <= P.nreg) v = madd(n == 2 ? P.om1 : (n == 3 ? P.om1_3 : P.om1_4), B[a][b], v);
          }
          C[a][b] = v * Real(sc);
        }
      }
    });
  });

  // plain storage: f*_i = w^_i + w_i (...); shifted: q*_i = s (f*_i / w_i - rho0) = (...)
  if constexpr (COLL == COLL_BGK) {
    // f* - ref = (1 - 1/tau)(f - ref) + (f^(0) - ref) / tau  (Sec. III.A)
    auto emit_bgk = [&](auto I, Real acc) {
      constexpr int i = LBM_CI(I);
      const Real dv = madd(P.om1, d[i], acc);
      const Real v = SHIFTED ? dv : Real(ref_weight<L, Sc>(i)) + dv;
      if constexpr (std::is_same<std::decay_t<Out>, KeepInQ>::value)
        q[i] = v;
      else
        out(I, v);
    };
    if constexpr (std::is_same<std::decay_t<Out>, KeepInQ>::value)
      rebuild<L, SHIFTED>(C, emit_bgk);
    else
      rebuild_rows<L, SHIFTED>(C, emit_bgk);
  } else {
    // f* = f^(0) + (1 - 1/tau) f^(1)  (Eq. RegularizedCollision)
    auto emit = [&](auto I, Real acc) {
      constexpr int i = LBM_CI(I);
      const Real v = SHIFTED ? acc : Real(ref_weight<L, Sc>(i)) + acc;
      if constexpr (std::is_same<std::decay_t<Out>, KeepInQ>::value)
        q[i] = v;
      else
        out(I, v);
    };
    if constexpr (std::is_same<std::decay_t<Out>, KeepInQ>::value)
      rebuild<L, SHIFTED>(C, emit);
    else
      rebuild_rows<L, SHIFTED>(C, emit);
  }
}

// Host side: the per-coefficient factors ka, kb and msn of CollParams for a 2D lattice L (coll: COLL_*).
template <class L, class Real>
inline void set_coef_factors(CollParams<Real>& p, int coll, int neq, int nreg, double omega, double om1,
                             double om1_3, double om1_4, double s) {
  using Sc = typename Scalar<Real>::type;
  for (int n = 0; n <= 4; ++n) {
    p.msn[n] = Real((Sc)(n <= neq ? -s : 0.0));
    const double om = n == 2 ? om1 : (n == 3 ? om1_3 : om1_4);
    for (int a = 0; a <= n; ++a) {
      const int b = n - a;
      const double sc = 1.0 / (factorial(a) * factorial(b) * ipow(L::CS2, n));
      double ka = n <= neq ? s * sc : 0.0;
      double kb = (n >= 2 && n <= nreg) ? om * sc : 0.0;
      if (coll == COLL_BGK) {
        ka *= omega;
        kb = 0.0;
      }
      p.ka[coef_index(a, b)] = Real((Sc)ka);
      p.kb[coef_index(a, b)] = Real((Sc)kb);
    }
  }
}

// ---------------------------------------------------------------------------
// Macroscopic fields of one cell's pulled populations (Sec. II.A), as the collision computes them: rho and
// u from the deviations (FP32 or FP64), theta from the FP64 energy moment on thermal lattices (1 otherwise).
// Used by the moments pass of the finite-difference variant.
// ---------------------------------------------------------------------------
template <class L, bool THERMAL, bool SHIFTED, class Real>
__device__ __forceinline__ void cell_macro(const Real (&q)[L::Q], const CollParams<Real>& P, Real& rho, Real& ux,
                                           Real& uy, Real& theta) {
  using Sc = typename Scalar<Real>::type;
  if constexpr (THERMAL) {
    double r = 0.0, jx = 0.0, jy = 0.0, e2 = 0.0;
    sfor<0, L::Q>([&](auto I) {
      constexpr int i = LBM_CI(I);
      constexpr double wi = L::W[i];
      double fi;
      if constexpr (SHIFTED)
        fi = wi * ((double)P.rho0 + (double)q[i] * (double)P.inv_s);
      else
        fi = (double)q[i];
      constexpr double cx = L::CX[i], cy = L::CY[i];
      r += fi;
      if constexpr (cx != 0.0) jx += cx * fi;
      if constexpr (cy != 0.0) jy += cy * fi;
      if constexpr (cx * cx + cy * cy != 0.0) e2 += (cx * cx + cy * cy) * fi;
    });
    const double uxd = jx / r, uyd = jy / r;
    rho = (Real)r;
    ux = (Real)uxd;
    uy = (Real)uyd;
    theta = (Real)((e2 / r - uxd * uxd - uyd * uyd) / (2.0 * L::CS2));
  } else {
    Real d0 = Real(0), dx = Real(0), dy = Real(0);
    sfor<0, L::Q>([&](auto I) {
      constexpr int i = LBM_CI(I);
      constexpr double wf = SHIFTED ? L::W[i] : 1.0;
      constexpr double cxw = L::CX[i] * wf, cyw = L::CY[i] * wf;
      Real di;
      if constexpr (SHIFTED)
        di = q[i];
      else
        di = q[i] - Real(ref_weight<L, Sc>(i));
      d0 = madd(Real(wf), di, d0);
      if constexpr (cxw != 0.0) dx = madd(Real(cxw), di, dx);
      if constexpr (cyw != 0.0) dy = madd(Real(cyw), di, dy);
    });
    if constexpr (SHIFTED) {
      d0 = d0 * P.inv_s;
      dx = dx * P.inv_s;
      dy = dy * P.inv_s;
      rho = P.rho0 + d0;
    } else {
      rho = Real(1) + d0 + Real(kappa<L, Sc>(0, 0));
      dx = dx + Real(kappa<L, Sc>(1, 0));
      dy = dy + Real(kappa<L, Sc>(0, 1));
    }
    const Real irho = Real(1) / rho;
    ux = dx * irho;
    uy = dy * irho;
    theta = Real(1);
  }
}

}  // namespace lbm
