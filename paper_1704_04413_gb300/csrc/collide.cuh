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
// Rebuild: out_i = sum_{(a,b) kept} K_i He(a, cx_i) He(b, cy_i) C[a][b], with
// K_i = w_i for plain storage and 1 for shifted storage (whose C carry the
// factor s and whose w_i cancels).  Factorised by rows of equal cy:
//   g[a](v) = sum_b He(b, v) C[a][b],   out_i = sum_a K_i He(a, cx_i) g[a](cy_i),
// and g[a](+-v) = E +- O with E/O the even/odd-b parts.
// ---------------------------------------------------------------------------
template <class L, bool SHIFTED, class Real, class F>
__device__ __forceinline__ void rebuild(const Real (&C)[5][5], F&& emit) {
  constexpr double c2 = L::CS2;
  constexpr int V = L::VMAX;
  Real g[5][2 * V + 1];
  sfor<0, V + 1>([&](auto VV) {
    constexpr int v = LBM_CI(VV);
    if constexpr (has_row<L>(v) || has_row<L>(-v)) {
      sfor<0, L::NMAX + 1>([&](auto Aa) {
        constexpr int a = LBM_CI(Aa);
        if constexpr (L::keep(a, 0)) {
        Real ev = Real(0), od = Real(0);
        sfor<0, L::NMAX + 1 - a>([&](auto Bb) {
          constexpr int b = LBM_CI(Bb);
          constexpr double h = he(b, v, c2);
          if constexpr (L::keep(a, b) && h != 0.0) {
            if constexpr (b % 2 == 0)
              ev = madd(Real(h), C[a][b], ev);
            else
              od = madd(Real(h), C[a][b], od);
          }
        });
        g[a][V + v] = ev + od;
        if constexpr (v != 0) g[a][V - v] = ev - od;
        }
      });
    }
  });
  sfor<0, L::Q>([&](auto I) {
    constexpr int i = LBM_CI(I);
    constexpr int v = L::CY[i];
    Real acc = Real(0);
    sfor<0, L::NMAX + 1>([&](auto Aa) {
      constexpr int a = LBM_CI(Aa);
      constexpr double h = he(a, L::CX[i], c2) * (SHIFTED ? 1.0 : L::W[i]);
      if constexpr (h != 0.0 && L::keep(a, 0)) acc = madd(Real(h), g[a][V + v], acc);
    });
    emit(I, acc);
  });
}

template <class L, bool SHIFTED, class Real, class F>
__device__ __forceinline__ void rebuild_rows(const Real (&C)[5][5], F&& emit) {
  constexpr double c2 = L::CS2;
  constexpr int V = L::VMAX;
  // rebuild() one row pair +-v at a time: its g[a](+-v) are made, its populations emitted, and the g die,
  // so that a caller storing each emitted population at once never holds more than one row pair's g
  sfor<0, V + 1>([&](auto VV) {
    constexpr int v = LBM_CI(VV);
    if constexpr (has_row<L>(v) || has_row<L>(-v)) {
      Real gp[5], gm[5];
      sfor<0, L::NMAX + 1>([&](auto Aa) {
        constexpr int a = LBM_CI(Aa);
        if constexpr (L::keep(a, 0)) {
          Real ev = Real(0), od = Real(0);
          sfor<0, L::NMAX + 1 - a>([&](auto Bb) {
            constexpr int b = LBM_CI(Bb);
            constexpr double h = he(b, v, c2);
            if constexpr (L::keep(a, b) && h != 0.0) {
              if constexpr (b % 2 == 0)
                ev = madd(Real(h), C[a][b], ev);
              else
                od = madd(Real(h), C[a][b], od);
            }
          });
          gp[a] = ev + od;
          if constexpr (v != 0) gm[a] = ev - od;
        }
      });
      sfor<0, L::Q>([&](auto I) {
        constexpr int i = LBM_CI(I);
        if constexpr (L::CY[i] == v || (v != 0 && L::CY[i] == -v)) {
          constexpr bool up = L::CY[i] == v;
          Real acc = Real(0);
          sfor<0, L::NMAX + 1>([&](auto Aa) {
            constexpr int a = LBM_CI(Aa);
            constexpr double h = he(a, L::CX[i], c2) * (SHIFTED ? 1.0 : L::W[i]);
            if constexpr (h != 0.0 && L::keep(a, 0)) {
              if constexpr (up)
                acc = madd(Real(h), gp[a], acc);
              else
                acc = madd(Real(h), gm[a], acc);
            }
          });
          emit(I, acc);
        }
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
template <class L, int COLL, bool THERMAL, bool SHIFTED, class Real, bool CLOSURE = false, bool FD = false,
          class Out = KeepInQ>
__device__ __forceinline__ void collide(Real (&q)[L::Q], const CollParams<Real>& P, const Real* da = nullptr,
                                        const Real* grad = nullptr, Out&& out = Out{}) {
  using Sc = typename Scalar<Real>::type;
  static_assert(!(THERMAL && !__is_same(Sc, Real)), "the thermal path computes one cell per thread");
  constexpr double c2 = L::CS2;
  // highest monomial order of f the mode needs (PR takes its orders >= 3 directly, hmom_direct below)
  constexpr int PM = (COLL == COLL_PR) ? 2 : (COLL == COLL_RR ? (THERMAL ? 3 : 2) : 1);
  const Real rho_ref = SHIFTED ? P.rho0 : Real(1);

  // deviations from the reference (plain storage); shifted storage holds them already
  Real d[L::Q];
  sfor<0, L::Q>([&](auto I) {
    constexpr int i = LBM_CI(I);
    if constexpr (SHIFTED)
      d[i] = q[i];
    else
      d[i] = q[i] - Real(ref_weight<L, Sc>(i));
  });

  // --- monomial moments of the deviations D[k][l] = sum_i d_i cx^k cy^l (Sec. II.A) ---
  Real D[5][5];
  sfor<0, 5>([&](auto K) {
    constexpr int k = LBM_CI(K);
    sfor<0, 5 - k>([&](auto Lq) {
      constexpr int l = LBM_CI(Lq);
      if constexpr (L::keep(k, l) && k + l <= PM) {
        Real acc = Real(0);
        sfor<0, L::Q>([&](auto I) {
          constexpr int i = LBM_CI(I);
          constexpr double c = ipow(L::CX[i], k) * ipow(L::CY[i], l) * (SHIFTED ? L::W[i] : 1.0);
          if constexpr (c != 0.0) acc = madd(Real(c), d[i], acc);
        });
        D[k][l] = SHIFTED ? acc * P.inv_s : acc;
      }
    });
  });

  // Hermite moments of f (see above)
  auto hmom = [&](auto Aa, auto Bb) -> Real {
    constexpr int a = LBM_CI(Aa);
    constexpr int b = LBM_CI(Bb);
    Real acc = Real(0);
    sfor<0, a + 1>([&](auto K) {
      constexpr int k = LBM_CI(K);
      sfor<0, b + 1>([&](auto Lq) {
        constexpr int l = LBM_CI(Lq);
        constexpr double h = he_coef(a, k, c2) * he_coef(b, l, c2);
        if constexpr (h != 0.0) acc = madd(Real(h), D[k][l], acc);
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
    Real acc = Real(0);
    sfor<0, L::Q>([&](auto I) {
      constexpr int i = LBM_CI(I);
      constexpr double c = he(a, L::CX[i], c2) * he(b, L::CY[i], c2) * (SHIFTED ? L::W[i] : 1.0);
      if constexpr (c != 0.0) acc = madd(Real(c), d[i], acc);
    });
    if constexpr (SHIFTED) {
      acc = acc * P.inv_s;
    } else {
      constexpr double kp = kappa<L, Sc>(a, b);
      if constexpr (kp != 0.0) acc += Real(kp);
    }
    return acc;
  };

  const Real drho = hmom(IC<0>{}, IC<0>{});  // rho - rho_ref
  Real rho = rho_ref + drho;
  Real ux, uy, e = Real(0);
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
    const Real irho = Real(1) / rho;
    ux = hmom(IC<1>{}, IC<0>{}) * irho;
    uy = hmom(IC<0>{}, IC<1>{}) * irho;
  }

  Real A[5][5];
  equilibrium_coefficients<L, THERMAL>(rho, ux, uy, e, A);

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
          if (n <= P.neq) v -= A[a][b];
          B[a][b] = v;
        }
      });
    });
  } else if constexpr (COLL == COLL_RR && FD) {
    const Real th = THERMAL ? Real(1) + e * Real(1.0 / c2) : Real(1);
    const Real pre = -P.tau * rho * Real(c2) * th;
    const Real div = THERMAL ? grad[0] + grad[3] : Real(0);
    B[2][0] = pre * (Real(2) * grad[0] - div);
    B[1][1] = pre * (grad[1] + grad[2]);
    B[0][2] = pre * (Real(2) * grad[3] - div);
    a1_third_from_second<L, THERMAL>(ux, uy, B);
    if constexpr (THERMAL && L::NMAX >= 3) {
      const Real mu_cs2 = P.tau3 * rho * Real(c2) * th * Real(c2);
      const Real gx = mu_cs2 * grad[4], gy = mu_cs2 * grad[5];
      B[3][0] -= Real(3) * gx;
      B[2][1] -= gy;
      B[1][2] -= gx;
      B[0][3] -= Real(3) * gy;
    }
    a1_fourth<L, THERMAL>(ux, uy, e, B);
  } else if constexpr (COLL == COLL_RR) {
    B[2][0] = hmom(IC<2>{}, IC<0>{}) - A[2][0];
    B[1][1] = hmom(IC<1>{}, IC<1>{}) - A[1][1];
    B[0][2] = hmom(IC<0>{}, IC<2>{}) - A[0][2];
    if constexpr (CLOSURE) {
      B[2][0] += da[0];
      B[1][1] += da[1];
      B[0][2] += da[2];
    }
    a1_third_from_second<L, THERMAL>(ux, uy, B);
    if constexpr (THERMAL && L::NMAX >= 3) {
      // App. C steps 2-4: projected a1^(3), averaged temperature-gradient terms, rebuilt a1^(3)
      const bool eq3 = 3 <= P.neq;
      const Real p30 = hmom(IC<3>{}, IC<0>{}) - (eq3 ? A[3][0] : Real(0));
      const Real p21 = hmom(IC<2>{}, IC<1>{}) - (eq3 ? A[2][1] : Real(0));
      const Real p12 = hmom(IC<1>{}, IC<2>{}) - (eq3 ? A[1][2] : Real(0));
      const Real p03 = hmom(IC<0>{}, IC<3>{}) - (eq3 ? A[0][3] : Real(0));
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

  // --- coefficients of the rebuilt populations (Eq. GenRegCollision), minus the reference ---
  Real C[5][5];
  sfor<0, L::NMAX + 1>([&](auto N) {
    constexpr int n = LBM_CI(N);
    sfor<0, n + 1>([&](auto Aa) {
      constexpr int a = LBM_CI(Aa);
      constexpr int b = n - a;
      if constexpr (L::keep(a, b)) {
        constexpr double sc = 1.0 / (factorial(a) * factorial(b) * ipow(c2, a + b));
        Real v;
        if constexpr (n == 0)
          v = drho;  // a0^(0) - rho_ref
        else
          v = (n <= P.neq) ? A[a][b] : Real(0);
        if constexpr (COLL == COLL_BGK) {
          v *= P.omega;
        } else if constexpr (n >= 2) {
          if (n <= P.nreg) v += (n == 2 ? P.om1 : (n == 3 ? P.om1_3 : P.om1_4)) * B[a][b];
        }
        if constexpr (SHIFTED) v *= P.s;
        C[a][b] = v * Real(sc);
      }
    });
  });

  // plain storage: f*_i = w^_i + w_i (...); shifted: q*_i = s (f*_i / w_i - rho0) = (...)
  if constexpr (COLL == COLL_BGK) {
    // f* - ref = (1 - 1/tau)(f - ref) + (f^(0) - ref) / tau  (Sec. III.A)
    auto emit_bgk = [&](auto I, Real acc) {
      constexpr int i = LBM_CI(I);
      const Real dv = P.om1 * d[i] + acc;
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
