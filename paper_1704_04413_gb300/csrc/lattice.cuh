// Lattice tables of the three 2D velocity sets (Tab. I) as compile-time
// constants.  Every per-population coefficient the kernels use (velocity
// components, weights, Hermite values) is a constant expression, so it is
// folded into the instruction stream as an immediate: no table is read from
// memory at run time.
//
// Velocity order is the library's own (exported by lbm_lattice_info).
#pragma once

namespace lbm {

template <int N>
struct IC {
  static constexpr int value = N;
};

// Compile-time loop: f(IC<B>{}), ..., f(IC<E-1>{}).
template <int B, int E, class F>
__host__ __device__ __forceinline__ void sfor(F&& f) {
  if constexpr (B < E) {
    f(IC<B>{});
    sfor<B + 1, E>(f);
  }
}

__host__ __device__ constexpr double ipow(double x, int n) {
  double r = 1.0;
  for (int k = 0; k < n; ++k) r *= x;
  return r;
}
__host__ __device__ constexpr double factorial(int n) {
  double r = 1.0;
  for (int k = 2; k <= n; ++k) r *= k;
  return r;
}

// One-dimensional factor of the 2D Hermite tensors (App. C, 2D forms): a
// tensor with a x-indices and b y-indices is He(a, xi_x) He(b, xi_y).
__host__ __device__ constexpr double he(int a, double x, double c2) {
  return a == 0 ? 1.0
       : a == 1 ? x
       : a == 2 ? x * x - c2
       : a == 3 ? (x * x - 3.0 * c2) * x
       : a == 4 ? x * x * x * x - 6.0 * c2 * x * x + 3.0 * c2 * c2
                : 0.0;
}
// Coefficient of x^k in he(a, x, c2).
__host__ __device__ constexpr double he_coef(int a, int k, double c2) {
  return (a == 0) ? (k == 0 ? 1.0 : 0.0)
       : (a == 1) ? (k == 1 ? 1.0 : 0.0)
       : (a == 2) ? (k == 2 ? 1.0 : k == 0 ? -c2 : 0.0)
       : (a == 3) ? (k == 3 ? 1.0 : k == 1 ? -3.0 * c2 : 0.0)
       : (a == 4) ? (k == 4 ? 1.0 : k == 2 ? -6.0 * c2 : k == 0 ? 3.0 * c2 * c2 : 0.0)
                  : 0.0;
}

// D2Q9 = E^9_{2,5}.  Complete basis: every He(a) He(b) with a, b <= 2.
struct D2Q9 {
  static constexpr int ID = 0;
  static constexpr int Q = 9;
  static constexpr int VMAX = 1;
  static constexpr int NMAX = 4;
  static constexpr int CX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  static constexpr int CY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  static constexpr double W[Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                                  1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
  static constexpr double CS2 = 1.0 / 3.0;
  __host__ __device__ static constexpr bool keep(int a, int b) { return a <= 2 && b <= 2; }
};

// D2V17 = E^17_{2,7}.  Basis: all tensors of order <= 3.
// Weights: (575+193 s)/8100, (3355-91 s)/18000, (655+17 s)/27000,
// (685-49 s)/54000, (1445-101 s)/162000 with s = sqrt(193); 1/c_s^2 = 5(25+s)/72.
struct D2V17 {
  static constexpr int ID = 1;
  static constexpr int Q = 17;
  static constexpr int VMAX = 3;
  static constexpr int NMAX = 3;
  static constexpr int CX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1, 2, -2, -2, 2, 3, 0, -3, 0};
  static constexpr int CY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1, 2, 2, -2, -2, 0, 3, 0, -3};
  static constexpr double W0 = 0.402005146909112625941664392459;
  static constexpr double W10 = 0.116154866497781543874035456626;
  static constexpr double W11 = 0.0330063536229869139497538259147;
  static constexpr double W22 = 0.0000790786021659181312371332405497;
  static constexpr double W30 = 0.00025841454978746755955748610405;
  static constexpr double W[Q] = {W0,  W10, W10, W10, W10, W11, W11, W11, W11,
                                  W22, W22, W22, W22, W30, W30, W30, W30};
  static constexpr double CS2 = 0.370251867018339849718915098632;
  __host__ __device__ static constexpr bool keep(int a, int b) { return a + b <= 3; }
};

// D2V37 = E^37_{2,9}.  Basis: all tensors of order <= 4.  1/c_s = 1.19697977039307435897239.
struct D2V37 {
  static constexpr int ID = 2;
  static constexpr int Q = 37;
  static constexpr int VMAX = 3;
  static constexpr int NMAX = 4;
  static constexpr int CX[Q] = {0,                                  // (0,0)
                                1,  0,  -1, 0,                      // (1,0)
                                1,  -1, -1, 1,                      // (1,1)
                                2,  0,  -2, 0,                      // (2,0)
                                2,  1,  -1, -2, -2, -1, 1,  2,      // (2,1)
                                2,  -2, -2, 2,                      // (2,2)
                                3,  0,  -3, 0,                      // (3,0)
                                3,  1,  -1, -3, -3, -1, 1,  3};     // (3,1)
  static constexpr int CY[Q] = {0,
                                0,  1,  0,  -1,
                                1,  1,  -1, -1,
                                0,  2,  0,  -2,
                                1,  2,  2,  1,  -1, -2, -2, -1,
                                2,  2,  -2, -2,
                                0,  3,  0,  -3,
                                1,  3,  3,  1,  -1, -3, -3, -1};
  static constexpr double W00 = 0.23315066913235250228650;
  static constexpr double W10 = 0.10730609154221900241246;
  static constexpr double W11 = 0.05766785988879488203006;
  static constexpr double W20 = 0.01420821615845075026469;
  static constexpr double W21 = 0.00535304900051377523273;
  static constexpr double W22 = 0.00101193759267357547541;
  static constexpr double W30 = 0.00024530102775771734547;
  static constexpr double W31 = 0.00028341425299419821740;
  static constexpr double W[Q] = {W00, W10, W10, W10, W10, W11, W11, W11, W11, W20, W20, W20, W20,
                                  W21, W21, W21, W21, W21, W21, W21, W21, W22, W22, W22, W22,
                                  W30, W30, W30, W30, W31, W31, W31, W31, W31, W31, W31, W31};
  static constexpr double ICS = 1.19697977039307435897239;
  static constexpr double CS2 = 1.0 / (ICS * ICS);
  __host__ __device__ static constexpr bool keep(int a, int b) { return a + b <= 4; }
};

// sum_i w_i cx_i^p cy_i^q (the constant part of a shifted-storage moment)
template <class L>
__host__ __device__ constexpr double weight_moment(int p, int q) {
  double s = 0.0;
  for (int i = 0; i < L::Q; ++i) s += L::W[i] * ipow(L::CX[i], p) * ipow(L::CY[i], q);
  return s;
}

// number of populations with velocity component cy == v
template <class L>
__host__ __device__ constexpr bool has_row(int v) {
  for (int i = 0; i < L::Q; ++i)
    if (L::CY[i] == v) return true;
  return false;
}

}  // namespace lbm
