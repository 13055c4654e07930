// Per-cell arithmetic of the regularized step on the 3D lattices of Tab. II, isothermal (theta = 1): the
// same scheme as the 2D collide() (Sec. II.A moments, App. B equilibrium, projection Sec. II.E or recursion
// Eq. MalaspinasRecursiveRelation, rebuild Eq. GenRegCollision with one relaxation time) with coefficients
// X[a][b][c] for a x-, b y- and c z-indices, multiplicity folded into 1 / (a! b! c! cs^2(a+b+c)).
//
// a1 of order >= 3 (RR) is the closed form of the isothermal recursion: the sum over index pairs of
// a1^(2)_pair times the velocity components of the other indices,
//   a1[a][b][c] = C(a,2) a1_xx ux^(a-2) uy^b uz^c + C(b,2) a1_yy ... + C(c,2) a1_zz ...
//               + a b a1_xy ux^(a-1) uy^(b-1) uz^c + a c a1_xz ... + b c a1_yz ...
#pragma once
#include "collide.cuh"
#include "lattice3.cuh"

namespace lbm {

template <class L, class Real>
__host__ __device__ constexpr double kappa3(int a, int b, int c) {
  double s = 0.0;
  for (int i = 0; i < L::Q; ++i)
    s += he(a, L::CX[i], L::CS2) * he(b, L::CY[i], L::CS2) * he(c, L::CZ[i], L::CS2) *
         ((double)(Real)L::W[i] - L::W[i]);
  return s;
}

__host__ __device__ constexpr int choose2(int n) { return n * (n - 1) / 2; }

// sum_i w_i H_(a,b,c)(xi_i) H_(d,e,f)(xi_i) / (d! e! f! cs^2(d+e+f)): the projection onto H_(a,b,c) of the
// expansion term of H_(d,e,f).  1 on the diagonal and 0 elsewhere on an orthonormal basis; D3Q19's
// third-order tensors that share their odd axis (H_xxy and H_yzz, ...) are the exception of Tab. II's
// bases, so PR subtracts the projection of the truncated f^(0) through this matrix, not a0 itself.
template <class L>
__host__ __device__ constexpr double gram3(int a, int b, int c, int d, int e, int f) {
  double s = 0.0;
  for (int i = 0; i < L::Q; ++i)
    s += L::W[i] * he(a, L::CX[i], L::CS2) * he(b, L::CY[i], L::CS2) * he(c, L::CZ[i], L::CS2) *
         he(d, L::CX[i], L::CS2) * he(e, L::CY[i], L::CS2) * he(f, L::CZ[i], L::CS2);
  s /= factorial(d) * factorial(e) * factorial(f) * ipow(L::CS2, d + e + f);
  if (a == d && b == e && c == f && s > 1.0 - 1e-12 && s < 1.0 + 1e-12) return 1.0;
  return (s > -1e-12 && s < 1e-12) ? 0.0 : s;
}

// Whether the kept tensors up to order `pm` need the monomial moment x^k y^l z^m.
template <class L>
__host__ __device__ constexpr bool needs_monomial(int k, int l, int m, int pm) {
  for (int a = k; a <= 4; ++a)
    for (int b = l; b <= 4; ++b)
      for (int c = m; c <= 4; ++c)
        if (a + b + c <= pm && L::keep(a, b, c) && (a - k) % 2 == 0 && (b - l) % 2 == 0 && (c - m) % 2 == 0)
          return true;
  return false;
}

template <class L, int COLL, bool SHIFTED, class Real>
__device__ __forceinline__ void collide3(Real (&q)[L::Q], const CollParams<Real>& P) {
  using Sc = typename Scalar<Real>::type;
  constexpr double c2 = L::CS2;
  constexpr int PM = COLL == COLL_PR ? L::NMAX : (COLL == COLL_RR ? 2 : 1);
  const Real rho_ref = SHIFTED ? P.rho0 : Real(1);

  Real d[L::Q];
  sfor<0, L::Q>([&](auto I) {
    constexpr int i = LBM_CI(I);
    [[maybe_unused]] constexpr double wr = (double)(Sc)L::W[i];
    if constexpr (SHIFTED)
      d[i] = q[i];
    else
      d[i] = q[i] - Real(wr);
  });

  // monomial moments of the deviations, D[k][l][m] = sum_i d_i cx^k cy^l cz^m (Sec. II.A)
  Real D[5][5][5];
  sfor<0, PM + 1>([&](auto K) {
    constexpr int k = LBM_CI(K);
    sfor<0, PM + 1 - k>([&](auto Lq) {
      constexpr int l = LBM_CI(Lq);
      sfor<0, PM + 1 - k - l>([&](auto M) {
        constexpr int m = LBM_CI(M);
        if constexpr (k <= 4 && l <= 4 && m <= 4 && needs_monomial<L>(k, l, m, PM)) {
          Real acc = Real(0);
          sfor<0, L::Q>([&](auto I) {
            constexpr int i = LBM_CI(I);
            constexpr double c = ipow(L::CX[i], k) * ipow(L::CY[i], l) * ipow(L::CZ[i], m) *
                                 (SHIFTED ? L::W[i] : 1.0);
            if constexpr (c != 0.0) acc = madd(Real(c), d[i], acc);
          });
          D[k][l][m] = SHIFTED ? acc * P.inv_s : acc;
        }
      });
    });
  });
  // Hermite moments of f: He expanded in monomials, plus the rounded-weight correction (plain storage)
  auto hmom = [&](auto Aa, auto Bb, auto Cc) -> Real {
    constexpr int a = LBM_CI(Aa), b = LBM_CI(Bb), c = LBM_CI(Cc);
    Real acc = Real(0);
    sfor<0, a + 1>([&](auto K) {
      constexpr int k = LBM_CI(K);
      sfor<0, b + 1>([&](auto Lq) {
        constexpr int l = LBM_CI(Lq);
        sfor<0, c + 1>([&](auto M) {
          constexpr int m = LBM_CI(M);
          constexpr double h = he_coef(a, k, c2) * he_coef(b, l, c2) * he_coef(c, m, c2);
          if constexpr (h != 0.0) acc = madd(Real(h), D[k][l][m], acc);
        });
      });
    });
    if constexpr (!SHIFTED) {
      constexpr double kp = kappa3<L, Sc>(a, b, c);
      if constexpr (kp != 0.0) acc += Real(kp);
    }
    return acc;
  };

  const Real drho = hmom(IC<0>{}, IC<0>{}, IC<0>{});
  const Real rho = rho_ref + drho;
  const Real irho = Real(1) / rho;
  const Real u[3] = {hmom(IC<1>{}, IC<0>{}, IC<0>{}) * irho, hmom(IC<0>{}, IC<1>{}, IC<0>{}) * irho,
                     hmom(IC<0>{}, IC<0>{}, IC<1>{}) * irho};
  Real pw[3][5];  // u_d^k
  sfor<0, 3>([&](auto Dd) {
    constexpr int dd = LBM_CI(Dd);
    pw[dd][0] = Real(1);
    sfor<1, 5>([&](auto K) {
      constexpr int k = LBM_CI(K);
      pw[dd][k] = pw[dd][k - 1] * u[dd];
    });
  });

  // a1^(2) (PR and RR); the six components xx, yy, zz, xy, xz, yz
  Real b2[6];
  if constexpr (COLL != COLL_BGK) {
    b2[0] = hmom(IC<2>{}, IC<0>{}, IC<0>{}) - rho * pw[0][2];
    b2[1] = hmom(IC<0>{}, IC<2>{}, IC<0>{}) - rho * pw[1][2];
    b2[2] = hmom(IC<0>{}, IC<0>{}, IC<2>{}) - rho * pw[2][2];
    b2[3] = hmom(IC<1>{}, IC<1>{}, IC<0>{}) - rho * pw[0][1] * pw[1][1];
    b2[4] = hmom(IC<1>{}, IC<0>{}, IC<1>{}) - rho * pw[0][1] * pw[2][1];
    b2[5] = hmom(IC<0>{}, IC<1>{}, IC<1>{}) - rho * pw[1][1] * pw[2][1];
  }

  // coefficients of the rebuilt populations minus the reference, per kept tensor
  Real C[5][5][5];
  sfor<0, 5>([&](auto Aa) {
    constexpr int a = LBM_CI(Aa);
    sfor<0, 5>([&](auto Bb) {
      constexpr int b = LBM_CI(Bb);
      sfor<0, 5>([&](auto Cc) {
        constexpr int c = LBM_CI(Cc);
        constexpr int n = a + b + c;
        if constexpr (n <= L::NMAX && L::keep(a, b, c)) {
          constexpr double sc = 1.0 / (factorial(a) * factorial(b) * factorial(c) * ipow(c2, n));
          Real v;
          if constexpr (n == 0)
            v = drho;
          else
            v = (n <= P.neq) ? rho * pw[0][a] * pw[1][b] * pw[2][c] : Real(0);
          if constexpr (COLL == COLL_BGK) {
            v *= P.omega;
          } else if constexpr (n >= 2) {
            Real a1;
            if constexpr (COLL == COLL_PR) {
              // a1 = sum_i H (f_i - f^(0)_i) (Sec. II.E): the projection of f minus that of the truncated
              // equilibrium, sum over the kept (d, e, f) of order <= N_eq of gram3 * a0_(d,e,f)
              a1 = hmom(IC<a>{}, IC<b>{}, IC<c>{});
              sfor<0, 5>([&](auto Dd) {
                constexpr int d = LBM_CI(Dd);
                sfor<0, 5>([&](auto Ee) {
                  constexpr int e = LBM_CI(Ee);
                  sfor<0, 5>([&](auto Ff) {
                    constexpr int f = LBM_CI(Ff);
                    constexpr int m = d + e + f;
                    if constexpr (m <= L::NMAX && L::keep(d, e, f)) {
                      constexpr double gm = gram3<L>(a, b, c, d, e, f);
                      if constexpr (gm != 0.0) {
                        if (m <= P.neq) a1 -= Real(gm) * rho * pw[0][d] * pw[1][e] * pw[2][f];
                      }
                    }
                  });
                });
              });
            } else {
              a1 = Real(0);
              if constexpr (a >= 2) a1 += Real(choose2(a)) * b2[0] * pw[0][a - 2] * pw[1][b] * pw[2][c];
              if constexpr (b >= 2) a1 += Real(choose2(b)) * b2[1] * pw[0][a] * pw[1][b - 2] * pw[2][c];
              if constexpr (c >= 2) a1 += Real(choose2(c)) * b2[2] * pw[0][a] * pw[1][b] * pw[2][c - 2];
              if constexpr (a >= 1 && b >= 1) a1 += Real(a * b) * b2[3] * pw[0][a - 1] * pw[1][b - 1] * pw[2][c];
              if constexpr (a >= 1 && c >= 1) a1 += Real(a * c) * b2[4] * pw[0][a - 1] * pw[1][b] * pw[2][c - 1];
              if constexpr (b >= 1 && c >= 1) a1 += Real(b * c) * b2[5] * pw[0][a] * pw[1][b - 1] * pw[2][c - 1];
            }
            if (n <= P.nreg) v += P.om1 * a1;
          }
          if constexpr (SHIFTED) v *= P.s;
          C[a][b][c] = v * Real(sc);
        }
      });
    });
  });

  // rebuild: out_i = K_i sum_{kept} He_a(cx_i) He_b(cy_i) He_c(cz_i) C[a][b][c] (K_i = w_i, or 1 shifted)
  sfor<0, L::Q>([&](auto I) {
    constexpr int i = LBM_CI(I);
    Real acc = Real(0);
    sfor<0, 5>([&](auto Aa) {
      constexpr int a = LBM_CI(Aa);
      sfor<0, 5>([&](auto Bb) {
        constexpr int b = LBM_CI(Bb);
        sfor<0, 5>([&](auto Cc) {
          constexpr int c = LBM_CI(Cc);
          if constexpr (a + b + c <= L::NMAX && L::keep(a, b, c)) {
            constexpr double h = he(a, L::CX[i], c2) * he(b, L::CY[i], c2) * he(c, L::CZ[i], c2) *
                                 (SHIFTED ? 1.0 : L::W[i]);
            if constexpr (h != 0.0) acc = madd(Real(h), C[a][b][c], acc);
          }
        });
      });
    });
    [[maybe_unused]] constexpr double wr = (double)(Sc)L::W[i];
    if constexpr (COLL == COLL_BGK) {
      const Real dv = P.om1 * d[i] + acc;  // f* - ref = (1 - 1/tau)(f - ref) + (f^(0) - ref)/tau
      q[i] = SHIFTED ? dv : Real(wr) + dv;
    } else {
      q[i] = SHIFTED ? acc : Real(wr) + acc;
    }
  });
}

}  // namespace lbm
