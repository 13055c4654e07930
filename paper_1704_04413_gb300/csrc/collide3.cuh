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

// Velocity-set grouping of the factorized rebuild: how many velocities have (cy, cz) = (y, z) (y out of
// [-VMAX, VMAX]: any cy), the j-th of them, and whether some kept tensor has x-order a and y-order b.
template <class L>
__host__ __device__ constexpr int count_yz(int y, int z) {
  int n = 0;
  for (int i = 0; i < L::Q; ++i)
    if ((y > L::VMAX || L::CY[i] == y) && L::CZ[i] == z) ++n;
  return n;
}

template <class L>
__host__ __device__ constexpr int member_yz(int y, int z, int j) {
  for (int i = 0; i < L::Q; ++i)
    if (L::CY[i] == y && L::CZ[i] == z && j-- == 0) return i;
  return 0;
}

template <class L>
__host__ __device__ constexpr bool has_ab(int a, int b) {
  for (int c = 0; c <= 4; ++c)
    if (a + b + c <= L::NMAX && L::keep(a, b, c)) return true;
  return false;
}

template <class L>
__host__ __device__ constexpr bool has_a(int a) {
  for (int b = 0; b <= 4; ++b)
    if (has_ab<L>(a, b)) return true;
  return false;
}

// Nonzero coefficients (multiply-adds) of the rebuild summed directly over populations x kept tensors,
// and of its axis-factorized form; the kernel takes the factorized form where it saves a fifth or more
// (D3Q27 216 against 512, D3Q103 1270 against 2734; D3V39's 21 (cy, cz) groups leave 437 against 464).
template <class L>
__host__ __device__ constexpr int rebuild_cost_direct() {
  int n = 0;
  for (int i = 0; i < L::Q; ++i)
    for (int a = 0; a <= 4; ++a)
      for (int b = 0; b <= 4; ++b)
        for (int c = 0; c <= 4; ++c)
          if (a + b + c <= L::NMAX && L::keep(a, b, c) &&
              he(a, L::CX[i], L::CS2) * he(b, L::CY[i], L::CS2) * he(c, L::CZ[i], L::CS2) != 0.0)
            ++n;
  return n;
}

template <class L>
__host__ __device__ constexpr int rebuild_cost_factorized() {
  int n = 0;
  for (int z = -L::VMAX; z <= L::VMAX; ++z) {
    if (count_yz<L>(L::VMAX + 1, z) == 0) continue;
    for (int a = 0; a <= 4; ++a)
      for (int b = 0; b <= 4; ++b)
        for (int c = 0; c <= 4; ++c)
          if (a + b + c <= L::NMAX && L::keep(a, b, c) && he(c, z, L::CS2) != 0.0) ++n;
    for (int y = -L::VMAX; y <= L::VMAX; ++y) {
      if (count_yz<L>(y, z) == 0) continue;
      for (int a = 0; a <= 4; ++a)
        for (int b = 0; b <= 4; ++b)
          if (has_ab<L>(a, b) && he(b, y, L::CS2) != 0.0) ++n;
    }
  }
  for (int i = 0; i < L::Q; ++i)
    for (int a = 0; a <= 4; ++a)
      if (has_a<L>(a) && he(a, L::CX[i], L::CS2) != 0.0) ++n;
  return n;
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

// Rebuild: out_i = K_i sum_{kept} He_a(cx_i) He_b(cy_i) He_c(cz_i) C[a][b][c] (K_i = w_i, or 1 shifted), each
// population handed to emit(I, acc) as soon as it is made.  Summed directly, or factorized by axis where that
// saves a fifth of the multiply-adds or more.
template <class L, bool SHIFTED, class Real, class Emit>
__device__ __forceinline__ void rebuild3(const Real (&C)[5][5][5], Emit&& emit) {
  constexpr double c2 = L::CS2;
  if constexpr (5 * rebuild_cost_factorized<L>() > 4 * rebuild_cost_direct<L>()) {
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
      emit(I, acc);
    });
  } else {
    // factorized by axis over the velocity set grouped by cz, then by (cy, cz):
    //   T[a][b] = sum_c He_c(cz) C[a][b][c],  U[a] = sum_b He_b(cy) T[a][b],  out_i = K_i sum_a He_a(cx_i) U[a]
    sfor<0, 2 * L::VMAX + 1>([&](auto Zi) {
      constexpr int zv = LBM_CI(Zi) - L::VMAX;
      if constexpr (count_yz<L>(L::VMAX + 1, zv) > 0) {
        Real T[5][5];
        sfor<0, 5>([&](auto Aa) {
          constexpr int a = LBM_CI(Aa);
          sfor<0, 5>([&](auto Bb) {
            constexpr int b = LBM_CI(Bb);
            if constexpr (has_ab<L>(a, b)) {
              Real acc = Real(0);
              sfor<0, 5>([&](auto Cc) {
                constexpr int c = LBM_CI(Cc);
                if constexpr (a + b + c <= L::NMAX && L::keep(a, b, c)) {
                  constexpr double h = he(c, zv, c2);
                  if constexpr (h != 0.0) acc = madd(Real(h), C[a][b][c], acc);
                }
              });
              T[a][b] = acc;
            }
          });
        });
        sfor<0, 2 * L::VMAX + 1>([&](auto Yi) {
          constexpr int yv = LBM_CI(Yi) - L::VMAX;
          if constexpr (count_yz<L>(yv, zv) > 0) {
            Real U[5];
            sfor<0, 5>([&](auto Aa) {
              constexpr int a = LBM_CI(Aa);
              Real acc = Real(0);
              sfor<0, 5>([&](auto Bb) {
                constexpr int b = LBM_CI(Bb);
                if constexpr (has_ab<L>(a, b)) {
                  constexpr double h = he(b, yv, c2);
                  if constexpr (h != 0.0) acc = madd(Real(h), T[a][b], acc);
                }
              });
              U[a] = acc;
            });
            sfor<0, count_yz<L>(yv, zv)>([&](auto J) {
              constexpr int i = member_yz<L>(yv, zv, LBM_CI(J));
              Real acc = Real(0);
              sfor<0, 5>([&](auto Aa) {
                constexpr int a = LBM_CI(Aa);
                if constexpr (has_a<L>(a)) {
                  constexpr double h = he(a, L::CX[i], c2) * (SHIFTED ? 1.0 : L::W[i]);
                  if constexpr (h != 0.0) acc = madd(Real(h), U[a], acc);
                }
              });
              emit(IC<i>{}, acc);
            });
          }
        });
      }
    });
  }
}

// First population with a nonzero coefficient in the monomial moment x^k y^l z^m (-1: none).
template <class L>
__host__ __device__ constexpr int first_pop3(int k, int l, int m) {
  for (int i = 0; i < L::Q; ++i)
    if (ipow(L::CX[i], k) * ipow(L::CY[i], l) * ipow(L::CZ[i], m) != 0.0) return i;
  return -1;
}

// Monomial moments of order <= 2, D[k][l][m] = sum_i cx^k cy^l cz^m d_i: summed directly over the
// populations, or in two stages over the velocity set grouped by (cy, cz),
//   R_k(y, z) = sum_{i: (cy_i, cz_i) = (y, z)} cx_i^k d_i,   D[k][l][m] = sum_(y, z) y^l z^m R_k(y, z),
// where that saves a fifth of the multiply-adds or more (D3Q27 130 against 171, D3Q103 570 against 751).
template <class L>
__host__ __device__ constexpr int moments_cost_direct() {
  int n = 0;
  for (int k = 0; k <= 2; ++k)
    for (int l = 0; l + k <= 2; ++l)
      for (int m = 0; m + l + k <= 2; ++m)
        if (needs_monomial<L>(k, l, m, 2))
          for (int i = 0; i < L::Q; ++i)
            if (ipow(L::CX[i], k) * ipow(L::CY[i], l) * ipow(L::CZ[i], m) != 0.0) ++n;
  return n;
}
// Whether the group (y, z) has a member with cx^k != 0, and the first such member (-1: none).
template <class L>
__host__ __device__ constexpr int group_first_k(int y, int z, int k) {
  for (int j = 0; j < count_yz<L>(y, z); ++j)
    if (ipow(L::CX[member_yz<L>(y, z, j)], k) != 0.0) return j;
  return -1;
}
template <class L>
__host__ __device__ constexpr int moments_cost_grouped() {
  int n = 0;
  for (int z = -L::VMAX; z <= L::VMAX; ++z)
    for (int y = -L::VMAX; y <= L::VMAX; ++y) {
      if (count_yz<L>(y, z) == 0) continue;
      for (int k = 0; k <= 2; ++k) {
        for (int j = 0; j < count_yz<L>(y, z); ++j)
          if (ipow(L::CX[member_yz<L>(y, z, j)], k) != 0.0) ++n;
        if (group_first_k<L>(y, z, k) < 0) continue;
        for (int l = 0; l + k <= 2; ++l)
          for (int m = 0; m + l + k <= 2; ++m)
            if (needs_monomial<L>(k, l, m, 2) && ipow(y, l) * ipow(z, m) != 0.0) ++n;
      }
    }
  return n;
}
// First group (as (z + VMAX) (2 VMAX + 1) + y + VMAX) with a term in D[k][l][m] (-1: none).
template <class L>
__host__ __device__ constexpr int first_group(int k, int l, int m) {
  for (int z = -L::VMAX; z <= L::VMAX; ++z)
    for (int y = -L::VMAX; y <= L::VMAX; ++y)
      if (count_yz<L>(y, z) > 0 && group_first_k<L>(y, z, k) >= 0 && ipow(y, l) * ipow(z, m) != 0.0)
        return (z + L::VMAX) * (2 * L::VMAX + 1) + y + L::VMAX;
  return -1;
}

// The RR collision (projected a1^(2), Eq. MalaspinasRecursiveRelation in the closed form above) of one cell,
// or of two cells in packed FP32x2, as a stream: ld(I) gives the pulled population i (storage representation
// as Real), and the monomial moments take it as it arrives, so that no population has to stay live through
// the collision; out(I, v) receives post-collision population i as soon as the rebuild makes it.
template <class L, bool SHIFTED, class Real, class Ld, class Out>
__device__ __forceinline__ void collide3_rr(Ld&& ld, const CollParams<Real>& P, Out&& out) {
  using Sc = typename Scalar<Real>::type;
  constexpr double c2 = L::CS2;
  const Real rho_ref = SHIFTED ? P.rho0 : Real(1);

  // monomial moments of order <= 2 of the deviations d_i (Sec. II.A), D[k][l][m] = sum_i d_i cx^k cy^l cz^m
  Real D[3][3][3];
  if constexpr (5 * moments_cost_grouped<L>() <= 4 * moments_cost_direct<L>()) {
    sfor<0, 2 * L::VMAX + 1>([&](auto Zi) {
      constexpr int zv = LBM_CI(Zi) - L::VMAX;
      sfor<0, 2 * L::VMAX + 1>([&](auto Yi) {
        constexpr int yv = LBM_CI(Yi) - L::VMAX;
        constexpr int gid = LBM_CI(Zi) * (2 * L::VMAX + 1) + LBM_CI(Yi);
        if constexpr (count_yz<L>(yv, zv) > 0) {
          Real R[3];
          sfor<0, count_yz<L>(yv, zv)>([&](auto J) {
            constexpr int j = LBM_CI(J);
            constexpr int i = member_yz<L>(yv, zv, j);
            [[maybe_unused]] constexpr double wr = (double)(Sc)L::W[i];
            Real di = ld(IC<i>{});
            if constexpr (!SHIFTED) di = di - Real(wr);
            sfor<0, 3>([&](auto K) {
              constexpr int k = LBM_CI(K);
              constexpr double c = ipow(L::CX[i], k) * (SHIFTED ? L::W[i] : 1.0);
              if constexpr (c != 0.0) add_term<j == group_first_k<L>(yv, zv, k)>(R[k], c, di);
            });
          });
          sfor<0, 3>([&](auto K) {
            constexpr int k = LBM_CI(K);
            if constexpr (group_first_k<L>(yv, zv, k) >= 0) {
              sfor<0, 3 - k>([&](auto Lq) {
                constexpr int l = LBM_CI(Lq);
                sfor<0, 3 - k - l>([&](auto M) {
                  constexpr int m = LBM_CI(M);
                  constexpr double h = ipow(yv, l) * ipow(zv, m);
                  if constexpr (needs_monomial<L>(k, l, m, 2) && h != 0.0)
                    add_term<gid == first_group<L>(k, l, m)>(D[k][l][m], h, R[k]);
                });
              });
            }
          });
        }
      });
    });
  } else {
  sfor<0, L::Q>([&](auto I) {
    constexpr int i = LBM_CI(I);
    [[maybe_unused]] constexpr double wr = (double)(Sc)L::W[i];
    Real di = ld(I);
    if constexpr (!SHIFTED) di = di - Real(wr);
    sfor<0, 3>([&](auto K) {
      constexpr int k = LBM_CI(K);
      sfor<0, 3 - k>([&](auto Lq) {
        constexpr int l = LBM_CI(Lq);
        sfor<0, 3 - k - l>([&](auto M) {
          constexpr int m = LBM_CI(M);
          if constexpr (needs_monomial<L>(k, l, m, 2)) {
            constexpr double c = ipow(L::CX[i], k) * ipow(L::CY[i], l) * ipow(L::CZ[i], m) *
                                 (SHIFTED ? L::W[i] : 1.0);
            if constexpr (c != 0.0) add_term<i == first_pop3<L>(k, l, m)>(D[k][l][m], c, di);
          }
        });
      });
    });
  });
  }
  if constexpr (SHIFTED) {
    sfor<0, 3>([&](auto K) {
      constexpr int k = LBM_CI(K);
      sfor<0, 3 - k>([&](auto Lq) {
        constexpr int l = LBM_CI(Lq);
        sfor<0, 3 - k - l>([&](auto M) {
          constexpr int m = LBM_CI(M);
          if constexpr (needs_monomial<L>(k, l, m, 2)) D[k][l][m] = D[k][l][m] * P.inv_s;
        });
      });
    });
  }
  // Hermite moments of order <= 2 of f: He expanded in monomials, plus the rounded-weight correction
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
  const Real irho = recip(rho);
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
  // a1^(2): xx, yy, zz, xy, xz, yz
  Real b2[6];
  b2[0] = hmom(IC<2>{}, IC<0>{}, IC<0>{}) - rho * pw[0][2];
  b2[1] = hmom(IC<0>{}, IC<2>{}, IC<0>{}) - rho * pw[1][2];
  b2[2] = hmom(IC<0>{}, IC<0>{}, IC<2>{}) - rho * pw[2][2];
  b2[3] = hmom(IC<1>{}, IC<1>{}, IC<0>{}) - rho * pw[0][1] * pw[1][1];
  b2[4] = hmom(IC<1>{}, IC<0>{}, IC<1>{}) - rho * pw[0][1] * pw[2][1];
  b2[5] = hmom(IC<0>{}, IC<1>{}, IC<1>{}) - rho * pw[1][1] * pw[2][1];

  // coefficients of the rebuilt populations minus the reference, with 1 / (a! b! c! cs^2n) folded into the
  // scaled powers e_d[k] = u_d^k / (k! cs^2k): equilibrium rho e_x[a] e_y[b] e_z[c]; a1 by the closed form,
  // g_xx e_x[a-2] e_y[b] e_z[c] + ... + g_xy e_x[a-1] e_y[b-1] e_z[c] + ... with g_xx = a1_xx / (2 cs^4),
  // g_xy = a1_xy / cs^4, grouped per (a, b) as P0 e_z[c] + P1 e_z[c-1] + P2 e_z[c-2]
  Real e[3][5];
  sfor<0, 3>([&](auto Dd) {
    constexpr int dd = LBM_CI(Dd);
    sfor<0, 5>([&](auto K) {
      constexpr int k = LBM_CI(K);
      e[dd][k] = pw[dd][k] * Real(1.0 / (factorial(k) * ipow(c2, k)));
    });
  });
  const Real mul_eq = SHIFTED ? P.s : Real(1);
  const Real rs = rho * mul_eq;
  const Real om1s = SHIFTED ? P.om1 * P.s : P.om1;
  Real g[6];
  sfor<0, 6>([&](auto Jj) {
    constexpr int j = LBM_CI(Jj);
    g[j] = b2[j] * (om1s * Real(j < 3 ? 0.5 / (c2 * c2) : 1.0 / (c2 * c2)));
  });
  Real C[5][5][5];
  sfor<0, 5>([&](auto Aa) {
    constexpr int a = LBM_CI(Aa);
    sfor<0, 5>([&](auto Bb) {
      constexpr int b = LBM_CI(Bb);
      if constexpr (has_ab<L>(a, b)) {
        const Real eab = e[0][a] * e[1][b];
        Real P0 = Real(0), P1 = Real(0);
        if constexpr (a >= 2) P0 = madd(g[0], e[0][a - 2] * e[1][b], P0);
        if constexpr (b >= 2) P0 = madd(g[1], e[0][a] * e[1][b - 2], P0);
        if constexpr (a >= 1 && b >= 1) P0 = madd(g[3], e[0][a - 1] * e[1][b - 1], P0);
        if constexpr (a >= 1) P1 = madd(g[4], e[0][a - 1] * e[1][b], P1);
        if constexpr (b >= 1) P1 = madd(g[5], e[0][a] * e[1][b - 1], P1);
        const Real P2 = g[2] * eab;
        sfor<0, 5>([&](auto Cc) {
          constexpr int c = LBM_CI(Cc);
          constexpr int n = a + b + c;
          if constexpr (n <= L::NMAX && L::keep(a, b, c)) {
            Real v;
            if constexpr (n == 0)
              v = drho * mul_eq;
            else
              v = (n <= P.neq) ? rs * (eab * e[2][c]) : Real(0);
            if constexpr (n >= 2) {
              Real a1 = P0 * e[2][c];
              if constexpr (c >= 1) a1 = madd(P1, e[2][c - 1], a1);
              if constexpr (c >= 2) a1 = madd(P2, e[2][c - 2], a1);
              if (n <= P.nreg) v += a1;
            }
            C[a][b][c] = v;
          }
        });
      }
    });
  });
  rebuild3<L, SHIFTED>(C, [&](auto Ii, Real acc) {
    constexpr int i = LBM_CI(Ii);
    [[maybe_unused]] constexpr double wr = (double)(Sc)L::W[i];
    out(Ii, SHIFTED ? acc : Real(wr) + acc);
  });
}

template <class L, int COLL, bool SHIFTED, class Real>
__device__ __forceinline__ void collide3(Real (&q)[L::Q], const CollParams<Real>& P) {
  if constexpr (COLL == COLL_RR) {
    collide3_rr<L, SHIFTED>([&](auto I) { return q[LBM_CI(I)]; }, P, [&](auto I, Real v) { q[LBM_CI(I)] = v; });
    return;
  }
  using Sc = typename Scalar<Real>::type;
  constexpr double c2 = L::CS2;
  // highest monomial order the mode needs (PR's projections of order >= 3 are summed directly, hmom_direct)
  constexpr int PM = COLL == COLL_PR ? 2 : 1;
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

  // Hermite moment summed directly over the populations (PR at orders >= 3): the monomial route would
  // subtract rounded sums of the slow populations' large deviations (He_3 = c^3 - 3 cs^2 c, ...)
  auto hmom_direct = [&](auto Aa, auto Bb, auto Cc) -> Real {
    constexpr int a = LBM_CI(Aa), b = LBM_CI(Bb), c = LBM_CI(Cc);
    Real acc = Real(0);
    sfor<0, L::Q>([&](auto I) {
      constexpr int i = LBM_CI(I);
      constexpr double h = he(a, L::CX[i], c2) * he(b, L::CY[i], c2) * he(c, L::CZ[i], c2) *
                           (SHIFTED ? L::W[i] : 1.0);
      if constexpr (h != 0.0) acc = madd(Real(h), d[i], acc);
    });
    if constexpr (SHIFTED) {
      acc = acc * P.inv_s;
    } else {
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

  // coefficients of the rebuilt populations minus the reference, per kept tensor, with the factor
  // 1 / (a! b! c! cs^2n) folded into scaled powers e_d[k] = u_d^k / (k! cs^2k):
  //   equilibrium  rho e_x[a] e_y[b] e_z[c]
  //   RR a1        g_xx e_x[a-2] e_y[b] e_z[c] + ... + g_xy e_x[a-1] e_y[b-1] e_z[c] + ...,
  //                g_xx = a1_xx / (2 cs^4), g_xy = a1_xy / cs^4 (the closed form above, rescaled)
  // grouped per (a, b) as P0 e_z[c] + P1 e_z[c-1] + P2 e_z[c-2].
  Real e[3][5];
  sfor<0, 3>([&](auto Dd) {
    constexpr int dd = LBM_CI(Dd);
    sfor<0, 5>([&](auto K) {
      constexpr int k = LBM_CI(K);
      e[dd][k] = pw[dd][k] * Real(1.0 / (factorial(k) * ipow(c2, k)));
    });
  });
  const Real mul_eq = (COLL == COLL_BGK ? P.omega : Real(1)) * (SHIFTED ? P.s : Real(1));
  const Real rs = rho * mul_eq;
  const Real om1s = SHIFTED ? P.om1 * P.s : P.om1;
  Real C[5][5][5];
  sfor<0, 5>([&](auto Aa) {
    constexpr int a = LBM_CI(Aa);
    sfor<0, 5>([&](auto Bb) {
      constexpr int b = LBM_CI(Bb);
      if constexpr (has_ab<L>(a, b)) {
        const Real eab = e[0][a] * e[1][b];
        sfor<0, 5>([&](auto Cc) {
          constexpr int c = LBM_CI(Cc);
          constexpr int n = a + b + c;
          if constexpr (n <= L::NMAX && L::keep(a, b, c)) {
            Real v;
            if constexpr (n == 0)
              v = drho * mul_eq;
            else
              v = (n <= P.neq) ? rs * (eab * e[2][c]) : Real(0);
            if constexpr (COLL == COLL_PR && n >= 2) {
              // a1 = sum_i H (f_i - f^(0)_i) (Sec. II.E): the projection of f minus that of the truncated
              // equilibrium, sum over the kept (d, e, f) of order <= N_eq of gram3 * a0_(d,e,f)
              Real a1;
              if constexpr (n <= 2)
                a1 = hmom(IC<a>{}, IC<b>{}, IC<c>{});
              else
                a1 = hmom_direct(IC<a>{}, IC<b>{}, IC<c>{});
              sfor<0, 5>([&](auto Dd) {
                constexpr int d = LBM_CI(Dd);
                sfor<0, 5>([&](auto Ee) {
                  constexpr int ee = LBM_CI(Ee);
                  sfor<0, 5>([&](auto Ff) {
                    constexpr int f = LBM_CI(Ff);
                    constexpr int m = d + ee + f;
                    if constexpr (m <= L::NMAX && L::keep(d, ee, f)) {
                      constexpr double gm = gram3<L>(a, b, c, d, ee, f);
                      if constexpr (gm != 0.0) {
                        if (m <= P.neq) a1 -= Real(gm) * rho * pw[0][d] * pw[1][ee] * pw[2][f];
                      }
                    }
                  });
                });
              });
              constexpr double sc = 1.0 / (factorial(a) * factorial(b) * factorial(c) * ipow(c2, n));
              if (n <= P.nreg) v += om1s * (a1 * Real(sc));
            }
            C[a][b][c] = v;
          }
        });
      }
    });
  });

  // rebuild: out_i = K_i sum_{kept} He_a(cx_i) He_b(cy_i) He_c(cz_i) C[a][b][c] (K_i = w_i, or 1 shifted)
  auto emit = [&](auto Ii, Real acc) {
    constexpr int i = LBM_CI(Ii);
    [[maybe_unused]] constexpr double wr = (double)(Sc)L::W[i];
    if constexpr (COLL == COLL_BGK) {
      const Real dv = P.om1 * d[i] + acc;  // f* - ref = (1 - 1/tau)(f - ref) + (f^(0) - ref)/tau
      q[i] = SHIFTED ? dv : Real(wr) + dv;
    } else {
      q[i] = SHIFTED ? acc : Real(wr) + acc;
    }
  };
  rebuild3<L, SHIFTED>(C, emit);
}

}  // namespace lbm
