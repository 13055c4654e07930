/*
 * FP64 CPU oracle for the RR lattice-Boltzmann step (arXiv 1704.04413).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU
 * baseline of the benchmark, never by the product path.  Plain, slow,
 * written in the paper's tensor-index form (see lbm_oracle.h).
 *
 * Parity pins live in tests/test_oracle_*.py.  Parity unpinned: none of the
 * functions below (the paper's figure curves are not reproduced here).
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TEN(a, n, t) ((a)[(n) * 16 + (t)]) /* rank-n tensor entry t in a [ORC_MAXN+1][16] block */

/* ------------------------------------------------------------------------ */
/* Lattices, Tab. I.  Each velocity group is listed by one representative;   */
/* the full group is its orbit under axis reflections and the x<->y swap.   */
/* D2Q9 weights: the printed column is shifted by one row; the reading used */
/* is 4/9 on (0,0), 1/9 on (1,0), 1/36 on (1,1) (the only one with          */
/* sum w xi_a xi_b = cs^2 delta_ab).                                        */
/* ------------------------------------------------------------------------ */
static int add_orbit(orc_lattice *L, int p, int q, double w) {
  int cand[8][2] = {{p, q}, {-p, q}, {p, -q}, {-p, -q}, {q, p}, {-q, p}, {q, -p}, {-q, -p}};
  int added = 0;
  for (int k = 0; k < 8; k++) {
    int dup = 0;
    for (int j = 0; j < L->V; j++)
      if (L->cx[j] == cand[k][0] && L->cy[j] == cand[k][1]) dup = 1;
    if (!dup) {
      L->cx[L->V] = cand[k][0];
      L->cy[L->V] = cand[k][1];
      L->w[L->V] = w;
      L->V++;
      added++;
    }
  }
  return added;
}

static int build_lattice(int lattice, orc_lattice *L) {
  memset(L, 0, sizeof(*L));
  if (lattice == ORC_D2Q9) {
    add_orbit(L, 0, 0, 4.0 / 9.0);
    add_orbit(L, 1, 0, 1.0 / 9.0);
    add_orbit(L, 1, 1, 1.0 / 36.0);
    L->cs2 = 1.0 / 3.0; /* 1/cs = sqrt(3) */
    L->nmax = 4;
    /* complete basis (Sec. II.F): every product of per-direction orders <= 2 */
    for (int a = 0; a <= 2; a++)
      for (int b = 0; b <= 2; b++) L->keep[a][b] = 1;
    return 0;
  }
  if (lattice == ORC_D2V17) {
    double s = sqrt(193.0);
    add_orbit(L, 0, 0, (575.0 + 193.0 * s) / 8100.0);
    add_orbit(L, 1, 0, (3355.0 - 91.0 * s) / 18000.0);
    add_orbit(L, 1, 1, (655.0 + 17.0 * s) / 27000.0);
    add_orbit(L, 2, 2, (685.0 - 49.0 * s) / 54000.0);
    add_orbit(L, 3, 0, (1445.0 - 101.0 * s) / 162000.0);
    L->cs2 = 72.0 / (5.0 * (25.0 + s)); /* 1/cs = sqrt(5(25+sqrt 193)/72) */
    L->nmax = 3;
    for (int a = 0; a <= 3; a++)
      for (int b = 0; a + b <= 3; b++) L->keep[a][b] = 1;
    return 0;
  }
  if (lattice == ORC_D2V37) {
    add_orbit(L, 0, 0, 0.23315066913235250228650);
    add_orbit(L, 1, 0, 0.10730609154221900241246);
    add_orbit(L, 1, 1, 0.05766785988879488203006);
    add_orbit(L, 2, 0, 0.01420821615845075026469);
    add_orbit(L, 2, 1, 0.00535304900051377523273);
    add_orbit(L, 2, 2, 0.00101193759267357547541);
    add_orbit(L, 3, 0, 0.00024530102775771734547);
    add_orbit(L, 3, 1, 0.00028341425299419821740);
    double ics = 1.19697977039307435897239;
    L->cs2 = 1.0 / (ics * ics);
    L->nmax = 4;
    for (int a = 0; a <= 4; a++)
      for (int b = 0; a + b <= 4; b++) L->keep[a][b] = 1;
    return 0;
  }
  return -1;
}

/* ------------------------------------------------------------------------ */
/* Index-tuple helpers                                                       */
/* ------------------------------------------------------------------------ */
static void tuple_to_alpha(int n, int t, int *alpha) {
  for (int k = 0; k < n; k++) alpha[k] = (t >> k) & 1;
}
static int alpha_to_tuple(int n, const int *alpha) {
  int t = 0;
  for (int k = 0; k < n; k++) t |= alpha[k] << k;
  return t;
}
/* alpha with entries `skip1` (and `skip2` if >= 0) removed: the beta_l / beta_lm of App. A */
static int drop_indices(int n, const int *alpha, int skip1, int skip2) {
  int beta[ORC_MAXN + 1], m = 0;
  for (int k = 0; k < n; k++)
    if (k != skip1 && k != skip2) beta[m++] = alpha[k];
  return alpha_to_tuple(m, beta);
}
static int count_y(int n, int t) {
  int c = 0;
  for (int k = 0; k < n; k++) c += (t >> k) & 1;
  return c;
}
static double fact(int n) {
  double r = 1.0;
  for (int k = 2; k <= n; k++) r *= k;
  return r;
}

/* ------------------------------------------------------------------------ */
/* Hermite tensors: Rodrigues relation of App. B,                            */
/*   xi_{a_n} H^(n-1)_{a_1..a_{n-1}} = H^(n)_{a_1..a_n}                      */
/*                                   + cs^2 sum_{l<n} delta_{a_l a_n} H^(n-2)_{beta_l}, */
/* solved for H^(n), with H^(0) = 1, H^(1) = xi.                             */
/* ------------------------------------------------------------------------ */
static double hermite_alpha(int n, const int *alpha, double xx, double xy, double cs2) {
  if (n == 0) return 1.0;
  double xi_last = alpha[n - 1] ? xy : xx;
  double v = xi_last * hermite_alpha(n - 1, alpha, xx, xy, cs2);
  for (int l = 0; l < n - 1; l++) {
    if (alpha[l] != alpha[n - 1]) continue;
    int beta[ORC_MAXN + 1], m = 0;
    for (int k = 0; k < n - 1; k++)
      if (k != l) beta[m++] = alpha[k];
    v -= cs2 * hermite_alpha(n - 2, beta, xx, xy, cs2);
  }
  return v;
}

double orc_hermite(int n, int tuple, double xx, double xy, double cs2) {
  int alpha[ORC_MAXN + 1];
  tuple_to_alpha(n, tuple, alpha);
  return hermite_alpha(n, alpha, xx, xy, cs2);
}

/* ------------------------------------------------------------------------ */
/* The three lattices and their Hermite tensors H^(n)_t(xi_i) are evaluated  */
/* once, when the library is loaded, by the functions above (a memo: the     */
/* values are exactly those the functions return).                           */
/* ------------------------------------------------------------------------ */
static orc_lattice g_lat[3];
static double g_herm[3][ORC_MAXQ][ORC_MAXN + 1][16];

__attribute__((constructor)) static void build_tables(void) {
  for (int id = 0; id < 3; id++) {
    build_lattice(id, &g_lat[id]);
    for (int i = 0; i < g_lat[id].V; i++)
      for (int n = 0; n <= ORC_MAXN; n++)
        for (int t = 0; t < (1 << n); t++)
          g_herm[id][i][n][t] = orc_hermite(n, t, g_lat[id].cx[i], g_lat[id].cy[i], g_lat[id].cs2);
  }
}

int orc_lattice_get(int lattice, orc_lattice *L) {
  if (lattice < 0 || lattice > 2) return -1;
  *L = g_lat[lattice];
  return 0;
}

/* H^(n)_t(xi_i) on lattice L: the memo when L is one of the three lattices, else evaluated. */
static double herm_at(const orc_lattice *L, int n, int t, int i) {
  for (int id = 0; id < 3; id++)
    if (g_lat[id].V == L->V && g_lat[id].cs2 == L->cs2) return g_herm[id][i][n][t];
  return orc_hermite(n, t, L->cx[i], L->cy[i], L->cs2);
}

/* ------------------------------------------------------------------------ */
/* Equilibrium coefficients, App. B:                                         */
/*   a0^(n)_{a_1..a_n} = u_{a_n} a0^(n-1)_{a_1..a_{n-1}}                      */
/*                     + (theta-1) cs^2 sum_{l<n} delta_{a_l a_n} a0^(n-2)_{beta_l}, a0^(0) = rho. */
/* ------------------------------------------------------------------------ */
void orc_a0(double cs2, double rho, double ux, double uy, double theta, int nmax, double *a0) {
  memset(a0, 0, sizeof(double) * (ORC_MAXN + 1) * 16);
  TEN(a0, 0, 0) = rho;
  for (int n = 1; n <= nmax; n++) {
    for (int t = 0; t < (1 << n); t++) {
      int alpha[ORC_MAXN + 1];
      tuple_to_alpha(n, t, alpha);
      double u_last = alpha[n - 1] ? uy : ux;
      double v = u_last * TEN(a0, n - 1, drop_indices(n, alpha, n - 1, -1));
      for (int l = 0; l < n - 1; l++)
        if (alpha[l] == alpha[n - 1]) v += (theta - 1.0) * cs2 * TEN(a0, n - 2, drop_indices(n, alpha, l, n - 1));
      TEN(a0, n, t) = v;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Off-equilibrium coefficients, recursive (Sec. II.E and App. A).           */
/* ------------------------------------------------------------------------ */
static int pair_tuple(int a, int b) { return a | (b << 1); }
static int triple_tuple(int a, int b, int c) { return a | (b << 1) | (c << 2); }

void orc_a1_recursive(double cs2, double rho, double ux, double uy, double theta, int thermal, int nmax,
                      const double *a0, double *a1) {
  double u[2] = {ux, uy};
  int nstart = thermal ? 4 : 3;
  for (int n = nstart; n <= nmax; n++) {
    for (int t = 0; t < (1 << n); t++) {
      int alpha[ORC_MAXN + 1];
      tuple_to_alpha(n, t, alpha);
      int an = alpha[n - 1];
      /* u_{a_n} a1^(n-1)_{a_1..a_{n-1}} */
      double v = u[an] * TEN(a1, n - 1, drop_indices(n, alpha, n - 1, -1));
      for (int l = 0; l < n - 1; l++) {
        int beta_l = drop_indices(n, alpha, l, n - 1);
        /* (1/rho) a0^(n-2)_{beta_l} a1^(2)_{a_l a_n} */
        v += TEN(a0, n - 2, beta_l) * TEN(a1, 2, pair_tuple(alpha[l], an)) / rho;
        /* thermal: cs^2 (theta-1) delta_{a_l a_n} a1^(n-2)_{beta_l} */
        if (thermal && alpha[l] == an) v += cs2 * (theta - 1.0) * TEN(a1, n - 2, beta_l);
      }
      if (thermal) {
        for (int l = 0; l < n - 1; l++)
          for (int m = l + 1; m < n - 1; m++) {
            int beta_lm = drop_indices(n - 1, alpha, l, m); /* drop a_l, a_m from a_1..a_{n-1} */
            int al = alpha[l], am = alpha[m];
            double bracket = TEN(a1, 3, triple_tuple(al, am, an)) - u[al] * TEN(a1, 2, pair_tuple(am, an)) -
                             u[am] * TEN(a1, 2, pair_tuple(al, an)) - u[an] * TEN(a1, 2, pair_tuple(al, am));
            v += TEN(a0, n - 3, beta_lm) * bracket / rho;
          }
      }
      TEN(a1, n, t) = v;
    }
  }
}

/* Thermal a1^(3) (App. C, steps 1-4).  Each a1^(3)_{b b g} of the
 * Chapman-Enskog form a1_{abg} = u_a a1_{bg} + u_b a1_{ag} + u_g a1_{ab}
 *                                - G_a delta_{bg} - G_b delta_{ag} - G_g delta_{ab}
 * (with G = mu cs^2 grad theta) gives one estimate of G_g when solved for it;
 * the D estimates are averaged (Eq. TempGradLBM) and a1^(3) is rebuilt. */
/* Eq. a1Rec (App. C step 4): a1^(3)_abg = u_a a1_bg + u_b a1_ag + u_g a1_ab - (delta_bg G_a + delta_ag G_b +
 * delta_ab G_g), with G_g = mu cs^2 d_g theta. */
static void a1_third_from_gradients(double ux, double uy, const double *a1_2, const double *G, double *a1_3) {
  double u[2] = {ux, uy};
  for (int t = 0; t < 8; t++) {
    int a = t & 1, b = (t >> 1) & 1, g = (t >> 2) & 1;
    double v = u[a] * a1_2[pair_tuple(b, g)] + u[b] * a1_2[pair_tuple(a, g)] + u[g] * a1_2[pair_tuple(a, b)];
    if (b == g) v -= G[a];
    if (a == g) v -= G[b];
    if (a == b) v -= G[g];
    a1_3[t] = v;
  }
}

void orc_a1_third_thermal(double ux, double uy, const double *a1_2, const double *a1_3_proj, double *a1_3) {
  const int D = 2;
  double u[2] = {ux, uy};
  double G[2];
  for (int g = 0; g < D; g++) {
    double acc = 0.0;
    for (int b = 0; b < D; b++) {
      double rhs = u[b] * a1_2[pair_tuple(b, g)] + u[b] * a1_2[pair_tuple(b, g)] + u[g] * a1_2[pair_tuple(b, b)] -
                   a1_3_proj[triple_tuple(b, b, g)];
      double mult = 1.0 + (b == g ? 2.0 : 0.0); /* number of deltas holding G_g in the (b,b,g) entry */
      acc += rhs / mult;
    }
    G[g] = acc / D;
  }
  a1_third_from_gradients(ux, uy, a1_2, G, a1_3);
}

/* ------------------------------------------------------------------------ */
/* Truncated Hermite expansion (Sec. II.C, Eq. GenRegCollision with a single */
/* tau): f_i = w_i sum_n 1/(n! cs^2n) sum_{alpha kept} H_alpha(xi_i) c_alpha. */
/* The multiplicity A^(n) of App. C arises from summing over all tuples.     */
/* ------------------------------------------------------------------------ */
void orc_expand(const orc_lattice *L, int nmin, int nmax, const double *coef, double *f) {
  for (int i = 0; i < L->V; i++) {
    double s = 0.0;
    for (int n = nmin; n <= nmax; n++) {
      double norm = fact(n) * pow(L->cs2, n);
      for (int t = 0; t < (1 << n); t++) {
        int ny = count_y(n, t), nx = n - ny;
        if (!L->keep[nx][ny]) continue;
        s += herm_at(L, n, t, i) * TEN(coef, n, t) / norm;
      }
    }
    f[i] = L->w[i] * s;
  }
}

/* Moments, Sec. II.A: rho = sum f, rho u = sum f xi, 2 rho E = sum f xi^2 with
 * rho E = rho (u^2 + D cs^2 theta) / 2 (p = rho r T, cs^2 = r T0). */
void orc_cell_moments(const orc_lattice *L, int thermal, const double *f, double *rho, double *ux, double *uy,
                      double *theta) {
  double r = 0, jx = 0, jy = 0, e2 = 0;
  for (int i = 0; i < L->V; i++) {
    r += f[i];
    jx += f[i] * L->cx[i];
    jy += f[i] * L->cy[i];
    e2 += f[i] * (double)(L->cx[i] * L->cx[i] + L->cy[i] * L->cy[i]);
  }
  *rho = r;
  *ux = jx / r;
  *uy = jy / r;
  if (thermal) {
    const int D = 2;
    *theta = (e2 / r - (*ux) * (*ux) - (*uy) * (*uy)) / (D * L->cs2);
  } else {
    *theta = 1.0;
  }
}

static int resolve_orders(const orc_params *p, const orc_lattice *L, int *neq, int *nreg) {
  *neq = p->hermite_order;
  *nreg = p->reg_order == 0 ? L->nmax : p->reg_order;
  if (*neq < 2 || *neq > L->nmax) return -1;
  if (*nreg < 2 || *nreg > L->nmax) return -1;
  if (p->thermal && p->lattice != ORC_D2V37) return -1;
  if (!(p->tau > 0.5)) return -1;
  if (p->tau3 < 0.0 || p->tau4 < 0.0 || (p->tau3 > 0.0 && !(p->tau3 > 0.5)) || (p->tau4 > 0.0 && !(p->tau4 > 0.5)))
    return -1;
  if (p->collision == ORC_BGK && (p->tau3 > 0.0 || p->tau4 > 0.0)) return -1;
  if (p->a1_source != 0 && (p->a1_source != 1 || p->collision != ORC_RR)) return -1;
  return 0;
}

/* Relaxation time of the order-n coefficients of f^(1) (n >= 2). */
static double tau_of_order(const orc_params *p, int n) {
  if (n == 3 && p->tau3 > 0.0) return p->tau3;
  if (n == 4 && p->tau4 > 0.0) return p->tau4;
  return p->tau;
}

/* ------------------------------------------------------------------------ */
/* Collision of one cell.                                                    */
/*  BGK (Sec. III.A): f* = f - (f - f^(0))/tau.                              */
/*  PR  (Sec. II.E):  a1^(n) = sum_i H^(n)_i (f_i - f_i^(0)), n = 2..N.      */
/*  RR  (Sec. II.E):  a1^(2) projected; isothermal a1^(n>=3) by Eq.          */
/*      (MalaspinasRecursiveRelation); thermal a1^(3) by App. C steps 1-4,   */
/*      a1^(n>=4) by Eq. (RecursiveRelation_ThermalCase).                    */
/*  PR/RR rebuild (Eq. GenRegCollision with one relaxation time per order,   */
/*      Sec. II.B): f* = f^(0) + sum_n (1 - 1/tau_n) f^(1,n), tau_2 = tau.   */
/* ------------------------------------------------------------------------ */
static int collide_cell(const orc_params *p, const double *f_in, const double *grad, const double *delta,
                        double *f_out);

int orc_collide(const orc_params *p, const double *f_in, double *f_out) {
  if (p->a1_source != 0) return -1;
  return collide_cell(p, f_in, NULL, NULL, f_out);
}

int orc_collide_fd(const orc_params *p, const double *f_in, const double *grad, double *f_out) {
  if (p->a1_source != 1 || !grad) return -1;
  return collide_cell(p, f_in, grad, NULL, f_out);
}

int orc_collide_delta(const orc_params *p, const double *f_in, const double *delta, double *f_out) {
  if (p->a1_source != 0 || p->collision != ORC_RR || p->thermal || !delta) return -1;
  return collide_cell(p, f_in, NULL, delta, f_out);
}

/* grad == NULL: a1 by projection; else a1^(2) (and the thermal temperature gradients) from grad.
 * delta != NULL (isothermal RR, projection): delta[0..2] = (xx, xy, yy) is added to the projected a1^(2)
 * (both xy and yx entries) before the recursion builds the higher orders. */
static int collide_cell(const orc_params *p, const double *f_in, const double *grad, const double *delta,
                        double *f_out) {
  orc_lattice L;
  if (orc_lattice_get(p->lattice, &L)) return -1;
  int neq, nreg;
  if (resolve_orders(p, &L, &neq, &nreg)) return -1;

  double rho, ux, uy, theta;
  orc_cell_moments(&L, p->thermal, f_in, &rho, &ux, &uy, &theta);

  double a0[(ORC_MAXN + 1) * 16];
  orc_a0(L.cs2, rho, ux, uy, theta, ORC_MAXN, a0);
  double feq[ORC_MAXQ];
  orc_expand(&L, 0, neq, a0, feq);

  if (p->collision == ORC_BGK) {
    for (int i = 0; i < L.V; i++) f_out[i] = f_in[i] - (f_in[i] - feq[i]) / p->tau;
    return 0;
  }

  /* projection of f - f^(0) onto every kept tensor of order 2..N */
  double a1p[(ORC_MAXN + 1) * 16];
  memset(a1p, 0, sizeof(a1p));
  for (int n = 2; n <= nreg; n++)
    for (int t = 0; t < (1 << n); t++) {
      double s = 0.0;
      for (int i = 0; i < L.V; i++) s += herm_at(&L, n, t, i) * (f_in[i] - feq[i]);
      TEN(a1p, n, t) = s;
    }

  double a1[(ORC_MAXN + 1) * 16];
  memset(a1, 0, sizeof(a1));
  if (p->collision == ORC_PR) {
    memcpy(a1, a1p, sizeof(a1));
  } else if (p->collision == ORC_RR && grad) {
    /* Chapman-Enskog forms of Sec. II.E (App. A) from the finite-difference gradients */
    const double th = p->thermal ? theta : 1.0;
    const double pre = -p->tau * rho * L.cs2 * th;
    const double div = p->thermal ? grad[0] + grad[3] : 0.0; /* (2/D) div u, D = 2 */
    TEN(a1, 2, pair_tuple(0, 0)) = pre * (2.0 * grad[0] - div);
    TEN(a1, 2, pair_tuple(1, 1)) = pre * (2.0 * grad[3] - div);
    TEN(a1, 2, pair_tuple(0, 1)) = pre * (grad[1] + grad[2]);
    TEN(a1, 2, pair_tuple(1, 0)) = pre * (grad[1] + grad[2]);
    if (p->thermal && nreg >= 3) {
      const double mu_cs2 = tau_of_order(p, 3) * rho * L.cs2 * theta * L.cs2;
      const double G[2] = {mu_cs2 * grad[4], mu_cs2 * grad[5]};
      a1_third_from_gradients(ux, uy, &TEN(a1, 2, 0), G, &TEN(a1, 3, 0));
    }
    orc_a1_recursive(L.cs2, rho, ux, uy, theta, p->thermal, nreg, a0, a1);
  } else if (p->collision == ORC_RR) {
    for (int t = 0; t < 4; t++) TEN(a1, 2, t) = TEN(a1p, 2, t);
    if (delta) {
      TEN(a1, 2, pair_tuple(0, 0)) += delta[0];
      TEN(a1, 2, pair_tuple(0, 1)) += delta[1];
      TEN(a1, 2, pair_tuple(1, 0)) += delta[1];
      TEN(a1, 2, pair_tuple(1, 1)) += delta[2];
    }
    if (p->thermal) {
      if (nreg >= 3) {
        /* the projected a1^(3) is needed whatever nreg: project it here if nreg == 3 did not */
        double proj3[8];
        for (int t = 0; t < 8; t++) {
          double s = 0.0;
          for (int i = 0; i < L.V; i++) s += herm_at(&L, 3, t, i) * (f_in[i] - feq[i]);
          proj3[t] = s;
        }
        orc_a1_third_thermal(ux, uy, &TEN(a1, 2, 0), proj3, &TEN(a1, 3, 0));
      }
    }
    orc_a1_recursive(L.cs2, rho, ux, uy, theta, p->thermal, nreg, a0, a1);
  } else {
    return -1;
  }

  for (int i = 0; i < L.V; i++) f_out[i] = feq[i];
  for (int n = 2; n <= nreg; n++) {
    double fn[ORC_MAXQ];
    orc_expand(&L, n, n, a1, fn);
    const double om1 = 1.0 - 1.0 / tau_of_order(p, n);
    for (int i = 0; i < L.V; i++) f_out[i] += om1 * fn[i];
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Streaming (Sec. III.A, method of characteristics on the on-grid lattice), */
/* written as a pull: f_i(x) <- f_i*(x - xi_i).  Periodic axes wrap; zero-   */
/* gradient axes clamp the source index into the domain.                     */
/* ------------------------------------------------------------------------ */
static int src_index(int x, int c, int n, int bc) {
  int s = x - c;
  if (bc == ORC_PERIODIC) {
    s %= n;
    if (s < 0) s += n;
  } else {
    if (s < 0) s = 0;
    if (s > n - 1) s = n - 1;
  }
  return s;
}

static void gather_cell(const orc_params *p, const orc_lattice *L, const double *f_in, int x, int y, double *fc) {
  long long plane = (long long)p->nx * p->ny;
  for (int i = 0; i < L->V; i++) {
    int xs = src_index(x, L->cx[i], p->nx, p->bc_x);
    int ys = src_index(y, L->cy[i], p->ny, p->bc_y);
    fc[i] = f_in[i * plane + (long long)ys * p->nx + xs];
  }
}

/* Moments rho, ux, uy, theta of every cell after streaming (the fields the collision sees), m[4][ny][nx]. */
static void stream_moments(const orc_params *p, const orc_lattice *L, const double *f_in, double *m) {
  long long plane = (long long)p->nx * p->ny;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < p->ny; y++) {
    double fc[ORC_MAXQ];
    for (int x = 0; x < p->nx; x++) {
      long long c = (long long)y * p->nx + x;
      gather_cell(p, L, f_in, x, y, fc);
      orc_cell_moments(L, p->thermal, fc, &m[c], &m[plane + c], &m[2 * plane + c], &m[3 * plane + c]);
    }
  }
}

/* Second-order central differences of ux, uy, theta at (x, y); neighbours follow the streaming rule (periodic
 * wrap, or the clamped edge cell on a zero-gradient axis, which makes the edge difference one-sided). */
static void central_gradients(const orc_params *p, const double *m, int x, int y, double *grad) {
  long long plane = (long long)p->nx * p->ny;
  int xp = src_index(x, -1, p->nx, p->bc_x), xm = src_index(x, 1, p->nx, p->bc_x);
  int yp = src_index(y, -1, p->ny, p->bc_y), ym = src_index(y, 1, p->ny, p->bc_y);
  const double *ux = m + plane, *uy = m + 2 * plane, *th = m + 3 * plane;
  long long ex = (long long)y * p->nx + xp, wx = (long long)y * p->nx + xm;
  long long ny_ = (long long)yp * p->nx + x, sy = (long long)ym * p->nx + x;
  grad[0] = 0.5 * (ux[ex] - ux[wx]);
  grad[1] = 0.5 * (ux[ny_] - ux[sy]);
  grad[2] = 0.5 * (uy[ex] - uy[wx]);
  grad[3] = 0.5 * (uy[ny_] - uy[sy]);
  grad[4] = 0.5 * (th[ex] - th[wx]);
  grad[5] = 0.5 * (th[ny_] - th[sy]);
}

int orc_step(const orc_params *p, const double *f_in, double *f_out) {
  orc_lattice L;
  if (orc_lattice_get(p->lattice, &L)) return -1;
  int neq, nreg;
  if (resolve_orders(p, &L, &neq, &nreg)) return -1;
  long long plane = (long long)p->nx * p->ny;
  double *m = NULL;
  if (p->a1_source == 1) {
    m = (double *)malloc(sizeof(double) * 4 * (size_t)plane);
    if (!m) return -1;
    stream_moments(p, &L, f_in, m);
  }
  int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
  for (int y = 0; y < p->ny; y++) {
    double fc[ORC_MAXQ], fo[ORC_MAXQ], grad[ORC_NGRAD];
    for (int x = 0; x < p->nx; x++) {
      gather_cell(p, &L, f_in, x, y, fc);
      if (m) central_gradients(p, m, x, y, grad);
      err |= collide_cell(p, fc, m ? grad : NULL, NULL, fo) != 0;
      for (int i = 0; i < L.V; i++) f_out[i * plane + (long long)y * p->nx + x] = fo[i];
    }
  }
  free(m);
  return err ? -1 : 0;
}

int orc_step_cells(const orc_params *p, const double *f_in, int ncell, const long long *cells, double *f_out) {
  orc_lattice L;
  if (orc_lattice_get(p->lattice, &L)) return -1;
  int neq, nreg;
  if (resolve_orders(p, &L, &neq, &nreg)) return -1;
  double *m = NULL;
  if (p->a1_source == 1) {
    m = (double *)malloc(sizeof(double) * 4 * (size_t)p->nx * (size_t)p->ny);
    if (!m) return -1;
    stream_moments(p, &L, f_in, m);
  }
  int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
  for (int k = 0; k < ncell; k++) {
    double fc[ORC_MAXQ], grad[ORC_NGRAD];
    int x = (int)(cells[k] % p->nx), y = (int)(cells[k] / p->nx);
    gather_cell(p, &L, f_in, x, y, fc);
    if (m) central_gradients(p, m, x, y, grad);
    err |= collide_cell(p, fc, m ? grad : NULL, NULL, f_out + (long long)k * L.V) != 0;
  }
  free(m);
  return err ? -1 : 0;
}

/* One step (pull streaming + RR collision) with a per-cell correction of a1^(2): delta[3][ny][nx] holds the
 * (xx, xy, yy) components added at each cell (orc_collide_delta). */
int orc_step_delta(const orc_params *p, const double *f_in, const double *delta, double *f_out) {
  orc_lattice L;
  if (orc_lattice_get(p->lattice, &L)) return -1;
  int neq, nreg;
  if (resolve_orders(p, &L, &neq, &nreg)) return -1;
  if (p->a1_source != 0 || p->collision != ORC_RR || p->thermal || !delta) return -1;
  long long plane = (long long)p->nx * p->ny;
  int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
  for (int y = 0; y < p->ny; y++) {
    double fc[ORC_MAXQ], fo[ORC_MAXQ];
    for (int x = 0; x < p->nx; x++) {
      long long c = (long long)y * p->nx + x;
      const double d[3] = {delta[c], delta[plane + c], delta[2 * plane + c]};
      gather_cell(p, &L, f_in, x, y, fc);
      err |= collide_cell(p, fc, NULL, d, fo) != 0;
      for (int i = 0; i < L.V; i++) f_out[i * plane + c] = fo[i];
    }
  }
  return err ? -1 : 0;
}

int orc_init(const orc_params *p, const double *rho, const double *ux, const double *uy, const double *T,
             const double *grad_u, double *f) {
  orc_lattice L;
  if (orc_lattice_get(p->lattice, &L)) return -1;
  int neq, nreg;
  if (resolve_orders(p, &L, &neq, &nreg)) return -1;
  long long plane = (long long)p->nx * p->ny;
#pragma omp parallel for schedule(static)
  for (long long c = 0; c < plane; c++) {
    double th = (T && p->thermal) ? T[c] : 1.0;
    double a0[(ORC_MAXN + 1) * 16], fe[ORC_MAXQ], fn[ORC_MAXQ];
    orc_a0(L.cs2, rho[c], ux[c], uy[c], th, ORC_MAXN, a0);
    orc_expand(&L, 0, neq, a0, fe);
    for (int i = 0; i < L.V; i++) fn[i] = 0.0;
    if (grad_u) {
      double g[2][2] = {{grad_u[0 * plane + c], grad_u[1 * plane + c]},   /* g[a][b] = d_b u_a */
                        {grad_u[2 * plane + c], grad_u[3 * plane + c]}};
      const double D = 2.0;
      double div = g[0][0] + g[1][1];
      double a1[(ORC_MAXN + 1) * 16];
      memset(a1, 0, sizeof(a1));
      for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) {
          double S = g[b][a] + g[a][b]; /* d_a u_b + d_b u_a */
          if (p->thermal && a == b) S -= (2.0 / D) * div;
          TEN(a1, 2, pair_tuple(a, b)) = -p->tau * rho[c] * L.cs2 * th * S;
        }
      if (p->thermal) {
        for (int t = 0; t < 8; t++) {
          int a = t & 1, b = (t >> 1) & 1, gg = (t >> 2) & 1;
          double uu[2] = {ux[c], uy[c]};
          TEN(a1, 3, t) = uu[a] * TEN(a1, 2, pair_tuple(b, gg)) + uu[b] * TEN(a1, 2, pair_tuple(a, gg)) +
                          uu[gg] * TEN(a1, 2, pair_tuple(a, b));
        }
      }
      orc_a1_recursive(L.cs2, rho[c], ux[c], uy[c], th, p->thermal, L.nmax, a0, a1);
      orc_expand(&L, 2, L.nmax, a1, fn);
    }
    for (int i = 0; i < L.V; i++) f[i * plane + c] = fe[i] + fn[i];
  }
  return 0;
}

int orc_moments(const orc_params *p, const double *f, double *rho, double *ux, double *uy, double *theta) {
  orc_lattice L;
  if (orc_lattice_get(p->lattice, &L)) return -1;
  long long plane = (long long)p->nx * p->ny;
#pragma omp parallel for schedule(static)
  for (long long c = 0; c < plane; c++) {
    double fc[ORC_MAXQ], r, u, v, th;
    for (int i = 0; i < L.V; i++) fc[i] = f[i * plane + c];
    orc_cell_moments(&L, p->thermal, fc, &r, &u, &v, &th);
    rho[c] = r;
    ux[c] = u;
    uy[c] = v;
    if (theta) theta[c] = th;
  }
  return 0;
}

int orc_conservation(const orc_params *p, const double *f, double *out4) {
  orc_lattice L;
  if (orc_lattice_get(p->lattice, &L)) return -1;
  long long plane = (long long)p->nx * p->ny;
  double m = 0, jx = 0, jy = 0, e = 0;
  for (long long c = 0; c < plane; c++)
    for (int i = 0; i < L.V; i++) {
      double v = f[i * plane + c];
      m += v;
      jx += v * L.cx[i];
      jy += v * L.cy[i];
      e += 0.5 * v * (double)(L.cx[i] * L.cx[i] + L.cy[i] * L.cy[i]);
    }
  out4[0] = m;
  out4[1] = jx;
  out4[2] = jy;
  out4[3] = e;
  return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
