/*
 * FP64 CPU oracle for the recursive-regularized (RR) lattice-Boltzmann step of
 * Coreixas et al., "Recursive regularization step for high-order lattice
 * Boltzmann methods" (arXiv 1704.04413).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
 * its Python binding) may include, link or call this code; only tests/, the
 * smoke check and the CPU-baseline leg of the benchmark do.  It shares no
 * source, table or helper with the CUDA path.
 *
 * Everything is written in the paper's tensor-index notation: a Hermite tensor
 * or coefficient of order n is stored for every index tuple
 * alpha = (alpha_1..alpha_n) in {x,y}^n, tuple t encoding alpha_k in bit k
 * (0 = x, 1 = y), so a rank-n tensor has 2^n entries.  Nothing is unrolled.
 *
 * Parity pins: every function here is checked by tests against something
 * other than itself (library Hermite polynomials, Gaussian quadrature of the
 * continuous Maxwellian, the Chapman-Enskog closed forms, conservation laws,
 * the exact Riemann solution, the viscous decay of a shear wave).
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_D2Q9 0
#define ORC_D2V17 1
#define ORC_D2V37 2

#define ORC_BGK 0
#define ORC_PR 1
#define ORC_RR 2

#define ORC_PERIODIC 0
#define ORC_ZERO_GRADIENT 1

#define ORC_MAXQ 64
#define ORC_MAXN 4 /* highest Hermite order handled (Sec. II.C: order 4 suffices) */

/* A two-dimensional lattice E^V_{2,Q} of Tab. I. */
typedef struct {
  int V;                 /* number of discrete velocities */
  int cx[ORC_MAXQ];      /* integer (on-grid) velocity components */
  int cy[ORC_MAXQ];
  double w[ORC_MAXQ];    /* quadrature weights */
  double cs2;            /* lattice constant c_s^2 = r T0 */
  int nmax;              /* highest Hermite order present in the kept basis */
  int keep[ORC_MAXN + 1][ORC_MAXN + 1]; /* keep[nx][ny]: tensor with nx x- and ny y-indices in the basis */
} orc_lattice;

typedef struct {
  int lattice;        /* ORC_D2Q9 / ORC_D2V17 / ORC_D2V37 */
  int hermite_order;  /* N of the equilibrium expansion f^(0),N */
  int reg_order;      /* N of the regularized f^(1),N; 0 = lattice maximum */
  int collision;      /* ORC_BGK / ORC_PR / ORC_RR */
  int thermal;        /* 1: theta from the energy moment (D2V37 only); 0: theta = 1 */
  int nx, ny;
  double tau;         /* relaxation time tau-bar of the discrete scheme (Sec. III.A); that of order 2 */
  int bc_x, bc_y;     /* ORC_PERIODIC / ORC_ZERO_GRADIENT */
  double tau3, tau4;  /* relaxation times of the order-3 and order-4 coefficients of f^(1) (Eq.
                         GenRegCollision with one time per order, Sec. II.B); 0 = tau.  PR/RR only */
  int a1_source;      /* RR only: 0 = a1^(2) (and the thermal a1^(3)) by projection of f - f^(0) (Eq. a12Proj,
                         Eq. TempGradLBM); 1 = by finite differences of the velocity (and temperature)
                         field (Sec. II.E allows finite differences in place of the projection) */
} orc_params;

/* Gradients handed to the finite-difference collision, per cell:
 * d ux/dx, d ux/dy, d uy/dx, d uy/dy, d theta/dx, d theta/dy. */
#define ORC_NGRAD 6

/* Lattice of Tab. I (0 on success, -1 for an unknown id). */
int orc_lattice_get(int lattice, orc_lattice *out);

/* Hermite tensor H^(n)_alpha evaluated at velocity (xx, xy) for lattice constant
 * cs2, by the Rodrigues recursion of App. B. */
double orc_hermite(int n, int tuple, double xx, double xy, double cs2);

/* Equilibrium Hermite coefficients a0^(n) for n = 0..nmax (App. B recursion).
 * a0 is [ORC_MAXN+1][16]; entry [n][t] is a0^(n)_alpha(t). */
void orc_a0(double cs2, double rho, double ux, double uy, double theta, int nmax, double *a0);

/* Recursive off-equilibrium coefficients from a1^(2) (and a1^(3) when thermal):
 * isothermal: Eq. (MalaspinasRecursiveRelation) for n = 3..nmax;
 * thermal:    a1^(3) given, Eq. (RecursiveRelation_ThermalCase) for n = 4..nmax.
 * a1 is [ORC_MAXN+1][16]; a1[2] (and a1[3] if thermal) are inputs. */
void orc_a1_recursive(double cs2, double rho, double ux, double uy, double theta, int thermal, int nmax,
                      const double *a0, double *a1);

/* Thermal a1^(3) rebuilt from projected a1^(2), a1^(3) (App. C steps 1-4). */
void orc_a1_third_thermal(double ux, double uy, const double *a1_2, const double *a1_3_proj, double *a1_3);

/* Truncated expansion w_i sum_{n=nmin..nmax} sum_alpha H_alpha a_alpha / (n! cs^2n) restricted to the kept basis. */
void orc_expand(const orc_lattice *L, int nmin, int nmax, const double *coef, double *f);

/* Moments of one cell: rho, ux, uy, theta (theta = 1 when !thermal). */
void orc_cell_moments(const orc_lattice *L, int thermal, const double *f, double *rho, double *ux, double *uy,
                      double *theta);

/* Collision of one cell (post-streaming f_in[V] -> post-collision f_out[V]). 0 on success; -1 when
 * p->a1_source asks for gradients (use orc_collide_fd). */
int orc_collide(const orc_params *p, const double *f_in, double *f_out);

/* The same with a1 built from the given gradients grad[ORC_NGRAD] (RR with a1_source = 1):
 *   a1^(2)_ab = -tau rho cs^2 theta (d_a u_b + d_b u_a - delta_ab div u)   (thermal; D = 2)
 *   a1^(2)_ab = -tau rho cs^2 (d_a u_b + d_b u_a)                           (isothermal)
 * and, thermal, mu cs^2 d_g theta = tau_3 rho cs^4 theta d_g theta in place of Eq. TempGradLBM. */
int orc_collide_fd(const orc_params *p, const double *f_in, const double *grad, double *f_out);

/* Isothermal RR collision of one cell with a correction of the non-equilibrium stress: delta[3] =
 * (xx, xy, yy) is added to the projected a1^(2) (xy to both off-diagonal entries), and the higher orders
 * follow by Eq. (MalaspinasRecursiveRelation) from the corrected a1^(2).  -1 unless RR, isothermal,
 * a1 by projection. */
int orc_collide_delta(const orc_params *p, const double *f_in, const double *delta, double *f_out);

/* One full step (pull streaming + collision) on f_in[V][ny][nx] -> f_out. */
int orc_step(const orc_params *p, const double *f_in, double *f_out);

/* Pull streaming + collision only at the listed cells (cell = y*nx + x);
 * f_out is [ncell][V]. */
int orc_step_cells(const orc_params *p, const double *f_in, int ncell, const long long *cells, double *f_out);

/* One step with orc_collide_delta at every cell, delta[3][ny][nx]. */
int orc_step_delta(const orc_params *p, const double *f_in, const double *delta, double *f_out);

/* Initial populations f^(0),N (+ f^(1) from analytic velocity gradients when
 * grad_u != NULL; grad_u is [4][ny][nx] = dux/dx, dux/dy, duy/dx, duy/dy).
 * T (theta) may be NULL (theta = 1). */
int orc_init(const orc_params *p, const double *rho, const double *ux, const double *uy, const double *T,
             const double *grad_u, double *f);

/* Fields rho, ux, uy, theta [ny][nx] of f (theta may be NULL). */
int orc_moments(const orc_params *p, const double *f, double *rho, double *ux, double *uy, double *theta);

/* Domain sums of mass, x- and y-momentum and total energy (1/2 sum f xi^2). */
int orc_conservation(const orc_params *p, const double *f, double *out4);

/* Number of OpenMP threads the oracle uses. */
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
