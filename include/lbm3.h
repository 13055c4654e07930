/* C ABI of the three-dimensional lattices of Tab. II (App. D of Coreixas et al., "Recursive
 * regularization step for high-order lattice Boltzmann methods", arXiv 1704.04413): D3Q19, D3Q27, D3V39
 * and D3Q103, isothermal (theta = 1), with the same collision modes as the 2D library (include/lbm.h):
 * BGK (Sec. III.A), projection regularization PR-N (Sec. II.E) and recursive regularization RR-N
 * (Eq. MalaspinasRecursiveRelation), rebuilt by Eq. GenRegCollision with one relaxation time.
 *
 * Conventions as in lbm.h: status codes LBM_OK / LBM_EINVAL / LBM_ENOMEM / LBM_ECUDA / LBM_EUNSTABLE, the
 * storage and compute constants, the boundary constants; no exception crosses the ABI; a context is not
 * thread-safe.  Fields are dense double arrays [nz][ny][nx] (x fastest); vectors are [3][nz][ny][nx]
 * (x, y, z components), velocity gradients [9][nz][ny][nx] with component 3a + b = d u_a / d x_b.
 * Pointers are host memory when on_device = 0, device memory of the context's device when on_device = 1
 * (read or written on the context's stream).  The caller owns every array it passes; the library owns
 * the populations.
 *
 * The paper runs no 3D simulation; these entry points extend its method to its own Tab. II lattices. */
#ifndef LBM3_H
#define LBM3_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Lattice ids (Tab. II), with the highest Hermite order of each kept basis:
 * D3Q19 3 (orders <= 3 without H_xxx-type and H_xyz), D3Q27 6 (every exponent <= 2: the complete basis),
 * D3V39 3 (every order-3 tensor), D3Q103 4 (every order-4 tensor). */
#define LBM_D3Q19 10
#define LBM_D3Q27 11
#define LBM_D3V39 12
#define LBM_D3Q103 13

typedef struct lbm3_ctx lbm3_ctx; /* opaque, owned by the library */

typedef struct {
  int lattice;       /* LBM_D3Q19 ... LBM_D3Q103 */
  int hermite_order; /* N of the equilibrium f^(0),N: 1..lattice maximum */
  int reg_order;     /* N of f^(1),N: 2..lattice maximum; 0 = lattice maximum */
  int collision;     /* LBM_BGK, LBM_PR, LBM_RR */
  int nx, ny, nz;    /* >= 1 */
  double nu, tau;    /* exactly one > 0: tau is tau-bar of the discrete scheme, nu = cs^2 (tau - 1/2) */
  int bc_x, bc_y, bc_z; /* LBM_PERIODIC or LBM_ZERO_GRADIENT (clamped pull source) */
  int storage;       /* LBM_F64, LBM_F32, LBM_F16_SHIFT, LBM_BF16_SHIFT, LBM_I16_SHIFT */
  int compute;       /* LBM_F64 (with LBM_F64 storage) or LBM_F32 (any other storage) */
  double rho0;       /* shifted storage reference density; 0 = 1 */
  double store_scale;/* shifted storage scale s, a power of two; 0 = 1 */
  void *stream;      /* cudaStream_t; NULL = legacy default stream */
} lbm3_params;

/* Velocities (cx, cy, cz), weights and cs^2 of a lattice, in the library's order; any output may be
 * NULL (cx, cy, cz, w hold at least 103 entries).  LBM_EINVAL for an unknown id. */
int lbm3_lattice_info(int lattice, int *V, int *cx, int *cy, int *cz, double *w, double *cs2);

/* Validate p, allocate the two population buffers (2 V nx ny nz sizeof(storage) bytes, rows padded to 128
 * bytes) on the current device.  LBM_EINVAL for invalid parameters (nothing allocated), LBM_ENOMEM. */
int lbm3_create(const lbm3_params *p, lbm3_ctx **out);
void lbm3_destroy(lbm3_ctx *c);

/* f = f^(0),N + f^(1) (Sec. III.B): f^(1) from a1^(2) = -tau rho cs^2 (grad u + grad u^T) and its recursion
 * to the lattice's highest order, or f = f^(0) when grad is NULL.  rho [cells], u [3][cells].  Host
 * arrays go through a device work area of 104 B per cell allocated on first use. */
int lbm3_init(lbm3_ctx *c, const double *rho, const double *u, const double *grad, int on_device);

/* n >= 0 time steps: pull streaming then collision fused in one pass per step, double-buffered.
 * Enqueued on the context's stream; does not synchronize.  Grids periodic in x with nx a multiple of
 * 16 bytes' worth of cells run the staged kernel (populations brought to shared memory by asynchronous
 * bulk copies a few row tiles ahead; D3Q103 excepted); the others the direct-load kernel, in one launch, or
 * on large grids two (the rows near the y and z faces separately).  All compute the same step. */
int lbm3_step(lbm3_ctx *c, int n);

/* rho [cells] and u [3][cells] of the current state; either may be NULL. */
int lbm3_moments(lbm3_ctx *c, double *rho, double *u, int on_device);

/* FP64 domain sums: out[0] mass, out[1..3] momentum.  Deterministic (fixed-order two-pass reduction);
 * synchronizes; LBM_EUNSTABLE (sums still written) when a sum is not finite; LBM_ETIMEOUT when a step
 * kernel gave up waiting (1 s unless lbm3_test_inject_copy_fault shortened it) on its own asynchronous
 * copies since the context was created (not expected: the word exists so that no wait is unbounded). */
int lbm3_conservation(lbm3_ctx *c, double out[4]);

/* Decoded populations f[V][nz][ny][nx] (library velocity order), and the inverse (encodes into the
 * storage format).  lbm3_get_populations synchronizes and reports the copy-wait status as
 * lbm3_conservation does. */
int lbm3_get_populations(lbm3_ctx *c, double *f, int on_device);
int lbm3_set_populations(lbm3_ctx *c, const double *f, int on_device);

/* The relaxation time tau-bar in use. */
double lbm3_tau(const lbm3_ctx *c);

/* Testing hook for the staged kernel's failure path, as lbm_test_inject_copy_fault in lbm.h: with
 * block >= 0 that thread block's producer announces the copies of its last tile but does not issue them,
 * so its compute warps' wait runs out after wait_seconds (0 < w <= 10, the limit of every wait of the
 * context's staged launches; default 1 s) and lbm3_conservation returns LBM_ETIMEOUT; block = -1 turns
 * it off.  Contexts that do not run the staged kernel ignore it.  No counterpart in the paper. */
int lbm3_test_inject_copy_fault(lbm3_ctx *c, int block, double wait_seconds);

#ifdef __cplusplus
}
#endif

#endif /* LBM3_H */
