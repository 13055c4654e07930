/*
 * liblbm: single-GPU (sm_103a) lattice-Boltzmann stream-and-collide with the
 * recursive-regularized (RR) collision of Coreixas, Wissocq, Puigt, Boussuge &
 * Sagaut, "Recursive regularization step for high-order lattice Boltzmann
 * methods" (arXiv 1704.04413), on the D2Q9, D2V17 and D2V37 lattices of its
 * Tab. I, with BGK (Sec. III.A) and projection regularization (PR, Sec. II.E)
 * as comparison modes.
 *
 * Conventions shared by every call:
 *  - Lattice units (Delta x = Delta t = 1, Sec. III.A).  Velocities are the
 *    integer on-grid vectors of Tab. I; cs^2 is the lattice constant.
 *  - Fields are row-major [ny][nx] arrays of double (x fastest).  Populations
 *    exchanged with the caller are [V][ny][nx] doubles in the library's
 *    velocity order (lbm_lattice_info).
 *  - theta is the temperature T/T0 in units of the lattice reference
 *    temperature (p = rho cs^2 theta).
 *  - `on_device` = 0: pointers are host memory (pageable or pinned); the call
 *    copies through the context's stream and returns when the data is usable.
 *    `on_device` = 1: pointers are device memory on the context's GPU (for
 *    example a torch tensor's data_ptr()); the call only enqueues work on the
 *    context's stream.
 *  - Return value: LBM_OK (0) or a negative LBM_E* code; no call aborts the
 *    process.  lbm_strerror() names a code; lbm_last_error() gives the detail
 *    of a context's last failure.
 *  - The caller owns every array it passes; the library copies what it needs.
 *    The library owns the device populations of a context.
 *  - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef LBM_H
#define LBM_H

#ifdef __cplusplus
extern "C" {
#endif

/* lattices (Tab. I) */
#define LBM_D2Q9 0
#define LBM_D2V17 1
#define LBM_D2V37 2

/* collision models */
#define LBM_BGK 0 /* f* = f - (f - f^(0)) / tau                      (Sec. III.A) */
#define LBM_PR 1  /* projected a1^(n), n = 2..N, Eq. RegularizedCollision (Sec. II.E) */
#define LBM_RR 2  /* a1^(2) projected, a1^(n>2) recursive (Eqs. MalaspinasRecursiveRelation,
                     RecursiveRelation_ThermalCase; App. C) */

/* boundary of an axis */
#define LBM_PERIODIC 0
#define LBM_ZERO_GRADIENT 1

#define LBM_A1_PROJECTION 0
#define LBM_A1_FINITE_DIFFERENCE 1 /* a pulled source outside the domain reads the nearest edge cell */

/* population storage / compute precision */
#define LBM_F64 0
#define LBM_F32 1
#define LBM_F16_SHIFT 2  /* binary16 of g_i = (f_i / w_i - rho0) * s */
#define LBM_BF16_SHIFT 3 /* bfloat16 of the same shifted deviation */
#define LBM_I16_SHIFT 4  /* 16-bit fixed point round(2^15 g) of the same g, |g| < 1 (saturating) */

/* status codes */
#define LBM_OK 0
#define LBM_EINVAL (-1)
#define LBM_ENOMEM (-2)
#define LBM_ECUDA (-3)
#define LBM_EUNSTABLE (-4)
#define LBM_ETIMEOUT (-5)
#define LBM_EIO (-6)

typedef struct lbm_ctx lbm_ctx; /* opaque, owned by the library */

typedef struct {
  int lattice;       /* LBM_D2Q9, LBM_D2V17, LBM_D2V37 */
  int hermite_order; /* N of the equilibrium f^(0),N (Sec. II.C): 2..lattice maximum (4, 3, 4) */
  int reg_order;     /* N of f^(1),N (Sec. II.D): 2..lattice maximum; 0 = lattice maximum */
  int collision;     /* LBM_BGK, LBM_PR, LBM_RR */
  int thermal;       /* 1: theta from the energy moment (D2V37 only); 0: theta = 1 */
  int nx, ny;        /* grid, each >= 1 */
  double nu;         /* kinematic viscosity; used when tau <= 0: tau = nu / cs^2 + 1/2 */
  double tau;        /* relaxation time of the discrete scheme (the shifted tau-bar of Sec. III.A), > 1/2 */
  int bc_x, bc_y;    /* LBM_PERIODIC or LBM_ZERO_GRADIENT */
  int storage;       /* LBM_F64, LBM_F32, LBM_F16_SHIFT, LBM_BF16_SHIFT, LBM_I16_SHIFT */
  int compute;       /* LBM_F64 (requires storage LBM_F64) or LBM_F32 (any other storage) */
  double rho0;       /* shifted storage reference density; 0 = 1 */
  double store_scale;/* shifted storage scale s, a power of two; 0 = 1 */
  void *stream;      /* cudaStream_t all work of the context is issued on; NULL = legacy default stream */
  double tau3, tau4; /* relaxation times tau-bar of the order-3 and order-4 coefficients of f^(1) (Eq.
                        GenRegCollision with one time per order, Sec. II.B: tau3 sets the heat
                        conductivity, Pr = (tau - 1/2) / (tau3 - 1/2)); 0 = tau.  Each > 1/2 when set;
                        PR and RR only (LBM_EINVAL with BGK) */
  int a1_source;     /* RR only: LBM_A1_PROJECTION (0, Eq. a12Proj and Eq. TempGradLBM) or
                        LBM_A1_FINITE_DIFFERENCE (1): a1^(2) = -tau rho cs^2 theta (grad u + grad u^T
                        [- div u I, thermal]) and the thermal temperature-gradient terms from second-order
                        central differences of the post-streaming fields (Sec. II.E).  Each step is then a
                        moments pass plus the step kernel; the context keeps 4 fields of the compute type
                        per cell for it.  LBM_EINVAL for other values, or with BGK / PR */
} lbm_params;

/* Lattice description in the library's velocity order (Tab. I).  Any output
 * pointer may be NULL; cx, cy, w must hold at least 37 entries.
 * Returns LBM_EINVAL for an unknown lattice. */
int lbm_lattice_info(int lattice, int *V, int *cx, int *cy, double *w, double *cs2);

/* Validate `p`, pick the kernels, allocate two population buffers of
 * V * ny * pitch elements on the current CUDA device.  No computation.
 * Errors: LBM_EINVAL (any field out of range, including tau <= 1/2,
 * thermal on a lattice other than D2V37, an order above the lattice's basis),
 * LBM_ENOMEM, LBM_ECUDA.  *out is NULL on failure. */
int lbm_create(const lbm_params *p, lbm_ctx **out);

/* Release the context and its device memory (NULL is accepted). */
void lbm_destroy(lbm_ctx *c);

/* Initial state f = f^(0),N(rho, u, theta) + f^(1) (Sec. III.B).  f^(1) is
 * built from the Chapman-Enskog a1^(2) of the supplied velocity gradients
 * (App. A: -tau rho cs^2 theta (S - (2/D) div u delta) thermal, -tau rho cs^2 S
 * isothermal) and the recursions for higher orders; grad_u = NULL gives
 * f = f^(0).  grad_u is [4][ny][nx] = d ux/dx, d ux/dy, d uy/dx, d uy/dy.
 * theta may be NULL (theta = 1).  Resets the step counter. */
int lbm_init(lbm_ctx *c, const double *rho, const double *ux, const double *uy, const double *theta,
             const double *grad_u, int on_device);

/* Advance n >= 0 time steps.  Each step is one fused kernel: pull streaming
 * (Sec. III.A, method of characteristics) then collision, double-buffered.
 * Enqueued on the context's stream; does not synchronize. */
int lbm_step(lbm_ctx *c, int n);

/* Macroscopic fields of the current state: rho, ux, uy and theta
 * (theta = 1 when isothermal); any output may be NULL.  Double precision: FP64 sums of
 * the populations, except FP32 storage, whose populations are summed in compensated
 * FP32 (about twice the FP32 precision, 1e-14 relative). */
int lbm_moments(lbm_ctx *c, double *rho, double *ux, double *uy, double *theta, int on_device);

/* FP64 domain sums: out[0] mass, out[1..2] momentum, out[3] total energy
 * (1/2 sum_i f_i |xi_i|^2), deterministic (fixed-order two-pass reduction).
 * Synchronizes.  Returns LBM_EUNSTABLE (sums still written) when a sum is not
 * finite. */
int lbm_conservation(lbm_ctx *c, double out[4]);

/* Flow diagnostics of Sec. III.B: out[0] = mean u^2, out[1] = std u^2,
 * out[2] = mean enstrophy density omega^2/2, out[3] = its std, with omega from
 * fourth-order centred differences (periodic wrap, clamped on zero-gradient
 * axes).  Synchronizes; LBM_EUNSTABLE when a value is not finite. */
int lbm_diagnostics(lbm_ctx *c, double out[4]);

/* Decoded populations f[V][ny][nx] (double) of the current state, and the
 * inverse (encodes into the storage format; rounding applies). */
int lbm_get_populations(lbm_ctx *c, double *f, int on_device);
int lbm_set_populations(lbm_ctx *c, const double *f, int on_device);

/* Number of steps since the last lbm_init / lbm_set_populations / lbm_load. */
long long lbm_step_count(const lbm_ctx *c);

/* Testing hook for the failure path of the staged step kernels (D2Q9 / D2V17
 * with binary16 or bfloat16 storage on x-periodic grids whose rows are whole
 * 16-byte units; other contexts never run them and ignore the hook).  Those
 * kernels copy population rows into shared memory asynchronously and wait for
 * the copies with a time limit; a wait that runs out records LBM_ETIMEOUT in
 * the context, which lbm_conservation / lbm_diagnostics then return.  With
 * block >= 0, the producer of that thread block announces the copies of its
 * last tile but does not issue them, so that block's compute warps give up
 * after wait_seconds (every earlier copy has been consumed, so none is in
 * flight when the block ends); block = -1 turns the hook off.  wait_seconds
 * (0 < w <= 10) replaces the default limit of 1 s for every wait of the
 * context's staged launches.  No counterpart in the paper.  LBM_EINVAL on bad
 * arguments. */
int lbm_test_inject_copy_fault(lbm_ctx *c, int block, double wait_seconds);

/* The relaxation time tau actually used (derived from nu when tau <= 0). */
double lbm_tau(const lbm_ctx *c);

/* Checkpoint: header (format tag, parameters, step count) and the raw stored
 * populations.  lbm_load requires a file written by a context with the same
 * lattice, grid, storage and collision parameters (LBM_EINVAL otherwise,
 * LBM_EIO on read/write failure); the restored state is bit-identical. */
int lbm_save(lbm_ctx *c, const char *path);
int lbm_load(lbm_ctx *c, const char *path);

/* Allocation-free conservation sums, for callers that cannot allocate device
 * memory when they need them: code whose device memory is owned by another
 * allocator (a framework pool), loops that forbid allocation after start-up,
 * hosts that hand out buffers but no allocation rights.  The paper has no
 * counterpart; this is a service entry point of the library.
 *
 * Computes the same four FP64 sums as lbm_conservation (mass, x- and
 * y-momentum, total energy), with the same kernels, from populations the
 * caller owns:
 *  - f: device pointer to populations in the storage format `storage`
 *    (LBM_F64 / LBM_F32 / LBM_F16_SHIFT / LBM_BF16_SHIFT / LBM_I16_SHIFT), SoA layout
 *    [V][ny][pitch] in the library's velocity order (lbm_lattice_info); plane
 *    stride ny * pitch elements, pitch >= nx.  rho0 and store_scale (0 = 1)
 *    describe shifted storage as in lbm_params.
 *  - out4: device pointer to 4 doubles, written on `stream` (cudaStream_t,
 *    NULL = legacy default stream); the call does not synchronize.
 * It allocates nothing: the per-block partial sums live in a static device
 * array of LBM_NOALLOC_MAX_CELLS / 256 * 4 doubles (2 MiB) that every GPU
 * loading the library holds until exit.  Grids above LBM_NOALLOC_MAX_CELLS
 * cells return LBM_EINVAL.  The first call on a device looks the array's
 * address up (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  All calls share the array: calls that
 * overlap on the GPU (other streams, other threads) race and must be ordered
 * by the caller.  The address is looked up once per device and kept: a
 * cudaDeviceReset of that device after its first call is not supported (the
 * module, and with it the array, may be reloaded elsewhere).  f and out4 must
 * be device (or managed) memory: host addresses return LBM_EINVAL; the sizes
 * of the buffers cannot be checked here.  Errors: LBM_EINVAL (bad argument,
 * size or pointer kind), LBM_ECUDA. */
#define LBM_NOALLOC_MAX_CELLS 16777216LL
int lbm_conservation_noalloc(int lattice, int storage, const void *f, int nx, int ny, int pitch, double rho0,
                             double store_scale, double *out4, void *stream);

/* ------------------------------------------------------------------------
 * Batched sweep: up to LBM_BATCH_MAX independent D2Q9 / D2V17 / isothermal
 * D2V37 grids of any sizes and relaxation times, mixed freely, advanced
 * together by one kernel launch per time step (recorded once in a CUDA graph
 * of two steps and replayed).  Per cell the arithmetic is that of lbm_step, so
 * a batched step is bit-identical to stepping each instance on its own.
 * ------------------------------------------------------------------------ */
#define LBM_BATCH_MAX 64
typedef struct lbm_batch lbm_batch; /* opaque, owned by the library */

/* One context per entry of ps[0..n-1] (lattice D2Q9, D2V17 or D2V37, isothermal,
 * compute LBM_F32 with any non-FP64 storage, a1 by projection; one collision model, one storage
 * format and one stream for all).  Errors as lbm_create; LBM_EINVAL for
 * n outside [1, LBM_BATCH_MAX] or mixed collision / storage / stream. */
int lbm_batch_create(const lbm_params *ps, int n, lbm_batch **out);
void lbm_batch_destroy(lbm_batch *b);

/* The i-th instance's context, owned by the batch: use it with lbm_init,
 * lbm_moments, lbm_conservation, ... (not lbm_destroy).  NULL if i is out of
 * range.  Stepping an instance alone with lbm_step puts it out of phase with
 * the others and makes lbm_batch_step return LBM_EINVAL. */
lbm_ctx *lbm_batch_context(lbm_batch *b, int i);

/* Advance every instance n >= 0 steps: graph replays of two steps each (the
 * graph is recorded on first use) plus one direct launch for an odd n.
 * Enqueued on the instances' stream; does not synchronize. */
int lbm_batch_step(lbm_batch *b, int n);

/* Launch shape of the batched kernel: threads per block (64, 128 or 256; each
 * thread updates two neighbouring cells of D2Q9 / D2V17, one of D2V37; a batch
 * holding D2V37 takes 128 only), rows per work item (1..64) and blocks per SM
 * of a persistent grid (0 = one block per work item). */
int lbm_batch_set_launch(lbm_batch *b, int threads, int rows, int blocks_per_sm);
int lbm_batch_get_launch(const lbm_batch *b, int *threads, int *rows, int *blocks_per_sm);

/* Autotuner: times every launch shape of the candidate set (threads
 * {64,128,256} (128 with D2V37) x rows {1,2,4,8} x blocks per SM {0 (one per item),2,4,8}) with 1 + `steps`
 * batched steps each and keeps the fastest; *best_ms (may be NULL) receives its
 * time per step.  Every timed step advances the instances, so tune before
 * lbm_init (or re-initialise afterwards).  Synchronizes. */
int lbm_batch_autotune(lbm_batch *b, int steps, double *best_ms);

/* ------------------------------------------------------------------------
 * Learned closure for coarse grids (a per-cell MLP, not part of the paper's
 * method; the plain RR step is both what it falls back to and the reference its
 * error is measured against).
 * Features of a cell: (rho - 1, ux, uy) / u0 of its 3x3 neighbourhood
 * (periodic), 27 values padded to LBM_CLOSURE_IN, BF16 row-major.  Outputs:
 * LBM_CLOSURE_OUT FP32 per cell, the first 3 being the subgrid stress
 * (xx, xy, yy) / u0^2 that a box filter of a finer grid leaves out of the
 * coarse equilibrium.  Network: IN -> HID -> HID -> HID -> OUT with GELU
 * (tanh form) on the hidden layers; BF16 weights and activations, FP32
 * accumulation (tensor-core MMA), FP32 master weights trained with Adam.
 * Parameter layout (LBM_CLOSURE_NPARAM floats): W1[HID][IN] b1[HID]
 * W2[HID][HID] b2[HID] W3[HID][HID] b3[HID] W4[OUT][HID] b4[OUT].
 * Array pointers are device memory unless named *_host.
 * ------------------------------------------------------------------------ */
#define LBM_CLOSURE_IN 32
#define LBM_CLOSURE_HID 64
#define LBM_CLOSURE_OUT 8
#define LBM_CLOSURE_NPARAM 10952
typedef struct lbm_closure lbm_closure;

/* Allocate a closure (weights zero, load them with lbm_closure_set_weights). */
int lbm_closure_create(lbm_closure **out);
void lbm_closure_destroy(lbm_closure *cl);
/* Host FP32 parameters (n must be LBM_CLOSURE_NPARAM); setting resets the Adam state. */
int lbm_closure_set_weights(lbm_closure *cl, const float *w_host, int n);
int lbm_closure_get_weights(lbm_closure *cl, float *w_host, int n);
/* y[n][OUT] = MLP(x[n][IN]) on `stream` (device buffers, both 16-byte aligned, else LBM_EINVAL), on the
 * 5th-generation tensor core (tcgen05 MMAs into tensor memory, 128 rows at a time).  Every wait on the tensor
 * core is bounded (1 s); a wait that ran out leaves NaN in the rows it did not finish. */
int lbm_closure_forward(lbm_closure *cl, const void *x, int n, float *y, void *stream);
/* One Adam step (lr, beta1 0.9, beta2 0.999) on the mean squared error of the 3 used outputs over
 * the n samples (x, y_target[n][OUT]); *loss_host (may be NULL) receives the loss before the step. */
int lbm_closure_train_step(lbm_closure *cl, const void *x, const float *y_target, int n, float lr,
                           float *loss_host, void *stream);
/* Gradient of that loss with respect to every parameter (host array of LBM_CLOSURE_NPARAM floats),
 * without updating; synchronizes. */
int lbm_closure_gradients(lbm_closure *cl, const void *x, const float *y_target, int n, float *grad_host,
                          float *loss_host);
/* Features of every cell of double fields rho, ux, uy [ny][nx] into x[nx*ny][IN]. */
int lbm_closure_features(const double *rho, const double *ux, const double *uy, int nx, int ny, double u0,
                         void *x, void *stream);
/* Box filter by `factor` of fine fields [ny][nx] (both divisible by factor): coarse rho, u (density-
 * weighted) into rho_c, ux_c, uy_c [ny/f][nx/f] and the subgrid stress / u0^2 into y[..][OUT]. */
int lbm_closure_coarsen(const double *rho, const double *ux, const double *uy, int nx, int ny, int factor,
                        double u0, double *rho_c, double *ux_c, double *uy_c, float *y, void *stream);
/* n RR steps of a D2Q9 FP32 context whose a1^(2) gets the closure's correction
 * Delta a1 = u0^2 y / (1 - 1/tau), y predicted each step from the current fields.  Two launches per
 * step (the moments, then features + network + collision fused per tile of 128 cells, the network on the
 * tensor core as in lbm_closure_forward); the result is bitwise that of lbm_moments +
 * lbm_closure_features + lbm_closure_forward + lbm_closure_apply.
 * Allocates a work area of 96 B per cell on first use.  LBM_EINVAL unless the context is D2Q9, RR,
 * isothermal, FP32 storage, a1 by projection. */
int lbm_step_closure(lbm_ctx *c, lbm_closure *cl, double u0, int n);
/* One RR step of such a context with a caller-supplied correction field y[nx*ny][LBM_CLOSURE_OUT]
 * (device, FP32; components 0..2 = xx, xy, yy of Delta a1 / u0^2 scaled as above), enqueued on the
 * context's stream.  No counterpart in the paper: the entry point of a closure computed elsewhere. */
int lbm_closure_apply(lbm_ctx *c, const float *y, double u0);

/* Text of a status code / of the context's last failure. */
const char *lbm_strerror(int code);
const char *lbm_last_error(const lbm_ctx *c);

#ifdef __cplusplus
}
#endif
#endif
