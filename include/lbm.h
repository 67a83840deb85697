/*
 * lbm.h - C ABI of the GB300 lattice Boltzmann library for the method of
 * Coelho, Ilha and Doria, "A lattice Boltzmann method based on generalized
 * polynomials and its application for electrons in metals" (arXiv:1510.07328).
 *
 * The library advances d2v9 populations with the K = 3 equilibrium expanded in
 * polynomials orthonormal under the Fermi-Dirac equilibrium itself
 * (Eq. (expansao0); the geometric-velocity form printed in Sect. "The Gaussian
 * quadrature"), relaxed by BGK (the LBGK equation of the same section) after
 * pull streaming.  Per cell and step it gathers the nine populations, forms
 * n = I_0, u_0 = j/n (the moment update after the LBGK equation) and the
 * energy E = sum f |e|^2, reads J_2 = 3 (E/n - |u_0|^2)/D, inverts the
 * Fermi-Dirac moment ratio J_2(x) = f_2^2/(f_1 f_3) for x = mu/theta
 * (I_2N = (2 pi)^{D/2} theta^{N+D/2} f_{N+D/2}(x), Sect. "Generalized
 * polynomials in D dimensions"), evaluates J_4 = f_3^2/(f_2 f_4), builds f_eq
 * and relaxes.
 *
 * The d1v3 lattice (D = 1, velocities 0, +1, -1, weights W_0 = n (1 - J_2/3),
 * W_+-1 = n J_2/6) runs the same calls with the theta = 0 or Maxwell-Boltzmann
 * closure (lbm_params.dim = 1).
 *
 * Conventions shared by every call:
 *  - Velocity order a = 0..8 on d2v9: rest; (1,0), (0,1), (-1,0), (0,-1);
 *    (1,1), (-1,1), (-1,-1), (1,-1).  On d1v3, a = 0..2: rest, +1, -1.
 *  - Arrays of per-cell values are row-major [ny][nx] (x fastest), one array
 *    per problem; populations are [Q][ny][nx] with Q = 9 (d2v9) or 3 (d1v3,
 *    ny = 1).
 *  - All calls are asynchronous on the context's CUDA stream unless stated;
 *    a call that writes host memory synchronises that stream before it returns.
 *  - Every call returns an lbm_status; nothing aborts or throws.  On failure
 *    lbm_last_error() returns a message (per context; lbm_last_error(NULL)
 *    gives the last failure of a call without a context).  An asynchronous CUDA error
 *    surfaces at the next call that synchronises (LBM_ECUDA).
 *  - Pointers are plain host or device addresses as stated per argument; the
 *    library never frees memory it did not allocate.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque; owned by the library */

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,       /* bad argument: NULL, size, tau <= 1/2, n <= 0, t out of range */
  LBM_ENOMEM = 2,       /* device or host allocation failed */
  LBM_ECUDA = 3,        /* a CUDA call failed (message in lbm_last_error) */
  LBM_ETIMEOUT = 4,     /* a bounded device wait gave up */
  LBM_EUNSUPPORTED = 5  /* valid but not implemented combination */
} lbm_status;

/* Statistics of the weight / equilibrium (Sect. "Generalized polynomials in D
 * dimensions").  FD: J_2 from the energy moment, J_4 from the inverted x.
 * FD_T0: the theta = 0 closure of Sect. "Numerical simulations for electrons
 * in metals", J_N = 1 + 2/(N + D) constant.  MB: J_N = 1, the Hermite D2Q9
 * limit.  FT: FD statistics at a temperature theta fixed per problem, the
 * literal reading of the moment update after the LBGK equation (which names
 * only I_0 and u_0): x follows from the density alone, n = 2 pi theta
 * f_1(x), and J_2, J_4 are the FD values at that x; energy is not conserved
 * by a collision.  theta = n_ref t_ref/(2 pi) of each problem (so n_ref and
 * t_ref are required at every precision).  d2v9 with the exact inversion and
 * without obstacles or forces only. */
typedef enum { LBM_STAT_FD = 0, LBM_STAT_FD_T0 = 1, LBM_STAT_MB = 2, LBM_STAT_FT = 3 } lbm_stat;

/* Population storage.  F64: f itself in FP64, all arithmetic FP64.
 * F32_DEV / BF16_DEV: the deviation g_a = f_a - W_a^ref from a per-problem
 * constant W^ref = w_a(J_2(t_ref)) n_ref, stored in FP32 / BF16, moment sums
 * and equilibrium in FP32.  These contexts also initialise in FP32 (the
 * step's deviation-form equilibrium, closure from t in FP32), and
 * lbm_moments takes x, t, T and mu from the FP32 inversion (n, u and the
 * diag sums stay FP64 sums of the stored values). */
typedef enum { LBM_F64 = 0, LBM_F32_DEV = 1, LBM_BF16_DEV = 2 } lbm_prec;

/* The Fermi-Dirac inversion J_2 -> (x, J_4) of Sect. "Generalized polynomials
 * in D dimensions" (J_2 = f_2^2/(f_1 f_3) solved for x, J_4 = f_3^2/(f_2 f_4)).
 * EXACT: in the storage's arithmetic (FP64 Newton for LBM_F64; FP32 fits in
 * delta = 3/2 - J_2 for deviation storage).  SURROGATE: the learned inversion
 * (lbm_surrogate_*).  EXACT_F64: deviation storage (FP32 or BF16) whose step
 * keeps FP32 populations, sums and equilibrium but inverts in FP64: delta from
 * the FP32 deviation moments, x by FP64 Newton to 1e-13, J_4 rounded once to
 * FP32; the initial closure J_2(t), J_4(t) and the T, mu, t that lbm_moments
 * reports come from the same FP64 functions.  LBM_STAT_FD on d2v9 only (else
 * LBM_EUNSUPPORTED); with LBM_F64 it is the same as EXACT.  No obstacles or
 * forces. */
typedef enum { LBM_INV_EXACT = 0, LBM_INV_SURROGATE = 1, LBM_INV_EXACT_F64 = 2 } lbm_inv;

typedef enum { LBM_BC_PERIODIC = 0, LBM_BC_BOUNCEBACK = 1 } lbm_bc;

/* One lattice.  bc_*: LBM_BC_*; halfway bounce-back walls sit half a cell
 * outside the first and last row/column.  n_ref, t_ref: the reference state
 * of the deviation storage (ignored for LBM_F64; n_ref > 0, t_ref in
 * [1e-3, 10]). */
typedef struct {
  int32_t nx, ny;
  double tau;
  int32_t bc_x, bc_y;
  double n_ref, t_ref;
} lbm_problem;

typedef struct {
  int32_t dim;       /* 2 (d2v9) or 1 (d1v3: every problem ny = 1, stat FD_T0 or MB,
                        exact inversion); other values -> LBM_EUNSUPPORTED */
  int32_t order;     /* 3 (K = 3 expansion); other values -> LBM_EUNSUPPORTED */
  int32_t stat;      /* lbm_stat */
  int32_t prec;      /* lbm_prec */
  int32_t inv;       /* lbm_inv */
  int32_t nproblems; /* >= 1; all problems advance together in one launch per step */
  const lbm_problem* problems; /* host array of nproblems entries, copied */
} lbm_params;

/* lbm_create: validate p, allocate the two population buffers and tables on
 * the current CUDA device, and bind the context to `cuda_stream` (a
 * cudaStream_t; NULL = legacy default stream).  Populations start at zero;
 * call lbm_init_riemann for every problem before stepping.
 * Errors: LBM_EINVAL (p or out NULL, nx or ny < 1, tau <= 0.5, bad enum,
 * reference state out of range, d1v3 problem with ny != 1), LBM_EUNSUPPORTED
 * (dim not 1 or 2, order != 3, d1v3 with LBM_STAT_FD: with three velocities
 * n, j and E fix every population, so no finite-temperature collision
 * exists; the learned inversion on d1v3), LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_create(const lbm_params* p, void* cuda_stream, lbm_ctx** out);

/* Initial state of one problem (the Riemann problems of Sect. "Numerical
 * simulations for electrons in metals" and their 2D analogues).  The
 * populations are set to the equilibrium f_eq(n, u_0, t) of each cell.
 *  HALF:     s[0] for x < x0, s[1] for x >= x0.
 *  QUADRANT: s[q], q = (x >= x0) + 2 (y >= y0).
 *  FIELD:    per-cell arrays n, ux, uy, t of nx*ny doubles each, host or
 *            device memory per field_on_device; read during the call only
 *            (with host arrays the call synchronises before it returns).
 *            Host arrays in page-locked memory that the GPU can address
 *            (cudaHostAlloc, or registered) are read in place by the kernel,
 *            over the coherent chip-to-chip link on a Grace-Blackwell node;
 *            pageable ones go through a staging copy.
 * t is T/T_F (T_F the theta = 0 chemical potential at the cell's density);
 * it must lie in [1e-3, 10] for LBM_STAT_FD and is ignored otherwise.  On
 * d1v3 QUADRANT is invalid and uy is ignored (FIELD still takes all four
 * arrays). */
typedef enum { LBM_INIT_HALF = 0, LBM_INIT_QUADRANT = 1, LBM_INIT_FIELD = 2 } lbm_init_kind;
typedef struct { double n, ux, uy, t; } lbm_state;
typedef struct {
  int32_t kind;
  int32_t x0, y0;
  lbm_state s[4];
  const double* n;
  const double* ux;
  const double* uy;
  const double* t;
  int32_t field_on_device;
} lbm_riemann_desc;

/* Errors: LBM_EINVAL (problem index, kind, NULL field, n <= 0 or t out of
 * range in a region state; per-cell field values are not checked on the
 * host; QUADRANT on d1v3), LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_init_riemann(lbm_ctx* ctx, int32_t problem, const lbm_riemann_desc* d);

/* Advance every problem by nsteps LBGK steps (pull stream + collide, one
 * kernel launch per step; repeated steps replay a captured CUDA graph).
 * Asynchronous.  Errors: LBM_EINVAL (nsteps < 0), LBM_ECUDA. */
lbm_status lbm_step(lbm_ctx* ctx, int32_t nsteps);

/* Tiling of the step launch.  A tile is 128 consecutive cells of
 * rows_per_tile consecutive rows of one problem (1, 2, 4 or 8 rows); every
 * problem of the context is cut into tiles and all tiles advance in one
 * launch per step.  ctas = 0 launches one CTA per tile; ctas > 0 launches that
 * many CTAs (a persistent grid) that walk the tiles in turn.  The default is
 * 4 rows, one CTA per tile. */
typedef struct {
  int32_t rows_per_tile;
  int32_t ctas;
  double ms_per_step; /* lbm_autotune: measured time of the chosen tiling */
} lbm_tiling;

/* Set the tiling (drops captured graphs).  Synchronises the context's stream.
 * Errors: LBM_EINVAL (rows not in {1, 2, 4, 8}, ctas < 0), LBM_ECUDA. */
lbm_status lbm_set_tiling(lbm_ctx* ctx, int32_t rows_per_tile, int32_t ctas);
lbm_status lbm_get_tiling(const lbm_ctx* ctx, lbm_tiling* out);

/* Time rows {1, 2, 4, 8} x ctas {one per tile, 4, 8 and 16 per SM} on the
 * context's own problems (steps_per_candidate timed steps each, after one
 * untimed step) and keep the fastest.  Each trial reads the current
 * populations and writes only the other buffer, so the state is unchanged.
 * Synchronises the stream; chosen may be NULL.  Errors: LBM_EINVAL, LBM_ECUDA. */
lbm_status lbm_autotune(lbm_ctx* ctx, int32_t steps_per_candidate, lbm_tiling* chosen);

/* Per-run diagnostics of lbm_moments: totals over the problem's cells (FP64,
 * summed in a fixed order, so identical states give identical sums) and
 * counts of cells whose inversion was clamped to t in [1e-3, 10] or whose
 * state is not finite. */
typedef struct {
  double sum_n, sum_jx, sum_jy, sum_E;
  int64_t clamped;
  int64_t nonfinite;
} lbm_diag;

/* Macroscopic fields of one problem from the current populations, each an
 * array of nx*ny doubles (any pointer may be NULL to skip that field):
 *  n; u_0 = (ux, uy) in lattice units; T = theta and mu in the paper's
 *  dimensionless units (m = k_B = hbar = 1); t = T/T_F.  For LBM_STAT_FD_T0,
 *  T = t = 0 and mu = T_F, the theta = 0 chemical potential at density n
 *  (n/(2 pi) on d2v9, n^2/8 on d1v3); for LBM_STAT_MB, T, mu, t are NaN;
 *  for LBM_STAT_FT, T = theta, t = 2 pi theta/n and mu = theta x(n), with no
 *  clamped cells counted.
 *  On d1v3 uy is 0 and diag.sum_E = sum of f e^2.
 * out_on_device != 0: the pointers are device memory and the call is
 * asynchronous; otherwise host memory and the call synchronises (host arrays
 * in page-locked memory that the GPU can address are written in place by the
 * kernel, pageable ones through a staging copy).  diag may be NULL; if not,
 * the call synchronises and fills it (host memory). */
lbm_status lbm_moments(lbm_ctx* ctx, int32_t problem, double* n, double* ux, double* uy,
                       double* T, double* mu, double* t, int32_t out_on_device, lbm_diag* diag);

/* FP32 field exchange for contexts with FP32 or BF16 deviation storage on
 * d2v9 (whose state carries FP32 precision): the FIELD initialisation and the
 * moments with float arrays, half the bytes of the double calls over the host
 * link.  The paper has no counterpart (an interface of this implementation).
 *
 * lbm_init_fields_f32: per-cell arrays n, ux, uy, t of nx*ny floats, host or
 * device memory per on_device, with the meaning, checks and host-memory
 * handling of FIELD in lbm_init_riemann; the result equals that of FIELD
 * given the same values as doubles.
 *
 * lbm_moments_f32: as lbm_moments, into float arrays: each value is the
 * double that lbm_moments reports, rounded once to float.  diag (FP64 sums)
 * as lbm_moments.
 *
 * Errors: as the double calls; LBM_EUNSUPPORTED for FP64 storage or d1v3. */
lbm_status lbm_init_fields_f32(lbm_ctx* ctx, int32_t problem, const float* n, const float* ux, const float* uy,
                               const float* t, int32_t on_device);
lbm_status lbm_moments_f32(lbm_ctx* ctx, int32_t problem, float* n, float* ux, float* uy, float* T, float* mu,
                           float* t, int32_t out_on_device, lbm_diag* diag);

/* Checkpoint / resume: copy the populations f_a (FP64, [Q][ny][nx]) of one
 * problem out of or into the library.  Storage of reduced precision converts
 * (f = W^ref + g on the way out, g = f - W^ref rounded on the way in).
 * on_device selects device or host memory for f; host copies synchronise. */
lbm_status lbm_get_populations(lbm_ctx* ctx, int32_t problem, double* f, int32_t on_device);
lbm_status lbm_set_populations(lbm_ctx* ctx, int32_t problem, const double* f, int32_t on_device);

/* Rigid obstacles and a constant body force (the porous-medium experiment of
 * Sect. "Numerical simulations for electrons in metals": electrons driven by
 * an external force through rigid obstacles, bounce-back on the obstacles).
 *
 * lbm_set_obstacles: solid = nx*ny bytes, row-major [ny][nx], nonzero marks a
 * solid cell; host or device memory per on_device, read during the call
 * only; NULL removes the problem's obstacles.  A fluid cell whose pull source
 * is solid takes the opposite population of its own cell (halfway
 * bounce-back, as at the walls); solid cells are not updated and
 * lbm_moments reports them as n = u = T = mu = t = 0, outside the diag sums.
 * The call also builds each cell's 16-bit pull code (which of its nine pull
 * sources are solid or beyond a wall, and whether it is solid itself), which
 * the FP32 / BF16 step pulls through.  The first call allocates three bytes
 * per cell of the context (mask and codes).
 *
 * lbm_set_force: force (fx, fy) per cell and step in lattice units, applied
 * by the exact difference method: after the BGK relaxation each fluid cell
 * receives f_eq(n, u_0 + F/n) - f_eq(n, u_0) on the same moments, which adds
 * exactly F of momentum and no mass.  lbm_moments then reports the velocity
 * at the time level, (j + F/2)/n.  With the FD closure the work of the force
 * heats the gas (the energy moment is conserved by the collision only).
 *
 * Both need d2v9 and the exact inversion (else LBM_EUNSUPPORTED), synchronise
 * the stream and drop captured graphs.  Errors: LBM_EINVAL (index, non-finite
 * force), LBM_EUNSUPPORTED, LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_set_obstacles(lbm_ctx* ctx, int32_t problem, const uint8_t* solid, int32_t on_device);
lbm_status lbm_set_force(lbm_ctx* ctx, int32_t problem, double fx, double fy);

/* Release everything the context owns (synchronises its stream first). */
lbm_status lbm_destroy(lbm_ctx* ctx);

/* Message of the last failure on ctx; with ctx NULL, of the last failure of a
 * call without a context (lbm_create, lbm_conservation_sums_static).  Valid
 * until the next call on the same context (or the next context-free call). */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Number of kernel launches issued by the library on this context since it
 * was created (graph replays count each captured kernel). */
int64_t lbm_launch_count(const lbm_ctx* ctx);

/* ---------------------------------------------------------------- learned inversion
 * A network stands in for the per-cell inversion J_2 -> x (x = mu/T) of the
 * FD moment ratio (the FD form of I_2N, Sect. "Generalized polynomials in D
 * dimensions"); the paper has no network, the model is this library's:
 *   inputs    (n, e), e = D n J_2/3 (D = 2) the internal energy in lattice
 *             units; fixed embedding n_hat = (n - 1.25)/0.75 and
 *             l_hat = (ln delta + 5.3)/3.7, delta = 3/2 - 3 e/(2 n)
 *   layers    h1 = silu(W1 x + b1), h2 = silu(W2 h1 + b2), y = W3 h2 + b3,
 *             64 hidden units each, silu(z) = z/(1 + e^{-z})
 *   outputs   ln T = 0.5 y_0 - 5.09, mu = 0.12 y_1 + 0.1985 (T, mu in the
 *             paper's units)
 *   parameters, FP32, in this order: W1 [64][2], b1 [64], W2 [64][64], b2 [64],
 *             W3 [2][64], b3 [2] (row-major [out][in]): 4482 values.
 * A context created with inv = LBM_INV_SURROGATE (FD statistics, FP32 or BF16
 * storage) evaluates the network per cell inside the step, polishes x = mu/T
 * by one third-order step on J_2(x) = J_2 and falls back to the exact
 * inversion when the first-order step is not below 2.5e-2 max(|x|, 1)
 * (see lbm_surrogate_engine). */
#define LBM_SURROGATE_NPARAM 4482

typedef struct {
  int32_t epochs;  /* passes over the training set (>= 1) */
  int32_t batch;   /* samples per step, a multiple of 128 */
  float lr;        /* Adam learning rate at the start (cosine decay) */
  float lr_final;  /* learning rate at the end (<= 0: lr/100) */
} lbm_train_cfg;

typedef struct {
  int64_t iterations;
  double loss_first, loss_last;  /* mean squared error of the normalised outputs, first and last batch */
  double val_rmse_lnT, val_rmse_mu, val_max_rel_x; /* on the validation set (-1 if none) */
  double seconds;
} lbm_train_report;

/* Features (n_hat, l_hat) and normalised targets of the exact forward map of
 * the method for states (n, t = T/T_F): x = x(t), J_2 = J_2(x), e = 2 n J_2/3,
 * T = n t/(2 pi), mu = T x.  feat, targ: count x 2 floats.  on_device: all
 * four arrays are device memory.  Synchronises.  Errors: LBM_EINVAL, LBM_ECUDA. */
lbm_status lbm_surrogate_targets(const double* n, const double* t, int64_t count, int32_t on_device, float* feat,
                                 float* targ, void* cuda_stream);

/* Mean squared error of the normalised outputs and its gradient with respect
 * to the 4482 parameters, over count samples (host arrays; count <= 2^24).
 * Synchronises.  Errors: LBM_EINVAL, LBM_ECUDA. */
lbm_status lbm_surrogate_loss_grad(const float* params, const float* feat, const float* targ, int64_t count,
                                   float* grad, double* loss, void* cuda_stream);

/* Train the network on states (n, t) (count >= 128; optional validation set)
 * with Adam; params (host, 4482 floats) holds the initial values on entry and
 * the trained ones on return.  Deterministic for fixed inputs.  on_device
 * refers to n, t, n_val, t_val.  Synchronises.  Errors: LBM_EINVAL, LBM_ECUDA. */
lbm_status lbm_surrogate_train(const double* n, const double* t, int64_t count, const double* n_val,
                               const double* t_val, int64_t count_val, int32_t on_device, const lbm_train_cfg* cfg,
                               float* params, lbm_train_report* rep, void* cuda_stream);

/* (T, mu) predicted by the network for count cells (n, e). */
lbm_status lbm_surrogate_eval(const float* params, const double* n, const double* e, int64_t count, double* T,
                              double* mu, int32_t on_device, void* cuda_stream);

/* Give a learned-inversion context its network (host array of 4482 floats,
 * copied; drops captured graphs).  Errors: LBM_EINVAL (not a learned-inversion
 * context, NULL, non-finite values), LBM_ENOMEM. */
lbm_status lbm_surrogate_load(lbm_ctx* ctx, const float* params);

/* Where the network runs:
 *  - LBM_SURROGATE_TENSOR_CORES (the default): its three layers as tcgen05
 *    MMAs over a tile row of 128 cells, FP16 operands with the inputs,
 *    layer-1 and layer-3 weights and all biases split into FP16 hi + lo
 *    parts, FP16 accumulation in tensor memory for the two hidden layers and
 *    FP32 for the output layer, SiLU in packed FP16 (a quarter of the pairs
 *    by a polynomial on the FMA pipe, the rest by the MUFU tanh);
 *  - LBM_SURROGATE_WARP_MMA: the same network, operands and splits, each warp
 *    on its own 32 cells with warp-level MMAs (mma.sync m16n8k8 / m16n8k16),
 *    FP16 accumulators in registers for the hidden layers (the layer-2 bias
 *    as their initial value) and FP32 ones for the output layer (its bias as
 *    the initial value), activations passed from layer to layer in
 *    registers;
 *  - LBM_SURROGATE_FP32_PIPE: per cell on the FP32 pipe (FP32 throughout).
 * In every case the network's x = mu/T is polished by one third-order step on
 * J_2(x) = J_2 (one evaluation of f_0..f_4) and accepted when the first-order
 * step is below 2.5e-2 max(|x|, 1).  Drops captured graphs.  Errors:
 * LBM_EINVAL (NULL context, unknown engine). */
enum { LBM_SURROGATE_FP32_PIPE = 0, LBM_SURROGATE_TENSOR_CORES = 1, LBM_SURROGATE_WARP_MMA = 2 };
lbm_status lbm_surrogate_engine(lbm_ctx* ctx, int32_t engine);

/* Cells that went through the network (n and delta = 3/2 - J_2 inside the
 * network's training domain: n in [0.5, 2], t = T/T_F in [0.005, 0.3]; the
 * other cells take the exact inversion directly), and those of them that fell
 * back to the exact inversion, since the context was created.  Synchronises.  Returns LBM_ETIMEOUT (counts still
 * filled) if a tensor-core wait ever gave up.  After a wait between layers
 * gave up, the CTA concerned served its remaining cells by the exact
 * inversion: the results stand.  If the wait for the last MMA before tensor
 * memory is freed also gave up (the message says so), tensor memory was
 * released while an MMA may still have been writing it, and the results of
 * the context's steps are not to be trusted. */
lbm_status lbm_surrogate_stats(lbm_ctx* ctx, int64_t* fallbacks, int64_t* evaluations);

/* The tensor-core engine's limit on the polls of each wait between its
 * layers (an mbarrier that the MMAs complete): polls >= 0 sets it, polls < 0
 * restores the default (4,194,304).  A wait that reaches the limit gives up
 * for its CTA as described under lbm_surrogate_stats; 0 makes every such wait
 * give up at once, which is how the recovery path is tested.  The final wait
 * before tensor memory is freed keeps the default limit.  The paper has no
 * counterpart (failure handling of this implementation).  Drops captured
 * graphs.  Errors: LBM_EINVAL (NULL context). */
lbm_status lbm_surrogate_wait_limit(lbm_ctx* ctx, int32_t polls);

/* lbm_conservation_sums_static - the paper has no counterpart to this call;
 * it exists for callers that cannot allocate device memory.
 *
 * Some callers may not call cudaMalloc at all: an application or plugin whose
 * device memory is owned by another allocator (a framework's caching
 * allocator or an arena sized at start-up), or a loop that must not allocate
 * while it runs.  lbm_moments allocates its per-block partial sums on first
 * use; this call computes the same conservation totals with its partial sums
 * in a fixed file-scope device array instead, and allocates nothing, on the
 * device or the host (its error message goes to a fixed buffer).
 *
 * f:     device pointer, FP64 populations [9][ny][nx] (the layout that
 *        lbm_get_populations writes), read only.
 * solid: device pointer to one byte per cell [ny][nx], nonzero for an
 *        obstacle cell (the mask given to lbm_set_obstacles), or NULL for
 *        none.  Obstacle cells are left out of every total, as lbm_moments
 *        leaves them out.
 * stat:  lbm_stat; for LBM_STAT_FD a cell counts as clamped when its finite
 *        J_2 lies outside the inversion's interval, the rule of lbm_moments;
 *        for the other closures (no inversion) the count is 0.
 * out:   device pointer to 6 doubles, written in stream order: sum n,
 *        sum j_x, sum j_y, sum E, clamped count, non-finite count (the fields
 *        of lbm_diag).
 * cuda_stream: cudaStream_t for the launches (NULL = legacy default stream).
 *
 * Limit: nx * ny <= LBM_STATIC_SUMS_MAX_CELLS (16,777,216 cells, a 4096 x 4096
 * lattice); larger sizes return LBM_EINVAL before any GPU work, with a message
 * in lbm_last_error(NULL).  The limit is a policy that bounds the work of one
 * call, not the capacity of the scratch array (the kernel is a grid-stride
 * loop over at most 4096 blocks, so the array would serve any size).  The
 * scratch array (192 KiB) lives on every GPU that loads the library until the
 * process exits.  The first call on each device looks up the array's device
 * address with cudaGetSymbolAddress and runs a one-thread set-up kernel,
 * synchronising the stream; make that first call before any stream capture.
 * The looked-up address is kept per device index for the life of the
 * process: after cudaDeviceReset it is stale, so do not call this entry point
 * again on a device that was reset.  All calls share the array: calls whose
 * kernels may overlap on the GPU (different streams or host threads) race and
 * must be serialised by the caller.  Asynchronous after the first call.
 * Errors (message in lbm_last_error(NULL)): LBM_EINVAL (NULL f or out, nx or
 * ny < 1, size above the limit, bad stat), LBM_EUNSUPPORTED (device index
 * >= 64), LBM_ECUDA (set-up or launch failed). */
#define LBM_STATIC_SUMS_MAX_CELLS 16777216
lbm_status lbm_conservation_sums_static(const double* f, int32_t nx, int32_t ny, const uint8_t* solid, int32_t stat,
                                        double* out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
