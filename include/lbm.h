/*
 * lbm.h - C ABI of the GB300 (sm_103a) D2Q9 pseudopotential lattice Boltzmann step.
 *
 * Method: Czelusniak, Cabezas Gomez & Wagner, "Effects of gravity induced
 * pressure variations for thermal liquid-gas phase-change simulations with the
 * pseudopotential lattice Boltzmann method" (arXiv 2301.12869), Sec. III:
 * pull streaming (Eq. LBE) on the D2Q9 set (Eq. VelocitySet), MRT collision
 * (Eqs. OperatorMRT, MatrixMRT, RelaxationMatrix) with Li's forcing scheme
 * (Eq. LiFS), density and velocity (Eqs. Density, Momentum), equilibrium
 * (Eq. EquilibriumDistribution), the Shan-Chen nearest-neighbour force
 * (Eq. ShanChenForce) with the Yuan-Schaefer potential (Eq. InteractionPotential)
 * of the Carnahan-Starling EOS (Sec. IV, Eq. EOS), and gravity as rho g
 * (Eq. Gravity_1) or (rho - <rho>) g (Eq. Gravity_2).
 *
 * Geometry: nx x ny nodes, x periodic, walls below row 0 and above row ny-1
 * (halfway bounce-back, the default) or on rows 0 and ny-1 (Zou-He wet nodes,
 * LBM_WALL_ZOU_HE); the Shan-Chen force is zero on rows 0 and ny-1.
 *
 * Beyond the step: the thermal variant (temperature field and the energy equation,
 * Eq. Energy_Equation), batched independent columns in one persistent launch
 * (lbm_batch_*), and a learned warm start for the columns (lbm_mlp_*, no counterpart in
 * the paper).
 *
 * Conventions for every function:
 *  - returns LBM_OK (0) or a negative LBM_E* code; lbm_last_error() gives text;
 *  - pointers are plain host or device addresses, as each argument states;
 *    nothing is retained after the call unless stated;
 *  - a handle is used from one host thread at a time;
 *  - all device work is issued on the handle's stream (borrowed at lbm_init);
 *    calls that return host data synchronise that stream.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ABI_VERSION 4

/* ---- status codes */
enum {
  LBM_OK = 0,
  LBM_EINVAL = -1,    /* invalid argument or parameter */
  LBM_ECUDA = -2,     /* a CUDA runtime call failed */
  LBM_ENONPHYS = -3,  /* the state became non-physical: rho <= 0, NaN, or
                         2 (p_EOS - rho/3)/G < 0 (psi undefined) */
  LBM_ETIMEOUT = -4,  /* a bounded device-side wait gave up */
  LBM_ENOMEM = -5     /* device allocation failed or workspace too small */
};

/* ---- enumerations */
enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_DOUBLE_FLOAT = 2 };        /* storage and arithmetic */
/* LBM_DOUBLE_FLOAT (batches only: lbm_batch_init, lbm_batch_convert): every real is the
 * unevaluated sum hi + lo of two FP32 numbers (8 bytes, about 48 significant bits) and all
 * arithmetic runs on FP32 instructions - FP64-class accuracy (~2^-46 relative per
 * operation) at GB300's FP32 rate; the residual is evaluated in FP64 as for FP64 batches. */
enum { LBM_GRAVITY_RHO_G = 1, LBM_GRAVITY_RHO_MINUS_MEAN_G = 2 }; /* Eq. Gravity_1 / _2 */
enum { LBM_HOST = 0, LBM_DEVICE = 1 };                            /* where a buffer lives */
/* walls below row 0 and above row ny-1 */
enum {
  LBM_WALL_BOUNCE_BACK = 0, /* halfway bounce-back: walls half a link beyond rows 0 and ny-1,
                               exact mass conservation */
  LBM_WALL_ZOU_HE = 1       /* Zou-He wet nodes (Sec. III): rows 0 and ny-1 are wall nodes
                               whose incoming populations give zero velocity (half force
                               included); mass is conserved only up to the wall closure */
};
enum {
  LBM_REDUCE_MASS = 0,        /* out[0] = sum over nodes of rho (FP64)                      */
  LBM_REDUCE_MEAN_RHO = 1,    /* out[0] = <rho> = mass / (nx ny), as used by Eq. Gravity_2   */
  LBM_REDUCE_RESIDUAL = 2,    /* out[0] = max |rho_now - rho_at_previous_RESIDUAL_call|;
                                 the first call after init/set_state returns +inf           */
  LBM_REDUCE_MAX_U = 3,       /* out[0] = max |u|                                            */
  LBM_REDUCE_INTERFACE_Y = 4, /* out[0] = first height (from y = 0, linear interpolation of
                                 the x-averaged rho) where rho crosses (rho_l + rho_v)/2 of
                                 the Maxwell rule at T; NaN if none                          */
  LBM_REDUCE_RHO_LV = 5       /* out[0] = max, out[1] = min of the x-averaged rho profile    */
};

/* ---- parameters (lattice units). Fill with lbm_params_default() first. */
typedef struct lbm_params {
  uint32_t size;          /* sizeof(lbm_params): versioning */
  int32_t precision;      /* LBM_FP64 or LBM_FP32 */
  int32_t nx, ny;         /* lattice size; nx must be a multiple of 16/sizeof(real) */
  double a, b, R;         /* Carnahan-Starling constants of Eq. EOS */
  double T;               /* absolute temperature */
  double G;               /* interaction parameter of Eqs. ShanChenForce/InteractionPotential (< 0) */
  double sigma;           /* sigma of Eq. LiFS */
  double tau_rho, tau_e, tau_varsigma, tau_j, tau_q, tau_nu; /* Eq. RelaxationMatrix */
  double gx, gy;          /* gravitational acceleration vector */
  int32_t gravity_form;   /* LBM_GRAVITY_RHO_G or LBM_GRAVITY_RHO_MINUS_MEAN_G */
  int32_t thermal;        /* 0: isothermal, T uniform. 1: thermal variant (Sec. III): a
                             temperature field T(x) enters Eq. EOS at every node and is
                             advanced after each LBM step by Eq. Energy_Equation */
  double rho_ref;         /* populations are stored as f_i - w_i rho_ref; NaN = choose
                             (mean of rho0 for FP32, 0 for FP64) */
  void* workspace;        /* optional caller-owned DEVICE buffer of lbm_workspace_bytes();
                             borrowed, must outlive the handle; NULL = library allocates */
  uint64_t workspace_bytes;
  /* thermal variant only (thermal = 1); Eq. Energy_Equation with constant kappa */
  double c_v;             /* specific heat at constant volume (> 0) */
  double kappa;           /* thermal conductivity (>= 0) */
  double T_bot, T_top;    /* wall temperatures below row 0 and above row ny-1 (> 0), imposed
                             half a link beyond the rows like the bounce-back walls */
  int32_t wall;           /* LBM_WALL_BOUNCE_BACK (default) or LBM_WALL_ZOU_HE (ny >= 3); with
                             Zou-He, <rho> of Eq. Gravity_2 is the stored state's mass / (nx ny) */
  int32_t reserved1;      /* must be 0 */
} lbm_params;

typedef struct lbm_handle lbm_handle;

/* Paper defaults: a = 0.5, b = 4, R = 1 (Sec. IV), G = -1, sigma = 1.385, all tau = 1
 * (Sec. IV), gravity off, form 1, FP64, rho_ref = NaN, no workspace, bounce-back walls, isothermal, with
 * c_v = 5 and kappa = 0.02 (Sec. IV) ready for thermal = 1. nx, ny, T, T_bot, T_top unset (0). */
void lbm_params_default(lbm_params* p);

/* Device bytes a handle needs for p (populations A/B, reduction partials, moments scratch). */
int lbm_workspace_bytes(const lbm_params* p, uint64_t* bytes);

/* Create a lattice. rho0 (nx*ny doubles, row-major [y][x]) is the initial density,
 * in host (LBM_HOST) or device (LBM_DEVICE) memory; the state is set to the rest
 * equilibrium f_i = f_i^eq(rho0, u = 0) of Eq. EquilibriumDistribution.
 * stream: a cudaStream_t (NULL = legacy default stream), borrowed.
 * Errors: LBM_EINVAL (bad sizes/parameters, NULL rho0/out), LBM_ENOMEM, LBM_ECUDA. */
int lbm_init(const lbm_params* p, const double* rho0, int rho0_where, void* stream, lbm_handle** out);

/* Advance nsteps >= 0 time steps (asynchronous on the handle's stream). Each step is
 * one launch of the fused kernel: stream (and, with Zou-He walls, rebuild the wall nodes'
 * incoming populations), rho, psi, <rho>, F_int, F_g, u, MRT + Li forcing, store. Device-side faults (non-physical state, timeouts) are recorded in a
 * sticky status returned by the next synchronising call.
 * Thermal variant: psi uses R T(x) of the current temperature field T^n, and the step
 * also stores its rho^n and u^n; then one launch advances T^n by Heun's second-order
 * Runge-Kutta (dt = 1) on Eq. Energy_Equation with those rho^n, u^n held fixed,
 * with isotropic D2Q9-weighted central differences and the wall temperatures T_bot, T_top
 * (ghost rows T(-1) = 2 T_bot - T(0), u(-1) = -u(0), likewise at the top; with Zou-He walls
 * the wall rows 0 and ny-1 hold T_bot and T_top). */
int lbm_step(lbm_handle* h, int64_t nsteps);

/* Macroscopic fields of the current state, as the next step evaluates them: the stored
 * post-collision populations are pulled (streamed) and rho (Eq. Density) and u
 * (Eq. Momentum, with F = F_int + F_g) computed. Outputs are nx*ny doubles [y][x] in
 * host or device memory per `where`; any pointer may be NULL to skip it. Synchronises
 * when where == LBM_HOST. */
int lbm_moments(lbm_handle* h, double* rho, double* ux, double* uy, int where);

/* FP64 reductions of the current state (see LBM_REDUCE_*). out: host array of 1
 * (2 for LBM_REDUCE_RHO_LV) doubles. Synchronises. */
int lbm_reduce(lbm_handle* h, int kind, double* out);

/* Full populations f_i (absolute, not deviations) as 9*nx*ny doubles [i][y][x] (i in
 * the order of Eq. VelocitySet), and the number of steps taken. */
int lbm_get_state(lbm_handle* h, double* f, int where, int64_t* steps_done);
int lbm_set_state(lbm_handle* h, const double* f, int where, int64_t steps_done);

/* Change T, G, sigma, tau_*, gx, gy, gravity_form (and c_v, kappa, T_bot, T_top of the
 * thermal variant) between steps (the paper's equilibrate-then-change protocol).
 * nx, ny, precision, rho_ref, a, b, R and thermal must match. */
int lbm_set_params(lbm_handle* h, const lbm_params* p);

/* Thermal variant: the temperature field, nx*ny doubles [y][x] in host or device memory
 * per `where` (stored in the handle's precision). lbm_init sets the steady conduction
 * profile T(y) = T_bot + (T_top - T_bot)(y + 1/2)/ny (Eq. Temp_Profile with constant kappa;
 * T_bot + (T_top - T_bot) y/(ny - 1) with Zou-He walls, whose wall rows keep T_bot, T_top).
 * The caller keeps T > 0. LBM_EINVAL on an isothermal handle. get synchronises when
 * where == LBM_HOST; set synchronises always. */
int lbm_set_temperature(lbm_handle* h, const double* T, int where);
int lbm_get_temperature(lbm_handle* h, double* T, int where);

/* Synchronise and return the sticky device status (LBM_OK, LBM_ENONPHYS, LBM_ETIMEOUT). */
int lbm_status(lbm_handle* h);

/* Release the handle and what it allocated. NULL is accepted. */
int lbm_destroy(lbm_handle* h);

/* Text of the last error on h (or of the last failed call without a handle when h is
 * NULL). Static storage owned by the library. */
const char* lbm_last_error(const lbm_handle* h);

/* ---- host-side thermodynamics of Eq. EOS (FP64, no device work) */
/* Critical point: dp/drho = d2p/drho2 = 0. */
int lbm_critical_point(double a, double b, double R, double* rho_c, double* T_c, double* p_c);
/* Coexistence densities and pressure at T < T_c by the Maxwell rule, Eqs. MaxwellRule. */
int lbm_coexistence(double a, double b, double R, double T, double* rho_v, double* rho_l, double* p_sat);

/* Launch configuration the handle uses for its fused step (for reports and tests):
 * grid CTAs, threads per CTA, dynamic shared bytes, band width (nodes along x per CTA),
 * strip height (rows per CTA), pipeline stages. Any pointer may be NULL. */
int lbm_launch_info(const lbm_handle* h, int* grid, int* block, int* smem_bytes,
                    int* band_width, int* strip_rows, int* stages);

/* Tile autotuner: times each tile variant of the fused kernel (band width and threads per
 * CTA) for `steps` launches on this lattice - every candidate reads the current state and
 * writes the spare buffer, so the state is unchanged - and keeps the fastest for later
 * lbm_step / lbm_moments calls. variant, ms (mean time per step of the winner): may be NULL.
 * A thermal or Zou-He handle considers only the variants that carry those kernels (variant 0
 * of each precision). Synchronises the handle's stream. */
int lbm_autotune(lbm_handle* h, int steps, int* variant, double* ms);

/* Number of tile variants of the fused kernel for a precision (LBM_EINVAL otherwise). */
int lbm_tile_variants(int precision);

/* Use tile variant `variant` (0 = default, as chosen by lbm_init) for later steps, e.g. a
 * result of lbm_autotune saved from an earlier run. LBM_EINVAL if out of range, or if the
 * handle is thermal or has Zou-He walls and the variant lacks those kernels (only variant 0
 * has them). */
int lbm_set_tiling(lbm_handle* h, int variant);

/* ---- batched independent columns: the 1-D liquid-column problem of Sec. IV for many
 * parameter sets at once, in one persistent launch
 *
 * A batch holds ncols independent lattices nx x ny_c (periodic x, walls at both ends) that
 * share nx, the precision, the EOS constants a, b, R, G, sigma and the relaxation times of
 * `p`, and differ in height, temperature, gravity and gravity form. */
typedef struct lbm_column {
  int32_t ny;            /* rows */
  int32_t gravity_form;  /* LBM_GRAVITY_RHO_G or LBM_GRAVITY_RHO_MINUS_MEAN_G */
  double T;              /* temperature */
  double gx, gy;         /* gravity */
} lbm_column;

typedef struct lbm_batch lbm_batch;

/* Create a batch. p: shared parameters (p->nx = column width <= 64; p->thermal must be 0; p->wall
 * LBM_WALL_BOUNCE_BACK or LBM_WALL_ZOU_HE for every column (Zou-He: ny_c >= 3);
 * p->ny, p->T, p->gx, p->gy, p->gravity_form and p->workspace are ignored; p->rho_ref NaN means: each column's
 * mean rho0 in FP32, 0 in FP64). cols: ncols descriptors (host). rho0: the columns' initial
 * densities concatenated, column c holding nx * ny_c doubles [y][x], in host or device
 * memory per rho0_where; the state is the rest equilibrium f_i^eq(rho0, 0). Each column
 * needs nx ny_c (sizeof(real) + 8) <= 200 KiB. stream: a cudaStream_t or NULL (the batch then
 * uses a private non-blocking stream). The library allocates the device memory.
 * Errors: LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA. */
int lbm_batch_init(const lbm_params* p, const lbm_column* cols, int ncols, const double* rho0, int rho0_where,
                   void* stream, lbm_batch** out);

/* Advance every column until its residual max_x |rho_t(x) - rho_(t-1)(x)|, evaluated every
 * check_every (>= 2) steps in FP64 from the stored populations, is <= tol, or until it has taken max_steps more steps. One
 * persistent launch over all columns (each CTA takes the tallest remaining column), issued
 * as a CUDA graph captured at the first run. Synchronises; seconds (may be NULL) receives
 * the device time of the launch. Per-column non-physical states are reported by
 * lbm_batch_results. */
int lbm_batch_run(lbm_batch* b, double tol, int64_t max_steps, int check_every, double* seconds);

/* As lbm_batch_run; a column also stops once stall_checks (> 0) consecutive checks with a
 * residual below 1e-6 (FP32) / 1e-13 (FP64) have not lowered its smallest residual of this
 * run by 1 % - its precision's rounding floor (FP32 columns floor near 1e-8; above those
 * levels transients may plateau and do not count). stall_checks = 0 is lbm_batch_run. The usual way to finish:
 * FP32 with tol = the final target and stall_checks ~10, then lbm_batch_convert to FP64 and
 * lbm_batch_run to the target. */
int lbm_batch_run_stall(lbm_batch* b, double tol, int64_t max_steps, int check_every, int stall_checks,
                        double* seconds);

/* Accelerate later runs of this batch by extrapolation (no counterpart in the paper: it
 * changes the way to each column's steady state, not the state). Every `checks` (>= 2)
 * residual checks a column's state is kept; after 6 such snapshots x_0..x_5 the fixed
 * point is estimated by minimal polynomial extrapolation of order 4 - the coefficients c
 * (c_4 = 1) minimising |sum_j c_j (x_{j+1} - x_j)| weight sum_j c_j x_j / sum_j c_j - which
 * captures the damped oscillations in which the columns' slow modes decay. The estimate
 * replaces the state when every density stays positive, and is undone when the next
 * residual check is worse than the one before it. checks = 0 turns it off. The library
 * allocates 6 x 9 x (total nodes) reals once. Not carried over by lbm_batch_convert. */
int lbm_batch_set_acceleration(lbm_batch* b, int checks);

/* Block size of the batched kernel (a runtime choice, no counterpart in the paper): threads
 * = 128, 256 (the default) or 512 per CTA; a CTA iterates one column at a time. Carried
 * over by lbm_batch_convert. LBM_EINVAL for another value. */
int lbm_batch_set_threads(lbm_batch* b, int threads);
/* Autotuner of the batched kernel's block size: on a copy of the batch's current state,
 * every column runs `steps` (>= 1) steps with no residual stop (after a 2-step warm-up) for
 * each candidate block size, timed with CUDA events on the batch's stream; the fastest is
 * kept (lbm_batch_set_threads). threads[3] and us[3] (host, may be NULL) receive the
 * candidates and their microseconds per step of the whole batch. The batch's own state,
 * step counts and residuals are not touched; the copy needs as much device memory as the
 * batch. Synchronises. */
int lbm_batch_autotune(lbm_batch* b, int steps, int* threads, double* us);

/* Per column (host arrays of ncols, any may be NULL): total steps taken, last residual
 * (+inf before the first check), status (LBM_OK or LBM_ENONPHYS). Returns LBM_ENONPHYS if
 * any column is non-physical. Synchronises. */
int lbm_batch_results(const lbm_batch* b, int64_t* steps, double* residual, int* status);

/* Per column (host array of ncols): device seconds that the persistent launches spent on the
 * column - from the moment a CTA took it to the moment it stopped - summed over every run
 * since lbm_batch_init (and carried over by lbm_batch_convert), from the GPU's global
 * timer. The time to steady state of one column, where a run's duration is the makespan
 * of all. Synchronises. */
int lbm_batch_column_seconds(const lbm_batch* b, double* seconds);

/* rho and u of every column as the next step evaluates them, concatenated like rho0, in
 * host or device memory per `where` (any pointer may be NULL). Synchronises. */
int lbm_batch_moments(lbm_batch* b, double* rho, double* ux, double* uy, int where);

/* Absolute populations of every column, concatenated [col][i][y][x] (9 nx ny_c doubles per
 * column), host or device. Synchronises. */
int lbm_batch_get_state(lbm_batch* b, double* f, int where);

/* Replace every column's populations by the rest state of its stored density field
 * rho = sum_i f_i (an initialisation with no counterpart in the paper, which gives only the
 * initial density profile): the forces F = F_int + F_g of Eqs. ShanChenForce and Gravity_1 /
 * Gravity_2 from rho (<rho> the column's mean), pre-collision populations with the moments
 * of the rest equilibrium f_eq(rho, 0) except the momentum -F/2, so that the velocity of
 * Eq. Momentum is zero, and one collision (Eqs. OperatorMRT, LiFS). The density is kept; the
 * momentum becomes +F/2. With every tau = 1 this is m* = m_eq(rho, 0) + S~(0, F)/2, which a
 * steady column satisfies up to its small residual velocity, so a start whose density is
 * close to the steady one starts close to the steady populations (f_eq(rho, 0), the state
 * lbm_batch_init sets, lacks the forcing terms). Call it after lbm_batch_init (or between
 * runs). A non-physical density sets the column's status. Synchronises. */
int lbm_batch_rest_state(lbm_batch* b);

/* A new batch with src's columns and current state in another precision (e.g. an FP32 run
 * continued in FP64 below the FP32 rounding floor); step counts carry over. */
int lbm_batch_convert(const lbm_batch* src, int precision, lbm_batch** out);

/* Release a batch. NULL is accepted. */
int lbm_batch_destroy(lbm_batch* b);

/* ---- learned warm start for the liquid columns (no counterpart in the paper)
 *
 * A 6 -> 128 -> 128 -> 128 -> 1 network with SiLU activations predicts the steady density
 * profile rho(z)/rho_c of a column from its descriptors (T/T_c, log10|g|, gravity form,
 * <rho>/rho_c, z/H, log2 H) with z = y + 1/2 and H = ny (the height places an interface of a
 * few lattice units' width, which z/H alone cannot). Its only use is to initialise columns;
 * the lattice Boltzmann run to the residual target alone decides the result.
 * Arithmetic: bfloat16 inputs, weights and activations as tensor-core operands (tcgen05,
 * FP32 accumulation in tensor memory), FP32 biases, output layer, loss and Adam; inputs
 * normalised as x_n = (x - c)/s with c = (0.825, -5, 1.5, 1.4, 0.5, 8), s = (0.125, 1, 0.5,
 * 1.1, 0.5, 2). Loss: mean squared error of rho/rho_c.
 *
 * Parameters: LBM_MLP_NPARAMS FP32 values, packed in this order:
 *   W1 [128][16] (input j < 6 used; the rest must be 0), b1 [128], W2 [128][128] ([out][in]),
 *   b2 [128], W3 [128][128], b3 [128], w4 [128], b4 [1].
 * Feature rows: 6 FP32 values (T/T_c, log10|g|, form, <rho>/rho_c, z/H, log2 H), raw (the network
 * normalises them). All feature/target/output arrays of these calls are DEVICE pointers. */
#define LBM_MLP_WIDTH 128
#define LBM_MLP_INPUTS 6
#define LBM_MLP_IN_PAD 16
#define LBM_MLP_NPARAMS (128 * 16 + 128 + 128 * 128 + 128 + 128 * 128 + 128 + 128 + 1)

typedef struct lbm_mlp lbm_mlp;

/* Create a network with the given parameters (host array), Adam state zero. batch_capacity
 * (a multiple of 128, <= 4194304) bounds the rows of one pass; the library allocates
 * ~(1.3 KB x batch_capacity + 0.7 MB) of device memory. stream: cudaStream_t or NULL. */
int lbm_mlp_create(const float* params, int batch_capacity, void* stream, lbm_mlp** out);
/* Replace the parameters (host array) and reset the Adam state; synchronises. */
int lbm_mlp_set_params(lbm_mlp* h, const float* params);
/* Current parameters into a host array; synchronises. */
int lbm_mlp_get_params(lbm_mlp* h, float* params);
/* Loss (mean over the n <= batch_capacity rows) and its gradient with respect to every
 * parameter (host array, packed like the parameters) for feature rows x [n][5] and targets
 * t [n] (device). No update. Synchronises. */
int lbm_mlp_gradients(lbm_mlp* h, const float* x, const float* t, int n, float* grads, double* loss);
/* iters Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr), each on `batch`
 * rows drawn with replacement from the n rows of x, t (device): row i of step k is
 * SplitMix64(k batch + i, seed) mod n, k counting every step since create/set_params.
 * losses (host, iters floats, may be NULL) receives each step's minibatch loss (then every
 * step synchronises). */
int lbm_mlp_train(lbm_mlp* h, const float* x, const float* t, long long n, int batch, int iters, float lr,
                  unsigned long long seed, float* losses);
/* y[i] = network(x[i]) (predicted rho/rho_c) for n rows (device arrays); synchronises. */
int lbm_mlp_predict(lbm_mlp* h, const float* x, long long n, float* y);
/* Feature rows of columns: row (c, y) of the concatenation over columns (sum of ny_c rows)
 * gets (T_c/T_crit, log10|g_c|, form_c, <rho>_c/rho_crit, (y + 1/2)/ny_c, log2 ny_c), with the critical
 * point of a, b, R. <rho>_c comes from rho when rho != NULL - the columns' density fields,
 * DEVICE, concatenated [col][y][x] with nx per column as lbm_batch_moments writes them -
 * else from mean_rho (host, one value per column). With rho and t != NULL, t receives the
 * targets rho(y, x = 0)/rho_crit. x, t: DEVICE. Synchronises `stream`. */
int lbm_mlp_features(const lbm_column* cols, int ncols, int nx, double a, double b, double R, const double* rho,
                     const double* mean_rho, float* x, float* t, void* stream);
/* Initial densities for lbm_batch_init: for each column the predicted profile p(y) times
 * rho_crit (floored at 1e-3), moved along y so that its mean equals mean_rho[c] (host): row y
 * takes p at y - s (linear between rows, the end values beyond them) with the shift s in
 * [-ny, ny] found by bisection, then a factor within rounding of 1 makes the mean exact
 * (a mean outside [p(ny - 1), p(0)] keeps s = 0 and scales the profile instead). Moving
 * rather than scaling keeps the predicted bulk densities. The same on every x; written to
 * rho0 (DEVICE, concatenated [col][y][x]). Synchronises. */
int lbm_mlp_warm_start(lbm_mlp* h, const lbm_column* cols, int ncols, int nx, double a, double b, double R,
                       const double* mean_rho, double* rho0);
/* The network's tensor-core matrix product on its own: C[M x N] = A[M x K] B[N x K]^T with A,
 * B bfloat16 bit patterns (DEVICE, row-major, K contiguous, lda/ldb multiples of 8, 16-byte
 * aligned, K a multiple of 16), C FP32 (DEVICE, ldc). accumulate = 0: C is overwritten;
 * accumulate = 1: C += the product, K split into ranges of k_split (a multiple of 64;
 * <= 0: no split) summed by atomic adds. Synchronises `stream`. */
int lbm_mlp_gemm(const uint16_t* A, int lda, const uint16_t* B, int ldb, float* C, int ldc, int M, int N, int K,
                 int k_split, int accumulate, void* stream);
/* lbm_mlp_gemm without synchronisation or allocation: the product is enqueued on `stream`
 * (so it can be captured in a CUDA graph) and nothing waits for it. status: caller-owned
 * DEVICE int that the kernel ORs a non-zero bit into when one of its bounded tensor-core
 * waits timed out (C is then incomplete); the caller zeroes it and reads it after the
 * stream completes. The arguments are checked as for lbm_mlp_gemm (LBM_EINVAL); a launch
 * error returns LBM_ECUDA. Text in lbm_last_error(NULL). */
int lbm_mlp_gemm_enqueue(const uint16_t* A, int lda, const uint16_t* B, int ldb, float* C, int ldc, int M, int N,
                         int K, int k_split, int accumulate, int* status, void* stream);
/* Release a network. NULL is accepted. */
int lbm_mlp_destroy(lbm_mlp* h);

/* ---- slabs of one domain across GPUs (one process per GPU; the paper has a single domain)
 *
 * The domain nx x p->ny is cut into horizontal slabs of rows. Slab s holds its own rows
 * [s->y0, s->y0 + s->ny_own) and LBM_SLAB_HALO ghost rows below and above in a caller-owned
 * DEVICE buffer real[9][ny_own + 2 LBM_SLAB_HALO][nx] (deviations f_i - w_i rho_ref, order of
 * Eq. VelocitySet; buffer row j is domain row y0 - LBM_SLAB_HALO + j). Two ghost rows are
 * what one step needs: pull streaming (Eq. LBE) reads the row next to the slab, and the
 * Shan-Chen force (Eq. ShanChenForce) on the slab's edge row needs psi of that row, which
 * pulls from the next one. Walls (p->wall) act where the slab meets row 0 or row p->ny - 1;
 * elsewhere the caller refreshes the ghost rows after every step with its neighbours' edge
 * rows (2 rows x 9 planes each way) and adds the slabs' mass partials element-wise for <rho>
 * of Eq. Gravity_2 over the whole domain (both by its own communication, e.g. NCCL). p->rho_ref must be the same
 * on every slab (NaN means 0). These calls allocate nothing, are asynchronous on `stream`
 * (a cudaStream_t, NULL = default) and take only device pointers; slab buffers start on a
 * 16-byte boundary (the step's bulk copies; else LBM_EINVAL). Isothermal only. A slab
 * with a neighbour needs ny_own >= LBM_SLAB_HALO. Errors: LBM_EINVAL, LBM_ECUDA. */
#define LBM_SLAB_HALO 2
typedef struct lbm_slab {
  int32_t y0;       /* first own row of the domain */
  int32_t ny_own;   /* own rows */
  int32_t reserved; /* must be 0 */
  int32_t reserved2;
} lbm_slab;

/* Number of FP64 partial sums (`part` below) a slab step writes. */
int lbm_slab_partials(const lbm_params* p, const lbm_slab* s, int* count);
/* Own rows of f = the rest equilibrium of rho0 (ny_own x nx doubles [y][x], device); ghost
 * rows untouched. */
int lbm_slab_init(const lbm_params* p, const lbm_slab* s, const double* rho0, void* f, void* stream);
/* The FP64 mass partials of the own rows of f (device): part[0 .. lbm_slab_partials) (npart >=
 * that, else LBM_EINVAL; the rest of part set to zero). Their sum, over all slabs, is
 * sum(rho - rho_ref) of the domain. */
int lbm_slab_mass(const lbm_params* p, const lbm_slab* s, const void* f, double* part, int npart, void* stream);
/* One time step of the own rows, f_out = step(f_in) (distinct buffers; f_in's ghost rows must
 * hold the neighbours' rows of the same state). part_in: device, npart_in doubles whose sum is
 * the domain-wide sum(rho - rho_ref) of f_in - the slabs' partials (lbm_slab_mass, or the
 * previous step's part_out) added element-wise over all slabs, zero-padded to a common length;
 * read for Eq. Gravity_2 only (may be NULL otherwise) and summed in a fixed order. Writes
 * part_out (device, distinct from part_in, npart_out >= lbm_slab_partials, else LBM_EINVAL;
 * entries beyond lbm_slab_partials set to zero): this slab's partials of f_out. status: device
 * int the kernel ORs LBM status bits into (1: non-physical, 2: a bounded wait timed out); the
 * caller zeroes it and reads it after the stream completes. */
int lbm_slab_step(const lbm_params* p, const lbm_slab* s, const void* f_in, void* f_out, const double* part_in,
                  int npart_in, double* part_out, int npart_out, int* status, void* stream);

/* ---- one step without device allocation (this entry point has no counterpart in the paper)
 *
 * Some callers cannot call cudaMalloc: a host loop that must not stall other streams on
 * the implicit device synchronisation an allocation can bring, a process whose device
 * memory is reserved up front by another allocator, or a plug-in that may not create
 * allocations of its own. lbm_step_noalloc runs one time step f_out = step(f_in) - the
 * same fused kernel as lbm_step - on caller-owned device arrays and allocates nothing.
 *
 * f_in, f_out: distinct DEVICE arrays (of the current device, or managed memory) of
 *   9*nx*ny reals (float for LBM_FP32, double for LBM_FP64), layout [i][y][x] in the order
 *   of Eq. VelocitySet, holding the deviations f_i - w_i rho_ref with rho_ref = p->rho_ref
 *   (NaN means 0), each starting on a 16-byte boundary. Caller-owned; read / written. A
 *   pointer that is not device memory, or not 16-byte aligned, is rejected (LBM_EINVAL);
 *   the element type and count cannot be checked here and are the caller's to get right
 *   (the Python binding checks them).
 * p: as for lbm_init, isothermal (thermal = 0), any wall; p->workspace is ignored. stream: a cudaStream_t (NULL = default).
 * Scratch: the FP64 partial mass sums that give <rho> (Eq. Gravity_2) and a status word
 *   live in a file-scope __device__ array of 65 792 bytes inside liblbm, held by every
 *   device that loads the library until the process exits. Its 4096 partial slots bound
 *   the step's grid: lattices wider than 4096 x-bands (nx > 4 194 304 in FP32, 2 097 152 in
 *   FP64) are rejected with LBM_EINVAL.
 * Cost: with Eq. Gravity_2 each call first reads f_in once more to form its mass partials
 *   (a handle keeps them from the previous step instead); with Eq. Gravity_1 it does not.
 * Every call shares that array and leaves its own values there; the status word is
 *   cleared at the start of each call. Calls that overlap on the GPU (several streams, or
 *   host threads without ordering) race on it: serialise them.
 * The first call on a device (per process) looks up the array's device address with
 *   cudaGetSymbolAddress and sets the kernels' shared-memory limit; make that first call
 *   before any stream capture. If that set-up fails, the call returns LBM_ECUDA and the
 *   next call on the device tries it again.
 * Synchronises `stream`. Returns LBM_OK, LBM_EINVAL, LBM_ECUDA, or the device status of
 *   this step (LBM_ENONPHYS, LBM_ETIMEOUT); text in lbm_last_error(NULL). */
int lbm_step_noalloc(const lbm_params* p, const void* f_in, void* f_out, void* stream);

/* Self-check of the failure path every device-side wait of the library takes (no
 * counterpart in the paper): one thread waits on an mbarrier that nothing arrives on,
 * bounded by `cycles` clock cycles (1 .. 2e9, about 1 ns each), then records the timeout in
 * a device status word that is read back - no trap, the context stays usable. Returns
 * LBM_ETIMEOUT, the expected outcome, or LBM_EINVAL / LBM_ECUDA; LBM_OK would mean the
 * wait did not give up. Allocates 4 device bytes on the current device; synchronises. */
int lbm_wait_bound_selftest(long long cycles);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
