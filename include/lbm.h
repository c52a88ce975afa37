/*
 * lbm.h -- C ABI of the GB300 (sm_103a) pseudo-potential lattice Boltzmann
 * library: the per-timestep D2Q9 MRT update of Kupershtokh et al.'s hybrid
 * pseudo-potential model with the kappa-scaled pressure-tensor modification
 * of Hu, Li & Uddin, "Surface tension adjustment in a pseudo-potential
 * lattice Boltzmann model" (arXiv:1412.7228), Sections 2 and 3.2.
 *
 * Conventions shared by every call
 *  - Every call returns an int: LBM_OK (0) or a negative LBM_E* code; the
 *    message of the last failure is lbm_last_error(ctx).
 *  - Fields are row-major with x fastest: node (x, y) is element y*nx + x of
 *    a host array of nx*ny doubles.  Lattice velocities e_0..e_8 are (0,0),
 *    (1,0), (0,1), (-1,0), (0,-1), (1,1), (-1,1), (-1,-1), (1,-1).
 *  - Moment order of Eq. 4: (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy);
 *    s[9] is the diagonal of Lambda (Eq. 2) in that order.
 *  - Host pointers belong to the caller and are only read or written during
 *    the call.  Device memory belongs to the context, unless the caller hands
 *    in dev_buf, which the library then uses but never frees.
 *  - Work is enqueued on the context's CUDA stream.  lbm_step() is
 *    asynchronous; every call that returns data to the host synchronises the
 *    stream.  Device-side faults of the method (a density outside the EOS's
 *    psi domain, NaN, a bounded wait that gave up) set a sticky per-instance
 *    status that the next synchronising call returns as LBM_EUNSTABLE or
 *    LBM_ETIMEOUT.
 *  - A context holds one or more independent lattices ("instances"); the
 *    single-lattice calls act on instance 0, the lbm_batch_* calls on
 *    instance i, and lbm_step() advances every instance.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define LBM_OK 0
#define LBM_EINVAL (-1)    /* bad argument; nothing was done */
#define LBM_ENOMEM (-2)    /* device buffer too small or allocation failed */
#define LBM_ECUDA (-3)     /* a CUDA runtime call failed */
#define LBM_EUNSTABLE (-4) /* sticky: a density left the psi domain or became NaN */
#define LBM_ETIMEOUT (-5)  /* sticky: a bounded device wait gave up */
#define LBM_EIO (-6)       /* checkpoint file could not be read or written */

/* Storage precision of the populations. */
#define LBM_FP32 1 /* FP32, stored as deviations f_a - t_a rho_ref */
#define LBM_FP64 2 /* FP64 */

/* Equations of state (the pressure law that sets psi through Eq. 10). */
#define LBM_EOS_CS 1  /* Carnahan-Starling: K(rho R T (1+n+n^2-n^3)/(1-n)^3 - a rho^2), n = b rho/4 */
#define LBM_EOS_VDW 2 /* van der Waals, Eq. 21: K(rho R T/(1 - b rho) - a rho^2) */
#define LBM_EOS_PR 3  /* Peng-Robinson, Eq. 29, with alpha(T) from omega and Tc */

/* Flags of lbm_set_params. */
#define LBM_FLAG_LI_EPS 0x1u /* third entry of C (Eq. 26) = -1.5 s_eps (Q_xx+Q_yy), Li et al.'s form */
/* Test hook: every CTA of the next steps also waits on a barrier phase that
 * nothing completes, with a 2 ms limit, and then reports LBM_ETIMEOUT. */
#define LBM_FLAG_TEST_FORCE_TIMEOUT 0x100u

/* Number of doubles written by lbm_batch_measure. */
#define LBM_MEASURE_N 8

typedef struct {
    int kind;      /* LBM_EOS_* */
    double a, b, R; /* EOS constants */
    double K;      /* scale of the whole law (Section 3, Eq. 21) */
    double T;      /* absolute temperature */
    double omega;  /* Peng-Robinson acentric factor (Eq. 29); else ignored */
    double Tc;     /* Peng-Robinson critical temperature in alpha(T); else ignored */
} lbm_eos;

typedef struct lbm_ctx lbm_ctx;

/* ---- Host-side EOS helpers (no GPU needed) ---------------------------- */

/* p_EOS(rho) of the law (Eq. 21, Eq. 29 or Carnahan-Starling). */
int lbm_eos_pressure(const lbm_eos* eos, double rho, double* p);

/* Critical point (rho_c, T_c, p_c) of the law, found numerically as the
 * temperature where min_rho dp/drho reaches 0; eos->T is ignored.  Used to
 * express temperatures as T/T_c (Section 3). */
int lbm_eos_critical(const lbm_eos* eos, double* rho_c, double* T_c, double* p_c);

/* Maxwell equal-area coexistence at eos->T: densities rho_g < rho_l and the
 * coexistence pressure p0.  Used to build initial droplet and slab fields.
 * LBM_EINVAL when eos->T is not below T_c. */
int lbm_eos_maxwell(const lbm_eos* eos, double* rho_g, double* rho_l, double* p0);

/* Least-squares line through (1/R_i, dp_i), Laplace's law Eq. 22:
 * dp = sigma / R + icpt; r2 is the coefficient of determination.  n >= 2. */
int lbm_laplace_fit(int n, const double* dp, const double* R, double* sigma, double* icpt,
                    double* r2);

/* Self-check of the FP64 step's reciprocal, division and square root (two
 * Newton-Raphson, resp. Goldschmidt, steps from the hardware estimates)
 * against IEEE-rounded 1/d, a/d and sqrt(d) on the current device: n values
 * of d spread evenly over [lo, hi], numerators a in [0.37, 0.87).  Writes
 * result[0..2] = the largest distances in units in the last place (rcp, div,
 * sqrt) and result[3] = 1 when sqrt(+0) = +0, sqrt(-0) = -0 and sqrt(-1) is
 * NaN.  Synchronous (legacy default stream).  LBM_EINVAL unless
 * 0 < lo < hi < inf, n >= 1 and result != NULL; LBM_ECUDA on a device
 * error. */
int lbm_fp64_math_check(double lo, double hi, long long n, unsigned long long result[4]);

/* Measured FP64 peak of the current device, the denominator of the FP64
 * step's roofline (the paper has no counterpart: it is a measurement aid).
 * Every resident thread of every SM runs 8 independent chains of `iters`
 * fused multiply-adds on `stream` (NULL: legacy default stream); one warm-up
 * launch, then the fastest of three launches timed with CUDA events.
 * flops_per_s = 2 x FMAs / seconds (an FMA is two floating-point operations);
 * seconds = that launch's duration.  Synchronous.  LBM_EINVAL unless
 * iters >= 1 and both outputs are given; LBM_ECUDA on a device error. */
int lbm_fp64_fma_rate(int iters, void* stream, double* flops_per_s, double* seconds);

/* ---- Context ------------------------------------------------------------ */

/* Bytes of device memory one context of these lattices needs when the caller
 * supplies dev_buf (populations of two time levels with their ghost layers,
 * per-instance descriptors, tile table, reduction and field scratch).
 * 0 on bad arguments (n < 1, any nx or ny outside [2, 2^20], unknown
 * precision). */
size_t lbm_required_bytes(int nx, int ny, int precision);
size_t lbm_batch_required_bytes(int n, const int* nx, const int* ny, int precision);

/* How the multi-step schedule (schedule 3 of lbm_set_schedule) groups a
 * batch of these lattices into launches: instances taken largest first
 * (index order among equal sizes) into as few chunks as 32 instances and
 * 80 MiB of populations (both time levels) per chunk allow, an instance
 * larger than that alone, with the bytes spread evenly over the chunks.
 * Writes the chunk of instance i to chunk_of[i] (caller-owned, n ints;
 * chunks numbered in launch order) and returns the number of chunks.  Host
 * arithmetic only: needs no device.  LBM_EINVAL for the shapes
 * lbm_batch_required_bytes refuses or a NULL chunk_of. */
int lbm_run_chunk_plan(int n, const int* nx, const int* ny, int precision, int* chunk_of);

/* Create a context of one nx x ny periodic lattice (lbm_create) or of n
 * independent lattices (lbm_batch_create) in the given precision; nx and ny
 * in [2, 2^20].  dev_buf: caller-owned device memory of at least the required
 * bytes, 256-byte aligned, or NULL to let the library allocate (and later
 * free) its own.  stream: a cudaStream_t, or NULL for the legacy default
 * stream.  Binds the context to the calling thread's current device.
 * Parameters must be set and a density initialised before the first
 * lbm_step.  Errors (*out stays NULL): LBM_EINVAL for a bad shape, precision
 * or a misaligned dev_buf; LBM_ENOMEM when buf_bytes is below the required
 * size or the allocation fails; LBM_ECUDA when no device is usable. */
int lbm_create(lbm_ctx** out, int nx, int ny, int precision, void* dev_buf, size_t buf_bytes,
               void* stream);
int lbm_batch_create(lbm_ctx** out, int n, const int* nx, const int* ny, int precision,
                     void* dev_buf, size_t buf_bytes, void* stream);

/* Release everything the context allocated (not a caller-owned dev_buf). */
void lbm_destroy(lbm_ctx* ctx);

/* Model parameters (Sections 2-3): EOS, hybrid-force weight A of Eq. 9,
 * surface-tension parameter kappa of Eq. 23, interaction strength G (only
 * its sign matters; G = 0 switches the interaction force and Q off),
 * relaxation rates s[9] (Eq. 2, moment order), the reference density rho_ref
 * subtracted from the FP32 populations, and LBM_FLAG_* flags.  LBM_EINVAL
 * (parameters unchanged) for an unknown EOS, T <= 0, a non-finite A, kappa,
 * G or rho_ref, or a rate outside (0, 2). */
int lbm_set_params(lbm_ctx* ctx, const lbm_eos* eos, double A, double kappa, double G,
                   const double s[9], double rho_ref, unsigned flags);
int lbm_batch_set_params(lbm_ctx* ctx, int i, const lbm_eos* eos, double A, double kappa,
                         double G, const double s[9], double rho_ref, unsigned flags);

/* Density-dependent shear viscosity (Section 4.2: gas and liquid of
 * different viscosity): with enable != 0, nu(rho) is linear between
 * (rho_gas, nu_gas) and (rho_liquid, nu_liquid) and clamped to that range, and
 * the shear rates become s_7 = s_8 = 1 / (3 nu(rho) + 1/2) at every node,
 * replacing s[7], s[8].  enable = 0 restores the fixed rates.  Call after
 * lbm_set_params; a later lbm_set_params keeps the law. */
int lbm_set_viscosity(lbm_ctx* ctx, int enable, double nu_gas, double nu_liquid, double rho_gas,
                      double rho_liquid);
int lbm_batch_set_viscosity(lbm_ctx* ctx, int i, int enable, double nu_gas, double nu_liquid,
                            double rho_gas, double rho_liquid);

/* Initial state f_a = M^-1 m_eq(rho, u) (Eq. 4) from host fields of nx*ny
 * doubles; ux, uy may be NULL (zero velocity).  Resets the step counter and
 * the instance's status.  The fields are copied to the device and checked
 * there first: a density that is not finite, positive and below the EOS's
 * upper limit (4/b Carnahan-Starling, 1/b otherwise; any positive density
 * when G = 0) or a velocity that is not finite returns LBM_EINVAL and leaves
 * the instance as it was.  A context of one lattice of 2^20 nodes or more
 * takes the fields in row bands, each band checked and its populations
 * written while the next band is copied.  Synchronous. */
int lbm_init_density(lbm_ctx* ctx, const double* rho, const double* ux, const double* uy);
int lbm_batch_init_density(lbm_ctx* ctx, int i, const double* rho, const double* ux,
                           const double* uy);
/* The same from fields of nx*ny floats (half the bytes to move): each value
 * is widened to FP64 exactly, then as above. */
int lbm_init_density_f32(lbm_ctx* ctx, const float* rho, const float* ux, const float* uy);
int lbm_batch_init_density_f32(lbm_ctx* ctx, int i, const float* rho, const float* ux,
                               const float* uy);

/* Enqueue n time steps (Eqs. 1, 9, 10, 23, 25, 26: density and psi, hybrid
 * force, modifying tensor, moment-space collision, streaming) of every
 * instance: one fused kernel launch per step (and per 64 instances),
 * replayed from CUDA graphs when graphs are on; with schedule 3 one launch
 * per call and chunk of instances, with schedule 4 one launch per call.
 * Asynchronous. */
int lbm_step(lbm_ctx* ctx, int n);

/* Wait for the stream; return the first sticky status of any instance. */
int lbm_sync(lbm_ctx* ctx);
/* Sticky status of instance i (synchronises). */
int lbm_status(lbm_ctx* ctx, int i);
/* Clear every instance's sticky status. */
int lbm_clear_status(lbm_ctx* ctx);

/* Macroscopic fields of the current state, each nx*ny doubles, any may be
 * NULL: rho = sum f, u = (sum f e + F/2)/rho (F of Eq. 9), psi of Eq. 10. */
int lbm_read_fields(lbm_ctx* ctx, double* rho, double* ux, double* uy, double* psi);
int lbm_batch_read_fields(lbm_ctx* ctx, int i, double* rho, double* ux, double* uy,
                          double* psi);
/* The same into fields of nx*ny floats (half the bytes to move): each value
 * is the FP64 result rounded to the nearest float. */
int lbm_read_fields_f32(lbm_ctx* ctx, float* rho, float* ux, float* uy, float* psi);
int lbm_batch_read_fields_f32(lbm_ctx* ctx, int i, float* rho, float* ux, float* uy, float* psi);

/* Pre-collision populations f_a(x, t) as 9*nx*ny doubles, index a*nx*ny + y*nx + x. */
int lbm_read_populations(lbm_ctx* ctx, double* f);
int lbm_batch_read_populations(lbm_ctx* ctx, int i, double* f);

/* Laplace-law sampling (Eq. 22) of a droplet centred at (cx, cy): mean
 * pressure p = p_EOS(rho) = rho/3 + G psi^2/2 (Eq. 10) over nodes within
 * r_in and beyond r_out (periodic minimum image), and the equimolar radius
 * R_eq = sqrt((sum rho - rho_out N)/(pi (rho_in - rho_out))).  Sums are FP64. */
int lbm_measure_pressure_jump(lbm_ctx* ctx, double cx, double cy, double r_in, double r_out,
                              double* p_in, double* p_out, double* R_eq);
/* Same for instance i; out[LBM_MEASURE_N] = {p_in, p_out, rho_in, rho_out,
 * R_eq, mass, n_in, n_out}. */
int lbm_batch_measure(lbm_ctx* ctx, int i, double cx, double cy, double r_in, double r_out,
                      double* out);

/* FP64 totals of the current state: mass sum rho, momentum sum rho u,
 * kinetic energy sum rho |u|^2 / 2, and max |u| (the peak spurious velocity
 * of a static droplet). */
int lbm_stats(lbm_ctx* ctx, double* mass, double* mom_x, double* mom_y, double* ke,
              double* umax);
int lbm_batch_stats(lbm_ctx* ctx, int i, double* out5);

/* Checkpoint: a header (sizes, precision, parameters, step count) and the
 * populations of every instance.  lbm_load needs a context of the same
 * shapes and precision and restores parameters, state and step count. */
int lbm_save(lbm_ctx* ctx, const char* path);
int lbm_load(lbm_ctx* ctx, const char* path);

/* Tile configurations of the fused step kernel for this precision: returns
 * their number; for index k writes tile width, height, threads per CTA and
 * pipeline stages (1: one tile per CTA; 2: persistent CTAs that prefetch the
 * next tile's TMA box while colliding the current one).  Any pointer may be
 * NULL. */
int lbm_tile_config_count(int precision);
int lbm_tile_config(int precision, int k, int* bx, int* by, int* threads, int* stages);
/* Select tile configuration k and CTA schedule (0: instance-major row
 * order, 1: the tiles of each launch's instances interleaved, 2: largest
 * instance first; a batch is stepped by one launch per 64 instances and
 * step).  Schedule 3 steps every instance through all n steps of an
 * lbm_step(n) call in one persistent launch per chunk of instances (up to 32
 * instances and 80 MiB of populations, the instances taken largest first and
 * spread evenly over as few chunks as that allows): CTAs take
 * (step, tile) items in step order from a counter in device memory and start
 * step s of a tile once every tile within two nodes of it (periodic) has
 * finished step s - 1 (each dependency wait bounded; one that gives up reports
 * LBM_ETIMEOUT); the launch is cooperative (every CTA resident), needs a
 * tile configuration of one tile box per CTA (stages 1; LBM_EINVAL
 * otherwise), and CUDA graphs are not used with it.  Schedule 4 holds a
 * single lattice (FP32: up to 64 nodes wide and 256 high, or 128 x 128; FP64:
 * up to 64 x 128; the last strip of 16 (FP32 up to 64 wide) or 8 rows at
 * least 2 rows high) in the shared memory of one thread-block cluster of up
 * to 16 CTAs for all n steps of an lbm_step call: one launch, strips of rows
 * per CTA, edge rows exchanged through distributed shared memory and one
 * cluster barrier per step (the tile configuration is ignored; LBM_EINVAL
 * for a batch, a lattice outside those sizes, or a device that cannot hold
 * the cluster).  Every schedule gives the same bits. */
int lbm_set_schedule(lbm_ctx* ctx, int tile_config, int schedule);
/* Time every (tile configuration, schedule) pair over `steps` steps of the
 * current state (which is restored afterwards) and keep the fastest (one
 * lattice: schedules 0 and 3, and 4 where the lattice fits a cluster).  Each
 * pair is timed as lbm_step runs it with the context's current graph
 * setting: with graphs on (lbm_use_graphs before this call), the one-step
 * schedules replay captured graphs and `steps` is rounded up to whole
 * replays.  A pair whose bounded device waits gave up is not chosen
 * (LBM_ETIMEOUT when no pair is left).  Writes the choice and its time per
 * step in milliseconds.  On an error the populations, counters and schedule
 * are put back as they were, as far as the device still allows. */
int lbm_autotune(lbm_ctx* ctx, int steps, int* tile_config, int* schedule, double* ms_per_step);

/* CUDA graphs for lbm_step: on (1) or off (0, the default).  With graphs on,
 * the one-step schedules run lbm_step(n) as replays of captured graphs of 32
 * steps, then of 16, 8, 4 and 2 steps as the rest's binary digits call for,
 * and a last odd step as a plain launch; a graph is captured on its first
 * use, and dropped when the parameters, schedule or graph setting change. */
int lbm_use_graphs(lbm_ctx* ctx, int on);
/* Capture, without running them, every graph lbm_step may replay for this
 * context (each length from either time level), so that no later lbm_step
 * pays for a capture (e.g. before a timed region).  Does nothing when graphs
 * are off or the schedule is 3.  Returns LBM_OK, LBM_EINVAL (an instance
 * without parameters or initial state) or LBM_ECUDA. */
int lbm_capture_graphs(lbm_ctx* ctx);

/* Steps done since the last init/load, and fused-step kernel launches
 * (graph replays count every kernel in them) since creation. */
long long lbm_steps_done(lbm_ctx* ctx);
long long lbm_kernel_launches(lbm_ctx* ctx);

/* Algorithmic bytes one lattice update moves: 9 population reads and 9
 * writes (72 for FP32, 144 for FP64). */
int lbm_bytes_per_update(int precision);

const char* lbm_last_error(lbm_ctx* ctx);

/* ---- Learned surrogate: MLP 3 -> 64 -> 64 -> 4 --------------------------
 * Maps (T/Tc, A, kappa) to (sigma, rho_l, rho_g, peak spurious velocity),
 * trained on droplet simulations of this library; its inverse picks the
 * kappa of Eq. 23 that gives a requested sigma.  Not in the paper.
 * GELU (exact, 0.5 z (1 + erf(z / sqrt 2))) after both hidden layers, FP32
 * weights and FP32 accumulation, mean-squared error on standardised targets,
 * Adam.  Parameters are one flat FP32 array of LBM_MLP_NPARAMS entries:
 * W1[64][3], b1[64], W2[64][64], b2[64], W3[4][64], b3[4] (row-major,
 * y = W x + b).  Inputs and targets are standardised inside with the
 * normalisation set by lbm_mlp_set_normalization (mean and std per column).
 * All host arrays are row-major FP32 (n x 3 inputs, n x 4 targets). */
#define LBM_MLP_IN 3
#define LBM_MLP_HIDDEN 64
#define LBM_MLP_OUT 4
#define LBM_MLP_NPARAMS 4676

typedef struct lbm_mlp lbm_mlp;

/* Create a network with seeded uniform(+-sqrt(6/(fan_in+fan_out))) weights and
 * zero biases on the given stream (NULL: legacy default); allocates its own
 * device buffers for up to max_samples training samples. */
int lbm_mlp_create(lbm_mlp** out, int max_samples, unsigned long long seed, void* stream);
void lbm_mlp_destroy(lbm_mlp* m);
int lbm_mlp_set_normalization(lbm_mlp* m, const float in_mean[3], const float in_std[3], const float out_mean[4],
                              const float out_std[4]);
int lbm_mlp_set_params(lbm_mlp* m, const float* params);
int lbm_mlp_get_params(lbm_mlp* m, float* params);
/* Mean-squared-error loss over n samples (standardised targets, mean over
 * samples and outputs) and its gradient with respect to every parameter,
 * computed by the training kernels without an update (gradient checks). */
int lbm_mlp_loss_grad(lbm_mlp* m, const float* X, const float* Y, int n, float* loss, float* grad);
/* One Adam step (lr, beta1, beta2, eps) on the full batch of n samples. */
int lbm_mlp_adam_step(lbm_mlp* m, const float* X, const float* Y, int n, float lr, float beta1, float beta2,
                      float eps);
/* Train for `epochs` passes over n samples in shuffled minibatches of
 * `batch` (seeded), Adam(lr, 0.9, 0.999, 1e-8); loss_per_epoch (nullable)
 * receives the mean minibatch loss of each epoch. */
int lbm_mlp_train(lbm_mlp* m, const float* X, const float* Y, int n, int epochs, int batch, float lr,
                  unsigned long long seed, float* loss_per_epoch);
/* Forward pass: n raw inputs -> n raw outputs (de-standardised). */
int lbm_mlp_predict(lbm_mlp* m, const float* X, int n, float* Y);
/* Inverse: for each of m targets (t_over_tc[i], A[i], sigma[i]) the kappa in
 * [kappa_lo, kappa_hi] whose predicted sigma equals sigma[i] (bisection on
 * the GPU; predicted sigma must decrease in kappa, as Eq. 28 has it).  NaN
 * where the target lies outside the predicted range. */
int lbm_mlp_invert_kappa(lbm_mlp* m, const float* t_over_tc, const float* A, const float* sigma, int count,
                         float kappa_lo, float kappa_hi, float* kappa_out);

/* ---- Allocation-free Laplace sampling of a device density field ----------
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory: one whose device memory is all owned by
 * another allocator (a framework's caching allocator or a fixed arena), or a
 * latency-critical loop that must not make an allocation call, which can
 * synchronise the whole device.
 *
 * The same sums as lbm_batch_measure, accumulated in FP64, but over a
 * density field d_rho of nx*ny doubles (row-major, x fastest) that the caller
 * keeps in device memory of the current device (make d_rho's device current
 * before the call); out receives LBM_MEASURE_N doubles in host memory {p_in,
 * p_out, rho_in, rho_out, R_eq, mass, n_in, n_out}, with p = p_EOS(rho) of
 * eos.  Work runs on `stream` (NULL: legacy default stream); the call copies
 * the totals to host memory and synchronises the stream before it returns.
 *
 * It allocates nothing: its scratch is a file-scope device array sized for at
 * most LBM_STATIC_MAX_NODES nodes (about 128 KiB, held by every GPU that loads
 * the library until the process exits).  Larger fields, a d_rho that is not
 * device memory of the current device, and an equation of state or
 * temperature that lbm_set_params would reject are refused with LBM_EINVAL
 * before any GPU work.  The first call on a device looks up the array's
 * device address with that device current; make that first call before any
 * stream capture.  Every call reuses the same array, so calls whose work
 * overlaps on the GPU (other streams, other host threads) race.
 * Returns LBM_OK, LBM_EINVAL or LBM_ECUDA. */
#define LBM_STATIC_MAX_NODES 16777216
int lbm_field_pressure_jump_static(const double* d_rho, int nx, int ny, const lbm_eos* eos, double cx,
                                   double cy, double r_in, double r_out, double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
