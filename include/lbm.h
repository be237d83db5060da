/*
 * lbm.h -- C ABI of the GB300 lattice Boltzmann library implementing the
 * second-order force scheme of Li, Duan & Shan, "Second-order force scheme for
 * lattice Boltzmann method" (arXiv:2212.07494).
 *
 * Problem statement (Sec. II of the paper): the discrete-velocity Boltzmann
 * equation with a body-force term F_i (Eq. dv), discretised in space and time
 * by the trapezoidal rule (Eq. implicityeq), which makes the stored variable
 *   fbar_i = f_i - Omega_i / 2 - F_i / 2                          (Eq. newf)
 * and the explicit update
 *   fbar_i(x + c_i, t + 1) = fbar_i(x, t) + Omega_i(x, t) + F_i(x, t)   (Eq. evolution)
 * with, for BGK, Eq. (explict_eq):
 *   fbar_i <- fbar_i - (fbar_i - f_i^eq)/tau + (1 - 1/(2 tau)) F_i
 * and, for SMRT, the order-by-order relaxation of the non-equilibrium central
 * (co-moving) Hermite moments, Eq. (RHS) in explicit form:
 *   d_p^(n) = (1 - 1/tau_n) d_1^(n) + (1 - 1/(2 tau_n)) d_F^(n),  d_F^(1) = rho g,
 * followed by the shift back to raw moments (Eq. bbd1), reconstruction and
 * streaming.  Macroscopic velocity: u = ubar + g/2 (Eq. half_F).
 *
 * Conventions shared by every entry point:
 *  - Units: lattice units (dx = dt = 1, c_s^2 = 1/3).  "tau" is the relaxation
 *    time appearing in the explicit update (the paper's tau-hat = tau + 1/2);
 *    the kinematic viscosity is nu = (tau_2 - 1/2)/3.  Every tau must be > 1/2.
 *  - Population order:
 *      D2Q9 : 0 (0,0); 1 (1,0); 2 (0,1); 3 (-1,0); 4 (0,-1);
 *             5 (1,1); 6 (-1,1); 7 (-1,-1); 8 (1,-1)
 *      D3Q19: 0 rest; 1..6 (1,0,0) (-1,0,0) (0,1,0) (0,-1,0) (0,0,1) (0,0,-1);
 *             7..18 (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1)
 *             (1,0,-1) (-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1)
 *      D3Q27: the D3Q19 order, then 19..26 (1,1,1) (-1,-1,-1) (1,1,-1)
 *             (-1,-1,1) (1,-1,1) (-1,1,-1) (-1,1,1) (1,-1,-1)
 *  - Host field layouts are structure-of-arrays with x fastest:
 *      populations f[i][z][y][x], velocity u[a][z][y][x] (a < D),
 *      per-node force g[a][z][y][x], per-row force g[y][a], solid[z][y][x].
 *  - Boundaries: an axis with periodic[k] = 0 has halfway bounce-back walls at
 *    -1/2 and n_k - 1/2; solid nodes (solid[x] != 0) bounce links back halfway
 *    too.  Solid nodes report rho = 1, u = 0 and are left out of totals.
 *  - Status codes: every call returns LBM_OK or a negative lbm_status; nothing
 *    throws across the ABI; lbm_last_error() returns a description of the
 *    last failure (per handle; thread-local for NULL).
 *  - Memory: the handle owns every device buffer it allocates (through the
 *    optional alloc/free callbacks, e.g. a PyTorch caching allocator, else
 *    cudaMalloc).  Input arrays are copied during the call; output arrays are
 *    caller-owned.  Calls are asynchronous on the handle's stream unless they
 *    return host data, in which case they synchronise that stream.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_NOT_CONVERGED = 1, /* per-channel status: max_steps reached above tol */
    LBM_OK = 0,
    LBM_ERR_ARG = -1,      /* invalid argument (sizes, tau <= 1/2, null pointer) */
    LBM_ERR_CUDA = -2,     /* a CUDA call failed; see lbm_last_error */
    LBM_ERR_OOM = -3,      /* device allocation failed */
    LBM_ERR_UNSTABLE = -4, /* a non-finite density or velocity was detected */
    LBM_ERR_TIMEOUT = -5,  /* a bounded device-side wait expired */
    LBM_ERR_STATE = -6     /* wrong state size / storage tag / handle kind */
} lbm_status;

typedef enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1, LBM_D3Q27 = 2 } lbm_lattice;
/* LBM_SMRT keeps the force's equilibrium part only, d_F^(1) = rho g and
 * d_F^(n>=2) = 0 (the scheme verified in Sec. III).  LBM_SMRT_FNEQ adds its
 * non-equilibrium contributions in the co-moving frame (Eq. Frc, third and
 * fourth terms): d_F^(n) = n g d^(n-1) for n = 3, 4, with d the central
 * moments of f recovered from those of fbar by inverting Eq. (newf),
 * d^(n) = (1 - 1/(2 tau_n)) (dbar_1^(n) + d_F^(n)/2).  LBM_MRT_RAW is the
 * raw-moment MRT of the appendix: the raw (not co-moving) non-equilibrium
 * moments relax order by order, a_p^(n) = a_0^(n) + (1 - 1/tau_n) a_1^(n)
 * + (1 - 1/(2 tau_n)) a_F^(n), with a_F^(n) = n F u^(n-1) and the fourth
 * order from the appendix's recursion.  All moment models start from the
 * same state; batches (lbm_batch_create) take all four. */
typedef enum { LBM_BGK = 0, LBM_SMRT = 1, LBM_SMRT_FNEQ = 2, LBM_MRT_RAW = 3 } lbm_collision;

/* Storage of the populations.  All modes store the deviation
 * delta_i = fbar_i - w_i; arithmetic is FP64 for LBM_F64 and FP32 otherwise.
 * FP16/BF16 conversions round to nearest even. */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16_SHIFT = 2, LBM_BF16_SHIFT = 3 } lbm_storage;

typedef enum {
    LBM_G_NONE = 0,    /* g = 0 */
    LBM_G_UNIFORM = 1, /* g: D doubles */
    LBM_G_ROWS = 2,    /* g: ny * D doubles, g[y][a] */
    LBM_G_FIELD = 3    /* g: D * nz * ny * nx doubles, g[a][z][y][x] */
} lbm_force_kind;

typedef struct lbm_handle lbm_handle;

typedef struct {
    int lattice;          /* lbm_lattice */
    int collision;        /* lbm_collision */
    int storage;          /* lbm_storage */
    int nx, ny, nz;       /* nz = 1 for D2Q9; nx * ny * nz < 2^31 / Q */
    int periodic[3];      /* per axis; 0 => halfway bounce-back walls */
    double tau[5];        /* tau per Hermite order n (index n); the moment models use tau[2..4]
                             (tau[0], tau[1] unused: orders 0 and 1 are conserved /
                             fixed by the force); BGK uses tau[2] */
    int force_kind;       /* lbm_force_kind */
    const double *g;      /* host, layout per force_kind; copied */
    const uint8_t *solid; /* host, nullable, nx*ny*nz bytes; copied */
    const double *rho0;   /* host, nullable (=> 1), nx*ny*nz; copied */
    const double *u0;     /* host, nullable (=> 0), D*nx*ny*nz; copied */
    void *stream;         /* cudaStream_t to run on; NULL => the library makes one */
    void *(*alloc)(size_t bytes, void *ctx); /* optional device allocator */
    void (*free_)(void *ptr, void *ctx);     /* its release function */
    void *alloc_ctx;
    double tau_bulk;      /* relaxation time of the trace (bulk) part of the
                             second-order moments, tau_{2,0} of Eq. (domg); the
                             traceless (shear) part keeps tau[2].  0 => tau[2].
                             Otherwise > 1/2, and a value other than tau[2] is
                             for LBM_SMRT / LBM_SMRT_FNEQ only (LBM_ERR_ARG).
                             The bulk viscosity is (2/D)(tau_bulk - 1/2)/3. */
} lbm_desc;

/* Create a lattice: validates the description, allocates two population
 * buffers, uploads g / solid / rho0 / u0 and initialises
 *   fbar = f_eq(rho0, u0) - F(rho0, u0)/2   (zero non-equilibrium part)
 * with the collision model's own equilibrium and force (Eq. newf with
 * Omega_i = 0).  On failure *out is NULL. */
lbm_status lbm_create(const lbm_desc *desc, lbm_handle **out);

/* Advance nsteps time steps (fused pull-stream, collide, store; Sec. II.B-C).
 * Asynchronous; long runs replay a captured CUDA graph. */
lbm_status lbm_step(lbm_handle *h, int64_t nsteps);

/* Macroscopic fields at the current step (Eq. half_F): rho (nx*ny*nz), u
 * (D planes) and totals {M, Px, Py, Pz} = sums over fluid nodes of rho and
 * rho*u (FP64, deterministic order).  Any output may be NULL.  Synchronises. */
lbm_status lbm_moments(lbm_handle *h, double *rho, double *u, double *totals);

/* Same on device pointers (FP64, same layouts); asynchronous. */
lbm_status lbm_moments_device(lbm_handle *h, double *rho_dev, double *u_dev,
                              double *totals_dev);

/* Advance K steps and return the K-step residual
 *   r = ||u(n) - u(n-K)||_2 / (K ||u(n)||_2)
 * over fluid nodes, accumulated in FP64.  Returns LBM_ERR_UNSTABLE if a
 * non-finite velocity appears.  Synchronises. */
lbm_status lbm_residual(lbm_handle *h, int K, double *r);

/* The periodic FP64 check of the state, asynchronously on the handle's
 * stream: writes 7 doubles to out_dev,
 *   {M, Px, Py, Pz, sum |u - u_snap|^2, sum |u|^2, number of non-finite nodes}
 * over fluid nodes, then stores u as the new snapshot u_snap.  The residual
 * of lbm_residual follows as sqrt(out[4]) / (K sqrt(out[5])) when the
 * previous check was K steps earlier; the snapshot starts at u = 0. */
lbm_status lbm_check_device(lbm_handle *h, double *out_dev);

/* Replace the body force (same kind and layout as at creation); takes effect
 * for the next step.  Asynchronous (the host array is copied first). */
lbm_status lbm_set_force(lbm_handle *h, const double *g);

/* Time-dependent uniform body force from a table, for forcing such as the
 * oscillating pressure gradient of the Womersley case (Sec. III.B) without a
 * host call per step: table[t][a] (period x D doubles, host, copied) is the
 * acceleration g of the t-th step after this call, repeating with the
 * given period, i.e. the collision of step s (and the velocity of
 * Eq. half_F reported at step s) uses table[s mod period], s counted from
 * this call.  The step counter lives on the device, so the schedule runs
 * inside the captured step graphs.  Requires LBM_G_UNIFORM at creation
 * (else LBM_ERR_STATE).  period = 0 removes the schedule (the force set
 * last by lbm_set_force or at creation applies again); lbm_set_force also
 * removes it.  The schedule's phase is not part of lbm_get_state's state.
 * Synchronises the handle's stream. */
lbm_status lbm_set_force_schedule(lbm_handle *h, const double *table, int64_t period);

/* Time-dependent scaling of the force of any kind (uniform, per row or per
 * node), for forcing of the form g(x, t) = s(t) g(x), such as the decaying
 * force of the forced Taylor-Green case (Sec. III.A): the collision of step
 * s (and the velocity of Eq. half_F at step s) uses scale[s mod period] times
 * the force set at creation or by lbm_set_force, s counted from this call.
 * scale: period doubles (host, copied).  The same device step counter as
 * lbm_set_force_schedule, so it runs inside the step graphs; either schedule
 * replaces the other.  period = 0 removes it; lbm_set_force also removes
 * it.  LBM_ERR_STATE without a force.  Synchronises the handle's stream. */
lbm_status lbm_set_force_scale_schedule(lbm_handle *h, const double *scale, int64_t period);

/* Pre-collision populations fbar_i(x, t) in FP64, host layout f[i][z][y][x]
 * (solid nodes: w_i).  Synchronises. */
lbm_status lbm_get_populations(lbm_handle *h, double *f);
/* Overwrite the state with the given pre-collision populations (rounded to the
 * storage format). */
lbm_status lbm_set_populations(lbm_handle *h, const double *f);

/* Raw checkpoint of the state in the storage format plus the step counter;
 * restore is bit-exact.  Layout of the lbm_state_bytes bytes: the deviations
 * fbar_{i,p} - w_i of the post-collision populations of the last step (the
 * values the next step pulls), in the storage type (double, float, IEEE
 * half or bfloat16), as [Q][nz][ny][nxp] with rows padded to
 * nxp = 32 * ceil(nx / 32) (padding entries are zero). */
size_t lbm_state_bytes(const lbm_handle *h);
lbm_status lbm_get_state(lbm_handle *h, void *host, size_t bytes, int64_t *step);
lbm_status lbm_set_state(lbm_handle *h, const void *host, size_t bytes, int64_t step);

/* Node layout of a thread in the fused stream-collide kernel (the pull of
 * Sec. II.C with the collision in between; the two compute the same values).
 *   LBM_LAYOUT_STRIDED: nodes_per_thread (1 or 2) nodes, block_x apart along
 *     x; each population of each node is one load.
 *   LBM_LAYOUT_VECTOR: nodes_per_thread consecutive nodes along x; each
 *     population of them is one aligned vector load and store (D2Q9: up to
 *     16 bytes), the one-node shift of the pull taken from the neighbouring
 *     lane.  Only without an obstacle mask and with Q * plane < 2^32 (plane
 *     as in lbm_get_state); the widths built per lattice and storage are
 *     given by lbm_launch_widths. */
typedef enum { LBM_LAYOUT_STRIDED = 0, LBM_LAYOUT_VECTOR = 1 } lbm_layout;

/* Launch shape of the fused stream-collide kernel: threads per block along x
 * (block_x: 32, 64, 128 or 256), nodes per thread along x and their layout.
 * Drops the captured step graphs;
 * synchronises the handle's stream.  The physics does not depend on the
 * shape; in FP32 arithmetic the results can differ in the last bits between
 * shapes (the FP32 storage modes collide nodes two at a time in packed FP32
 * where a thread has two, which may pair fused multiply-adds differently
 * from one node at a time).  A new handle starts with the shape measured
 * fastest on GB300 for its lattice and storage: the vector layout at its
 * wider width for FP16 and BF16 storage and for D3Q27 in FP32 when the layout
 * applies, else the strided layout.  LBM_ERR_ARG for a shape not listed. */
lbm_status lbm_set_launch_layout(lbm_handle *h, int block_x, int nodes_per_thread, int layout);
/* lbm_set_launch_layout with LBM_LAYOUT_STRIDED (nodes_per_thread 1 or 2). */
lbm_status lbm_set_launch(lbm_handle *h, int block_x, int nodes_per_thread);
/* The current launch shape (outputs nullable). */
lbm_status lbm_get_launch(const lbm_handle *h, int *block_x, int *nodes_per_thread, int *layout);
/* The two vector widths (nodes per thread; equal when only one is built) of
 * LBM_LAYOUT_VECTOR for a lattice and storage (outputs nullable). */
lbm_status lbm_launch_widths(int lattice, int storage, int *lo, int *hi);

/* Time every supported launch shape over `trials` launches each (CUDA events
 * on the handle's stream; the kernel reads the current state and writes the
 * spare buffer, so the state does not advance): the strided shapes, and the
 * vector shapes (blocks of 32, 64, 128; both widths) where
 * that layout applies.  Keep the fastest and return its block_x and
 * nodes_per_thread (outputs nullable; lbm_get_launch gives its layout) with
 * its mean launch time in milliseconds.  Synchronises. */
lbm_status lbm_autotune(lbm_handle *h, int trials, int *block_x, int *nodes_per_thread, double *ms);

/* Information (outputs nullable): D, Q, the step counter, and the
 * algorithmic bytes of one node update, 2 Q times the storage size (the
 * populations read and written by one step). */
lbm_status lbm_info(const lbm_handle *h, int *D, int *Q, int64_t *step, size_t *bytes_per_node);

/* Speed above which one time step of the body force is lost to the rounding
 * of the stored deviations: the regime in which a reduced storage format
 * can carry a forced flow.  Each step adds the force to the first moment of
 * the populations (Sec. II.C: after the collision the first central moment
 * is F/2, before it the pull brought -F/2), so the stored deviation
 * delta_i of a population changes by about 3 w_i c_i . g, while a fluid
 * moving at u holds delta_i ~ 3 w_i c_i . u.  Rounding to nearest with a
 * p-bit significand drops every change below half an ulp of the stored
 * value, which is at least 2^-(p+1) of it; so once |u| exceeds
 *   u_stall = 2^(p+1) max|g|     (p = 53, 24, 11, 8 for F64, F32, F16, BF16)
 * the force increments round away and the flow stops gaining speed from the
 * force (the stored state stagnates).  A flow accelerated from rest, u ~ g t,
 * gets there after about 2^(p+1) steps: 512 in BF16, 4096 in FP16, 3.4e7 in
 * FP32.  +inf without a force (or a zero one).  The maximum is over the
 * force given at creation, by lbm_set_force, or by a schedule.  lbm_create
 * leaves a note in lbm_last_error(h) when the initial velocity already
 * exceeds u_stall. */
lbm_status lbm_force_resolution(const lbm_handle *h, double *u_stall);

void lbm_destroy(lbm_handle *h);
const char *lbm_last_error(const lbm_handle *h);

/* ---------------------------------------------------------------- batches
 * Many independent D2Q9 lattices ("channels") of different sizes, relaxation
 * times and forces, advanced together by ONE persistent kernel launch
 * (captured in a CUDA graph): each time step of a channel is split into
 * tiles of rows that any CTA may claim; a channel's next step starts when
 * all tiles of its current step are done.  Every K steps a channel computes
 * its residual r_K (as lbm_residual) and retires once r_K <= tol.
 * Channels share lattice (D2Q9), collision (any lbm_collision; one tau per
 * order, no split bulk time) and storage (LBM_F32 or LBM_F64);
 * each takes its own nx, ny, periodic flags, tau, uniform (or no) force and
 * optional solid mask (halfway bounce-back at solid nodes).  The descriptions' rho0/u0 are copied.  The stream of
 * descs[0] is used (NULL => the library makes one). */
typedef struct lbm_batch lbm_batch;

lbm_status lbm_batch_create(const lbm_desc *descs, int n, lbm_batch **out);

/* Run every channel until r_K <= tol (status LBM_OK), a non-finite residual
 * (LBM_ERR_UNSTABLE) or max_steps more steps (LBM_NOT_CONVERGED).  Outputs
 * (n entries each, nullable): steps completed (the channel stops one step
 * after the check that met tol), status, last residual.  Returns
 * LBM_ERR_TIMEOUT if the kernel's bounded scan for work saw no progress
 * anywhere for the scan limit (see lbm_batch_set_spin_limit); the channels
 * then hold the state they had reached.  Synchronises.
 * The tail of a run: once at most lbm_batch_set_handoff's number of channels
 * still run, each of them leaves the kernel at its next step boundary and
 * the library continues it as a plain lattice (lbm_create / lbm_step /
 * lbm_check_device on a stream of its own, all such channels concurrently),
 * with the same check cadence, residual and stopping rules; the final state
 * returns to the batch, so the outputs and lbm_batch_moments read the same
 * as without the handoff. */
lbm_status lbm_batch_run_to_steady(lbm_batch *b, double tol, int K, int64_t max_steps, int64_t *steps_out,
                                   int *st_out, double *r_out);

/* Advance every channel nsteps more steps (same launch, no convergence). */
lbm_status lbm_batch_step(lbm_batch *b, int64_t nsteps);

/* Re-initialise every channel from its description (step counters to 0). */
lbm_status lbm_batch_reset(lbm_batch *b);

/* Macroscopic fields / FP64 pre-collision populations of channel i (host
 * layouts as for a single lattice).  Synchronise. */
lbm_status lbm_batch_moments(lbm_batch *b, int i, double *rho, double *u);
lbm_status lbm_batch_get_populations(lbm_batch *b, int i, double *f);

/* Tiling: threads per CTA (64, 128, 256) and target nodes per tile (rows of a
 * channel per tile = ceil(tile_nodes / nx)).  lbm_batch_autotune times every
 * (block, tile) pair over `steps` steps, keeps the fastest, then resets the
 * channels (tuning advances them). */
lbm_status lbm_batch_set_tiles(lbm_batch *b, int block, int tile_nodes);
lbm_status lbm_batch_autotune(lbm_batch *b, int steps, int *block, int *tile_nodes, double *ms_per_step);

/* Channels left running when the tail moves to plain lattices (default 8;
 * 0: the kernel runs every channel to the end).  A lone small channel costs
 * a whole scheduling round of the persistent kernel per step, a plain
 * lattice one graph-launched kernel. */
lbm_status lbm_batch_set_handoff(lbm_batch *b, int channels);

/* Scans for work without progress anywhere before the kernel stops with
 * LBM_ERR_TIMEOUT (default 2^26). */
lbm_status lbm_batch_set_spin_limit(lbm_batch *b, int64_t scans);

lbm_status lbm_batch_info(const lbm_batch *b, int i, int64_t *steps, int *tiles, int *rows);
const char *lbm_batch_last_error(const lbm_batch *b);
void lbm_batch_destroy(lbm_batch *b);

/* ---------------------------------------------------------------- surrogate
 * The steady-flow surrogate of the warm start: a U-Net on an H x W grid
 * (H, W multiples of 8) mapping per-node inputs x[n][y][x][cin] (FP32,
 * 1 <= cin <= 16) to outputs y[n][y][x][3] (FP32).  Every 3x3 convolution
 * pads with zeros along y and, when periodic_x = 1, wraps around along x
 * (a channel periodic in x), else pads with zeros.  Architecture: 4 levels of widths
 * 32/64/128/256, two 3x3 convolutions + ReLU per level, 2x2 average pooling
 * down, nearest 2x upsampling + 3x3 conv + ReLU up, concatenation
 * [up path, skip], linear 3x3 head.  BF16 weights and activations, FP32
 * accumulation on the tensor cores (every convolution and input-gradient
 * convolution but the 3-output head as an implicit GEMM on tcgen05 with TMEM
 * accumulators, the weight gradients too where H divides 64 or is a multiple
 * of 64; the head and the other weight gradients on mma.sync), FP32 master
 * weights and Adam moments.  A tcgen05 convolution whose bounded wait
 * expires is reported as LBM_ERR_TIMEOUT by the next lbm_unet_grad or
 * lbm_unet_get_params (the calls that synchronise).
 * Loss: sum_p m[p] sum_c (y - t)^2 * scale (scale = 1 / (3 sum m) gives the
 * weighted mean).  Parameters (host, FP32) in the canonical layout: per layer
 * W[co][ky][kx][ci] then b[co], layers in the order enc1a enc1b enc2a enc2b
 * enc3a enc3b bota botb up3 dec3a dec3b up2 dec2a dec2b up1 dec1a dec1b head.
 * All *_dev pointers are device arrays of n * H * W pixels. */
typedef struct lbm_unet lbm_unet;

/* H, W multiples of 8; 1 <= cin <= 16; max_batch * H <= 65535.  stream: the
 * cudaStream_t every call runs on (NULL: the library makes one). */
lbm_status lbm_unet_create(int H, int W, int cin, int periodic_x, int max_batch, void *stream, lbm_unet **out);
int64_t lbm_unet_num_params(const lbm_unet *u);
lbm_status lbm_unet_set_params(lbm_unet *u, const float *host);  /* resets Adam */
lbm_status lbm_unet_get_params(lbm_unet *u, float *host);
lbm_status lbm_unet_forward(lbm_unet *u, const float *x_dev, float *y_dev, int n);
/* Loss and parameter gradient (host outputs nullable; synchronises if given). */
lbm_status lbm_unet_grad(lbm_unet *u, const float *x_dev, const float *t_dev, const float *m_dev, int n,
                         float scale, double *loss_host, float *grad_host);
/* One Adam step from the last gradient (Kingma & Ba, bias-corrected). */
lbm_status lbm_unet_adam(lbm_unet *u, float lr, float beta1, float beta2, float eps);
/* Forward, backward and Adam (beta 0.9 / 0.999, eps 1e-8); loss to loss_dev
 * (nullable).  Asynchronous. */
lbm_status lbm_unet_train_step(lbm_unet *u, const float *x_dev, const float *t_dev, const float *m_dev, int n,
                               float scale, float lr, double *loss_dev);
/* Which kernel computes the weight gradients: LBM_UNET_WGRAD_AUTO (the
 * default) takes the tcgen05 one wherever the shape allows, and
 * LBM_UNET_WGRAD_MMA_SYNC the mma.sync one everywhere.  Both compute the
 * same sums in FP32 in different orders.  Synchronises the network's
 * stream; LBM_ERR_ARG for another kind. */
enum { LBM_UNET_WGRAD_AUTO = 0, LBM_UNET_WGRAD_MMA_SYNC = 1 };
lbm_status lbm_unet_set_wgrad(lbm_unet *u, int kind);
const char *lbm_unet_last_error(const lbm_unet *u);
void lbm_unet_destroy(lbm_unet *u);

/* Arithmetic peak of the current device's CUDA cores, measured: one launch
 * of a full wave of threads (8 blocks of 256 per SM), each running 8
 * independent chains of `iters` fused multiply-adds, timed with CUDA events
 * after one untimed launch.  precision: LBM_F32 or LBM_F64.  Outputs
 * (nullable): TFLOP/s (2 flops per FMA) and the timed launch's duration.
 * The ceilings of the step kernels that HBM does not bound: FP32 FMA for
 * the collision arithmetic of the FP32, FP16 and BF16 modes (an FP32 FMA
 * per lane per clock is also one warp instruction issued per scheduler per
 * clock), FP64 FMA for the FP64 mode.  Measurement only; allocates and frees
 * its own output buffer, synchronises. */
lbm_status lbm_alu_peak(int precision, int64_t iters, double *tflops, double *ms);

/* ------------------------------------------------------------------------
 * Split domains: the domain decomposition of the stream step (Sec. II.C).
 *
 * The pull f_i(x, t + 1) = f_i,p(x - c_i, t) couples a node only to its
 * neighbours one layer away, so a domain split into slabs along its
 * outermost axis (y in 2-D, z in 3-D) needs, per time step, one exchange:
 * each slab's first and last owned layer pull the populations that cross the
 * cut from a halo layer holding the neighbouring slab's layer.  Those with
 * c = +1 along the axis fill the lower halo, those with c = -1 the upper.
 * The FP64 check is the sum of the slabs' checks (an all-reduce of the mass,
 * the momentum and the residual terms).  The result is the same, bit for
 * bit, as the whole domain's: every node runs the same arithmetic on the
 * same values.
 *
 * Here every slab lives on the current device, in its own population
 * buffers, and all share the stream of desc (the library's own when NULL);
 * the exchange is one kernel over a table of layer copies.
 */
typedef struct lbm_split lbm_split;

/* Slab layout and exchange schedule of `parts` slabs of an axis of n_all
 * layers (host only, no device work).  Slab p owns the global layers
 * [layers[2p], layers[2p] + layers[2p + 1]): n_all / parts each, the first
 * n_all % parts one more.  Local layer 0 and n + 1 of a slab with n layers
 * are its halo layers, 1 .. n its own.  copies (5 ints each: destination
 * slab, destination local layer, source slab, source local layer,
 * population index) lists the copies of one exchange in order; with
 * periodic = 0 none crosses the domain's ends.  Outputs nullable;
 * *n_copies receives the count; LBM_ERR_ARG if max_copies is too small, if
 * parts < 1 or parts > n_all. */
lbm_status lbm_split_schedule(int lattice, int n_all, int parts, int periodic, int *layers, int *copies,
                              int max_copies, int *n_copies);
/* Create the whole domain of desc (as lbm_create; its initial state) and
 * `parts` slabs of it along the outermost axis.  Device memory: the whole
 * domain's buffers plus every slab's (n + 2 layers each). */
lbm_status lbm_split_create(const lbm_desc *desc, int parts, lbm_split **out);
/* nsteps time steps: every slab's stream-collide step, then the exchange.
 * Asynchronous on the split's stream. */
lbm_status lbm_split_step(lbm_split *s, int64_t nsteps);
/* The FP64 check of lbm_check_device summed over the slabs in slab order
 * (each slab keeps its own velocity snapshot), 7 device doubles at out_dev.
 * Asynchronous. */
lbm_status lbm_split_check_device(lbm_split *s, double *out_dev);
/* The slabs' layers assembled into the whole domain, then lbm_moments,
 * lbm_get_state (layout of lbm_get_state; *step nullable) or
 * lbm_get_populations on it.  Synchronise. */
lbm_status lbm_split_moments(lbm_split *s, double *rho, double *u, double *totals);
size_t lbm_split_state_bytes(const lbm_split *s);
lbm_status lbm_split_get_state(lbm_split *s, void *host, size_t bytes, int64_t *step);
lbm_status lbm_split_get_populations(lbm_split *s, double *f);
/* lbm_set_launch_layout on every slab. */
lbm_status lbm_split_set_launch_layout(lbm_split *s, int block_x, int nodes_per_thread, int layout);
/* Last error message of s (of the calling thread when s is NULL). */
const char *lbm_split_last_error(const lbm_split *s);
void lbm_split_destroy(lbm_split *s);

/* lbm_check_noalloc -- the FP64 check of lbm_check_device for callers that
 * cannot allocate device memory.  The paper has no counterpart: it is a
 * service of this library.
 *
 * Who needs it: code that receives device pointers but may not own device
 * memory (plug-ins driven by a host framework), processes whose device
 * memory is already reserved by a pooling allocator, and fixed-budget or
 * latency-critical loops where cudaMalloc (which can fail and synchronises
 * the device) is not allowed.  lbm_create allocates, so such callers hold the
 * state in their own buffer and call this function with it.
 *
 * Inputs: desc (lattice, storage, nx, ny, nz, periodic, force_kind and, for
 * LBM_G_UNIFORM, the D host values in desc->g; collision and tau are not
 * used; desc->stream is ignored), state_dev: a device buffer in the
 * lbm_get_state layout above.  Output: out_dev, 7 device doubles
 *   {M, Px, Py, Pz, sum |u - u_snap|^2, sum |u|^2, non-finite nodes}
 * as lbm_check_device writes them.  stream: cudaStream_t or NULL.
 *
 * Limits: no solid mask (LBM_ERR_ARG), force NONE or UNIFORM only, and the
 * velocity snapshot D * nx * ny * nz * (8 for LBM_F64, else 4) bytes must fit
 * in 16 MiB - 128 KiB (about 2.08 million nodes for D2Q9 in FP32);
 * larger problems are rejected with LBM_ERR_ARG before any device work.
 *
 * Memory: nothing is allocated.  Scratch (partial sums, the force, the
 * snapshot) lives in one static 16 MiB device array that every GPU which
 * loads this library holds until the process exits.  The first call on a
 * device sets up that device (looks up the array's address and clears it,
 * synchronously), so make it before any stream capture on that device.
 * All calls on a device share the array, which keeps the last call's
 * snapshot: the residual entries compare with the velocity of the previous
 * call on the same device, if that call had the same lattice, storage, nx,
 * ny and nz.  The first call on a device, and a call whose layout differs
 * from the previous call's, compare with zero instead (the call clears the
 * snapshot on its stream first), so there sum |u - u_snap|^2 = sum |u|^2.
 * Calls that overlap on the GPU (different streams without ordering) race
 * on the array. */
lbm_status lbm_check_noalloc(const lbm_desc *desc, const void *state_dev, double *out_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_GB300_H */
