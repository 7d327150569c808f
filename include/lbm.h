/*
 * lbm.h -- C ABI of the GB300 (sm_103a) thermal compressible lattice
 * Boltzmann library: one fused pull-stream / BGK-collide step with the
 * Hermite-expanded body force of Li & Shan, "Body-force modelling in thermal
 * compressible flows with lattice Boltzmann method" (arXiv 2302.04741).
 *
 * What one step computes (Sec. 2):
 *   f~_i(x, t+1) = f*_i(x - e_i, t)                              (pull stream)
 *   f*_i = f~_i - (f~_i - f0_i)/tau + (1 - 1/(2 tau)) F_i          (Eq. lbm)
 * with f0_i the Hermite-expanded equilibrium (4th order on D2Q37, 3rd on
 * D3Q39) and F_i the discrete body force up to the third moment (Eq. fi,
 * without the deviatoric-stress terms), both evaluated at the mid-point
 * state rho, u + g/2, theta; tau is the collision divisor tau-hat of Eq. lbm
 * (tau-hat = tau + 1/2 in the paper's notation, so the kinematic viscosity is
 * theta (tau - 1/2) in lattice units where the lattice spacing is c).
 *
 * Conventions for every entry point:
 *   - Returns an lbm_status (0 = LBM_OK, negative = error); no exception
 *     crosses the ABI.  lbm_last_error() gives the message of the last error
 *     of a context.
 *   - The library owns all device memory of a context (cudaMalloc at create,
 *     cudaFree at destroy).  Caller arrays are only read or written during
 *     the call; the caller keeps ownership.
 *   - Array arguments may be host or device pointers (detected with
 *     cudaPointerGetAttributes); device pointers must be on the context's
 *     device.  Fields are row-major [nz][ny][nx], x fastest, N = nx*ny*nz
 *     sites; vector fields are component-major: u[a*N + site].
 *   - Velocities and accelerations are in units of sqrt(theta_0), theta_0 = 1
 *     (the units in which the quadrature is exact); the lattice spacing is c
 *     (lbm_lattice_info) and the time step is 1.
 *   - All work is issued on the context's stream.  lbm_step returns without
 *     synchronising; calls that hand results to the caller (lbm_moments,
 *     lbm_conserved, lbm_get_*) synchronise that stream before returning.
 *   - One context must not be used from two host threads at once; separate
 *     contexts are independent.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

/* Velocity sets (Sec. 3: D2Q37, ninth-order Gauss-Hermite rule with lattice
 * constant c ~ 1.19698; D3Q39: seventh-order rule, c = sqrt(3/2)). */
typedef enum { LBM_D2Q37 = 0, LBM_D3Q39 = 1 } lbm_lattice;

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = -1,    /* bad argument (message says which)                   */
  LBM_ENOMEM = -2,    /* device or host allocation failed                    */
  LBM_ECUDA = -3,     /* a CUDA runtime call failed (message has the code)   */
  LBM_EUNSTABLE = -4, /* lbm_conserved found NaN/Inf or rho <= 0 or T <= 0   */
  LBM_ETIMEOUT = -5,  /* a bounded device wait ran out (reported by the next
                         lbm_conserved; the results of that step are void)   */
  LBM_ESTATE = -6,    /* call out of order (e.g. lbm_step before lbm_init)   */
  LBM_EIO = -7        /* checkpoint file could not be read or written        */
} lbm_status;

/* Body-force acceleration g(x) (the g of Eq. BGK). */
enum { LBM_G_UNIFORM = 0, /* g = g0                                             */
       LBM_G_SINE = 1,    /* g = g0 * sin(2 pi x_a / n_a), a = wave_axis        */
       LBM_G_FIELD = 2 }; /* g = field[a*N + site], D components, caller-owned,
                             copied to the device at lbm_create                */
typedef struct {
  int kind;
  double g0[3];
  int wave_axis;
  const double *field;
} lbm_gfield;

/* Population storage (the codec wraps the pull and the store of a step). */
enum { LBM_FP64 = 0,         /* f_i in IEEE double, arithmetic in double          */
       LBM_FP32_SHIFTED = 1, /* f_i - w_i rho0 (rho0 = 1) in float, arithmetic in float */
       LBM_FP16_SCALED = 2 };/* half(s (f_i - w_i) / w_i), one scale s per grid chosen
                                at lbm_init, arithmetic in float               */

/* Boundary condition per axis.  Walls are allowed on the LAST axis only (y on
 * D2Q37, z on D3Q39), at x_a = -1/2 and n_a - 1/2, and need n_a >= 6.  The
 * paper's multi-speed boundary rule is unpublished (Sec. 3), so the library
 * uses its own mass-conserving rules:
 *   BOUNCE_BACK:  f~_i(x) = f*_{-i}(x') with x' the same column and the wall
 *                 coordinate mirrored, x'_a = e_ia - 1 - x_a at the low wall
 *                 (2 n_a - 1 - (x_a - e_ia) at the high wall);
 *   THERMAL_WALL: diffuse reflection: those slots receive
 *                 rho_w f0_i(1, 0, T_wall), rho_w chosen per column so that the
 *                 column's incoming mass equals its outgoing mass. */
enum { LBM_PERIODIC = 0, LBM_BOUNCE_BACK = 1, LBM_THERMAL_WALL = 2 };

typedef struct {
  int precision;     /* LBM_FP64 | LBM_FP32_SHIFTED | LBM_FP16_SCALED         */
  int force_order;   /* the paper's N in Eq. F: force terms n <= N+1.
                        0: n = 1 only; 1: n <= 2 (the Guo scheme, Sec. 2);
                        2: n <= 3, the third-moment term of Eq. fi (default)  */
  int include_sigma; /* 1: keep the deviatoric stress in the force's second
                        coefficient, a^(2) = a^(2)_0 - sigma-bar (Eq. f2, the
                        sigma terms of Eq. fi), with sigma-bar = -(1 - 1/(2
                        tau-hat)) sum_i (f~_i - f0_i)(xi_i - u)(xi_i - u).
                        Acts at force_order 2 only (it enters the n = 3 term);
                        runs in the plain step kernel (LBM_KERNEL_TMA and
                        LBM_KERNEL_PREFETCH are rejected) and not in batches.
                        0: neglected, as in the paper's runs (default)       */
  int bc[3];         /* per axis: LBM_PERIODIC | LBM_BOUNCE_BACK | LBM_THERMAL_WALL */
  double T_lo[3];    /* wall temperature at x_a = -1/2 (THERMAL_WALL)         */
  double T_hi[3];    /* wall temperature at x_a = n_a - 1/2                   */
  void *stream;      /* cudaStream_t to issue work on; NULL = a stream the
                        library creates for the context                      */
  int block_x;       /* threads per block along x for the step kernel
                        (0 = library default; multiple of 32, <= 256)        */
  int graph_steps;   /* > 0: lbm_step replays a captured CUDA graph of this
                        many steps (even); 0 = plain launches                */
  int kernel;        /* step kernel: LBM_KERNEL_AUTO (= plain), LBM_KERNEL_PLAIN
                        (one thread per site, direct loads), or LBM_KERNEL_TMA
                        (persistent, TMA-staged shared-memory ring; error if
                        the grid does not qualify: FP32/FP16 storage and
                        nx * sizeof(element) a multiple of 16 bytes)          */
  int tma_stages;    /* shared-memory ring depth of the TMA-staged kernel
                        (0 = library default, else 2..8)                     */
  double mu;         /* > 0: constant dynamic viscosity mu; every site relaxes
                        with tau-hat = mu / (rho theta) + 1/2 at its mid-point
                        state (the paper's validation runs set tau = mu/(rho
                        theta) so that mu and the conductivity stay uniform,
                        Sec. 3.1); the tau argument of lbm_create is then
                        unused.  0: constant tau-hat = tau (default)          */
  int overlap_steps; /* 1: each plain step kernel is launched as a programmatic
                        dependent of the previous kernel on the stream, so its
                        blocks are scheduled while that kernel drains; they
                        wait for its completion and memory (griddepcontrol.
                        wait) before the first population load.  0: plain
                        stream order.  -1 (default): on for grids of at least
                        LBM_OVERLAP_MIN_SITES sites (on grids too small to
                        fill the GPU its effect was within run-to-run noise).
                        Results are identical either way.                    */
  int storage_probe; /* LBM_FP64 storage only: 0 (default) off; LBM_FP32_SHIFTED
                        or LBM_FP16_SCALED: after every step (and at lbm_init)
                        each stored deviation f*_i - w_i is rounded to that
                        codec's format (float; half of s (f - w)/w with the
                        scale s chosen at lbm_init as for LBM_FP16_SCALED),
                        the arithmetic staying in double.  Such a run has the
                        storage precision of the named codec and exact
                        arithmetic: its distance from the plain FP64 run is
                        the codec's storage floor.  Plain step kernel only.  */
  int fp64_arith;    /* LBM_FP64 storage: arithmetic of the step kernel.
                        LBM_ARITH_DOUBLE (0, default): IEEE double.
                        LBM_ARITH_FLOAT_PAIR (1): float-float (an unevaluated
                        sum of two floats, ~48 significant bits) on the FP32
                        pipe; populations stay doubles in memory and every
                        other call of the context is unchanged.  On GPUs whose
                        FP64 rate is a small fraction of the FP32 rate (GB300:
                        1/73) the double step is bound by the FP64 units; the
                        float-float step moves that bound.  Per population it
                        agrees with the double step to about 1e-14.  Plain
                        step kernel, no solid sites, no storage probe.        */
} lbm_options;

enum { LBM_ARITH_DOUBLE = 0, LBM_ARITH_FLOAT_PAIR = 1 };

#define LBM_OVERLAP_MIN_SITES 131072

enum { LBM_KERNEL_AUTO = 0, LBM_KERNEL_PLAIN = 1, LBM_KERNEL_TMA = 2,
       LBM_KERNEL_PREFETCH = 3 /* persistent; each thread prefetches its next tile's
                                  populations into shared memory with cp.async while
                                  colliding the current one (FP32-shifted only) */,
       LBM_KERNEL_WAVE = 4     /* several steps per launch: persistent blocks take
                                  (step, line, tile) items in step-major order and
                                  wait, with bounded polls, until the 3 lines on each
                                  side finished the previous step; FP32-shifted and
                                  FP16-scaled storage, no sigma-bar terms; results
                                  identical to the plain kernel */ };

/* Fills *opt with the defaults: FP64, force_order 2, no sigma, fully periodic,
 * wall temperatures 1, NULL stream, library block shape, no graph. */
void lbm_default_options(lbm_options *opt);

/* sizeof(lbm_options) as compiled into the library, so that a binding can
 * check its own copy of the struct layout before passing one in. */
size_t lbm_options_size(void);

/* Velocity set of a lattice: D, Q, c, the integer vectors e (Q*3, the
 * library's direction order: rest first, then opposite pairs), the weights w
 * (Q).  Any output pointer may be NULL.  Host pointers only. */
int lbm_lattice_info(lbm_lattice lat, int *D, int *Q, double *c, int *e, double *w);

/* Creates a context on the current CUDA device for an nx*ny*nz grid (nz must
 * be 1 on D2Q37): the discrete problem of Sec. 2 -- the distribution f_i on
 * the Gauss-Hermite abscissae xi_i = c e_i (Eq. rut1 and the quadrature that
 * precedes it), advanced by Eq. lbm with collision divisor tau = tau-hat
 * > 1/2 and the body-force acceleration g of Eq. BGK.  g may be NULL (no
 * force).  opt may be NULL (defaults).  Allocates two population buffers
 * (ping-pong), the force table and reduction scratch; the context owns them
 * until lbm_destroy.  *out receives the context, or NULL on error
 * (LBM_EINVAL for an invalid argument, checked before any allocation;
 * LBM_ENOMEM / LBM_ECUDA when the device refuses). */
int lbm_create(lbm_lattice lat, int nx, int ny, int nz, double tau, const lbm_gfield *g,
               const lbm_options *opt, lbm_ctx **out);

/* Sets the state to the Maxwellian with the given density, velocity and
 * temperature (the physical fields at t = 0): it stores
 * f~_i = f0_i(rho, u, T) - F_i(rho, u, T)/2 (the auxiliary distribution of the
 * second-order scheme, Sec. 2) at the slots the next pull reads, so that
 * lbm_moments right after lbm_init returns the given fields (exactly up to
 * round-off for periodic and bounce-back boundaries).  rho: N, u: D*N,
 * T: N, doubles, host or device (page-locked host arrays are read in place
 * by the kernel; with any host array the call returns after the state is
 * written, so the arrays may be reused at once).  For LBM_FP16_SCALED this
 * also fixes the grid's scale.  Resets the step counter. */
int lbm_init(lbm_ctx *ctx, const double *rho, const double *u, const double *T);

/* Marks solid sites: walls of any shape as a staircase of sites (the
 * curved walls of the paper's concentric-cylinder test, Sec. 3.2; the paper
 * leaves the wall rule unpublished, so this is the library's own).  solid: N
 * bytes, non-zero = solid; T_wall: N doubles, the wall temperature of each
 * solid site (> 0; ignored at fluid sites); host memory, copied.  A fluid
 * site x whose pull source y = x - e_i is solid receives the diffuse-wall
 * population rho_w(x) f0_i(1, 0, T_y); rho_w(x) makes the mass the walls emit
 * into x equal the mass x sends into solid sites in the same step, so every
 * fluid site keeps its mass.  Solid sites are not stepped and report zeros
 * from lbm_moments and lbm_get_populations; lbm_conserved sums fluid sites.
 * Requires all axes periodic, FP64 or FP32-shifted storage and the plain
 * step kernel (batches reject such contexts), and must precede lbm_init
 * (LBM_ESTATE after it).  Not stored by lbm_save: set it again before
 * lbm_load. */
int lbm_set_solid(lbm_ctx *ctx, const unsigned char *solid, const double *T_wall);

/* Advances n >= 0 steps of Eq. lbm (Sec. 2): per step and site, the pull
 * f~_i(x) = f*_i(x - e_i), the moments of Eq. rut1, the mid-point state
 * rho, u + g/2, theta, the equilibrium (Eq. fN with the Maxwellian
 * coefficients) and the force of Eq. fi, and the relaxation
 * f*_i = f~_i - (f~_i - f0_i)/tau + (1 - 1/(2 tau)) F_i -- one fused launch
 * per step, or graph replays.  Asynchronous on the context's stream.
 * LBM_EINVAL for n < 0, LBM_ESTATE before lbm_init or on a batch member. */
int lbm_step(lbm_ctx *ctx, int n);

/* Physical mid-point moments of the current state, in double: rho (N),
 * u (D*N) = sum f~ xi / rho + g/2, T (N) = theta, and the heat flux q (D*N),
 * q = 1/2 (1 - 1/(2 tau)) sum_i (f~_i - f0_i + F_i/2) |xi_i - u|^2 (xi_i - u)
 * (the physical non-equilibrium part, Sec. 2).  Any output may be NULL.
 * Host or device pointers; page-locked host outputs are written in place by
 * the kernel over the host link (no staging copy), pageable ones through a
 * device buffer.  Synchronises the stream. */
int lbm_moments(lbm_ctx *ctx, double *rho, double *u, double *T, double *q);

/* lbm_moments without synchronising: the same fields (Sec. 2), enqueued on
 * the context's stream and written when the stream reaches them.  Outputs
 * must be device memory or page-locked host memory (LBM_EINVAL otherwise);
 * the caller waits for the stream (or an event recorded after this call)
 * before reading them.  Lets a caller overlap the readout with other work,
 * e.g. the next steps of a batch this context has left. */
int lbm_moments_async(lbm_ctx *ctx, double *rho, double *u, double *T, double *q);

/* Changes the collision divisor tau (tau-hat of Eq. lbm, > 1/2) and the
 * uniform body-force acceleration g (Eq. BGK; NULL = no force) of a context
 * created with a uniform or no force, for the steps that follow.  The
 * buffers stay: a caller that serves many simulations of one grid size can
 * re-use a context (lbm_set_params, then lbm_init) without any device
 * allocation.  LBM_EINVAL for tau <= 1/2 or a non-uniform force. */
int lbm_set_params(lbm_ctx *ctx, double tau, const lbm_gfield *g);

/* Global sums over the grid (deterministic for a fixed grid) of the
 * conserved moments of Eq. rut (discrete form Eq. rut1): mass = sum rho,
 * mom[D] = sum rho u, energy = sum rho (|u|^2 + D theta)/2, all physical
 * mid-point values (with a force, Eq. lbm changes the momentum by sum rho g
 * and the energy by sum rho g.u per step, Sec. 2).  Per-site moments and the compensated
 * (two-sum) per-thread, block and grid merges run in the storage's
 * arithmetic precision (double for LBM_FP64, float pairs otherwise, about
 * 48 bits), in a fixed order; the totals are combined in double.  Any output
 * may be NULL (host pointers).
 * Returns LBM_EUNSTABLE if any site has a non-finite moment, rho <= 0 or
 * theta <= 0 (the sums are still written).  Synchronises the stream. */
int lbm_conserved(lbm_ctx *ctx, double *mass, double *mom, double *energy);

/* The pulled (pre-collision) distribution f~ of the current state, decoded to
 * double: out[i*N + site], Q*N values, library direction order. */
int lbm_get_populations(lbm_ctx *ctx, double *out);

/* The stored post-collision state f* decoded to double (Q*N), and its inverse
 * (values are rounded to the storage precision).  With lbm_step(ctx, 1) these
 * give one step of the method from an arbitrary state. */
int lbm_get_state(lbm_ctx *ctx, double *out);
int lbm_set_state(lbm_ctx *ctx, const double *in);

/* Step kernel in use: LBM_KERNEL_PLAIN, LBM_KERNEL_TMA or LBM_KERNEL_PREFETCH. */
int lbm_step_kernel(const lbm_ctx *ctx);

/* Steps taken since lbm_init / lbm_load. */
long long lbm_step_count(const lbm_ctx *ctx);

/* Scale s of the LBM_FP16_SCALED codec (0 for the other codecs). */
double lbm_fp16_scale(const lbm_ctx *ctx);

/* Checkpoint: writes / reads the raw population buffer, the codec scale, the
 * step counter and the grid description.  lbm_load requires a context created
 * with the same lattice, grid and precision; the continuation after a load is
 * bitwise identical to the uninterrupted run. */
int lbm_save(lbm_ctx *ctx, const char *path);
int lbm_load(lbm_ctx *ctx, const char *path);

/* Device bytes held by a context. */
size_t lbm_device_bytes(const lbm_ctx *ctx);

/* Message of the last error on ctx (or, when ctx is NULL, of the last failed
 * call made without a context: lbm_create, lbm_conserved_static).  Never NULL. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Frees all device memory of the context (the populations of Eq. lbm, the
 * force table and the reduction scratch allocated by lbm_create) and the
 * context itself, after the context's stream has drained; a batch member is
 * removed from its batch first.  NULL is a no-op.  Never fails. */
void lbm_destroy(lbm_ctx *ctx);

/* ---- Batches: many grids, one launch per step. ----
 *
 * Not in the paper (whose runs are single grids): independent simulations of
 * differing sizes and parameters are stepped together by one kernel whose
 * blocks stride over the tiles of all member grids, so small grids
 * share the GPU instead of each paying a full launch.  Every site goes
 * through the same device code as lbm_step, so a grid's state after n batch
 * steps is bit-identical to n lbm_step calls on it alone.
 *
 * Members must be initialised contexts of the batch's lattice, precision
 * (FP32-shifted or FP16-scaled) and force order, created with the batch's
 * stream and on its device; a context belongs to at most one batch, and
 * lbm_step on a member returns LBM_ESTATE (lbm_moments, lbm_conserved,
 * lbm_get_* and lbm_init still work; they are ordered on the shared stream).
 * lbm_destroy on a member removes it from its batch first. */
typedef struct lbm_batch lbm_batch;

/* capacity: maximum number of members (device table size). */
int lbm_batch_create(lbm_lattice lat, int precision, int force_order, void *stream, int capacity,
                     lbm_batch **out);
int lbm_batch_add(lbm_batch *b, lbm_ctx *ctx);
int lbm_batch_remove(lbm_batch *b, lbm_ctx *ctx);
int lbm_batch_size(const lbm_batch *b);

/* Launch configuration: threads per block along x (multiple of 32, <= 256),
 * sites per thread (1 or 2; a tile is block_x * sites_per_thread sites of
 * one row), and graph_steps > 0 (even) to replay a captured CUDA graph of
 * that many launches.  Defaults: 128, 1, 0. */
int lbm_batch_set_config(lbm_batch *b, int block_x, int sites_per_thread, int graph_steps);
int lbm_batch_get_config(const lbm_batch *b, int *block_x, int *sites_per_thread, int *graph_steps);

/* Advances every member by n steps (asynchronous on the batch's stream). */
int lbm_batch_step(lbm_batch *b, int n);

/* Halo staging (FP32-shifted batches, sites_per_thread 1): staged = 1 steps
 * the batch with a kernel that, while it collides one tile of sites, copies
 * the populations its threads pull for their next tile into shared memory
 * with cp.async (two stages of Q x block_x floats; warps whose pulls wrap
 * around x or reach a wall load directly).  The results are bit-identical
 * to the plain batch kernel.  Returns LBM_EINVAL for FP16-scaled storage or
 * sites_per_thread 2 (and lbm_batch_set_config rejects sites_per_thread 2
 * while staging is on).  Default 0. */
int lbm_batch_set_staging(lbm_batch *b, int staged);
int lbm_batch_get_staging(const lbm_batch *b, int *staged);

/* Autotuner: times trial_steps (even) batch steps for each block width in
 * {64, 128, 256} with 1 or 2 sites per thread and, for FP32-shifted storage,
 * with halo staging (one site per thread), keeps the fastest, and caches the
 * choice per (lattice, precision, force order, member grid shapes) for the
 * process.  The trials are real steps: every member advances by
 * 9 * (trial_steps + 2) steps (FP32-shifted) or 6 * (trial_steps + 2) steps
 * (FP16-scaled) when the timing runs (0 on a cache hit).  The chosen block
 * width and sites per thread are returned (may be NULL); the staging choice
 * is read with lbm_batch_get_staging.  graph_steps is kept. */
int lbm_batch_tune(lbm_batch *b, int trial_steps, int *block_x, int *sites_per_thread);

const char *lbm_batch_last_error(const lbm_batch *b);
void lbm_batch_destroy(lbm_batch *b);

/* ---- Slabs: one grid split along its last axis. ----
 *
 * Eq. lbm is local (Sec. 2): a step at site x reads f*_i(x - e_i) with
 * |e_ia| <= 3, so a grid cut into slabs of its last axis (y on D2Q37, z on
 * D3Q39) steps each slab on its own once the three layers beyond each cut
 * are known.  A slab context holds global layers [a_begin, a_end) of that
 * axis plus three ghost layers on each side that is not a wall (a periodic
 * axis wraps: the first slab's lower neighbour is the last slab).  Per step:
 * lbm_step on every slab, then one halo exchange per cut, which copies into
 * each neighbour's ghost layers the planes its sites pull (populations
 * pointing across the cut, up to three layers deep).  The slabs then
 * reproduce the undivided grid bit for bit (same kernels, same inputs).
 *
 * lbm_create_slab: nx, ny, nz, tau, g and opt as for lbm_create on the
 *   whole grid; 0 <= a_begin < a_end <= n_axis, at least 3 layers.  Caller
 *   arrays of lbm_init, lbm_moments, lbm_get_populations, lbm_get_state and
 *   lbm_set_state, and an LBM_G_FIELD force, cover the slab's own layers only
 *   (N_slab = nx * (a_end - a_begin) sites on D2Q37, nx * ny * (a_end -
 *   a_begin) on D3Q39, same layouts); lbm_conserved sums the slab's own
 *   sites.  Plain step kernel, graph_steps = 0 (a step is followed by an
 *   exchange), no solid sites, no batches.  After lbm_init no exchange is
 *   needed before the first step (the init writes every slot the slab's
 *   sites pull); after lbm_set_state or lbm_load of a single slab, exchange
 *   before stepping.  LBM_EINVAL on a bad range or option.
 * lbm_slab_exchange: both directions of the cut between lo and hi (hi holds
 *   the layers after lo's, or lo ends the axis and hi starts it on a
 *   periodic axis); same device, issued on lo's stream (order the two
 *   slabs' steps before it, e.g. one stream for all slabs).  FP16 slabs must
 *   share one scale (lbm_set_fp16_scale).
 * lbm_slab_halo_pack / unpack: the same exchange through a message, for
 *   slabs on different devices or processes (the caller moves the message,
 *   e.g. with NCCL send / recv): pack side 1 writes the message for the
 *   neighbour above, side 0 for the one below; unpack side 0 reads the
 *   message from the neighbour below, side 1 from above.  The message is
 *   lbm_slab_halo_bytes(ctx) bytes of device memory (same on both sides of a
 *   cut); asynchronous on the slab's stream.  LBM_EINVAL when the side is a
 *   wall.
 * lbm_slab_info: the slab's range and ghost layers (a whole-grid context
 *   reports [0, n_axis) and no ghosts). */
int lbm_create_slab(lbm_lattice lat, int nx, int ny, int nz, int a_begin, int a_end, double tau,
                    const lbm_gfield *g, const lbm_options *opt, lbm_ctx **out);
int lbm_slab_exchange(lbm_ctx *lo, lbm_ctx *hi);
size_t lbm_slab_halo_bytes(const lbm_ctx *ctx);
int lbm_slab_halo_pack(lbm_ctx *ctx, int side, void *dst);
int lbm_slab_halo_unpack(lbm_ctx *ctx, int side, const void *src);
int lbm_slab_info(const lbm_ctx *ctx, int *a_begin, int *a_end, int *ghosts_below, int *ghosts_above);

/* Sets the FP16 scale s of an initialised LBM_FP16_SCALED context to a power
 * of two, rescaling the stored half values exactly (a power-of-two factor
 * only shifts their exponents; values that leave the normal half range are
 * rounded).  Used to give FP16 slabs of one grid the scale the undivided
 * grid would choose (the smallest of their own).  LBM_EINVAL for another
 * codec or a scale that is not a power of two. */
int lbm_set_fp16_scale(lbm_ctx *ctx, double scale);

/* ---- Allocation-free conservation sums (no counterpart in the paper). ----
 *
 * For callers that must not allocate device memory: a plugin inside an
 * application that owns every device byte through its own pool, a runtime
 * whose memory budget is reserved up front, or a latency-sensitive loop that
 * cannot afford cudaMalloc / cudaFree (they synchronise the whole device).
 * Such callers cannot create an lbm_ctx, so this call takes the raw state and
 * computes what lbm_conserved computes, with the same kernels and order.
 *
 *   f    device pointer to a post-collision population buffer in the
 *        library's layout (Q*N values f[i*N + site], library direction
 *        order) and storage format: double f_i (LBM_FP64), float f_i - w_i
 *        (LBM_FP32_SHIFTED) or half s (f_i - w_i) / w_i (LBM_FP16_SCALED,
 *        s = fp16_scale, ignored otherwise);
 *   opt  precision, bc, T_lo / T_hi and stream are used (NULL: defaults);
 *   g    NULL, LBM_G_UNIFORM, or LBM_G_FIELD with a DEVICE pointer of D*N
 *        doubles (LBM_G_SINE is rejected: pass it as a field);
 *   out  device pointer to 6 doubles: mass, momentum[3], energy, and the
 *        number of sites with a non-finite moment, rho <= 0 or T <= 0.
 *
 * Solid sites (lbm_set_solid) are not supported: every site is summed as
 * fluid and pulled with the plain rule, so on a state from a context with
 * solid sites the sums differ from lbm_conserved.
 *
 * f, out and a field force must be device (or managed) memory of the
 * current device; host addresses and memory of another GPU are rejected with
 * LBM_EINVAL before any launch.
 *
 * Nothing is allocated: the per-block partial sums live in a static device
 * array of LBM_STATIC_MAX_TILES row tiles (128 sites along x each; 3.0 MB
 * held by every GPU that loads the library until the process exits).  Grids
 * needing more tiles, ceil(nx/128)*ny*nz > LBM_STATIC_MAX_TILES, are rejected
 * with LBM_EINVAL.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  All calls on a device share the one
 * array: calls that overlap on the GPU (different streams, no ordering) race
 * and give wrong sums.  Every partial a call reads is written by that call
 * first, so nothing has to be cleared between calls.  Asynchronous on
 * opt->stream; errors are described by lbm_last_error(NULL). */
#define LBM_STATIC_MAX_TILES 32768
int lbm_conserved_static(lbm_lattice lat, int nx, int ny, int nz, const lbm_options *opt,
                         const lbm_gfield *g, double fp16_scale, const void *f, double *out);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
