/*
 * lcs.h -- C ABI of the GB300 particle library (liblcs.so).
 *
 * The library advances inertial point particles through a frozen periodic
 * Eulerian velocity field and keeps them grouped by the virtual subdomain
 * that contains them, following Tominaga & Onishi, "LCS.jl" (arXiv
 * 2604.11008):
 *   - particle equations of motion, Sec. 2.2, Eqs. (5)-(6), with the drag
 *     factor f = 1 (Stokes drag) and an optional constant gravity g;
 *   - fluid velocity at the particle by trilinear interpolation from the
 *     eight surrounding cell-centre values, Sec. 2.2;
 *   - two-stage second-order Runge-Kutta time integration, Sec. 2.2 (Heun);
 *   - periodic cube of side L with grid spacing L/N, Sec. 2.1;
 *   - 3-D domain decomposition, Sec. 2.1, with particle migration by
 *     mask computation -> prefix scan -> parallel pack, Sec. 2.3.3, and
 *     unpack with compaction, Sec. 3.2.2.
 * The P = Px*Py*Pz subdomains are virtual: they are segments of one array
 * in one GPU's memory, and "communication" is a device-memory scatter.
 *
 * Conventions
 *   - All pointers marked "device" must be CUDA device pointers of the
 *     current device; "host" means ordinary host memory; "any" accepts both
 *     (copied with cudaMemcpyDefault).
 *   - Vectors are structure-of-arrays: a [3][n] double array holds all x
 *     components, then all y, then all z.
 *   - The field is [3][N][N][N] doubles, cell (i, j, k) of component c at
 *     c*N^3 + i + N*(j + N*k) (x fastest); its value belongs to the cell
 *     centre ((i+1/2)dx, (j+1/2)dx, (k+1/2)dx), dx = L/N.
 *   - Particle i of a subdomain p = (px, py, pz) has its containing cell
 *     c_s = min(floor(x_s * N/L), N-1) in [px*N/Px, (px+1)*N/Px) etc., and
 *     p is numbered px + Px*(py + Py*pz).
 *   - The library keeps positions in fixed point in cell units (52 fraction
 *     bits: the FP64 product x_s * N/L given to lcs_init / lcs_set_state is
 *     held exactly, and its integer part is the cell above) and velocities as
 *     float pairs (48 significant bits).  lcs_get_state returns them rounded
 *     to FP64: a position read back is within one unit in the last place of
 *     the value set, and the cell of a position read back can differ from
 *     the library's only when it lies within that rounding of a cell face.
 *   - Every call returns an lcs_status; nothing is thrown across the ABI.
 *     Errors detected inside kernels are latched in a device status word
 *     and reported by the next synchronising call (lcs_sync, lcs_get_state,
 *     lcs_backward); once an error is latched the context answers
 *     LCS_ERR_STATE to every call except lcs_last_error and lcs_destroy.
 *     A call on a live context that refuses its arguments (LCS_ERR_ARG)
 *     does nothing and latches nothing; the context stays usable.
 *   - A context is not thread safe; all its work is ordered on the stream
 *     given to lcs_init.
 */
#ifndef LCS_H_
#define LCS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lcs_ctx lcs_ctx;

typedef enum {
  LCS_OK = 0,
  LCS_ERR_ARG = 1,          /* invalid argument (message in lcs_last_error) */
  LCS_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  LCS_ERR_OOM = 3,          /* device allocation failed */
  LCS_ERR_CAPACITY = 4,     /* a subdomain segment outgrew its capacity */
  LCS_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
  LCS_ERR_NONFINITE = 6,    /* a particle position or velocity became NaN/Inf */
  LCS_ERR_DISPLACEMENT = 7, /* a particle moved by >= L/2, or beyond a neighbouring subdomain, in one step */
  LCS_ERR_STATE = 8         /* the context holds an earlier error */
} lcs_status;

typedef enum {
  LCS_F64 = 0,   /* field kept in FP64 (see field_kernel) */
  LCS_F32 = 1,   /* field rounded to FP32 (nearest even); FP32 interpolation */
  LCS_BF16 = 2   /* field rounded to BF16 (nearest even); FP32 interpolation */
} lcs_dtype;

typedef enum {
  LCS_KERNEL_AUTO = 0,   /* library choice: LCS_KERNEL_DF for LCS_F64 */
  LCS_KERNEL_FP64 = 1,   /* FP64 field, all arithmetic in FP64 */
  LCS_KERNEL_DF = 2      /* FP64 field stored as an unevaluated float pair
                            (hi + lo, 48 significant bits); interpolation and
                            the Heun increments in float-float arithmetic
                            (error-free FP32 transformations), added exactly
                            to the fixed-point positions and in float-float to
                            the velocity pairs: no FP64 instruction on the
                            Stokes path */
} lcs_kernel;

typedef enum {
  LCS_DRAG_STOKES = 0,   /* f = 1 in Eq. (6) */
  LCS_DRAG_NONLINEAR = 1 /* f = 1 + 0.15 Re_p^0.687, Re_p = 2 r |V - U| / nu, with the
                            radius r from tau_p = (2/9)(rho_p/rho) r^2 / nu (Sec. 2.2,
                            Eq. 7); forward only (no lcs_backward) */
} lcs_drag;

/* One ensemble: a field, its particles and its parameters. */
typedef struct {
  int n;                  /* grid points per axis N (the grid is N^3), 2 <= N <= 1024
                             (the fixed-point positions hold N 2^52 < 2^63) */
  double box;             /* side L of the periodic cube (> 0) */
  int sub[3];             /* virtual subdomains (Px, Py, Pz); N % P_s == 0 */
  int64_t np;             /* number of particles, 0 <= np < 2^31 */
  lcs_dtype field_dtype;  /* storage precision of the library's field copy */
  lcs_kernel field_kernel;/* arithmetic of the step for LCS_F64 */
  const double *field;    /* device [3][N][N][N]; read during lcs_init only */
  const double *x0;       /* device [3][np] finite positions; values outside
                             [0, L) are folded into the box (see lcs_init) */
  const double *v0;       /* device [3][np] velocities */
  const double *tau;      /* device [np] relaxation times tau_p > 0, or NULL */
  double tau_const;       /* tau_p of every particle when tau == NULL */
  const uint32_t *ids;    /* device [np] particle ids, or NULL for 0..np-1 */
  double dt;              /* time step, 0 < dt <= tau_p for every particle */
  double g[3];            /* constant acceleration added to dV/dt (gravity) */
  int sort_every;         /* cell sort after every k-th step (0: never) */
  int sort_brick;         /* brick edge B of the cell order (0: 8; 1: x-fastest) */
  int track_images;       /* 1: keep per-axis periodic image counts */
  int ckpt_every;         /* > 0: tape checkpoints every k steps for lcs_backward */
  lcs_drag drag;          /* drag law (LCS_DRAG_STOKES when zero-initialised) */
  double nu;              /* kinematic viscosity, > 0 (LCS_DRAG_NONLINEAR only) */
  double density_ratio;   /* rho_p / rho, > 0; 0 selects 843 (water, Sec. 2.2) */
  /* Evolving field: with field_next != NULL the fluid velocity is linear in
   * time between `field` (time t_field[0]) and field_next (time t_field[1]):
   * U(X, t) = (1 - th) U_0(X) + th U_1(X), th = (t - t_field[0]) /
   * (t_field[1] - t_field[0]); step n (from 0) starts at t = t_start + n dt
   * and its Heun stages see t and t + dt.  lcs_set_field pushes the next
   * snapshot.  NULL: the frozen field.  Forward only (no lcs_backward). */
  const double *field_next; /* device [3][N][N][N] or NULL; read during the call only */
  double t_start;         /* time of the initial state */
  double t_field[2];      /* times of field and field_next, t_field[1] > t_field[0] */
  /* 1: migrate after each Runge-Kutta stage, as the paper does (Sec. 3.2.2):
   * after the predictor X* (folded into the box) and again after X'; the
   * stage velocity V* travels with the particle.  Trajectories equal those of
   * the default single migration after the step up to rounding; only the
   * storage order differs.  All ensembles of a context must agree.  Not with
   * ckpt_every (the deferred-scatter step kernel with 256 threads only). */
  int migrate_per_stage;
  /* 1: owned-field mode, the memory pattern of the multi-GPU decomposition
   * (Sec. 2.1, 2.3): every subdomain interpolates only from its own copy of
   * the field cells it owns plus a halo of two cells per side (its brick,
   * (N/P_s + 4) cells per axis, built from the field at lcs_init).  A
   * stencil outside the brick -- a particle moved more than one cell beyond
   * its subdomain within a stage -- is reported as LCS_ERR_DISPLACEMENT.
   * Results equal those of the shared field bit for bit otherwise.  With
   * field_next the second snapshot has bricks too (rebuilt by
   * lcs_set_field).  All ensembles of a context must agree.  Not with
   * LCS_KERNEL_FP64 or ckpt_every; the step kernel is then mode
   * LCS_STEP_OWNED_FIELD.  0: every subdomain reads the one field copy. */
  int owned_field;
} lcs_desc;

/* Create a context for n_ens ensembles (1 <= n_ens <= 1024, all with the same
 * field_dtype and field_kernel) working on `stream`
 * (a cudaStream_t, may be NULL for the legacy default stream).  Copies the
 * particles into library-owned device memory, converts the field into the
 * library's layout and precision, and places every particle in the segment
 * of its subdomain: the particles of a subdomain keep the order in which
 * they were given (a stable partition by subdomain).  A position outside
 * [0, L) is folded into the periodic box (Sec. 2.1): x - k L with
 * k = floor(x / L), one rounding, moved by one more image if that rounding
 * lands on L or below 0; with track_images, k starts the particle's image
 * count, so unwrapped positions read back (lcs_get_state_by_id) continue
 * from the positions given.  Validates 2 <= N <= 1024, 0 <= np < 2^31,
 * N % P_s == 0, P <= 4096, tau_p >= dt, finite positions no more than 2^30
 * boxes away (LCS_ERR_ARG otherwise).  On success *out owns all device
 * memory until lcs_destroy. */
lcs_status lcs_init(const lcs_desc *ens, int n_ens, void *stream, lcs_ctx **out);

/* Enqueue nsteps time steps (asynchronous).  One step of every ensemble:
 * interpolate, integrate (Heun) and wrap every particle, flag it by
 * destination subdomain, and migrate (prefix scan, pack, unpack); after
 * steps whose 1-based count is a multiple of sort_every, sort every
 * subdomain's particles stably by cell.  A step is one persistent
 * step-kernel launch per group of ensembles that share a step configuration
 * (their tiles share one work counter), then one tail kernel for all
 * ensembles; twice that with migration per stage.
 * Runs of consecutive steps are recorded as CUDA graphs and replayed: with a
 * step period Q (the least common multiple of the ensembles' sort_every and
 * ckpt_every, stretched to at least 8, at most 64) a run ends at the next
 * multiple of Q, at a checkpoint step or at the end of the call, so a call
 * of n steps costs about n / Q graph launches (one per sort period); with
 * no such period, one graph launch per step.  The first run of each kind is
 * recorded when it is first needed.
 * Under LCS_STEP_DEFERRED and LCS_STEP_OWNED_FIELD the sort after a step
 * computes only the permutation: the next step kernel reads its records
 * through it, so the sorted records are written once, by that step.  A
 * permutation still pending when another call needs the records in sorted
 * order is read through (lcs_get_state) or applied then (lcs_get_state_by_id,
 * lcs_migrate, lcs_pair_histogram, a checkpoint); none of this is visible in
 * any result. */
lcs_status lcs_step(lcs_ctx *ctx, int64_t nsteps);

/* Standalone migration pass on the current state (asynchronous): a stable
 * partition by destination subdomain -- each subdomain keeps its own
 * particles in order, then receives the others in order of their source
 * subdomain and, within one source, in storage order (Sec. 2.3.3 / 3.2.2).
 * Works for any destinations, not only neighbours. */
lcs_status lcs_migrate(lcs_ctx *ctx);

/* Standalone cell sort (asynchronous): stable sort of every subdomain's
 * segment by cell key.  The key orders the cells of a subdomain brick by
 * brick (B^3 bricks, brick-major x-fastest, x-fastest inside a brick). */
lcs_status lcs_sort(lcs_ctx *ctx);

/* Replace the particles of ensemble `ens` (np unchanged).  Pointers are
 * "any"; x and v are [3][np]; tau ([np]) is required when the context was
 * created with per-particle tau_p and ignored otherwise; img ([3][np]
 * int32) may be NULL (zeros).  seg (host, Ptot+1 int64) gives
 * the segments; particles need not lie in their segment's subdomain until
 * the next lcs_migrate.  Positions outside [0, L) are folded as in lcs_init,
 * the folds added to img.  Synchronising. */
lcs_status lcs_set_state(lcs_ctx *ctx, int ens, const double *x, const double *v,
                         const double *tau, const uint32_t *ids, const int32_t *img,
                         const int64_t *seg);

/* Copy the current particles of ensemble `ens` in storage order (segments
 * contiguous, subdomain 0 first).  Pointers are "any" and may be NULL to
 * skip an array; seg (Ptot+1 int64) receives the segment bounds.
 * Synchronising; returns the latched device status. */
lcs_status lcs_get_state(lcs_ctx *ctx, int ens, double *x, double *v, double *tau,
                         uint32_t *ids, int32_t *img, int64_t *seg);

/* Copy the current particles of ensemble `ens` ordered by particle id
 * (ascending; equal ids keep their storage order).  Pointers are "any" and
 * may be NULL to skip an array: x and v are [3][np], ids [np] receives the
 * ids in that order.  With track_images the positions are unwrapped,
 * RN(x + RN(L img)) with img the periodic images crossed since the
 * positions were given (lcs_init / lcs_set_state, including the folds of
 * positions given outside the box); without, they are the positions in
 * [0, L) that lcs_get_state returns.  This is the final state X_T, V_T of
 * the problem statement (Sec. 2.2) in the order the particles were given
 * (ids NULL at lcs_init numbers them 0..np-1).  Synchronising; returns the
 * latched device status. */
lcs_status lcs_get_state_by_id(lcs_ctx *ctx, int ens, double *x, double *v, uint32_t *ids);

/* Copy the field as the kernels of ensemble `ens` see it (after rounding to
 * the storage precision), expanded to FP64 [3][N][N][N] ("any" pointer).
 * Synchronising. */
lcs_status lcs_get_field(lcs_ctx *ctx, int ens, double *out);

/* Particle statistics: counts[b] (host, nbins <= 4096) = number of unordered
 * pairs of particles of ensemble `ens` whose separation r (minimum image in
 * the periodic box, positions as lcs_get_state returns them,
 * r = sqrt((dx dx + dy dy) + dz dz) in FP64) is below r_max, with
 * b = min(floor(r * (nbins / r_max)), nbins - 1): the counts behind the
 * radial distribution function g(r) (particle-phase validation of Sec. 3),
 * g_b = counts[b] / (np (np - 1) / 2 * shell volume_b / L^3).  Requires N >= 3
 * and 0 < r_max <= L/N (pairs then lie in neighbouring cells).  Scratch is
 * allocated with cudaMallocAsync on the context's stream.  Synchronising. */
lcs_status lcs_pair_histogram(lcs_ctx *ctx, int ens, double r_max, int nbins, int64_t *counts);

/* The radial distribution function of ensemble `ens` from the same counts:
 * g[b] (host, nbins doubles) = counts[b] / (np (np - 1) / 2 * V_b / L^3),
 * V_b = (4/3) pi (r_{b+1}^3 - r_b^3) with r_b = b r_max / nbins, and r[b]
 * (host, may be NULL) the bin centres (r_b + r_{b+1}) / 2; g[b] = 0 where
 * the expected count is 0 (np < 2).  counts (host, may be NULL) receives the
 * counts.  Same requirements as lcs_pair_histogram.  Synchronising. */
lcs_status lcs_pair_rdf(lcs_ctx *ctx, int ens, double r_max, int nbins, double *r, double *g,
                        int64_t *counts);

/* Evolving field: the second snapshot of ensemble `ens` becomes the first,
 * `field` (device [3][N][N][N] FP64, read during the call) at time t becomes
 * the second (t must exceed the current second snapshot's time); the step
 * graphs are rebuilt.  LCS_ERR_ARG for an ensemble created with a frozen
 * field.  Synchronising. */
lcs_status lcs_set_field(lcs_ctx *ctx, int ens, const double *field, double t);

/* Gradients of a scalar loss of the final state of ensemble 0 with respect
 * to the field and the initial state, by the hand-written adjoint of the
 * Heun step (reverse of the recorded steps, recomputing every segment of
 * ckpt_every steps from its checkpoint).  Requires ckpt_every > 0 and
 * track_images = 1 at init.  gx, gv (device [3][np], in particle-id order)
 * hold dLoss/dX_T and dLoss/dV_T of the final unwrapped positions and
 * velocities; gU (device [3][N][N][N], accumulated into -- zero it first),
 * gx0 and gv0 (device [3][np], id order, overwritten) receive the
 * gradients.  The tape covers the steps since lcs_init.  Synchronising. */
lcs_status lcs_backward(lcs_ctx *ctx, const double *gx, const double *gv, double *gU,
                        double *gx0, double *gv0);

/* Kernel classes reported by lcs_profile_steps. */
enum {
  LCS_PROF_STEP = 0,    /* fused interpolate + integrate + scan + pack kernel */
  LCS_PROF_TAIL = 1,    /* step tail: unpack, next layout, buffer swap (one kernel) */
  LCS_PROF_SORT = 2,    /* the cell-sort kernels (keys, radix passes, and the
                           permutation of the records where no step kernel
                           reads through it) */
  LCS_PROF_N = 3
};

/* Tracing: enqueue nsteps steps like lcs_step but without the graph, with
 * a CUDA event pair around every kernel (class) on the context's stream.
 * Synchronising.  ms[k] (host, LCS_PROF_N doubles) receives the summed
 * device time of class k in milliseconds, count[k] (host, may be NULL) the
 * number of timed intervals (for LCS_PROF_STEP: step-kernel launches).  The particle state advances exactly as lcs_step. */
lcs_status lcs_profile_steps(lcs_ctx *ctx, int64_t nsteps, double *ms, int64_t *count);

/* Step-kernel modes (all give identical results):
 *   LCS_STEP_PLAIN          records and field read from global memory;
 *   LCS_STEP_STAGED_FIELD   each tile first copies the box of field cells
 *                           around its particles into shared memory (64 KB;
 *                           a tile whose box is larger reads global memory);
 *                           not available with LCS_KERNEL_FP64;
 *   LCS_STEP_PREFETCH       the records of a block's next tile are brought
 *                           into shared memory by bulk asynchronous copies
 *                           while the current tile is processed;
 *   LCS_STEP_DEFERRED       a block integrates its next tile before it
 *                           resolves the scan prefix of the previous one,
 *                           which waits parked in shared memory and is then
 *                           written out with coalesced stores;
 *   LCS_STEP_OWNED_FIELD    LCS_STEP_DEFERRED reading the subdomains' own
 *                           field bricks (owned_field contexts only, which
 *                           use no other mode). */
#define LCS_STEP_PLAIN 0
#define LCS_STEP_STAGED_FIELD 1
#define LCS_STEP_PREFETCH 2
#define LCS_STEP_DEFERRED 3
#define LCS_STEP_OWNED_FIELD 4

/* Number of step-kernel configurations lcs_tune tries. */
#define LCS_TUNE_CONFIGS 14

/* Autotuner: time every step-kernel configuration on steps_per_trial real
 * steps of all ensembles and keep, for every class of ensembles, the fastest
 * for that class; then rebuild the step graphs.  A class is the ensembles of
 * one grid size N whose particle counts lie in the same decade (10^k <= np <
 * 10^(k+1)).  During the trials every class runs in launches of its own, so
 * that each class's step kernel is timed alone; afterwards the ensembles
 * that share a configuration share launches (at most 42 ensembles per
 * launch), so a context runs one step-kernel launch per configuration in
 * use (and per 42 ensembles).  The configurations, in order, as (threads per block, particles per
 * thread, mode): (256,2,0) (256,1,0) (128,2,0) (256,2,1) (128,2,1)
 * (256,2,2) (128,2,2) (256,1,2) (256,2,3) (128,2,3) (256,1,3) (128,1,3)
 * (256,1,4) (256,2,4).  The first two numbers fix the scan tile.
 * Configurations of mode LCS_STEP_STAGED_FIELD are skipped for the all-FP64
 * kernel, every mode but LCS_STEP_DEFERRED for an evolving field or
 * migration per stage (then with 256 threads only), and every mode but
 * LCS_STEP_OWNED_FIELD for an owned_field context (and that mode for any
 * other).  The trial steps advance the simulation (steps_per_trial steps per
 * tried configuration, recorded like any other step); results do not depend
 * on the choice.  *block, *items, *mode (may be NULL) receive the choice
 * for the class of ensemble 0 (lcs_step_config_of reports any ensemble's);
 * trial_ms (host, LCS_TUNE_CONFIGS doubles, may be NULL) the step-kernel
 * milliseconds of each configuration in that order, summed over all
 * classes, -1 for one skipped.  Synchronising. */
lcs_status lcs_tune(lcs_ctx *ctx, int steps_per_trial, int *block, int *items, int *mode,
                    double *trial_ms);

/* Step-kernel configuration of ensemble `ens` (host outputs, may be NULL):
 * threads per block, particles per thread, mode. */
lcs_status lcs_step_config_of(lcs_ctx *ctx, int ens, int *block, int *items, int *mode);

/* Select one of the LCS_TUNE_CONFIGS step-kernel configurations by hand for
 * every ensemble (the values lcs_tune chooses among); the step graphs are
 * rebuilt.
 * Results do not depend on the choice.  LCS_ERR_ARG for a combination not
 * in the list or one that lcs_tune skips for this context (see there).
 * Synchronising. */
lcs_status lcs_set_step_config(lcs_ctx *ctx, int block, int items, int mode);

/* Number of step tiles, summed over the ensembles since lcs_init, whose
 * field cells were read from a shared-memory box (LCS_STEP_STAGED_FIELD
 * only; tiles whose box did not fit read global memory and are not
 * counted).  *count is host memory.  Synchronising. */
lcs_status lcs_staged_tiles(lcs_ctx *ctx, int64_t *count);

/* Wait for all enqueued work; return the latched device status. */
lcs_status lcs_sync(lcs_ctx *ctx);

/* Human-readable description of the last error of ctx (never NULL); with
 * ctx == NULL, the last error of this thread's most recent failed call,
 * e.g. the reason lcs_init refused its arguments. */
const char *lcs_last_error(lcs_ctx *ctx);

/* Release every resource of ctx (NULL is ignored). */
void lcs_destroy(lcs_ctx *ctx);

/* Number of kernel launches enqueued by ctx since lcs_init. */
int64_t lcs_launch_count(lcs_ctx *ctx);

/* Number of CUDA graph launches lcs_step has issued since lcs_init (one per
 * recorded run of steps, see lcs_step). */
int64_t lcs_graph_launch_count(lcs_ctx *ctx);

/* Stable partition of n keys into nbins bins -- a counting sort; the
 * paper's mask -> prefix scan -> parallel pack (Sec. 2.3.3) is the case
 * nbins = 2, where the rank of a mask-1 element within bin 1 is its
 * exclusive scan value.  perm[r] receives the index of the key placed at
 * rank r (bins ascending, equal keys in input order); bin_off (nbins+1)
 * receives the bin starts.  keys, perm, bin_off are device pointers;
 * 1 <= nbins <= 65536, 0 <= n < 2^31.  A key >= nbins is placed in bin
 * nbins-1 and, if status (device int32, may be NULL) is given, LCS_ERR_ARG
 * is written there (LCS_OK otherwise).  Scratch is allocated and freed with
 * cudaMallocAsync / cudaFreeAsync on `stream`.  Asynchronous. */
lcs_status lcs_partition(const uint32_t *keys, int64_t n, int nbins, uint32_t *perm,
                         int64_t *bin_off, int32_t *status, void *stream);

/* Largest n accepted by lcs_partition_noalloc. */
#define LCS_PARTITION_NOALLOC_MAX_N (1 << 20)

/* lcs_partition for callers that cannot allocate device memory where they
 * call it: code running while its stream is captured into a CUDA graph,
 * code under a fixed device-memory budget, or latency-critical loops that
 * cannot afford the synchronisation of cudaMalloc / cudaFree.  Same
 * arguments, results and asynchrony as lcs_partition, but no allocation of
 * any kind: the scratch is a file-scope device array of about 13.6 MB that
 * every GPU loading the library keeps until the process exits.
 * Limits: n <= LCS_PARTITION_NOALLOC_MAX_N (larger n returns LCS_ERR_ARG
 * before any work is enqueued), 1 <= nbins <= 65536.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it with the id of the device's current
 * context; a call in a different context (after cudaDeviceReset, say) looks
 * it up again.  Make the first call on a device, and the first call after
 * such a change, before any stream capture on that device.  All calls share the one array, so two
 * calls that may run at the same time on the GPU (different streams without
 * ordering, or different host threads) race and corrupt each other's
 * results; order them on one stream.  The paper has no counterpart of this
 * entry point: it is an interface variant of lcs_partition. */
lcs_status lcs_partition_noalloc(const uint32_t *keys, int64_t n, int nbins, uint32_t *perm,
                                 int64_t *bin_off, int32_t *status, void *stream);

/* Self-test of the bounded device-side waits (failure detection without a
 * GPU fault).  Runs, in one small kernel on `stream`, the two waits the step
 * kernels use against partners that never answer: the decoupled look-back
 * of a tile whose predecessor never publishes, and an mbarrier wait for
 * bulk copies that were never issued.  Both waits must give up after their
 * iteration limits (about a second at most) and report it; the kernel then
 * returns normally.  *lookback and *mbarrier (host) receive LCS_ERR_TIMEOUT
 * when the respective wait gave up as designed (LCS_OK if it had not).
 * Synchronising; LCS_ERR_ARG for NULL outputs, LCS_ERR_CUDA if the launch
 * failed.  No context is involved. */
lcs_status lcs_selftest_waits(void *stream, int32_t *lookback, int32_t *mbarrier);

#ifdef __cplusplus
}
#endif

#endif /* LCS_H_ */
