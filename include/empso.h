/*
 * empso.h - C ABI of the GB300 EMPSO fitness-evaluation library.
 *
 * Method: arXiv 1905.12795 ("Towards automatically building starting models
 * for FWI using global optimization methods: a PSO approach via DEAP +
 * Devito").  A particle is a small grid of velocity control nodes; it is
 * interpolated onto the finite-difference grid (two-grid strategy, section
 * "Testing approach"), every shot is forward-modelled with a 2nd-order-in-time,
 * 4th/8th-order-in-space acoustic FD scheme with a damping layer (JSON nbpml)
 * and a Ricker source, and the L2 misfit against the observed traces is the
 * particle's fitness.  An elitist-mutated PSO (section "Theory", Eq. 1-3 and
 * the EMPSO figure) then moves the swarm.
 *
 * Conventions shared by every entry point:
 *  - All device work is enqueued on the caller's `stream` (a cudaStream_t
 *    passed as void*; NULL = legacy default stream) and is stream-ordered;
 *    nothing synchronises the host unless stated.
 *  - Buffers marked "device" are caller-owned device memory; the library
 *    never frees or keeps them beyond the call.  Buffers marked "host" are
 *    read before the call returns.
 *  - The library owns only its context: per-grid tables, workspace (model
 *    fields, wavefield slots, partial misfits), swarm state and surrogate.
 *  - No C++ exception crosses this boundary; every call returns a status and
 *    leaves a message for empso_last_error().  On error nothing is enqueued
 *    unless the status is EMPSO_CUDA_ERROR.
 *  - One context serves one host thread at a time.
 *
 * Units: metres, seconds, hertz, metres per second.  Float arrays are
 * row-major with x fastest.
 */
#ifndef EMPSO_H
#define EMPSO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t empso_status;
#define EMPSO_OK              0
#define EMPSO_INVALID_ARG     1  /* a size, pointer, position or enum is out of range */
#define EMPSO_OOM             2  /* device or pinned allocation failed */
#define EMPSO_CUDA_ERROR      3  /* a CUDA call failed; the context may be unusable */
#define EMPSO_NONFINITE       4  /* a misfit was NaN/Inf (reported as +inf, strict mode only) */
#define EMPSO_TIMEOUT         5  /* a bounded device-side wait gave up */
#define EMPSO_UNSUPPORTED     6  /* e.g. space order not in {2,4,8}, swarm too large */
#define EMPSO_NOT_INITIALIZED 7  /* swarm or surrogate used before its init call */
#define EMPSO_IO_ERROR        8  /* checkpoint file unreadable, unwritable or invalid */

typedef struct empso_ctx empso_ctx;

/* One modelling grid ("Testing approach": FD grid, nbpml damping cells, space
 * order, record length, Ricker peak frequency).  Node (i, j) of the physical
 * nx x nz grid sits at (i hx, j hz); `pad` damping cells surround it on all
 * four sides.  dt <= 0 selects dt = T / (nt - 1) with
 * nt = ceil(T / (0.9 dt_cfl)) + 1, dt_cfl = 2 / (vmax sqrt(rho (1/hx^2 + 1/hz^2)))
 * and rho the extreme eigenvalue of the 1-D stencil.  Interpolated models are
 * clipped to [vmin, vmax]; vmax also sets the damping strength.  A particle on
 * this grid has kz x kx control nodes (index k = kz_i * kx + kx_i) spanning
 * the physical domain edge to edge, interpolated by a natural cubic spline
 * (interp_mode 0) or bilinearly (interp_mode 1, the paper's two-grid rule). */
typedef struct {
    int32_t nx, nz;
    int32_t pad;
    int32_t space_order;
    float hx, hz;
    float t_rec;
    float f0;
    float dt;
    float vmin, vmax;
    int32_t kx, kz;
    int32_t interp_mode;
} empso_grid;

/* One shot ("Testing approach": acquisition geometry).  Source at (sx, sz),
 * receivers rec_xz[rec_begin .. rec_begin + nrec) of the table given to
 * empso_create, all inside the physical domain.  `weight` scales this shot's
 * misfit in the particle's sum (1 for the paper's plain sum). */
typedef struct {
    float sx, sz;
    int32_t rec_begin;
    int32_t nrec;
    int32_t grid_id;
    float weight;
} empso_shot;

/* EMPSO parameters ("Theory": Eq. 1-3, EM figure; "Testing approach": NM,
 * p_em, start iteration, c1, c2; JSON lambda for the velocity clamp).
 * P particles of D dimensions; EM on the floor(nm_frac P) worst particles from
 * generation em_start (1-based) on when em_enabled; seed keys Philox4x32-10. */
typedef struct {
    int32_t P, D;
    double c1, c2, lambda, p_em, nm_frac;
    int32_t em_start, em_enabled;
    uint64_t seed;
} empso_pso;

/* Create a context.  grids: host [ngrids]; rec_xz: host [nrec_total][2]
 * receiver table (copied); pso: host, may be NULL when no swarm is needed;
 * xmin/xmax: host [pso->D] search box (ignored when pso is NULL).  On success
 * *out owns device tables and must be released with empso_destroy.
 * Errors: INVALID_ARG (bad sizes/positions), UNSUPPORTED (space order),
 * OOM, CUDA_ERROR. */
empso_status empso_create(const empso_grid *grids, int32_t ngrids,
                          const float *rec_xz, int32_t nrec_total,
                          const empso_pso *pso, const double *xmin,
                          const double *xmax, empso_ctx **out);

/* Release the context and everything it allocated (synchronises the device). */
void empso_destroy(empso_ctx *ctx);

/* Time axis chosen for a grid: dt (s) and number of steps/trace samples nt.
 * dt, nt: host, either may be NULL. */
empso_status empso_grid_info(const empso_ctx *ctx, int32_t grid_id, float *dt,
                             int32_t *nt);

/* The same without a context: validates `grid` (host) with the rules of
 * empso_create and returns the time axis it gets (CFL rule of the scheme in
 * "Testing approach" unless grid->dt > 0).  Host only, no device work.
 * dt, nt: host, either may be NULL.
 * Errors: INVALID_ARG (bad sizes/bounds or NULL grid), UNSUPPORTED (space order);
 * the message is in empso_last_error(NULL). */
empso_status empso_time_axis(const empso_grid *grid, float *dt, int32_t *nt);

/* Two-grid parameterisation ("Testing approach"): particles device [P][K]
 * (K = kz kx of the grid, m/s) -> vel_out device [P][nz][nx] (m/s), clipped
 * to [vmin, vmax].  Exposed for tests; eval_fitness does this internally. */
empso_status empso_interp(empso_ctx *ctx, int32_t grid_id, const float *particles,
                          int32_t P, float *vel_out, void *stream);

/* Forward-model M gridded models on every shot ("Testing approach": FD
 * modelling of each shot) and write the traces.  vel: device [M][nz][nx]
 * (m/s) of the one grid all shots use; shots: host [S]; traces: device, for
 * each model the concatenation over shots of [nt][nrec_s] float samples, so
 * model m starts at m * sum_s nt nrec_s.  Trace sample n is the wavefield at
 * t_{n+1} = (n + 1) dt, bilinearly sampled after step n; the source term of
 * step n is r(n dt). */
empso_status forward_traces(empso_ctx *ctx, const float *vel, int32_t M,
                            const empso_shot *shots, int32_t S, float *traces,
                            void *stream);

/* Misfit of M gridded models: misfit[m] = sum_s weight_s * phi_ms with
 * phi = 1/2 sum_n sum_r (d - d_obs)^2 ("Testing approach": l2 norm).
 * vel: device [M][nz][nx]; d_obs: device, concatenation over shots of
 * [nt][nrec_s]; misfit: device [M] doubles.  Non-finite misfits become +inf. */
empso_status eval_models(empso_ctx *ctx, const float *vel, int32_t M,
                         const empso_shot *shots, int32_t S, const float *d_obs,
                         double *misfit, void *stream);

/* Fitness of P particles (the method's fitness evaluation): each particle is
 * interpolated onto the grid of every shot, every (particle, shot) instance
 * is modelled in one persistent launch, and misfit[p] = sum_s weight_s phi_ps
 * is reduced in fixed shot order.  particles: device [P][K] (K of the shots'
 * grids, which must agree); shots: host [S] (grids may differ); d_obs:
 * device, concatenation over shots of [nt_g(s)][nrec_s]; misfit: device [P]. */
empso_status eval_fitness(empso_ctx *ctx, const float *particles, int32_t P,
                          const empso_shot *shots, int32_t S, const float *d_obs,
                          double *misfit, void *stream);

/* Initialise the swarm ("Theory": random positions, randomized velocities):
 * x ~ U(xmin, xmax), v ~ U(-vmax, vmax), vmax = lambda (xmax - xmin), pbest
 * fitness +inf, generation 0.  particles_out: device [P][D] floats (x), may be
 * NULL.  Errors: NOT_INITIALIZED if the context has no swarm. */
empso_status pso_init(empso_ctx *ctx, float *particles_out, void *stream);

/* One EMPSO generation given the fitness of the current positions ("Theory",
 * Eq. 1-3 and the EM figure): generation k += 1; strict personal-best update;
 * global best = lowest-index argmin; if EM is on and k >= em_start, the
 * floor(nm_frac P) worst particles of a stable ascending sort of the fitness
 * take g_d + 0.1 VR_d N(0,1) with probability p_em (else g_d) per coordinate,
 * velocities unchanged; all others follow Eq. 1 (constriction Eq. 3, clamp to
 * +-vmax) and Eq. 2; positions are clamped to the box.  misfit: device [P];
 * particles_out: device [P][D] floats, may be NULL; gbest_out: HOST int, may
 * be NULL - when given, the call synchronises the stream to fill it. */
empso_status pso_step(empso_ctx *ctx, const double *misfit, float *particles_out,
                      int32_t *gbest_out, void *stream);

/* Copy the swarm state into caller buffers (any may be NULL): x, v, p device
 * [P][D] doubles; pf device [P]; order device [P] ints (the last sort, or the
 * identity when EM did not run); gk device int[2] = {g, k}. */
empso_status pso_get_state(empso_ctx *ctx, double *x, double *v, double *p,
                           double *pf, int32_t *order, int32_t *gk, void *stream);

/* Overwrite the swarm state from caller device buffers (x, v, p [P][D], pf
 * [P]) with global-best index g and generation k (host values). */
empso_status pso_set_state(empso_ctx *ctx, const double *x, const double *v,
                           const double *p, const double *pf, int32_t g,
                           int32_t k, void *stream);

/* One whole EMPSO generation as a CUDA graph: fitness of the swarm's current
 * positions (as eval_fitness, on every shot) followed by pso_step.  The first
 * call for a given shot list, d_obs and misfit_out pointer (and kernel
 * settings) plans the launch - it may allocate workspace and synchronises
 * `stream` - and captures the work into a graph; later calls replay that
 * graph on `stream` with one launch.  d_obs: device, as for eval_fitness;
 * misfit_out: device [P] doubles receiving this generation's fitness, or
 * NULL.  The swarm dimension must equal the grids' control-node count.
 * The shots' host array is read at capture time only. */
empso_status empso_generation(empso_ctx *ctx, const empso_shot *shots, int32_t S,
                              const float *d_obs, double *misfit_out, void *stream);

/* Autotuner: times the streaming kernel, the on-chip kernel at every cluster
 * size and rows-per-thread shape the batch fits, and the L2 cluster kernel at
 * cluster sizes 4, 8, 10, 12 and 16 (one warm-up and one timed launch each,
 * CUDA events on `stream`) on this exact batch (particles device [P][K],
 * shots, d_obs; misfit device [P] is used as scratch output), and keeps the
 * fastest for every later batch with the same grids, shot counts and P.  With
 * a kernel kind selected (empso_set_kernel), only that kind's candidates are
 * timed.  The choice is returned in *kind_out / *cluster_out (host, may be
 * NULL) and appended to the tuning cache file (with its rows per thread) if
 * one is set.  Synchronises `stream`. */
empso_status empso_autotune(empso_ctx *ctx, const float *particles, int32_t P,
                            const empso_shot *shots, int32_t S, const float *d_obs,
                            double *misfit, int32_t *kind_out, int32_t *cluster_out,
                            void *stream);

/* Tuning cache: a JSON-lines file (one object per tuned batch: gpu, key,
 * kind, cluster, ms).  Entries of this GPU are loaded now and used for
 * matching batches; empso_autotune appends to it.  NULL or "" disables it. */
empso_status empso_set_tuning_cache(empso_ctx *ctx, const char *path);

/* pso_step with a separate key for the elitist-mutation sort: `rank` (device
 * [P], may be NULL = misfit) orders the particles for EM while `misfit` alone
 * drives the personal and global bests.  Used by surrogate pre-screening,
 * where particles that were not modelled carry misfit +inf and their
 * predicted misfit as rank key. */
empso_status pso_step_ranked(empso_ctx *ctx, const double *misfit, const double *rank,
                             float *particles_out, int32_t *gbest_out, void *stream);

/* ---- Surrogate pre-screening (not in the paper) ----------------------------
 * A K -> H -> H -> 1 ReLU perceptron (K = swarm dimension) predicts the log
 * misfit of a particle from its control nodes scaled to [-1, 1] with the
 * swarm's bounds.  Dense layers run on BF16 tensor cores with FP32
 * accumulation; master weights and Adam moments are FP32.  It is trained
 * online on a device replay buffer of (particle, log misfit) pairs,
 * standardised with the buffer's mean and deviation.  Parameters, flat FP32,
 * in the order W1 [H][K], b1 [H], W2 [H][H], b2 [H], w3 [H], b3 [1]. */

/* Create the network: hidden width H (multiple of 16, <= 1024), replay
 * capacity (pairs), Adam learning rate, seed of the weights and minibatches.
 * Needs a swarm.  Allocates; synchronises the device. */
empso_status surrogate_init(empso_ctx *ctx, int32_t hidden, int32_t capacity, float lr,
                            uint64_t seed);

/* Training in pre-screening generations of surrogate_generation: with
 * enable = 0 (default) the network trains after the generation's modelling
 * on the pairs of all generations so far; with enable = 1 it trains on the
 * pairs of the earlier generations on a second stream while the selected
 * particles are modelled (one generation of lag, shorter generations). */
empso_status surrogate_set_overlap(empso_ctx *ctx, int32_t enable);

/* Pre-screening policy (engineering choices of this library; the paper has
 * no surrogate): recent > 0 draws half of every training minibatch from the
 * newest `recent` pairs of the replay buffer (the swarm's current
 * neighbourhood), the other half from all of it (0: all uniform, the
 * default).  min_rank_corr > 0: after a pre-screened generation whose
 * predictions rank its modelled particles with a Spearman correlation below
 * min_rank_corr against their true misfits, the next surrogate_generation
 * models the whole swarm (true modelling stays the fallback; 0: never, the
 * default).  patience > 0: after that many pre-screened generations in a row
 * that did not lower the swarm's best misfit, the next surrogate_generation
 * models the whole swarm (0: never, the default); each call synchronises
 * `stream` once more to read the best misfit.  Errors: INVALID_ARG (recent <
 * 0, min_rank_corr outside [-1, 1], patience < 0), NOT_INITIALIZED. */
empso_status surrogate_set_policy(empso_ctx *ctx, int32_t recent, float min_rank_corr, int32_t patience);

/* Spearman correlation of the last pre-screened generation (predicted vs
 * true misfit of its modelled particles).  rho: host; synchronises `stream`. */
empso_status surrogate_last_rank_corr(empso_ctx *ctx, float *rho, void *stream);

/* Tensor-core path of this context's dense layers: 1 = tcgen05.mma with
 * the accumulator in tensor memory (default), 0 = mma.sync.  Both compute
 * BF16 products with FP32 accumulation. */
empso_status surrogate_set_backend(empso_ctx *ctx, int32_t kind);

/* Predicted log misfit: particles device [P][K] -> logphi device [P]. */
empso_status surrogate_predict(empso_ctx *ctx, const float *particles, int32_t P, float *logphi,
                               void *stream);

/* Append pairs to the replay buffer (ring): particles device [n][K], misfit
 * device [n]; pairs with a non-finite or non-positive misfit are skipped. */
empso_status surrogate_add(empso_ctx *ctx, const float *particles, const double *misfit,
                           int32_t n, void *stream);

/* `steps` Adam steps on minibatches of `batch` pairs drawn uniformly from the
 * buffer (Philox stream of the seed); refreshes the standardisation first. */
empso_status surrogate_train(empso_ctx *ctx, int32_t steps, int32_t batch, void *stream);

/* Read (get, device [n_params]) and/or overwrite (set) the FP32 parameters;
 * *n_params (host, may be NULL) receives their count. */
empso_status surrogate_params(empso_ctx *ctx, float *get, const float *set, int32_t *n_params,
                              void *stream);

/* Gradient of L = 1/(2n) sum (y - target)^2 on one batch, without updating:
 * particles device [n][K] (raw positions), target device [n] (standardised
 * units), grad device [n_params], loss device [1] (may be NULL). */
empso_status surrogate_grad(empso_ctx *ctx, const float *particles, const float *target,
                            int32_t n, float *grad, float *loss, void *stream);

/* One surrogate-assisted EMPSO generation.  While the replay buffer holds
 * fewer than `warm` pairs, every particle is modelled; afterwards only the
 * round(keep_frac P) particles with the smallest predicted misfit are
 * modelled (eval_fitness on them), their pairs join the buffer, the network
 * takes `train_steps` Adam steps of `batch`, and pso_step_ranked moves the
 * swarm with +inf fitness for the others and their predictions as EM keys.
 * misfit_out: device [P] (may be NULL) = the fitness used (+inf where not
 * modelled); *n_modelled (host, may be NULL) = particles modelled.
 * Synchronises `stream` once (to read the buffer count). */
empso_status surrogate_generation(empso_ctx *ctx, const empso_shot *shots, int32_t S,
                                  const float *d_obs, double keep_frac, int32_t warm,
                                  int32_t train_steps, int32_t batch, double *misfit_out,
                                  int32_t *n_modelled, void *stream);

/* Modelling kernel selection for the persistent launch:
 *   EMPSO_KERNEL_AUTO       the tuned choice for this batch (empso_autotune),
 *                           else the on-chip variant when every grid fits a
 *                           cluster of <= 16 CTAs, else the L2 cluster
 *                           variant, else the streaming variant;
 *   EMPSO_KERNEL_STREAMING  wavefields in global memory, one CTA per
 *                           instance;
 *   EMPSO_KERNEL_RESIDENT   wavefields in distributed shared memory, one
 *                           thread-block cluster per instance (calls return
 *                           UNSUPPORTED when a grid does not fit);
 *   EMPSO_KERNEL_CLUSTER_L2 wavefields in a per-cluster global buffer, one
 *                           thread-block cluster per instance, with few
 *                           enough instances in flight to stay in L2 (for
 *                           grids too large for the on-chip variant).
 * All compute the same scheme; results agree to FP32 rounding. */
#define EMPSO_KERNEL_AUTO      0
#define EMPSO_KERNEL_STREAMING 1
#define EMPSO_KERNEL_RESIDENT  2
#define EMPSO_KERNEL_CLUSTER_L2 3
empso_status empso_set_kernel(empso_ctx *ctx, int32_t kind);

/* Cluster size (CTAs per instance) of the on-chip kernel: 0 lets the library
 * pick the size that keeps the most SMs busy; 1..16 forces it (calls return
 * UNSUPPORTED when the batch does not fit that size). */
empso_status empso_set_cluster(empso_ctx *ctx, int32_t ctas);

/* Rows per thread of the on-chip kernel (EMPSO_KERNEL_RESIDENT): each thread
 * updates a run of at most `rows` consecutive rows of one 4-point column
 * group per step.  0 (default): the planner's or the autotuner's choice
 * (among 13, 11, 9, 8, 6); 4..8 run with up to 512 threads per CTA, 9..13
 * with up to 384 (more registers per thread).  An engineering choice of this
 * library (the paper has no such parameter).  Errors: INVALID_ARG for any
 * other value. */
empso_status empso_set_tile_rows(empso_ctx *ctx, int32_t rows);

/* Co-resident groups of the last modelling launch: thread-block clusters of
 * the cluster kernels (times the cluster size = SMs busy), CTAs of the
 * streaming kernels.  groups: host. */
empso_status empso_last_clusters(const empso_ctx *ctx, int32_t *groups);

/* Rows per thread of the last on-chip launch (0 if the last launch used
 * another kernel).  rows: host. */
empso_status empso_last_tile_rows(const empso_ctx *ctx, int32_t *rows);

/* Which modelling kernel the last launch used: *kind = EMPSO_KERNEL_STREAMING
 * or EMPSO_KERNEL_RESIDENT (0 before any launch), *cluster = CTAs per
 * instance.  Either pointer may be NULL (host ints). */
empso_status empso_last_launch(const empso_ctx *ctx, int32_t *kind, int32_t *cluster);

/* Work units of the last on-chip launch that ran two instances at once, one
 * on each half of the cluster (instances of a grid that fits half the
 * cluster without raising the launch's shared memory or threads, e.g. the
 * coarse grid of a mixed-resolution batch); 0 for other kernels. */
empso_status empso_last_paired_units(const empso_ctx *ctx, int32_t *paired);

/* Device-function name of the last modelling launch's kernel
 * ("wave_resident_kernel", "wave_stream_kernel" for the streaming kernel
 * with bulk asynchronous row copies, "wave_kernel" for the plain streaming
 * kernel; "" before any launch): what a profiler's kernel filter matches.
 * The string is static. */
const char *empso_last_kernel_name(const empso_ctx *ctx);

/* Device-side status of the launches since the last call: a bounded wait
 * inside a kernel that gave up (EMPSO_TIMEOUT) - the instance concerned then
 * reports misfit +inf.  Synchronises `stream`, then clears the word.
 * status: host int. */
empso_status empso_device_error(empso_ctx *ctx, int32_t *status, void *stream);

/* Kernel timing: when enable != 0, eval_fitness / eval_models /
 * forward_traces record CUDA events on their stream around the model-field
 * kernels, the persistent modelling launch and the misfit reduction. */
empso_status empso_set_timing(empso_ctx *ctx, int32_t enable);

/* Durations of the last timed call in milliseconds (host double[3]):
 * [0] model fields (interpolation), [1] modelling launch, [2] misfit
 * reduction.  Waits for the last recorded event.  NOT_INITIALIZED if no
 * timed call ran since timing was enabled. */
empso_status empso_read_timing(empso_ctx *ctx, double *ms3);

/* Misfits of M gridded models on one grid WITHOUT ANY ALLOCATION.  The paper
 * has no counterpart: this entry point exists for callers that may not
 * allocate device memory - code running where the CUDA allocator must not be
 * touched (a host that owns and budgets all device memory itself, a plugin
 * inside another runtime's memory pool, a real-time loop that forbids
 * allocation after start-up).  It needs no context.
 *
 * grid: host; rec_xz: host [nrec_total][2] (<= 1024 receivers); vel: device
 * [M][nz][nx]; shots: host [S] (<= 64, all with grid_id 0); d_obs: device,
 * concatenation over shots of [nt][nrec_s]; misfit: device [M].  Same result
 * as eval_models (same kernels, streaming variant).
 *
 * Scratch: a fixed 16 MiB device array inside the library (held by every GPU
 * that loads it, until exit).  It must hold the model fields of all M models
 * plus two wavefield buffers of at least one instance; larger requests return
 * EMPSO_UNSUPPORTED with the needed size in empso_last_error(NULL).  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents (the call
 * clears what must start at zero itself); calls that overlap on the GPU -
 * different streams, or different host threads, on one device - race on it
 * and must be serialised by the caller.  Errors: INVALID_ARG, UNSUPPORTED,
 * CUDA_ERROR; message in empso_last_error(NULL). */
empso_status eval_models_noalloc(const empso_grid *grid, const float *rec_xz,
                                 int32_t nrec_total, const float *vel, int32_t M,
                                 const empso_shot *shots, int32_t S,
                                 const float *d_obs, double *misfit, void *stream);

/* Human-readable name of a status code (static storage). */
const char *empso_status_string(empso_status s);

/* Message of the last failed call on this context (static storage of the
 * context; empty string if none).  ctx may be NULL for empso_create errors. */
const char *empso_last_error(const empso_ctx *ctx);

/* ---- irregular control grid ("Testing approach") -----------------------
 * The paper's two-grid strategy with a variable node spacing: L depth
 * levels at level_z[l] (metres, strictly increasing), level l holding
 * level_count[l] >= 1 nodes at x positions node_x[o_l .. o_l + level_count[l])
 * (strictly increasing; o_l = sum of the earlier counts).  A particle on
 * this grid has K = sum level_count values in that order.  The FD-grid
 * velocity at (x, z) is bilinear level-wise: on the two levels bracketing
 * z, linear in x between that level's neighbouring nodes (end values held
 * beyond the ends), then linear in z between the two levels (the first or
 * last level held above or below); then clipped to [vmin, vmax].
 * empso_set_levels switches grid `grid_id` to this rule (interp_mode 2),
 * computing its per-point taps on the device; it synchronises the device
 * and drops captured generations.  K <= 1024.  Errors: INVALID_ARG,
 * UNSUPPORTED (K > 1024), OOM/CUDA_ERROR. */
empso_status empso_set_levels(empso_ctx *ctx, int32_t grid_id, int32_t n_levels,
                              const float *level_z, const int32_t *level_count,
                              const float *node_x);

/* Fixed water layer (the prior information of "Testing approach"): every
 * FD point of grid `grid_id` at depth z <= water_depth takes v_water (then
 * the clip), whatever the particle; water_depth <= 0 removes the layer.
 * Applies to every interpolation mode; synchronises the device and drops
 * captured generations. */
empso_status empso_set_water(empso_ctx *ctx, int32_t grid_id, float water_depth, float v_water);

/* Depth-dependent search ranges ("Testing approach"): the first and last
 * levels get [v (1 - lo), v (1 + hi)] around the prior 1-D velocity v_first
 * / v_last of that level; every intermediate level's limits lie on the
 * straight lines, in depth, through the first and last levels' minima and
 * maxima.  All nodes of a level share its range.  Host function (no
 * context): xmin, xmax host [sum level_count].  INVALID_ARG on bad input. */
empso_status empso_level_bounds(int32_t n_levels, const float *level_z,
                                const int32_t *level_count, double v_first, double v_last,
                                double lo_first, double hi_first, double lo_last,
                                double hi_last, double *xmin, double *xmax);

/* ---- observed-data preprocessing ("Testing approach") ------------------
 * Band-limited resampling of traces: in device [S][nt_in][nrec] sampled at
 * n dt_in (n = 0 .. nt_in - 1, zero outside), out device [S][nt_out][nrec]
 * at m dt_out, out[s][m][r] = dt_in sum_n in[s][n][r] h(m dt_out - n dt_in)
 * with the Blackman-windowed sinc h(tau) = 2 f_cut sinc(2 f_cut tau)
 * w(tau / half_width), w(u) = 0.42 + 0.5 cos(pi u) + 0.08 cos(2 pi u) for
 * |u| < 1.  With dt_out = dt_in it is a zero-phase low-pass below f_cut; with
 * another dt_out it also moves the traces onto that time axis (e.g. data
 * recorded on a fine grid onto the inversion grid's steps).  The transition
 * band is about 3 / half_width Hz wide.  in and out must not overlap.
 * Errors: INVALID_ARG, UNSUPPORTED (window of more than the shared memory
 * holds: half_width / dt_in too large). */
empso_status empso_lowpass(empso_ctx *ctx, const float *in, int32_t S, int32_t nt_in,
                           int32_t nrec, double dt_in, float *out, int32_t nt_out,
                           double dt_out, double f_cut, double half_width, void *stream);

/* ---- local FWI ("Testing approach": the EMPSO model starts a descent-based
 * full-waveform inversion) ---------------------------------------------
 * empso_gradient: misfit phi_m = sum_s w_s / 2 |R u_s - d_obs,s|^2 and its
 * gradient dphi_m/dv at every physical node of M gridded models vel device
 * [M][nz][nx] (m/s), all shots on one grid.  Computed by the exact discrete
 * adjoint of the modelling scheme: a forward pass that keeps, for every
 * (model, shot), the Laplacian L u^n of every step in device memory (all the
 * adjoint pass needs of the forward field; (nt + 1) x padded-grid floats
 * each, e.g. 0.78 GB per shot of a 461 x 151 grid with 40 damping cells and
 * 1414 steps), then the adjoint pass backward
 * in time accumulating sum_k mu^k f (L u^{k-1} + s^{k-1}), folded from the
 * damping pad onto the edge nodes and chained through a = v^2 dt^2.  The
 * forward pass runs on the on-chip kernel (history streamed out) when the
 * kernel selection is EMPSO_KERNEL_AUTO or EMPSO_KERNEL_RESIDENT and the grid
 * fits a cluster (RESIDENT: else UNSUPPORTED); else on the L2 cluster kernel
 * (also streaming the history out) when the selection is EMPSO_KERNEL_AUTO or
 * EMPSO_KERNEL_CLUSTER_L2 and the grid fits it (CLUSTER_L2: else
 * UNSUPPORTED); otherwise (EMPSO_KERNEL_STREAMING) as one launch per time
 * step.  All agree to FP32 rounding.
 * misfit: device [M] doubles or NULL; grad: device [M][nz][nx].  d_obs as
 * for eval_models.  Synchronises `stream` once (instance table upload).
 * Errors: INVALID_ARG, OOM (history does not fit), UNSUPPORTED, CUDA_ERROR. */
empso_status empso_gradient(empso_ctx *ctx, const float *vel, int32_t M,
                            const empso_shot *shots, int32_t S, const float *d_obs,
                            double *misfit, float *grad, void *stream);

/* Chains of the gradient's backward pass: its (model, shot) instances are
 * independent, so they run as n chains (1..8) of consecutive instances on
 * separate streams inside the captured graph, one chain's memory waits and
 * launch gaps overlapping another's work; 0 (default): 4 chains from 16
 * instances up, else 1 (measured on the 461 x 151 grid: 16 shots 35.6 ->
 * 33.3 ms with 4 chains, 4 shots 15.7 -> 18.1 ms).  Results do not depend on
 * n (each instance's arithmetic is the same).  A cluster size set by
 * empso_set_cluster also applies to the gradient's on-chip forward pass.
 * An engineering choice of this library (the paper has no such parameter).
 * Errors: INVALID_ARG outside 0..8. */
empso_status empso_set_gradient_chains(empso_ctx *ctx, int32_t chains);

/* Steepest-descent FWI of one model vel device [nz][nx] (in place), the
 * paper's local inversion: iteration k moves v <- clip(v - alpha g, vmin,
 * vmax) along the adjoint gradient g.  The first step length makes the
 * largest change 1 % of the mean velocity; later ones are the
 * Barzilai-Borwein length s.s / s.y (s = model change, y = gradient change;
 * kept when s.y <= 0); a step is accepted when the misfit decreases by at
 * least 1e-4 g.(v - v_new) (Armijo), else halved, at most 10 times, after
 * which the inversion stops.  history: host [iters + 1] misfits (initial
 * and after each accepted iteration) or NULL; *done: accepted iterations.
 * A multiscale inversion calls this once per frequency band, with that
 * band's grid (Ricker f0) and low-passed d_obs (empso_lowpass).
 * Synchronises `stream` every iteration. */
empso_status empso_fwi(empso_ctx *ctx, float *vel, const empso_shot *shots, int32_t S,
                       const float *d_obs, int32_t iters, float vmin, float vmax,
                       double *history, int32_t *done, void *stream);

/* ---- non-finite misfits ------------------------------------------------
 * A particle whose misfit sum is NaN or infinite (a diverging or
 * non-finite model) gets misfit +inf, so it never becomes a personal or
 * global best (Eq. 1-2 compare misfits), and is counted. */

/* Running count of non-finite misfits since the context was created (or
 * last reset): read after the work already queued on `stream`, which this
 * call synchronises; reset != 0 zeroes the count after reading it. */
empso_status empso_nonfinite_count(empso_ctx *ctx, int64_t *count, int32_t reset, void *stream);

/* Strict mode (off by default).  When on, eval_models, eval_fitness,
 * empso_generation and surrogate_generation synchronise their stream after
 * the work and return EMPSO_NONFINITE when that call produced a non-finite
 * misfit; the outputs are still written, those misfits as +inf. */
empso_status empso_set_strict(empso_ctx *ctx, int32_t enable);

/* ---- checkpoints ------------------------------------------------------
 * empso_save writes the swarm state (positions x, velocities v, personal
 * bests p and their misfits pf, global-best index g, generation counter k,
 * the last sort order) and, when the surrogate is initialised, its
 * parameters, Adam moments and step, replay buffer and target statistics to
 * `path` (written to `path`.tmp and renamed, so an existing checkpoint is
 * replaced only by a complete one).  The RNG needs no state: its streams are
 * counters keyed by (seed, k, particle, dimension).  empso_load restores
 * them into a context created with the same swarm (P, D, seed, xmin, xmax)
 * and, if the file holds a surrogate, the same surrogate shape (K, hidden,
 * capacity); a run resumed from a checkpoint continues bit for bit as the
 * uninterrupted run would.  Both synchronise the device.  Errors:
 * EMPSO_IO_ERROR (file cannot be opened, read, written or renamed; bad
 * magic, version, length or checksum), EMPSO_INVALID_ARG (shape, seed or
 * bounds mismatch), EMPSO_NOT_INITIALIZED (no swarm, or a surrogate in the
 * file but none in the context).  The context is left unchanged on error. */
empso_status empso_save(empso_ctx *ctx, const char *path);
empso_status empso_load(empso_ctx *ctx, const char *path);

#ifdef __cplusplus
}
#endif

#endif /* EMPSO_H */
