/*
 * dsmc.h -- C ABI of the GB300 (sm_103a) DSMC library for force-driven rarefied
 * flow between two parallel plates: the micro model of the Micro-Macro-Surrogate
 * method of arXiv 2311.14140 ("A DSMC-CFD coupling method using surrogate
 * modelling for low-speed rarefied gas flows").
 *
 * The problem (Sec. 2.1): a monatomic gas between two plates held at a constant
 * temperature, driven by an external acceleration F parallel to the plates, in
 * steady, fully developed, one-dimensional flow.  Everything is nondimensional as in
 * Eq. 6: lengths in the plate gap H (walls at y = 0 and y = 1), speeds in
 * v0 = sqrt(2 k T0 / m) with T0 the wall temperature, time in H / v0, body force
 * in v0^2 / H, stress in P0.  The Knudsen number enters through the viscosity,
 * mu0 v0 / (P0 H) = 2 Kn / sqrt(pi) (Eq. 7 against Eq. 2).  The DSMC method itself
 * is Bird's, which the paper cites (Sec. 1, Sec. 2) without describing it.
 *
 * One time step (a call to dsmc_step advances n of them), in this order:
 *   1. within each cell, NTC collisions of hard-sphere or VHS molecules in
 *      consecutive groups of at most `group_size` sorted particles, with the cell
 *      moments sampled half before and half after the collisions when the step is
 *      at or past `sample_start`;
 *   2. free flight of every particle for dt with the body force along x, and fully
 *      diffuse re-emission at the walls (any number of bounces, up to 64);
 *   3. a stable counting sort of the particles into cells (ties keep their previous
 *      order).
 * Random numbers are Philox4x32-10 keyed on the seed with counters built from
 * (stream, step, slot, bounce) for the flight and (stream, step, cell, group,
 * candidate) for collisions, so a run is a deterministic function of its inputs.
 *
 * Memory and ownership.  All particle and cell data live on the device.  The
 * library allocates them with cudaMalloc in dsmc_create and frees them in
 * dsmc_destroy, or uses a caller-owned device workspace given to dsmc_create_in
 * (dsmc_workspace_bytes says how large), which it never frees.  Output buffers of
 * the copy functions are caller-owned; they may be host memory (pageable or pinned)
 * or device memory.
 *
 * Streams and errors.  Work is enqueued on the stream of the options (NULL: the
 * legacy default stream) and is asynchronous unless a function says it
 * synchronises.  Every function returns a dsmc_status; dsmc_last_error() gives a
 * message for the last failure on the calling thread.  Device-side limits (bounce
 * count, rejection-sampling attempts) never trap: kernels record them in a device
 * error word, and the next synchronising call returns DSMC_E_DEVICE_LIMIT.
 * One handle must not be used from two threads at once.
 */
#ifndef DSMC_H
#define DSMC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DSMC_API __attribute__((visibility("default")))
#else
#define DSMC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Gas species.  Only omega enters the nondimensional problem: the Knudsen number
 * fixes n * sigma (Eq. 7), so mass, d_ref and T_ref are informational and only
 * checked for sign.  omega is the VHS viscosity index, 0.5 <= omega <= 1
 * (0.5 = hard sphere). */
typedef struct dsmc_gas {
  double mass;  /* kg, > 0 */
  double d_ref; /* m, > 0 */
  double omega; /* VHS viscosity index */
  double T_ref; /* K, > 0 */
} dsmc_gas;

typedef enum dsmc_status {
  DSMC_OK = 0,
  DSMC_E_INVAL = 1,        /* bad argument (message in dsmc_last_error) */
  DSMC_E_NOMEM = 2,        /* device allocation failed or workspace too small */
  DSMC_E_CUDA = 3,         /* a CUDA call failed */
  DSMC_E_DEVICE_LIMIT = 4, /* a kernel hit a bounded loop's limit (error word) */
  DSMC_E_STATE = 5         /* call not valid in the handle's current state */
} dsmc_status;

/* Arithmetic of the per-cell moment sums (dsmc_options.accum).  Both forms products of
 * the binary32 velocities; a group's sums are then combined exactly (fixed point in
 * the cell's grid, integer addition), so the sums do not depend on which warp takes
 * which group, and accumulated over steps in binary64.
 *   DSMC_ACCUM_FP32: each lane adds its particles' products in binary32 (second and
 *     third moments by fused multiply-add) and the warp sums them in binary32: at most
 *     28 roundings of relative size 2^-24 on partial sums bounded by the sum of
 *     |products|.  The default.
 *   DSMC_ACCUM_FP64: every product is rounded to binary32 (as a plain CPU DSMC forms
 *     it) and added in binary64 from the first addition on. */
typedef enum dsmc_accum { DSMC_ACCUM_FP32 = 0, DSMC_ACCUM_FP64 = 1 } dsmc_accum;

/* Options.  Get the defaults from dsmc_default_options and change fields. */
typedef struct dsmc_options {
  double dt_factor;       /* dt = dt_factor / nu, nu = n sigma_ref <g> the equilibrium
                             collision frequency, <g> = 2 sqrt(2/pi); default 0.2 */
  double dt;              /* > 0: time step in H / v0, overriding dt_factor (required
                             when Kn is infinite); default 0 */
  long long sample_start; /* steps numbered from 1; steps >= sample_start are
                             sampled; default 0 (every step) */
  int group_size;         /* collision group G: even, 2 <= G <= 512; default 256 */
  int collisions;         /* 0 turns collisions off; default 1 */
  int profile;            /* 1: time every kernel launch with CUDA events (then
                             dsmc_step synchronises at its end); default 0 */
  int span_particles;     /* particles per span (CTA) of the step passes at the
                             initial density: 0 keeps the partition in use (at creation
                             4096, or fewer down to 1024 when the handle holds less than
                             two such spans per SM; or what dsmc_autotune chose), else
                             1024..2^24.
                             Only the work split changes: results are identical for
                             every value; default 0 */
  int cta_warps;          /* warps per CTA of the collide/move pass: 0 keeps the shape
                             in use (8 at creation, 4 for a pool, or what dsmc_autotune
                             chose), else 4 or 8; results are identical; default 0 */
  int span_rows;          /* sort-matrix rows per span, one per equal part of its
                             slots, each scattered by its own warp: 0 keeps the value
                             in use (1 at creation, or what dsmc_autotune chose), else
                             1 or 2; results are identical; default 0 */
  int graph;              /* 1: dsmc_step replays the launches of 16 steps as one
                             CUDA graph (captured on first use; needs a stream other
                             than the legacy default; off while profiling); results
                             are identical; default 0 */
  int accum;              /* dsmc_accum: arithmetic of the moment sums; default
                             DSMC_ACCUM_FP32 */
  void* stream;           /* cudaStream_t for all work; default NULL */
} dsmc_options;

/* What one instance of a handle computes with: the binary32 values are exactly those
 * the kernels use. */
typedef struct dsmc_info {
  long long n_particles;
  int n_cells;
  int ppc;
  long long step;      /* steps completed */
  long long n_samples; /* sampled steps in the accumulators */
  double Kn, omega, body_force;
  double nsigma;       /* n sigma_ref H (Eq. 7 with the VHS viscosity) */
  double dt;           /* binary64 time step */
  float dt_f, F_f;     /* binary32 time step and body force */
  float coef;          /* n sigma_ref dt / (2 ppc): NTC candidate factor */
  float cvhs, vexp;    /* sigma g / sigma_ref = cvhs * g^vexp (HS: 1, 1) */
  float vinv;          /* 1 / vexp (0 when omega = 1) */
  float lncv;          /* ln cvhs */
  float smax0;         /* initial (sigma g)_max / sigma_ref */
  size_t device_bytes; /* device memory the whole handle uses */
  int n_instances;     /* instances in the handle */
  int span_particles;  /* particles per span of the partition in use */
  int cta_warps;       /* warps per CTA of the collide/move pass in use */
  int span_rows;       /* sort-matrix rows per span in use */
  int cells_per_span;  /* this instance's cells per span of the step passes */
  int n_spans;         /* this instance's spans (CTAs of the collide/move pass) */
  int total_spans;     /* spans of all instances */
  int first_slot;      /* the instance's first particle slot in the handle */
  int first_cell;      /* the instance's first row in dsmc_sample_moments_all */
} dsmc_info;

/* One member of a batch: the arguments of dsmc_create. */
typedef struct dsmc_instance {
  dsmc_gas gas;
  double Kn;
  double wall_T;
  double body_force;
  int n_cells;
  int ppc;
  uint64_t seed;
} dsmc_instance;

typedef struct dsmc_sim* dsmc_handle;

/* Number of raw moment sums per cell returned by dsmc_sample_moments. */
#define DSMC_NMOM 13

DSMC_API dsmc_status dsmc_default_options(dsmc_options* opt);

/* Device bytes dsmc_create_in needs for n_cells * ppc particles. */
DSMC_API size_t dsmc_workspace_bytes(int n_cells, int ppc);

/* Create a run: n_cells cells of width 1/n_cells across the gap (Sec. 3 uses
 * Delta y = 0.005), ppc particles per cell at start, each placed uniformly in its
 * cell with velocity components N(0, 1/2) (the gas at rest at the wall
 * temperature, Sec. 2.1), then sorted into cells.  Kn > 0 (+INFINITY: collisionless,
 * then options.dt must be set); wall_T > 0 is the reference temperature T0;
 * body_force is F = F' H / v0^2 (Eq. 6); 1 <= n_cells <= 16384, ppc >= 1,
 * n_cells * ppc <= 2^31 - 2^24 (with group_size 512 and more than ~12,000 cells the
 * step's shared memory may not fit: DSMC_E_INVAL).  The library allocates the device memory.  Initialisation
 * is enqueued on the legacy default stream and completed before return. */
DSMC_API dsmc_status dsmc_create(const dsmc_gas* gas, double Kn, double wall_T,
                        double body_force, int n_cells, int ppc, uint64_t seed,
                        dsmc_handle* out);

/* As dsmc_create, with options applied from the start (their stream is used for
 * initialisation) and the caller's device workspace of workspace_bytes >=
 * dsmc_workspace_bytes(n_cells, ppc), 256-byte aligned; NULL workspace: the
 * library allocates.  The library never frees a caller's workspace. */
DSMC_API dsmc_status dsmc_create_in(const dsmc_gas* gas, double Kn, double wall_T,
                           double body_force, int n_cells, int ppc, uint64_t seed,
                           const dsmc_options* opt, void* workspace,
                           size_t workspace_bytes, dsmc_handle* out);

/* Replace the options.  Takes effect for the next step. */
DSMC_API dsmc_status dsmc_set_options(dsmc_handle h, const dsmc_options* opt);

/* Enqueue n_steps >= 0 steps.  Asynchronous (unless profiling); returns an error
 * latched by an earlier synchronising call, else DSMC_OK. */
DSMC_API dsmc_status dsmc_step(dsmc_handle h, int n_steps);

/* Wait for the handle's stream and check the device error word. */
DSMC_API dsmc_status dsmc_sync(dsmc_handle h);

/* Copy the n_cells x DSMC_NMOM raw sums, row-major per cell, into out (binary64):
 *   [count, vx, vy, vz, vx^2, vy^2, vz^2, vx vy, vx vz, vy vz, vx|v|^2, vy|v|^2, vz|v|^2]
 * summed over the particles of the cell and the sampled steps, each step counted
 * half before and half after its collisions.  Velocities in v0.  *n_samples gets
 * the number of sampled steps.  Synchronises. */
DSMC_API dsmc_status dsmc_sample_moments(dsmc_handle h, double* out, long long* n_samples);

/* Number of cell fields returned by dsmc_cell_fields. */
#define DSMC_NFIELD 9

/* Cell fields from raw moment sums: the time averages the paper reports for its DSMC
 * (Sec. 3), in the units of Eq. 6.  sums holds n_cells x DSMC_NMOM raw sums (the layout
 * of dsmc_sample_moments) over n_samples >= 1 sampled steps of a run with ppc >= 1
 * particles per cell at start; out gets n_cells x DSMC_NFIELD values, row-major per
 * cell:
 *   [0] n   = count / (n_samples ppc)        density relative to the initial one
 *   [1..3] u_i = sum v_i / count              mean velocity (v0)
 *   [4] T   = (2/3) (<|v|^2> - |u|^2)         temperature (T0)
 *   [5] Pxy = 2 n (<vx vy> - ux uy)           shear stress (P0 = n0 k T0; rho/P0 = 2/v0^2)
 *   [6..8] q_i = n <c_i |c|^2>, c = v - u     heat flux (P0 v0)
 * A cell without samples gives n = 0 and NaN elsewhere.  Host memory; binary64. */
DSMC_API dsmc_status dsmc_cell_fields(const double* sums, long long n_samples, int ppc,
                                      int n_cells, double* out);

/* The same fields from instance i's own sums (computed on the device); out (host or
 * device memory) gets its n_cells x DSMC_NFIELD values.  Synchronises. */
DSMC_API dsmc_status dsmc_cell_fields_of(dsmc_handle h, int i, double* out);

/* Zero the moment sums and collision counters (enqueued). */
DSMC_API dsmc_status dsmc_reset_samples(dsmc_handle h);

/* Copy the particle state in cell order (N floats each; any pointer may be NULL to
 * skip it).  Synchronises. */
DSMC_API dsmc_status dsmc_copy_state(dsmc_handle h, float* y, float* vx, float* vy, float* vz);

/* Copy cell data: offset[n_cells + 1] (first slot of each cell in the sorted state),
 * smax[n_cells] ((sigma g)_max / sigma_ref), ncand[n_cells] and nacc[n_cells]
 * (collision candidates and accepted collisions since the last reset).  Any pointer
 * may be NULL.  Synchronises. */
DSMC_API dsmc_status dsmc_copy_cells(dsmc_handle h, int* offset, float* smax,
                            unsigned long long* ncand, unsigned long long* nacc);

/* Replace the particle state (N floats each, any order, y in [0, 1]; values outside
 * are moved onto the nearest wall), the per-cell (sigma g)_max (NULL: keep) and the
 * step counter, then sort into cells.  This restores a checkpoint bit-exactly.
 * Synchronises. */
DSMC_API dsmc_status dsmc_load_state(dsmc_handle h, const float* y, const float* vx,
                            const float* vy, const float* vz, const float* smax,
                            long long step);

DSMC_API dsmc_status dsmc_get_info(dsmc_handle h, dsmc_info* info);

/* Batches: many independent runs advanced by the same launches.
 *
 * The paper's method trains its surrogate on many micro-simulations at different
 * (Kn, force) points (Sec. 2.3-2.4); a batch runs them together so that small runs
 * fill the GPU.  Instance i of a batch evolves bit for bit as dsmc_create_in with
 * instances[i] and the same options would: its random numbers are keyed on its own
 * seed, step, cells and slots.  Instances may differ in gas, Kn, wall_T, force,
 * n_cells and ppc; options (dt_factor or dt, group size, sampling start, stream) are
 * shared.  Particle slots, cells and sort matrices are concatenated in one device
 * workspace (dsmc_batch_workspace_bytes); every step is the same four launches as
 * for one run, over the spans of all instances.  The functions without `_of` act on
 * instance 0, dsmc_step and dsmc_reset_samples on all instances. */

/* Device bytes dsmc_create_batch needs (0 for invalid sizes). */
DSMC_API size_t dsmc_batch_workspace_bytes(const dsmc_instance* instances, int n_instances);

/* Create n_instances (1..65535) runs in one handle; each instance is validated as by
 * dsmc_create (messages name the failing instance), and all particles, each instance
 * padded to a multiple of 64, must total <= 2^31 - 2^24.  workspace as for
 * dsmc_create_in (NULL: the library allocates).  Synchronises. */
DSMC_API dsmc_status dsmc_create_batch(const dsmc_instance* instances, int n_instances,
                                       const dsmc_options* opt, void* workspace,
                                       size_t workspace_bytes, dsmc_handle* out);

/* Number of active instances (0 for NULL). */
DSMC_API int dsmc_batch_size(dsmc_handle h);

/* Per-instance forms of the functions above, for instance id i (0 <= i < batch size for
 * dsmc_create_batch; the id from dsmc_pool_add for pools). */
DSMC_API dsmc_status dsmc_sample_moments_of(dsmc_handle h, int i, double* out,
                                            long long* n_samples);
DSMC_API dsmc_status dsmc_reset_samples_of(dsmc_handle h, int i);
DSMC_API dsmc_status dsmc_copy_state_of(dsmc_handle h, int i, float* y, float* vx, float* vy,
                                        float* vz);
/* offset[] is relative to the instance's first slot, as for a run of its own. */
DSMC_API dsmc_status dsmc_copy_cells_of(dsmc_handle h, int i, int* offset, float* smax,
                                        unsigned long long* ncand, unsigned long long* nacc);
DSMC_API dsmc_status dsmc_load_state_of(dsmc_handle h, int i, const float* y, const float* vx,
                                        const float* vy, const float* vz, const float* smax,
                                        long long step);
DSMC_API dsmc_status dsmc_get_info_of(dsmc_handle h, int i, dsmc_info* info);

/* The moment sums of all instances in one copy: out holds (cell capacity of the
 * handle) x DSMC_NMOM binary64 values; instance i's rows start at its
 * dsmc_info.first_cell (for dsmc_create_batch: instance after instance, no gaps).
 * n_samples (NULL or dsmc_id_bound entries) gets each instance's sampled steps (0 for
 * unused ids).  Synchronises. */
DSMC_API dsmc_status dsmc_sample_moments_all(dsmc_handle h, double* out, long long* n_samples);

/* One more than the largest instance id the handle has handed out. */
DSMC_API int dsmc_id_bound(dsmc_handle h);

/* Per instance id < dsmc_id_bound: out[2 id] = sampled particle count and
 * out[2 id + 1] = sum of vx over all cells and sampled steps (zeros for unused ids).
 * The channel-mean velocity of the samples is their ratio.  Synchronises. */
DSMC_API dsmc_status dsmc_channel_sums(dsmc_handle h, double* out);

/* Pools: a handle whose instances come and go while it runs (continuous batching).
 * Capacity is fixed at creation; dsmc_pool_add places an instance in free ranges of
 * the handle's arrays (DSMC_E_NOMEM "no room" when they are taken) and
 * dsmc_pool_remove frees them.  An added instance is set up on the device by the next
 * dsmc_step or synchronising call, exactly as dsmc_create would set it up, and from
 * then on evolves as it would alone (the counter-based random numbers are keyed on its
 * own seed, step, cells and slots).  Removal takes effect for the next launch; work
 * already enqueued finishes first.  Ids of removed instances are reused.  Options are
 * shared by all instances; sample_start counts each instance's own steps. */
typedef struct dsmc_pool_limits {
  long long max_particles;    /* slots, each instance padded to a multiple of 64 */
  int max_cells;              /* cells of all instances together */
  int max_instances;          /* instances at once, 1..65535 */
  int max_cells_per_instance; /* 1..16384 */
} dsmc_pool_limits;

/* Device bytes dsmc_pool_create needs (0 for invalid limits). */
DSMC_API size_t dsmc_pool_workspace_bytes(const dsmc_pool_limits* limits);
DSMC_API dsmc_status dsmc_pool_create(const dsmc_pool_limits* limits, const dsmc_options* opt,
                                      void* workspace, size_t workspace_bytes,
                                      dsmc_handle* out);
/* *id gets the new instance's id (-1 on failure). */
DSMC_API dsmc_status dsmc_pool_add(dsmc_handle h, const dsmc_instance* instance, int* id);
DSMC_API dsmc_status dsmc_pool_remove(dsmc_handle h, int id);

/* Serving: micro-solve requests run to a target standard error.
 *
 * A request is one run (dsmc_instance) that arrives at `arrival` seconds after the
 * start of dsmc_serve and is finished when the relative standard error of its
 * channel-mean velocity (sum vx / count over all sampled particles and steps) is at
 * most target_se, or after max_steps steps.  The standard error is taken by batch means:
 * the sampled epochs (epoch_steps steps each, sampling from the pool's
 * options.sample_start on, counted in each instance's own steps) are split into
 * `batches` consecutive batches, each gives a mean, and the error is their standard
 * deviation over sqrt(batches).  The paper runs its micro-solves at the (Kn, force)
 * points its surrogate asks for (Sec. 2.3-2.4); the request loop is this library's. */
typedef struct dsmc_request {
  dsmc_instance instance;
  double arrival;      /* seconds after the start, non-decreasing along the array */
  double target_se;    /* relative standard error to reach, > 0 (0.01 = 1 %) */
  long long max_steps; /* >= 1 */
} dsmc_request;

typedef struct dsmc_serve_options {
  int epoch_steps;   /* steps between reads of the channel sums; default 32 */
  int batches;       /* batches of the batch-means error, >= 2; default 16 */
  int max_active;    /* instances on the device at once, 0: as many as fit; default 0 */
  double time_limit; /* seconds, 0: none; default 0 */
} dsmc_serve_options;

typedef struct dsmc_request_result {
  double admitted;   /* seconds after the start (-1: never admitted) */
  double finished;   /* seconds after the start (-1: not finished in the time limit) */
  long long steps;   /* steps run */
  double u_mean;     /* channel-mean velocity of the samples (v0) */
  double u_se;       /* its batch-means standard error (v0); INFINITY if too few epochs */
  double count;      /* final channel sums: sampled particle count ... */
  double sum_vx;     /* ... and sum of vx */
  int converged;     /* 1 target met, 0 step or time limit, -1 rejected (invalid or too
                        large for the pool) */
  int id;            /* pool id it ran under */
} dsmc_request_result;

DSMC_API dsmc_status dsmc_default_serve_options(dsmc_serve_options* so);

/* Continuous batching of `requests` on an empty pool handle (dsmc_pool_create), in
 * real time: a request is admitted once it has arrived and the pool has room (in
 * order of arrival), all admitted instances advance together epoch_steps at a time,
 * and every instance whose target is met after an epoch is removed, its result
 * recorded, and its memory given to the next waiting requests.  Each instance's
 * trajectory is that of the same run alone.  results[n_requests] are filled.
 * Returns when every request is finished or the time limit has passed. */
DSMC_API dsmc_status dsmc_serve(dsmc_handle pool, const dsmc_request* requests, int n_requests,
                                const dsmc_serve_options* so, dsmc_request_result* results);

/* One request solved as a plain run of its own (dsmc_create_in with `opt`, the library
 * allocating), epoch by epoch to the same criterion; times are seconds after the call
 * (admitted: after creation).  For comparison with dsmc_serve. */
DSMC_API dsmc_status dsmc_solve(const dsmc_request* request, const dsmc_options* opt,
                                const dsmc_serve_options* so, dsmc_request_result* result);

/* Open boundary (the MMS hybrid's DSMC-CFD interface, Sec. 2 and Sec. 3.2): from the
 * next step on, the boundary of instance i at y = 1 is a reservoir of gas in the
 * first-order Chapman-Enskog state of a shear flow with bulk velocity u (along x) and
 * shear stress P (Eq. 6 units, |P| <= 0.25), instead of a wall.  Each particle that
 * crosses it is re-emitted into the run from the flux-weighted half-range distribution
 * exp(-c^2) (1 + 2 P c_x c_y) |c_y|, c_y < 0 (c the peculiar velocity), so the number
 * of particles is conserved; the boundary at y = 0 stays a diffuse wall.  u and P are
 * rounded once to binary32; call again to update them (e.g. every hybrid iteration). */
DSMC_API dsmc_status dsmc_set_open_top(dsmc_handle h, int i, double u, double P);

/* The device address of instance i's moment sums (n_cells x DSMC_NMOM binary64, the
 * layout of dsmc_sample_moments), valid until the handle is destroyed or the instance
 * removed; its contents change with every step.  For consumers on the device. */
DSMC_API dsmc_status dsmc_device_moments_of(dsmc_handle h, int i, const double** acc);

/* The surrogate stage (Sec. 2.3, Appendix A): training samples from windows of DSMC
 * moment sums, Bayesian ridge regression with evidence maximisation for the boundary
 * models (no-slip Eq. 11, first-order slip Eq. 12) and the constitutive models C0..C3
 * (Eq. 13 with the stress correction Eq. 14 and Table 1 exponents), selection by
 * Eq. 17 with equal priors, and the corrected macroscopic solve (Eq. 8 with Eqs. 9-10)
 * with Monte Carlo uncertainty bands from the posteriors.  All arithmetic binary64.
 *
 * A training sample is one window of sampled steps of a run with n_cells cells of
 * ppc particles: per cell u = sum vx / N and P_xy = 2 n (<vx vy> - <vx><vy>),
 * n = N / (steps ppc); the constitutive targets are E_i = P_i + (2 Kn / sqrt(pi)) du/dy
 * at the cells with two neighbours (central differences), the boundary targets the
 * wall velocities extrapolated linearly from the two nearest cells, with
 * P^CFD(wall) = F (2y - 1) = -F, +F.  The regression has no intercept and flat
 * hyperpriors; a weight precision above 1e30 switches the weights off. */
typedef struct dsmc_surrogate* dsmc_surrogate_handle;

typedef struct dsmc_surrogate_fit {
  long long n_samples;      /* training samples (windows) */
  double n_v, n_c;          /* data points of the boundary and constitutive models */
  double log_evidence_v[2]; /* no-slip, slip */
  double prob_v[2];
  double alpha_v[2], beta_v[2];
  double sigma_p, sigma_p_var; /* slip coefficient: posterior mean and variance */
  int iterations_v;
  double log_evidence_c[4]; /* C0..C3 */
  double prob_c[4];
  double alpha_c[4], beta_c[4];
  double m_c[4][3];         /* posterior means a_1..a_k of C_k */
  double S_c[4][9];         /* posterior covariances (k x k block of a row-major 3x3) */
  int iterations_c[4];
  int sel_v, sel_c;         /* selected models: 0 no-slip / 1 slip; k of C_k (the
                               lowest index among log evidences within 1e-9 relative
                               of the best) */
  double b[3];              /* exponents used */
} dsmc_surrogate_fit;

/* Table 1 exponents at the tabulated Kn nearest in log Kn (b[3]). */
DSMC_API dsmc_status dsmc_surrogate_exponents(double Kn, double* b);

/* A surrogate for runs of n_cells (>= 3) cells with ppc particles per cell at Kn with
 * body force F != 0; b = NULL takes Table 1.  Device work goes on `stream`. */
DSMC_API dsmc_status dsmc_surrogate_create(double Kn, double F, int n_cells, int ppc,
                                           const double* b, void* stream,
                                           dsmc_surrogate_handle* out);
/* A surrogate trained from runs that cover only the Knudsen layer next to the bottom
 * wall (the MMS hybrid's DSMC sub-domain): the runs span y in [0, length] of the
 * channel (0 < length < 1) with n_cells cells; the constitutive targets come from the
 * cells 1 .. n_train - 1 of the training region (the rest is the buffer next to the
 * interface) and the slip model from the bottom wall alone (x = -P(0) = F). */
DSMC_API dsmc_status dsmc_surrogate_create_region(double Kn, double F, int n_cells, int ppc,
                                                  double length, int n_train,
                                                  const double* b, void* stream,
                                                  dsmc_surrogate_handle* out);
DSMC_API dsmc_status dsmc_surrogate_destroy(dsmc_surrogate_handle s);
/* Forget all training samples. */
DSMC_API dsmc_status dsmc_surrogate_reset(dsmc_surrogate_handle s);
/* One training sample from a window's raw sums (n_cells x DSMC_NMOM, host or device)
 * of n_steps sampled steps. */
DSMC_API dsmc_status dsmc_surrogate_add_window(dsmc_surrogate_handle s, const double* acc,
                                               long long n_steps);
/* One training sample from the sums instance i of h has accumulated since its last
 * reset (read in place on the device), then resets them: calls after every window of
 * steps give consecutive samples.  Synchronises. */
DSMC_API dsmc_status dsmc_surrogate_add_run(dsmc_surrogate_handle s, dsmc_handle h, int i);
/* Fit and select all models on the samples so far.  Synchronises. */
DSMC_API dsmc_status dsmc_surrogate_train(dsmc_surrogate_handle s, dsmc_surrogate_fit* out);
/* The stress correction S(y) (Eq. 14) of a fit's selected constitutive model (posterior
 * means, the fit's exponents) at the n + 1 faces y = f / n of an n-cell CFD grid
 * (host or device output; zeros for C0).  Synchronises. */
DSMC_API dsmc_status dsmc_surrogate_correction(const dsmc_surrogate_fit* fit, int n,
                                               double* S_faces, void* stream);
/* Monte Carlo bands (Sec. 2.3): n_trials trials, each drawing the selected models'
 * weights as m + L z (S = L L^T) with z the trial's row of 4 standard normals
 * (slip coefficient, a_1..a_3; host or device), solving Eq. 8 on n_cfd cells
 * (cell-centred finite volume, wall values through ghost cells); u_mean and u_std
 * (NULL to skip; sample standard deviation) get n_cfd values.  fit = NULL uses the
 * last dsmc_surrogate_train.  Synchronises. */
DSMC_API dsmc_status dsmc_surrogate_profile(dsmc_surrogate_handle s,
                                            const dsmc_surrogate_fit* fit, int n_cfd,
                                            const double* z, int n_trials, double* u_mean,
                                            double* u_std);

/* The MMS hybrid (Sec. 2, Sec. 3.2): DSMC only in the Knudsen layer next to the bottom
 * wall (two mean free paths, Kn in channel units, rounded up to whole cells of width dy,
 * plus `buffer` cells next to the interface; by symmetry it stands for both walls),
 * open to the CFD through the Chapman-Enskog interface of dsmc_set_open_top, its
 * windows training the surrogates (dsmc_surrogate_create_region) that correct the
 * CFD, iterated.  Iteration k: interface velocity = the CFD's at y = L_d (mean of the
 * two cells next to that face), stress F (2 L_d - 1); `steps` sampled steps (after
 * `warmup` unsampled ones in the first iteration), one training sample per `window`
 * steps, samples accumulating over iterations; retrain; CFD with the selected models.
 * The first CFD profile is no-slip Navier-Stokes. */
#define DSMC_MMS_MAX_ITER 64

typedef struct dsmc_mms_params {
  dsmc_gas gas;
  double Kn;         /* channel Knudsen number */
  double body_force; /* F of the channel (Eq. 6 units), != 0 */
  double wall_T;
  double dy;         /* DSMC cell width in channel units (Sec. 3: 0.005) */
  int ppc;           /* particles per cell (Sec. 3: 50) */
  int buffer;        /* buffer cells next to the interface (Sec. 3.2: 5) */
  int iterations;    /* 1..DSMC_MMS_MAX_ITER */
  int steps;         /* sampled steps per iteration */
  int window;        /* steps per training sample (Sec. 3: 100) */
  int warmup;        /* unsampled steps before the first samples */
  int n_cfd;         /* CFD cells over the channel */
  uint64_t seed;
  int group_size;    /* 0: 256 */
} dsmc_mms_params;

typedef struct dsmc_mms_result {
  int n_train, n_sub;          /* cells of the training region and of the sub-domain */
  double L_d;                  /* sub-domain height (channel units) */
  double b[3];                 /* exponents used (Table 1) */
  int iterations_done;
  double u_interface[DSMC_MMS_MAX_ITER]; /* interface velocity and stress of each */
  double p_interface[DSMC_MMS_MAX_ITER]; /* iteration (the binary32 values used) */
  long long samples;           /* training samples */
  dsmc_surrogate_fit fit;      /* the last fit */
} dsmc_mms_result;

DSMC_API dsmc_status dsmc_default_mms_params(dsmc_mms_params* p);

/* Runs the hybrid on `stream`.  profile[n_cfd] gets the final CFD profile with the
 * selected models' posterior means; with n_trials > 0, z (n_trials x 4 standard
 * normals, as for dsmc_surrogate_profile) gives band_sd[n_cfd] (NULL to skip), the
 * Monte Carlo standard deviation.  Synchronises. */
DSMC_API dsmc_status dsmc_mms_run(const dsmc_mms_params* p, void* stream, double* profile,
                                  const double* z, int n_trials, double* band_sd,
                                  dsmc_mms_result* out);

/* Gaussian-process variant of the surrogate stage (not the paper's method): GP
 * regression (Rasmussen and Williams 2006, Ch. 2) over n <= DSMC_GP_MAX_POINTS design
 * points X (n x 2, row-major, inputs scaled to the unit square) with m output columns Y
 * (n x m, row-major), squared-exponential covariance
 * exp(-1/2 ((dx_1 / l_1)^2 + (dx_2 / l_2)^2)) plus noise s2 on the diagonal, each column
 * standardised (mean, population standard deviation) and sharing the covariance.
 * dsmc_gp_fit evaluates the summed log marginal likelihood at each of n_grid
 * hyperparameter points grid[3 g .. 3 g + 2] = (l_1, l_2, s2) (one CTA each, Cholesky in
 * binary64 on the device), keeps the best (lml[n_grid] and *best, either may be NULL)
 * and alpha = K^-1 y there.  Inputs may be host or device memory.  Synchronises. */
#define DSMC_GP_MAX_POINTS 128
typedef struct dsmc_gp* dsmc_gp_handle;
DSMC_API dsmc_status dsmc_gp_fit(const double* X, const double* Y, int n, int m,
                                 const double* grid, int n_grid, void* stream,
                                 dsmc_gp_handle* out, double* lml, int* best);
/* Predictive means at ns points Xs (ns x 2) into out (ns x m).  Synchronises. */
DSMC_API dsmc_status dsmc_gp_predict(dsmc_gp_handle gp, const double* Xs, int ns, double* out);
DSMC_API dsmc_status dsmc_gp_hyper(dsmc_gp_handle gp, double* l1, double* l2, double* s2);
DSMC_API dsmc_status dsmc_gp_destroy(dsmc_gp_handle gp);

/* The cell-centred finite-volume solve of Eq. 8 on n cells with the stress correction
 * S given at the n + 1 faces and the wall values of Eq. 9 (slip = 0) or Eq. 10 with
 * coefficient sigma_p (slip = 1): u[n] (host or device).  Synchronises. */
DSMC_API dsmc_status dsmc_cfd_faces(double Kn, double F, int n, int slip, double sigma_p,
                                    const double* S_faces, double* u, void* stream);

/* Tuner of the step's work split.  For CTA shapes of 8 and 4 warps, 1 or 2 sort rows per
 * span, and span sizes 1024, 2048, ... particles (those whose shared memory fits,
 * skipping sizes that give the same partition) it runs one untimed and steps_per_trial
 * timed steps, keeps the fastest, and stores it in the handle's options (cta_warps,
 * span_rows, span_particles).  The trial steps are real steps of the run: they
 * advance every instance, and since the partition does not change results the run is
 * the same as without tuning.  *best_span_particles and *best_ms_per_step (either may
 * be NULL) get the choice and its time per step.  Synchronises. */
DSMC_API dsmc_status dsmc_autotune(dsmc_handle h, int steps_per_trial, int* best_span_particles,
                                   double* best_ms_per_step);

/* Kernel timing (options.profile = 1).  For kernel id k < dsmc_kernel_count():
 * total milliseconds and launches since the last dsmc_reset_kernel_times. */
DSMC_API int dsmc_kernel_count(void);
DSMC_API const char* dsmc_kernel_name(int k);
DSMC_API dsmc_status dsmc_kernel_times(dsmc_handle h, double* total_ms, long long* launches);
DSMC_API dsmc_status dsmc_reset_kernel_times(dsmc_handle h);

/* Release the handle and the device memory it allocated.  NULL is accepted. */
DSMC_API dsmc_status dsmc_destroy(dsmc_handle h);

/* Stable sort of a particle state into cells that allocates nothing.  The paper has
 * no counterpart: this is a service for callers that cannot allocate device memory
 * when they need the sort, such as plug-ins inside a runtime that owns all device
 * memory and lends them no allocator, or latency-sensitive loops that must avoid the
 * device-wide synchronisation of cudaMalloc/cudaFree.
 * Inputs y, vx, vy, vz and outputs y_out, vx_out, vy_out, vz_out (n_particles floats
 * each) and offset_out (n_cells + 1 ints) are caller-owned device memory; an output
 * that overlaps an input or another output is rejected (DSMC_E_INVAL).  On completion
 * (asynchronously, on `stream`) the outputs hold the state ordered by cell,
 * cell = trunc(y * n_cells) clamped to [0, n_cells - 1], particles of one cell in their
 * input order, and offset_out[c] is the first slot of cell c
 * (offset_out[n_cells] = n_particles), exactly as dsmc_load_state sorts.  Device-side
 * failure: if the inputs changed while the sort ran (for instance an overlapping call
 * on the shared scratch), the kernels write no record outside the outputs and set
 * offset_out[n_cells] = -1 instead; read it with the outputs after synchronising.
 * Scratch: a fixed 8 MiB array compiled into the library, held by every GPU that
 * loads it until the process exits.  Calls on one GPU that overlap in time (other
 * streams or threads) share it and race.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture on the device.  Limits: 1 <= n_cells <= 51200,
 * 1 <= n_particles <= 2^31 - 2^24; anything else returns DSMC_E_INVAL with a message
 * in dsmc_last_error().  No cudaMalloc, cudaFree or allocating library call is made. */
DSMC_API dsmc_status dsmc_sort_cells_static(const float* y, const float* vx, const float* vy,
                                           const float* vz, float* y_out, float* vx_out,
                                           float* vy_out, float* vz_out, int* offset_out,
                                           int n_particles, int n_cells, void* stream);

DSMC_API const char* dsmc_last_error(void);
DSMC_API const char* dsmc_status_string(dsmc_status s);

#ifdef __cplusplus
}
#endif

#endif /* DSMC_H */
