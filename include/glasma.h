/*
 * glasma.h -- C ABI of the GB300 colored-particle-in-cell (CPIC) library:
 * boost-invariant SU(3) Glasma fields coupled to Wong test particles
 * (Avramescu, Baran, Greco, Ipp, Mueller, Ruggieri, arXiv:2303.05599).
 *
 * One context holds one event: an N x N periodic transverse lattice with the
 * Glasma fields and an ensemble of test particles of up to GL_MAX_SPECIES
 * species.  All device memory lives in ONE workspace that the CALLER
 * allocates (cudaMalloc, or a PyTorch tensor) and owns; the library never
 * allocates device memory.  The context itself is a small host object owned
 * by the library (gl_create / gl_destroy).
 *
 * Every call is enqueued on the CUDA stream given to gl_create and returns
 * without waiting, except the uploads and downloads (gl_upload, gl_download,
 * gl_upload_native, gl_download_native, gl_batch_upload*) and the
 * observables, which wait for the stream.  Calls on one context must not overlap from several host
 * threads.  Errors are returned as gl_status; gl_error_string gives the last
 * message of a context.  No call aborts the process.
 *
 * Units.  The configuration is given in physical units (fm, GeV).  Inside,
 * everything is in lattice units with a = L/N: t = tau/a, dt = dtau/a,
 * momenta p a, masses m a.  The fields are stored as
 *   phi = g A_eta, pi = g a^2 P^eta, e_i = g a P^i   (Sec. 2.1),
 * Hermitian traceless, given by their 8 components X^a = 2 tr(X T^a) with
 * T^a = lambda^a/2.  The site fields are E^ = g a^2 E, B^ = g a^2 B (Sec. 3.2).
 *
 * Canonical host layouts used by gl_upload / gl_download (always double):
 *   GL_BUF_LINKS      [2][N*N][18]  U_x, U_y at step n; site s = y*N + x;
 *                                   3x3 complex row-major, (re, im) pairs
 *   GL_BUF_PHI        [N*N][8]      phi(n)
 *   GL_BUF_E          [2][N*N][8]   e_x, e_y at n - 1/2
 *   GL_BUF_PI         [N*N][8]      pi at n - 1/2
 *   GL_BUF_SITE       [6][N*N][8]   E_x, E_y, E_eta, B_x, B_y, B_eta at the
 *                                   last pushed time t_{n-1} (download only;
 *                                   GL_ERR_STATE before the first push, or
 *                                   when field steps since it overwrote them)
 *   GL_BUF_PARTICLES  [np][16]      x, y, eta, p^x, p^y, P_eta, Q^1..Q^8,
 *                                   p_T^2 at formation, species index;
 *                                   x, y in [0, N); P_eta = tau^2 p^eta
 *                                   (static and eikonal species: accumulated
 *                                   lab p_z)
 *   GL_BUF_JETS       [n_jets][44]  light-like jet-correlator probes: x0, y0,
 *                                   W (3x3 complex, row-major re/im), X_x, X_y,
 *                                   X_z (8 components each), see gl_config
 *   GL_BUF_ENERGY     [N*N]         energy density of the Glasma fields at the
 *                                   last pushed time t_{n-1}, under the same
 *                                   condition as GL_BUF_SITE (Figs. 6 and 9
 *                                   background): tr(E_x^2 + E_y^2 + E_eta^2 +
 *                                   B_x^2 + B_y^2 + B_eta^2) of the site fields,
 *                                   lattice units; the physical value is this
 *                                   / (g^2 a^4) (download only)
 *   GL_BUF_PTAU       [np]          temporal-constraint diagnostic (with the
 *                                   GL_CFG_PTAU_DIAGNOSTIC flag): p^tau of each
 *                                   particle integrated from its own equation of
 *                                   motion (Sec. 3.1, Euler with the state at t_n,
 *                                   started at the mass shell at the first push;
 *                                   NaN before that, and always for static and
 *                                   eikonal species), caller's order; compare
 *                                   with the mass shell of the GL_BUF_PARTICLES
 *                                   record; upload after GL_BUF_PARTICLES (which
 *                                   resets it to NaN)
 */
#ifndef GLASMA_H
#define GLASMA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GL_ABI_VERSION 1
#define GL_MAX_SPECIES 8

typedef enum {
    GL_OK = 0,
    GL_ERR_ARG = 1,      /* invalid argument or configuration */
    GL_ERR_CUDA = 2,     /* a CUDA runtime call or kernel launch failed */
    GL_ERR_STATE = 3,    /* call out of order (e.g. push without field step) */
    GL_ERR_TIMEOUT = 4,  /* a bounded device wait gave up */
    GL_ERR_NUMERIC = 5,  /* non-finite values or failed link matching at init */
    GL_ERR_SIZE = 6      /* workspace or host buffer of the wrong size */
} gl_status;

typedef enum { GL_FP64 = 0, GL_FP32_2ROW = 1 } gl_precision;

typedef enum {
    GL_BUF_LINKS = 0,
    GL_BUF_PHI = 1,
    GL_BUF_E = 2,
    GL_BUF_PI = 3,
    GL_BUF_SITE = 4,
    GL_BUF_PARTICLES = 5,
    GL_BUF_JETS = 6,
    GL_BUF_ENERGY = 7,
    GL_BUF_PTAU = 8
} gl_buffer;

/* One MV event (Sec. 2, parameters of Sec. 7.1). */
typedef struct {
    int32_t N;              /* lattice sites per transverse direction, >= 4 */
    int32_t Ns;             /* colour sheets per nucleus (eq. for the regularised correlator) */
    int32_t precision;      /* gl_precision */
    int32_t reunit_every;   /* FP32: re-unitarise links in FP64 every k steps (0: never); on GB300 an
                               FP64 re-unitarising step costs about 2.5 normal steps, 64 is a good period */
    double L_fm;            /* transverse box length */
    double g2mu_GeV;        /* MV parameter g^2 mu */
    double mIR_GeV;         /* infrared regulator of the Poisson kernel */
    double LambdaUV_GeV;    /* ultraviolet cutoff of the Poisson kernel (<= 0: none) */
    double dtau_over_a;     /* leapfrog time step in units of a */
    uint64_t seed;          /* Philox key of this event's random numbers */
    int32_t sort_every;     /* reorder particles by lattice row, motion class (Wong, static,
                               eikonal) and cell every k pushes (0: never); only the memory
                               order changes, downloads keep the caller's order */
    int32_t n_jets;         /* light-like jet-correlator probes (Sec. 5.2, light-like jets), >= 0:
                               each starts at a uniform (x0, y0) at tau = 0 (Philox counters
                               (j, 0, 4, 0)) and moves along +x at the speed of light, carrying
                               the Wilson line W of the x links it crosses (links at t_{n+1})
                               and X_i = sum dt W f_i W^+, f = (E_x, E_y - B_eta, E_eta + B_y)
                               at its cell at t_n; advanced by every push; single events only */
    uint32_t flags;         /* GL_CFG_* options, 0 for none */
    int32_t reserved;       /* must be 0 */
} gl_config;

/* gl_config.flags: integrate p^tau of every Wong particle from its own
 * equation of motion beside the mass shell (the temporal-constraint
 * diagnostic, GL_BUF_PTAU); costs one more read and write per particle and
 * push. */
#define GL_CFG_PTAU_DIAGNOSTIC 1u

/* One species of test particles (Sec. 3.2 and 7.1). */
typedef struct {
    double mass_GeV;        /* INFINITY: infinitely massive static quark (Sec. 5.1) */
    double tau_form_fm;     /* formation time; pushed from the first t_n >= tau_form */
    int64_t count;
    int32_t rep;            /* 0: fundamental charge (q2 = 4, q3 = 10/3); 1: adjoint (24, 0) */
    int32_t mom_mode;       /* 0: |p_T| = p0, uniform azimuth; 1: |p_T| ~ U[p0, p1], uniform
                               azimuth; 2: p^x = p0, p^y = 0; 3: eikonal light-like parton
                               along +x (Sec. 5.2): the path x = x0 + t is fixed, y and eta
                               stay, the momenta start at 0 and accumulate the kicks
                               dt Q.(E_x, E_y - B_eta, E_eta + B_y) (p^x, p^y, lab p_z in the
                               P_eta slot), and Q is rotated by the crossed x links; the mass
                               is not used */
    double p0_GeV, p1_GeV;
} gl_species;

/* Ensemble and field observables (Sec. 3.1 eq. for momentum broadening). */
typedef struct {
    int64_t step;                       /* field step n of the context */
    double tau_fm;                      /* tau of the particle state */
    int32_t n_species;
    uint32_t what;                      /* GL_OBS_* parts computed; the others are NaN (counts 0) */
    int64_t n_active[GL_MAX_SPECIES];   /* particles pushed at the last step */
    double sum_px2[GL_MAX_SPECIES];     /* sums over active particles, GeV^2 */
    double sum_py2[GL_MAX_SPECIES];
    double sum_pL2[GL_MAX_SPECIES];     /* p_L = lab p^z (static: accumulated) */
    double sum_dpT2[GL_MAX_SPECIES];    /* sum of p_T^2 - p_T^2(tau_form) */
    double casimir2_dev[GL_MAX_SPECIES];/* max |q2 - q2(R)| over particles */
    double casimir3_dev[GL_MAX_SPECIES];/* max |q3 - q3(R)| */
    double gauss_max;                   /* max over sites of |G(x)|, lattice units */
    double gauss_rms;
    double unitarity_max;               /* max over links of ||U U^+ - 1||_F */
    double mean_trE_T2;                 /* lattice means of tr(E_x^2 + E_y^2), tr E_eta^2, */
    double mean_trE_L2;                 /* tr(B_x^2 + B_y^2), tr B_eta^2 at the last pushed */
    double mean_trB_T2;                 /* time, lattice units (E^ = g a^2 E); NaN when */
                                        /* GL_BUF_SITE could not be downloaded */
    double mean_trB_L2;
} gl_obs;

typedef struct gl_ctx gl_ctx;

/* Bytes of device workspace a context with this configuration needs.
 * Returns 0 for an invalid configuration. */
size_t gl_workspace_bytes(const gl_config* cfg, const gl_species* species, int32_t n_species);

/* Create a context on the current CUDA device.  d_workspace: caller-owned
 * device memory of at least gl_workspace_bytes() bytes, 256-byte aligned,
 * kept alive until gl_destroy.  stream: a cudaStream_t (NULL = default). */
gl_status gl_create(const gl_config* cfg, const gl_species* species, int32_t n_species, void* d_workspace,
                    size_t workspace_bytes, void* stream, gl_ctx** out);

/* Release the host context (the workspace stays the caller's). */
gl_status gl_destroy(gl_ctx* ctx);

/* Message for the last error of ctx (or of gl_create when ctx is NULL). */
const char* gl_error_string(const gl_ctx* ctx);

/* MV initial condition at tau = 0 (Sec. 2.1): Gaussian colour charges on Ns
 * sheets per nucleus, Poisson solve by FFT, path-ordered Wilson lines, the
 * pure-gauge links of both nuclei, the Glasma links from the lattice matching
 * condition and E_eta(0).  Sets the step to 0.  GL_ERR_NUMERIC if the link
 * matching did not converge somewhere. */
gl_status glasma_init(gl_ctx* ctx);

/* Sample all particles (Sec. 3.2 and 4.2): uniform transverse positions,
 * eta = 0, momenta per species mode, classical charges Q = U Q0 U^+ with U
 * Haar-distributed. */
gl_status wong_init(gl_ctx* ctx);

/* Copy a host buffer in the canonical layout into the context (waits).
 * count = number of doubles; GL_ERR_SIZE if it does not match. */
gl_status gl_upload(gl_ctx* ctx, gl_buffer which, const double* host, size_t count);

/* Copy a context buffer out in the canonical layout (waits). */
gl_status gl_download(gl_ctx* ctx, gl_buffer which, double* host, size_t count);

/* Native snapshots: one part of a context's state as the bytes of its device
 * layout in the context's precision, for checkpoints that are restored into a
 * context created with the same gl_config and species (the bytes are opaque
 * and valid only there).  A native round trip restores the state bitwise,
 * particle order and p^tau diagnostic included, and moves fewer bytes than
 * the canonical layout (FP32: 224 B per site and 76 B per particle, against
 * 544 B and 128 B).
 *   GL_NATIVE_FIELDS     U, phi, e, pi of the current time slice
 *   GL_NATIVE_PARTICLES  every particle array, in device order (sorted), with
 *                        the species and original indices */
typedef enum { GL_NATIVE_FIELDS = 0, GL_NATIVE_PARTICLES = 1 } gl_native_part;

/* Size in bytes of a native part (0 for a NULL context or an unknown part). */
size_t gl_native_bytes(const gl_ctx* ctx, gl_native_part part);

/* Copy a native part to host memory of exactly gl_native_bytes() bytes
 * (waits).  GL_ERR_SIZE if bytes does not match, GL_ERR_ARG for an unknown
 * part. */
gl_status gl_download_native(gl_ctx* ctx, gl_native_part part, void* host, size_t bytes);

/* Copy a native part from host memory into the context (waits).  Like
 * gl_upload, it sets neither the step (gl_set_step) nor the site fields.
 * Particles: every species index must lie in [0, n_species) and every
 * original index in [0, np); the device checks both after the copy, and if
 * any is out of range it sets that entry to species 0 / its own position and
 * returns GL_ERR_ARG (the particle state is then unspecified, but every
 * later call stays within its arrays). */
gl_status gl_upload_native(gl_ctx* ctx, gl_native_part part, const void* host, size_t bytes);

/* Set the field step index n (t_n = n dt) of the uploaded state; the
 * particles are taken to be at the same time.  The uploaded fields stay the
 * current ones, so uploads may come before or after this call. */
gl_status gl_set_step(gl_ctx* ctx, int64_t step);

/* Advance the fields n_steps leapfrog steps (Sec. 2.1 equations of motion).
 * Particles that are then more than one step behind can no longer be pushed
 * (wong_push returns GL_ERR_STATE). */
gl_status glasma_step(gl_ctx* ctx, int32_t n_steps);

/* Interpolate E and B to the lattice sites at the particles' time t_n
 * (Sec. 3.2 formulas; GL_BUF_SITE).  Needs exactly one glasma_step since the
 * particles' time (the momenta at n - 1/2 and n + 1/2 are both used).
 * wong_push calls it itself when it has not been called for this step. */
gl_status wong_site_fields(gl_ctx* ctx);

/* Push the particles from t_n to t_{n+1} (Sec. 3.1 and 3.2: site E/B
 * interpolation, Euler step of Wong's equations, NGP colour rotation with the
 * crossed links and the rapidity Wilson line).  Needs exactly one preceding
 * glasma_step since the particles' time. */
gl_status wong_push(gl_ctx* ctx);

/* n_steps coupled steps: glasma_step(1) + wong_push each. */
gl_status gl_step_coupled(gl_ctx* ctx, int32_t n_steps);

/* Choose the launch shape of the field kernel and the push block size (64,
 * 128, 256) for this context from timed trial launches.  FP32 field shapes
 * (the strip kernel: a warp walks up a strip of 32 columns): 0 = 16 warps per
 * SM, 1 = 12, 2 = 8 (more registers per thread each).  FP64 tiles: 1 = 32x4,
 * 2 = 32x2.  Results do not depend on the shape.  Waits.  Needs the
 * particles at the fields' time; the trials write only buffers that the next
 * coupled step rewrites.  Outputs may be NULL. */
gl_status gl_autotune(gl_ctx* ctx, int32_t* tile_shape, int32_t* push_block);

/* Trial timings of the last gl_autotune, ms: field_ms[4] by field shape,
 * push_ms[3] by block size (0 where not tried). */
gl_status gl_tuning(const gl_ctx* ctx, float* field_ms, float* push_ms);

/* Ensemble sums and field checks at the current time (waits): the same as
 * gl_observables_ex(ctx, GL_OBS_ALL, out). */
gl_status observables(gl_ctx* ctx, gl_obs* out);

/* Parts of gl_obs to compute.  GL_OBS_PARTICLES: the per-species sums and
 * Casimir drifts (a pass over the particles; per-particle values in the
 * context's precision, accumulated in FP64).  GL_OBS_FIELDS: Gauss residual,
 * link unitarity and the site-field means (an FP64 pass over the lattice,
 * which on GPUs with slow FP64 costs more than a coupled step: meant for
 * report intervals). */
#define GL_OBS_PARTICLES 1u
#define GL_OBS_FIELDS 2u
#define GL_OBS_ALL 3u

/* Jet-correlator result (waits): out[i] = mean over the probes of X_i . X_i
 * = sum_a (X_i^a)^2 for i = x, y, z, in GeV^2.  A parton of charge Q0 on a
 * probe's path receives the kicks Q0 . X_i, so the charge-averaged momentum
 * broadening of a light-like parton in representation R is
 * <delta p_i^2> = (q2(R) / 8) out[i] (q2 = 4 fundamental, 24 adjoint).
 * GL_ERR_STATE if the context has no probes. */
gl_status gl_jets_observables(gl_ctx* ctx, double* out3);

/* observables() restricted to the parts in `what` (waits).  The values of the
 * other parts are NaN and their counts 0; out->what records the parts
 * computed.  GL_ERR_ARG for a null pointer or unknown bits in `what`. */
gl_status gl_observables_ex(gl_ctx* ctx, uint32_t what, gl_obs* out);

/* ---- Batches of events ------------------------------------------------
 * Many independent MV events (the paper averages its observables over many
 * events, Sec. 7.1), possibly of different N, advanced together: one coupled
 * step of the whole batch is one field launch over the sites of every event
 * and one push launch over the particles of every event, captured once in a
 * CUDA graph and replayed; the field launch of step s runs concurrently with
 * the push of step s - 1 (the schedule is chosen by gl_batch_autotune).  All
 * events share the precision, the time step dtau/a and the re-unitarisation
 * period; they start at tau = 0 together.  Each event's particles are sorted
 * by row, motion class and cell when sampled or uploaded and every sort_every steps (all events in
 * one launch per sort stage).  Jet-correlator probes (n_jets > 0) are not
 * supported in batches (GL_ERR_ARG). */
typedef struct gl_batch gl_batch;

/* Workspace bytes for n_events events; cfgs[n_events], species
 * [n_events][n_species] (event e's species at species + e * n_species). */
size_t gl_batch_workspace_bytes(const gl_config* cfgs, const gl_species* species, int32_t n_species,
                                int32_t n_events);

/* Create a batch in one caller-owned workspace (256-byte aligned); stream must
 * be a non-default stream (graph capture). */
gl_status gl_batch_create(const gl_config* cfgs, const gl_species* species, int32_t n_species, int32_t n_events,
                          void* d_workspace, size_t workspace_bytes, void* stream, gl_batch** out);
gl_status gl_batch_destroy(gl_batch* batch);
const char* gl_batch_error_string(const gl_batch* batch);

/* Context of event e (owned by the batch): use it for uploads, downloads and
 * per-event observables. */
gl_ctx* gl_batch_event(gl_batch* batch, int32_t e);

/* glasma_init and wong_init of every event. */
gl_status gl_batch_init(gl_batch* batch);

/* Choose the launch shapes and the step schedule from timed trial launches
 * that do not change the state (waits).  Chosen: the field launch shape (FP32
 * strips: 0 = 16 warps per SM, 1 = 12, 2 = 8, the rows of all events' strips
 * split evenly among the resident warps; FP64 batches use the 32x4 tile, 1),
 * by the whole step as for the push; the block size (128,
 * 256, 512) and chunk (particles per block: 128, 256, 512, 1024) of the
 * separate push kernel, by the time of the whole overlapped step, not of the
 * push alone; and the steady-state step, either
 *   - the field and push kernels on two streams, the push with one block per
 *     chunk of particles or (push_grid 1, 2) that many resident 128-thread
 *     blocks per SM launched ahead of the field kernel (chunks of 1024), or
 *   - one persistent fused launch that interleaves field items (FP32: 24
 *     rows of a strip for each of a block's 8 warps; FP64: 32x4 tiles) and
 *     push chunks of 512, 1024 or 2048 particles.
 * The push and whole-step trials run on copies of the particles in the spare
 * particle buffers that sorting provides; if an event with particles has
 * sort_every = 0, only the field launch shape is tuned.  Outputs may be NULL. */
gl_status gl_batch_autotune(gl_batch* batch, int32_t* tile_shape, int32_t* push_block);

/* Set the launch shapes and schedule directly (values as above: push_chunk
 * 128, 256, 512, 1024 or 2048; fused 0 or 1; push_grid 0, 1 or 2, ignored
 * when fused).  Results do not depend on them.
 * GL_ERR_ARG for other values or a tile other than 32x4 (1) in an FP64 batch. */
gl_status gl_batch_set_launch(gl_batch* batch, int32_t tile_shape, int32_t push_block, int32_t push_chunk,
                              int32_t fused, int32_t push_grid);

/* The launch shapes and schedule in use.  Outputs may be NULL. */
gl_status gl_batch_get_launch(const gl_batch* batch, int32_t* tile_shape, int32_t* push_block,
                              int32_t* push_chunk, int32_t* fused, int32_t* push_grid);

/* FP32 batches: the rows per strip segment of the field kernel that the next
 * step launches (the unit of work of one warp: the strips of all events are
 * cut into segments of this length and spread over the resident warps; set by
 * gl_batch_set_segment_rows, chosen by gl_batch_autotune from trial launches,
 * or else by a cost model of the launch shape's resident warps).  Results do
 * not depend on it.  0 for FP64 batches or NULL. */
int32_t gl_batch_segment_rows(const gl_batch* batch);

/* FP32 batches: fix the rows per strip segment for the current field launch
 * shape (set the shape first, with gl_batch_set_launch); 0 returns to the cost
 * model's choice.  Results do not depend on it.  GL_ERR_ARG for rows < 0 or
 * > 65536, or a non-zero value in an FP64 batch. */
gl_status gl_batch_set_segment_rows(gl_batch* batch, int32_t rows);

/* Trial timings of the last autotune, ms (0 where not tried): field_ms[3] by
 * field launch shape (the fastest of its segment lengths); push_ms[3] by push
 * block size; step_ms[8] for a whole step: [0] two streams (the fastest field
 * shape, push block and chunk sizes), [1..3] fused with push chunks of 512,
 * 1024, 2048, [4..7] two streams with push_grid 1 beside field shape 0 (FP64:
 * the 32x8 slot) and 1, then push_grid 2 beside the same (the best of the
 * other FP32 shapes in the first slot). */
gl_status gl_batch_tuning(const gl_batch* batch, float* field_ms, float* push_ms, float* step_ms);

/* n_steps coupled steps of every event (all events at one common step). */
gl_status gl_batch_step(gl_batch* batch, int32_t n_steps);

/* The same n_steps with direct launches and CUDA events around every field
 * and push launch; field_ms and push_ms receive the summed kernel durations
 * (waits).  For measurement. */
gl_status gl_batch_step_timed(gl_batch* batch, int32_t n_steps, double* field_ms, double* push_ms);

/* gl_upload of buffer `which` of every event: host[e] holds count[e] doubles
 * in the canonical layout for event e.  The copies and conversions of all
 * events are enqueued on the batch stream and waited for once, at the end, so
 * a restore of many events pays one wait per buffer instead of one per event
 * (waits).  Errors as gl_upload, reported for the first failing event; the
 * events before it are uploaded. */
gl_status gl_batch_upload(gl_batch* batch, gl_buffer which, const double* const* host, const size_t* count);

/* gl_upload_native of part `part` of every event: host[e] holds bytes[e]
 * bytes for event e.  Events alternate between two streams, as in
 * gl_batch_upload, with one wait at the end (waits).  Errors as
 * gl_upload_native, reported for the first failing event. */
gl_status gl_batch_upload_native(gl_batch* batch, gl_native_part part, const void* const* host, const size_t* bytes);

/* observables() of every event into out[n_events] (waits). */
gl_status gl_batch_observables(gl_batch* batch, gl_obs* out);

/* gl_observables_ex of every event into out[n_events] (waits).  The particle
 * sums of all events are reduced by one launch pair and the results of all
 * events come back in one device-to-host copy; each event's values are
 * bitwise those of gl_observables_ex on that event alone. */
gl_status gl_batch_observables_ex(gl_batch* batch, uint32_t what, gl_obs* out);

/* gl_batch_observables_ex in two halves, so that the results of one step can
 * be read back while the next runs.  _begin enqueues the reductions of the
 * events' current state (`what`: GL_OBS_* bits) and their copy into one of
 * two pinned host slots, and returns without waiting; _end waits for the
 * oldest outstanding request and fills out[n_events] with its results,
 * bitwise those gl_batch_observables_ex would have given at the time of the
 * _begin.  At most two requests are outstanding (a third _begin, an _end
 * with none, or gl_batch_observables_ex with one outstanding: GL_ERR_STATE).
 * Steps enqueued between _begin and _end run after the request on the
 * batch's stream.  gl_batch_destroy waits for outstanding requests. */
gl_status gl_batch_observables_begin(gl_batch* batch, uint32_t what);
gl_status gl_batch_observables_end(gl_batch* batch, gl_obs* out);

/* Bytes of one event's results in the one device-to-host copy of a batch
 * observables request: GL_MAX_SPECIES x 7 per-species values and the 7 field
 * check values, FP64, which the host unpacks into the event's gl_obs record.
 * Host only: no GPU work, no error. */
size_t gl_batch_obs_row_bytes(void);

/* Largest particle count gl_ensemble_sums_noalloc accepts. */
#define GL_NOALLOC_MAX_PARTICLES 2097152

/* Per-species ensemble sums for callers that cannot allocate device memory
 * (a host that owns every device allocation itself, or a process that must not
 * grow its device footprint after start-up).  The paper has no counterpart:
 * this is a service of the library, computing the particle sums of
 * observables() from particle records the caller already holds on the device.
 *
 * d_particles: device array of np canonical FP64 records [np][16] (the
 *   GL_BUF_PARTICLES layout, lattice units); np <= GL_NOALLOC_MAX_PARTICLES,
 *   GL_ERR_SIZE otherwise.
 * mass, rep, kind: host arrays of n_species entries (1..GL_MAX_SPECIES):
 *   lattice mass m a, charge representation (0 F, 1 A) and motion class
 *   (0 Wong particle, 1 static quark of infinite mass, 2 eikonal light-like
 *   parton of mom_mode 3).  p_L is the lab p_z built from P_eta = tau^2 p^eta
 *   for class 0 and the accumulated longitudinal momentum in the P_eta slot
 *   for classes 1 and 2, as in observables().  Other values: GL_ERR_ARG.
 * active_mask: bit s set if species s is included; t: lattice time t_n used
 *   for p_L.
 * A NaN in a record propagates: into the sums, and into the Casimir maxima.
 * d_out: device array of n_species x 7 doubles per species: count, sum p_x^2,
 *   sum p_y^2, sum p_L^2, sum (p_T^2 - p_T^2 at formation), max |q2 - q2(R)|,
 *   max |q3 - q3(R)|  (lattice units).
 * stream: cudaStream_t.  Asynchronous on the stream.
 *
 * Allocates nothing: its scratch is a fixed 917,504-byte array compiled into
 * the library, which every GPU that loads the library keeps until the process
 * exits.  The first call on a device looks up that array's device address; make
 * that first call before any stream capture.  All calls share the one array, so
 * calls that overlap on the GPU (different streams, or different host threads
 * on one device) race and must be serialised by the caller. */
gl_status gl_ensemble_sums_noalloc(const double* d_particles, int64_t np, int32_t n_species, const double* mass,
                                   const int32_t* rep, const int32_t* kind, uint32_t active_mask, double t,
                                   double* d_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif
