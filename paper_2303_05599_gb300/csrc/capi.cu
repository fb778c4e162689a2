// C ABI of the library (declared in include/glasma.h): context, workspace
// carving, call ordering and status codes.  Every numerical step runs in the
// kernels of field.cu, particles.cu, init.cu and obs.cu.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "internal.h"

namespace gl {
size_t init_scratch_bytes(int64_t Vn);
void launch_parts_convert(int prec, void* parts, int64_t np, double* stg, int to_device, cudaStream_t st);
}  // namespace gl

using namespace gl;

static const double HBARC = 0.1973269804;  // GeV fm
static const int MAX_BLOCKS = FIELD_OBS_MAX_BLOCKS;  // rows of per-block partial results

struct gl_ctx {
    gl_config cfg;
    int ns;
    gl_species sp[GL_MAX_SPECIES];
    int N;
    int prec;
    int64_t Vn, np;
    int64_t off[GL_MAX_SPECIES + 1];
    double a_fm, aG, dt, g2mu_a, m_a, Lambda_a;
    double t_form[GL_MAX_SPECIES];
    double p0[GL_MAX_SPECIES], p1[GL_MAX_SPECIES];
    int rep[GL_MAX_SPECIES], mode[GL_MAX_SPECIES];
    SpeciesParams spp;
    double q0[2][8];
    double q2ref[GL_MAX_SPECIES], q3ref[GL_MAX_SPECIES];
    cudaStream_t stream;
    cudaStream_t aux;   // push stream of the overlapped coupled step (created on first use)
    cudaEvent_t ev_f, ev_p;
    char* ws;
    size_t ws_bytes;
    void* field[2];
    void* site_buf[2];  // site fields at t_n live in site_buf[n & 1]
    void* parts;
    void* parts_alt;    // second particle buffer for the cell sort
    void* sort_scratch;
    int sort_ok;
    int64_t n_jets;       // light-like jet-correlator probes (0: none)
    void* jets;
    double* jet_partials; // 1024 x 3 block partials, then the 3 results
    void* scratch;
    size_t scratch_bytes;
    double* partials;
    double* obs_dev;
    int* d_bad;
    int cur;
    int64_t step, pstep;
    int64_t site_time[2];  // time index n whose site fields site_buf[n & 1] holds (-1: none)
    int tile;           // field-kernel launch shape (gl_autotune)
    int seg;            // FP32: rows per strip segment (gl_autotune; 0: the cost model's)
    int push_block;     // push block size (gl_autotune)
    float tune_field_ms[4], tune_push_ms[3];
    char err[256];
};

static char g_create_err[256] = "";

// site-field buffer of time t_n
static inline void* site_at(const gl_ctx* c, int64_t n) { return c->site_buf[n & 1]; }
// the site fields of time n are held (written by a field step or site_once
// and not overwritten since)
static inline bool site_holds(const gl_ctx* c, int64_t n) { return n >= 0 && c->site_time[n & 1] == n; }
static inline void site_forget(gl_ctx* c) { c->site_time[0] = c->site_time[1] = -1; }

extern "C" {
static uint32_t active_mask(const gl_ctx* c, int64_t n);
static void observables_launch(gl_ctx* c, uint32_t what);
static gl_status observables_read(gl_ctx* c, uint32_t what, gl_obs* o);
static gl_status transfer_enqueue(gl_ctx* c, gl_buffer which, double* host, size_t count, int to_device);
static void observables_fill(const gl_ctx* c, uint32_t what, const double* host, gl_obs* o);
static gl_status native_upload_enqueue(gl_ctx* c, int part, const void* host, size_t bytes, cudaStream_t st);
static gl_status native_check(gl_ctx* c, int part, const void* host, size_t bytes);
}

static size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

static gl_status fail(gl_ctx* c, gl_status s, const char* msg) {
    char* dst = c ? c->err : g_create_err;
    snprintf(dst, 256, "%s", msg);
    return s;
}

static gl_status check_cuda(gl_ctx* c, const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char m[256];
        snprintf(m, sizeof m, "%s: %s", where, cudaGetErrorString(e));
        return fail(c, GL_ERR_CUDA, m);
    }
    return GL_OK;
}

static const char* validate(const gl_config* cfg, const gl_species* sp, int32_t ns) {
    if (!cfg) return "null config";
    if (cfg->N < 4 || cfg->N > 32768) return "N must be in [4, 32768]";
    if (cfg->Ns < 1) return "Ns must be >= 1";
    if (cfg->precision != GL_FP64 && cfg->precision != GL_FP32_2ROW) return "unknown precision";
    if (!(cfg->L_fm > 0) || !(cfg->dtau_over_a > 0)) return "L_fm and dtau_over_a must be positive";
    if (ns < 0 || ns > GL_MAX_SPECIES) return "n_species must be in [0, 8]";
    if (ns > 0 && !sp) return "null species";
    int64_t np = 0;
    for (int k = 0; k < ns; k++) {
        if (sp[k].count < 0) return "negative particle count";
        if (sp[k].rep != 0 && sp[k].rep != 1) return "rep must be 0 or 1";
        if (sp[k].mom_mode < 0 || sp[k].mom_mode > 3) return "mom_mode must be 0, 1, 2 or 3";
        if (!(sp[k].mass_GeV >= 0)) return "mass must be >= 0 or INFINITY";
        np += sp[k].count;
    }
    if (np >= ((int64_t)1 << 31)) return "at most 2^31 - 1 particles";
    if (cfg->n_jets < 0 || cfg->n_jets > (1 << 24)) return "n_jets must be in [0, 2^24]";
    if (cfg->flags & ~GL_CFG_PTAU_DIAGNOSTIC) return "unknown flags";
    if (cfg->reserved != 0) return "reserved must be 0";
    return nullptr;
}

struct Carve {
    size_t field, site, parts, parts_alt, sort, jets, jet_partials, scratch, partials, obs, bad, total;
};

static Carve carve(const gl_config* cfg, int64_t np, int ns) {
    const int64_t Vn = (int64_t)cfg->N * cfg->N;
    const int prec = cfg->precision;
    Carve c;
    size_t o = 0;
    c.field = o; o += 2 * a256(field_bytes(prec, Vn));
    c.site = o; o += 2 * a256(site_bytes(prec, Vn));
    c.parts = o; o += a256(particle_bytes(prec, np));
    const bool sorting = cfg->sort_every > 0 && np > 0 && sort_supported(Vn, ns, np);
    c.parts_alt = o; o += sorting ? a256(particle_bytes(prec, np)) : 0;
    c.sort = o; o += sorting ? a256(sort_scratch_bytes(Vn, np, ns)) : 0;
    const size_t nj = cfg->n_jets > 0 ? (size_t)cfg->n_jets : 0;
    c.jets = o; o += nj ? a256(nj * JET_LEN * (prec == 0 ? 8 : 4)) : 0;
    c.jet_partials = o; o += nj ? a256((1024 * 3 + 3) * sizeof(double)) : 0;
    size_t sc = init_scratch_bytes(Vn);
    size_t stg = (size_t)Vn * 6 * 8 * sizeof(double);
    if (stg > sc) sc = stg;
    if ((size_t)np * 16 * sizeof(double) > sc) sc = (size_t)np * 16 * sizeof(double);
    if (nj * JET_LEN * sizeof(double) > sc) sc = nj * JET_LEN * sizeof(double);
    c.scratch = o; o += a256(sc);
    c.partials = o; o += a256((size_t)MAX_BLOCKS * (GL_MAX_SPECIES * PO_N + FO_N) * sizeof(double));
    c.obs = o; o += a256((GL_MAX_SPECIES * PO_N + FO_N) * sizeof(double));
    c.bad = o; o += 256;
    c.total = o;
    return c;
}

// Q0 of the fundamental classical charge: Q^8 = s is the root near -1.06 of
// s^3 - 12 s - 20/sqrt(3) = 0 (q2 = 4, q3 = 10/3 with only Q^5, Q^8 nonzero),
// taken from the trigonometric form of the depressed-cubic roots; Q^5 = -sqrt(4 - s^2).
static void q0_vectors(double q0[2][8]) {
    memset(q0, 0, sizeof(double) * 16);
    const double p = -12.0, q = -20.0 / sqrt(3.0);
    const double r = 2.0 * sqrt(-p / 3.0);
    const double th = acos((3.0 * q / (2.0 * p)) * sqrt(-3.0 / p)) / 3.0;
    const double s = r * cos(th - 2.0 * M_PI / 3.0);
    q0[0][7] = s;
    q0[0][4] = -sqrt(4.0 - s * s);
    q0[1][0] = sqrt(24.0);
}

namespace gl {
// read-only view of a context for the batch (batch.cu)
void ctx_view(const gl_ctx* c, CtxView* v) {
    v->field[0] = c->field[0];
    v->field[1] = c->field[1];
    v->site[0] = c->site_buf[0];
    v->site[1] = c->site_buf[1];
    v->parts = c->parts;
    v->N = c->N;
    v->prec = c->prec;
    v->cur = c->cur;
    v->step = c->step;
    v->pstep = c->pstep;
    v->np = c->np;
    v->dt = c->dt;
    for (int k = 0; k < GL_MAX_SPECIES; k++) {
        v->mass[k] = c->spp.mass[k];
        v->motion[k] = c->spp.motion[k];
        v->t_form[k] = c->t_form[k];
    }
    v->ns = c->ns;
    v->parts_alt = c->parts_alt;
    v->sort_every = c->sort_ok ? c->cfg.sort_every : 0;
    v->ptau_diag = c->spp.ptau_diag;
    v->sort_scratch = c->sort_scratch;
}
// record that the batch advanced this event by `steps` coupled steps
void ctx_advance(gl_ctx* c, int64_t steps) {
    c->step += steps;
    c->pstep += steps;
    c->cur = (int)(c->step & 1);
    // the last push of the batch read the site fields of pstep - 1, written
    // by the field step of that time; the other buffer is not tracked
    c->site_time[(c->pstep - 1) & 1] = c->pstep - 1;
    c->site_time[c->pstep & 1] = -1;
}
size_t ctx_workspace_bytes(const gl_config* cfg, const gl_species* sp, int32_t ns) {
    return gl_workspace_bytes(cfg, sp, ns);
}
// the particle-observables launch of a context, for the batched reduction
void ctx_obs_event(const gl_ctx* c, ObsEvent* o) {
    const int64_t pushed = c->pstep > 0 ? c->pstep - 1 : -1;
    o->parts = c->parts;
    o->np = c->np;
    o->t = c->pstep * c->dt;
    o->mask = pushed >= 0 ? active_mask(c, pushed) : 0u;
    o->sp = c->spp;
    for (int k = 0; k < GL_MAX_SPECIES; k++) { o->q2ref[k] = c->q2ref[k]; o->q3ref[k] = c->q3ref[k]; }
    o->partials = c->partials;
    o->out = c->obs_dev;
    o->fo.fields = c->field[c->cur];
    o->fo.site = site_at(c, c->pstep - 1);
    o->fo.N = c->N;
    o->fo.block_begin = 0;
    o->fo.nblocks = field_obs_blocks(c->N);
    o->fo.partials = c->partials + (size_t)MAX_BLOCKS * GL_MAX_SPECIES * PO_N;
    o->fo.out = c->obs_dev + GL_MAX_SPECIES * PO_N;
}
gl_status ctx_upload_enqueue(gl_ctx* c, gl_buffer which, const double* host, size_t count, cudaStream_t st) {
    const cudaStream_t own = c->stream;
    c->stream = st;  // the copy, the conversion and a particle sort go to st
    const gl_status s = ::transfer_enqueue(c, which, (double*)host, count, 1);
    c->stream = own;
    return s;
}
gl_status ctx_upload_native_copy(gl_ctx* c, int part, const void* host, size_t bytes, cudaStream_t st) {
    if (gl_status s = ::native_check(c, part, host, bytes)) return s;
    if (bytes == 0) return GL_OK;
    cudaMemcpyAsync(part == GL_NATIVE_FIELDS ? c->field[c->cur] : c->parts, host, bytes, cudaMemcpyHostToDevice, st);
    return check_cuda(c, "gl_batch_upload_native");
}
PartsCheckEv ctx_parts_check_event(const gl_ctx* c) {
    PartsCheckEv e;
    e.parts = c->parts;
    e.np = c->np;
    e.ns = c->ns;
    e.block_begin = 0;
    e.nblocks = parts_check_blocks(c->np);
    return e;
}
void ctx_obs_fill(const gl_ctx* c, uint32_t what, const double* host, gl_obs* o) {
    ::observables_fill(c, what, host, o);
}
}  // namespace gl

extern "C" {

size_t gl_workspace_bytes(const gl_config* cfg, const gl_species* sp, int32_t ns) {
    if (validate(cfg, sp, ns)) return 0;
    int64_t np = 0;
    for (int k = 0; k < ns; k++) np += sp[k].count;
    return carve(cfg, np, ns).total;
}

gl_status gl_create(const gl_config* cfg, const gl_species* sp, int32_t ns, void* d_workspace, size_t bytes,
                    void* stream, gl_ctx** out) {
    if (!out) return fail(nullptr, GL_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (const char* m = validate(cfg, sp, ns)) return fail(nullptr, GL_ERR_ARG, m);
    if (!d_workspace || ((uintptr_t)d_workspace & 255)) return fail(nullptr, GL_ERR_ARG, "workspace must be 256-byte aligned");
    gl_ctx* c = new (std::nothrow) gl_ctx;
    if (!c) return fail(nullptr, GL_ERR_ARG, "host allocation failed");
    memset(c, 0, sizeof *c);
    c->cfg = *cfg;
    c->ns = ns;
    c->N = cfg->N;
    c->prec = cfg->precision;
    c->Vn = (int64_t)cfg->N * cfg->N;
    c->np = 0;
    c->off[0] = 0;
    for (int k = 0; k < ns; k++) {
        c->sp[k] = sp[k];
        c->np += sp[k].count;
        c->off[k + 1] = c->np;
    }
    Carve cv = carve(cfg, c->np, ns);
    if (bytes < cv.total) {
        delete c;
        return fail(nullptr, GL_ERR_SIZE, "workspace smaller than gl_workspace_bytes()");
    }
    c->ws = (char*)d_workspace;
    c->ws_bytes = bytes;
    c->field[0] = c->ws + cv.field;
    c->field[1] = c->ws + cv.field + a256(field_bytes(c->prec, c->Vn));
    c->site_buf[0] = c->ws + cv.site;
    c->site_buf[1] = c->ws + cv.site + a256(site_bytes(c->prec, c->Vn));
    c->parts = c->ws + cv.parts;
    c->sort_ok = cfg->sort_every > 0 && c->np > 0 && sort_supported(c->Vn, ns, c->np);
    c->parts_alt = c->sort_ok ? c->ws + cv.parts_alt : nullptr;
    c->sort_scratch = c->sort_ok ? c->ws + cv.sort : nullptr;
    c->n_jets = cfg->n_jets;
    c->jets = c->n_jets ? c->ws + cv.jets : nullptr;
    c->jet_partials = c->n_jets ? (double*)(c->ws + cv.jet_partials) : nullptr;
    c->scratch = c->ws + cv.scratch;
    c->scratch_bytes = cv.partials - cv.scratch;
    c->partials = (double*)(c->ws + cv.partials);
    c->obs_dev = (double*)(c->ws + cv.obs);
    c->d_bad = (int*)(c->ws + cv.bad);
    c->stream = (cudaStream_t)stream;
    // lattice units (same expressions as the Python workload definitions)
    c->a_fm = cfg->L_fm / cfg->N;
    c->aG = cfg->L_fm / cfg->N / HBARC;
    c->dt = cfg->dtau_over_a;
    c->g2mu_a = cfg->g2mu_GeV * (cfg->L_fm / cfg->N / HBARC);
    c->m_a = cfg->mIR_GeV * (cfg->L_fm / cfg->N / HBARC);
    c->Lambda_a = cfg->LambdaUV_GeV > 0 ? cfg->LambdaUV_GeV * (cfg->L_fm / cfg->N / HBARC) : 0.0;
    q0_vectors(c->q0);
    c->spp.n_species = ns;
    c->spp.ptau_diag = (cfg->flags & GL_CFG_PTAU_DIAGNOSTIC) != 0;
    for (int k = 0; k < GL_MAX_SPECIES; k++) {
        const bool on = k < ns;
        const bool st = on && isinf(sp[k].mass_GeV);
        c->spp.motion[k] = st ? MOTION_STATIC : (on && sp[k].mom_mode == 3 ? MOTION_EIKONAL : MOTION_WONG);
        c->spp.mass[k] = on ? (st ? INFINITY : sp[k].mass_GeV * c->aG) : 0.0;
        c->t_form[k] = on ? sp[k].tau_form_fm * cfg->N / cfg->L_fm : 0.0;
        c->p0[k] = on ? sp[k].p0_GeV * c->aG : 0.0;
        c->p1[k] = on ? sp[k].p1_GeV * c->aG : 0.0;
        c->rep[k] = on ? sp[k].rep : 0;
        c->mode[k] = on ? sp[k].mom_mode : 0;
        c->q2ref[k] = c->rep[k] == 1 ? 24.0 : 4.0;
        c->q3ref[k] = c->rep[k] == 1 ? 0.0 : 10.0 / 3.0;
    }
    c->cur = 0;
    c->step = c->pstep = 0;
    site_forget(c);
    c->tile = 0;
    c->seg = 0;
    c->push_block = 128;
    *out = c;
    return GL_OK;
}

gl_status gl_destroy(gl_ctx* c) {
    if (!c) return GL_ERR_ARG;
    if (c->aux) {
        cudaStreamSynchronize(c->aux);
        cudaEventDestroy(c->ev_f);
        cudaEventDestroy(c->ev_p);
        cudaStreamDestroy(c->aux);
    }
    delete c;
    return GL_OK;
}

const char* gl_error_string(const gl_ctx* c) { return c ? c->err : g_create_err; }

// reorder the particles by row, motion class and cell (memory order only)
static void sort_particles(gl_ctx* c) {
    if (!c->sort_ok) return;
    launch_sort(c->prec, c->parts, c->parts_alt, c->np, c->N, c->ns, c->spp.motion, c->sort_scratch, c->stream);
    void* tmp = c->parts;
    c->parts = c->parts_alt;
    c->parts_alt = tmp;
}
}  // extern "C"
void gl::ctx_sort(gl_ctx* c) { sort_particles(c); }
void gl::ctx_swap_parts(gl_ctx* c) {
    void* tmp = c->parts;
    c->parts = c->parts_alt;
    c->parts_alt = tmp;
}
extern "C" {

static uint32_t active_mask(const gl_ctx* c, int64_t n) {
    uint32_t m = 0;
    const double t = n * c->dt;
    for (int k = 0; k < c->ns; k++)
        if (t >= c->t_form[k]) m |= 1u << k;
    return m;
}

gl_status glasma_init(gl_ctx* c) {
    gl::ApiRange range_("glasma_init");
    if (!c) return GL_ERR_ARG;
    launch_mv_init(c->prec, c->field[c->cur], c->scratch, c->N, c->cfg.Ns, c->g2mu_a, c->m_a, c->Lambda_a,
                   c->cfg.seed, c->d_bad, c->stream);
    for (int k = 0; k < 2; k++) cudaMemsetAsync(c->site_buf[k], 0, site_bytes(c->prec, c->Vn), c->stream);
    if (gl_status s = check_cuda(c, "glasma_init")) return s;
    int bad = 0;
    cudaMemcpyAsync(&bad, c->d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return check_cuda(c, "glasma_init sync");
    c->step = c->pstep = 0;
    site_forget(c);
    if (bad) {
        char m[128];
        snprintf(m, sizeof m, "link matching did not converge on %d links", bad);
        return fail(c, GL_ERR_NUMERIC, m);
    }
    return GL_OK;
}

gl_status wong_init(gl_ctx* c) {
    gl::ApiRange range_("wong_init");
    if (!c) return GL_ERR_ARG;
    launch_sample(c->prec, c->parts, c->np, c->N, c->cfg.seed, c->off, c->ns, c->rep, c->mode, c->p0, c->p1, c->q0,
                  c->stream);
    sort_particles(c);
    if (c->n_jets) launch_jets_init(c->prec, c->jets, c->n_jets, c->N, c->cfg.seed, c->stream);
    c->pstep = c->step;
    return check_cuda(c, "wong_init");
}

static size_t expected_count(const gl_ctx* c, gl_buffer which) {
    switch (which) {
        case GL_BUF_LINKS: return (size_t)2 * c->Vn * 18;
        case GL_BUF_PHI: return (size_t)c->Vn * 8;
        case GL_BUF_E: return (size_t)2 * c->Vn * 8;
        case GL_BUF_PI: return (size_t)c->Vn * 8;
        case GL_BUF_SITE: return (size_t)6 * c->Vn * 8;
        case GL_BUF_PARTICLES: return (size_t)c->np * 16;
        case GL_BUF_JETS: return (size_t)c->n_jets * JET_LEN;
        case GL_BUF_ENERGY: return (size_t)c->Vn;
        case GL_BUF_PTAU: return (size_t)c->np;
    }
    return 0;
}

// the copies and conversions of one transfer, enqueued on the context's
// stream (the caller waits)
static gl_status transfer_enqueue(gl_ctx* c, gl_buffer which, double* host, size_t count, int to_device) {
    if (!c || (!host && count)) return GL_ERR_ARG;
    if ((int)which < 0 || (int)which > GL_BUF_PTAU) return fail(c, GL_ERR_ARG, "unknown buffer");
    if (count != expected_count(c, which)) return fail(c, GL_ERR_SIZE, "host buffer size does not match");
    if (to_device && (which == GL_BUF_SITE || which == GL_BUF_ENERGY))
        return fail(c, GL_ERR_ARG, "site fields and energy density are download-only");
    if ((which == GL_BUF_SITE || which == GL_BUF_ENERGY) && !site_holds(c, c->pstep - 1))
        return fail(c, GL_ERR_STATE, "the site fields of the last pushed time are not held (no push yet, or later "
                                     "field steps overwrote them)");
    if (count == 0) return GL_OK;
    double* stg = (double*)c->scratch;
    if (to_device) cudaMemcpyAsync(stg, host, count * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (which == GL_BUF_PARTICLES) {
        launch_parts_convert(c->prec, c->parts, c->np, stg, to_device, c->stream);
        if (to_device) sort_particles(c);
    } else if (which == GL_BUF_JETS) {
        launch_jets_convert(c->prec, c->jets, c->n_jets, stg, to_device, c->stream);
    } else if (which == GL_BUF_ENERGY) {
        launch_energy(c->prec, site_at(c, c->pstep - 1), c->N, stg, c->stream);
    } else if (which == GL_BUF_PTAU) {
        launch_ptau_convert(c->prec, c->parts, c->np, stg, to_device, c->stream);
    } else launch_convert(c->prec, which, to_device, which == GL_BUF_SITE ? site_at(c, c->pstep - 1) : c->field[c->cur], stg, c->N, c->np,
                        c->stream);
    if (!to_device) cudaMemcpyAsync(host, stg, count * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    return check_cuda(c, to_device ? "gl_upload" : "gl_download");
}

static gl_status transfer(gl_ctx* c, gl_buffer which, double* host, size_t count, int to_device) {
    if (gl_status s = transfer_enqueue(c, which, host, count, to_device)) return s;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return check_cuda(c, "transfer sync");
    return GL_OK;
}

gl_status gl_upload(gl_ctx* c, gl_buffer which, const double* host, size_t count) {
    gl::ApiRange range_("gl_upload");
    return transfer(c, which, (double*)host, count, 1);
}

gl_status gl_download(gl_ctx* c, gl_buffer which, double* host, size_t count) {
    gl::ApiRange range_("gl_download");
    return transfer(c, which, host, count, 0);
}

// ------------------------------------------------------------ native snapshots
static size_t native_bytes(const gl_ctx* c, int part) {
    if (part == GL_NATIVE_FIELDS) return field_bytes(c->prec, c->Vn);
    if (part == GL_NATIVE_PARTICLES) return particle_bytes(c->prec, c->np);
    return 0;
}

static gl_status native_check(gl_ctx* c, int part, const void* host, size_t bytes) {
    if (!c || (!host && bytes)) return GL_ERR_ARG;
    if (part != GL_NATIVE_FIELDS && part != GL_NATIVE_PARTICLES) return fail(c, GL_ERR_ARG, "unknown native part");
    if (bytes != native_bytes(c, part)) return fail(c, GL_ERR_SIZE, "host buffer size does not match gl_native_bytes()");
    return GL_OK;
}

// the copy into the current field slice or the particle arrays, then (for
// particles) the index check into c->d_bad, all on st
static gl_status native_upload_enqueue(gl_ctx* c, int part, const void* host, size_t bytes, cudaStream_t st) {
    if (gl_status s = native_check(c, part, host, bytes)) return s;
    if (bytes == 0) return GL_OK;
    void* dst = part == GL_NATIVE_FIELDS ? c->field[c->cur] : c->parts;
    cudaMemcpyAsync(dst, host, bytes, cudaMemcpyHostToDevice, st);
    if (part == GL_NATIVE_PARTICLES) {
        cudaMemsetAsync(c->d_bad, 0, sizeof(int), st);
        launch_parts_validate(c->prec, c->parts, c->np, c->ns, c->d_bad, st);
    }
    return check_cuda(c, "gl_upload_native");
}

size_t gl_native_bytes(const gl_ctx* c, gl_native_part part) { return c ? native_bytes(c, (int)part) : 0; }

gl_status gl_download_native(gl_ctx* c, gl_native_part part, void* host, size_t bytes) {
    gl::ApiRange range_("gl_download_native");
    if (gl_status s = native_check(c, (int)part, host, bytes)) return s;
    if (bytes == 0) return GL_OK;
    const void* src = part == GL_NATIVE_FIELDS ? c->field[c->cur] : c->parts;
    cudaMemcpyAsync(host, src, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return check_cuda(c, "gl_download_native sync");
    return check_cuda(c, "gl_download_native");
}

gl_status gl_upload_native(gl_ctx* c, gl_native_part part, const void* host, size_t bytes) {
    gl::ApiRange range_("gl_upload_native");
    if (gl_status s = native_upload_enqueue(c, (int)part, host, bytes, c->stream)) return s;
    int bad = 0;
    if (part == GL_NATIVE_PARTICLES && bytes > 0)
        cudaMemcpyAsync(&bad, c->d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return check_cuda(c, "gl_upload_native sync");
    if (bad) return fail(c, GL_ERR_ARG, "native particles: species or original index out of range (repaired)");
    return GL_OK;
}

gl_status gl_set_step(gl_ctx* c, int64_t step) {
    if (!c || step < 0) return GL_ERR_ARG;
    // the current fields stay current; their buffer takes the index of the
    // new step's parity, as after any sequence of field steps
    if ((int)(step & 1) != c->cur) {
        void* f = c->field[0];
        c->field[0] = c->field[1];
        c->field[1] = f;
        c->cur = (int)(step & 1);
    }
    c->step = c->pstep = step;
    site_forget(c);
    return GL_OK;
}

// One leapfrog step on stream st; the same kernel interpolates E, B at the
// fields' time t_step into the site buffer of that time's parity.  FP32 links
// of row y are re-unitarised in the steps n with (n + 1 + y) % reunit_every
// == 0, a rule of the step index alone, so a resumed run re-unitarises where
// an uninterrupted one does.
static void one_field_step(gl_ctx* c, cudaStream_t st) {
    const int every = c->prec == GL_FP32_2ROW ? c->cfg.reunit_every : 0;
    launch_fused_step(c->prec, c->field[c->cur], c->field[1 - c->cur], site_at(c, c->step), c->N, c->step, c->dt,
                      every, c->tile, c->seg, st);
    c->site_time[c->step & 1] = c->step;
    c->cur = 1 - c->cur;
    c->step++;
}

gl_status glasma_step(gl_ctx* c, int32_t n) {
    gl::ApiRange range_("glasma_step");
    if (!c || n < 0) return GL_ERR_ARG;
    for (int k = 0; k < n; k++) one_field_step(c, c->stream);
    return check_cuda(c, "glasma_step");
}

static gl_status site_once(gl_ctx* c) {
    if (c->pstep != c->step - 1) return fail(c, GL_ERR_STATE, "needs exactly one field step since the particles' time");
    launch_site_fields(c->prec, c->field[1 - c->cur], c->field[c->cur], site_at(c, c->pstep), c->N, c->pstep * c->dt,
                       c->stream);
    c->site_time[c->pstep & 1] = c->pstep;
    return GL_OK;
}

gl_status wong_site_fields(gl_ctx* c) {
    gl::ApiRange range_("wong_site_fields");
    if (!c) return GL_ERR_ARG;
    if (site_holds(c, c->pstep) && c->pstep == c->step - 1) return GL_OK;  // written by the field step
    if (gl_status s = site_once(c)) return s;
    return check_cuda(c, "wong_site_fields");
}

// push of the particles at t_pstep on stream st: reads the site fields of
// t_pstep and the links and scalar of t_{pstep+1} (field buffer of that time)
static gl_status push_once(gl_ctx* c, cudaStream_t st, void* bn1) {
    const double t = c->pstep * c->dt;
    if (c->np) launch_push(c->prec, site_at(c, c->pstep), bn1, c->parts, c->np, c->N, t, c->dt, active_mask(c, c->pstep),
                           c->spp, st, c->push_block);
    if (c->n_jets) launch_jets_step(c->prec, site_at(c, c->pstep), bn1, c->jets, c->n_jets, c->N, t, c->dt, st);
    c->pstep++;
    if (c->sort_ok && c->pstep % c->cfg.sort_every == 0) {
        launch_sort(c->prec, c->parts, c->parts_alt, c->np, c->N, c->ns, c->spp.motion, c->sort_scratch, st);
        void* tmp = c->parts;
        c->parts = c->parts_alt;
        c->parts_alt = tmp;
    }
    return GL_OK;
}

gl_status wong_push(gl_ctx* c) {
    gl::ApiRange range_("wong_push");
    if (!c) return GL_ERR_ARG;
    if (c->pstep != c->step - 1) return fail(c, GL_ERR_STATE, "wong_push needs exactly one field step since the particles' time");
    if (!site_holds(c, c->pstep))
        if (gl_status s = site_once(c)) return s;
    if (gl_status s = push_once(c, c->stream, c->field[c->cur])) return s;
    return check_cuda(c, "wong_push");
}

static gl_status ensure_aux(gl_ctx* c) {
    if (c->aux) return GL_OK;
    if (cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_f, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_p, cudaEventDisableTiming) != cudaSuccess)
        return check_cuda(c, "stream creation");
    return GL_OK;
}

// n coupled steps with the field step of t_s overlapped with the push of the
// particles at t_{s-1} (second stream): the field kernel of step s reads the
// buffers of time s and writes those of s+1 and the site fields of t_s, while
// the push of s-1 reads the site fields of t_{s-1} and the links and scalar of
// time s; the field step s+1, which rewrites the buffers of time s-1, waits
// for that push.  The caller's stream waits for the last push.
gl_status gl_step_coupled(gl_ctx* c, int32_t n) {
    gl::ApiRange range_("gl_step_coupled");
    if (!c || n < 0) return GL_ERR_ARG;
    if (n == 0) return GL_OK;
    if (c->pstep != c->step) return fail(c, GL_ERR_STATE, "particles are not at the fields' time");
    if (c->np == 0) {
        for (int k = 0; k < n; k++) one_field_step(c, c->stream);
        c->pstep = c->step;
        return check_cuda(c, "gl_step_coupled");
    }
    if (gl_status s = ensure_aux(c)) return s;
    one_field_step(c, c->stream);
    for (int k = 1; k <= n; k++) {
        cudaEventRecord(c->ev_f, c->stream);          // field step of pstep + 1 done
        cudaStreamWaitEvent(c->aux, c->ev_f, 0);
        void* bn1 = c->field[c->cur];                 // buffers of time pstep + 1
        if (gl_status s = push_once(c, c->aux, bn1)) return s;
        if (k == n) break;
        if (k >= 2) cudaStreamWaitEvent(c->stream, c->ev_p, 0);  // push of the step before
        one_field_step(c, c->stream);
        cudaEventRecord(c->ev_p, c->aux);
    }
    cudaEventRecord(c->ev_p, c->aux);
    cudaStreamWaitEvent(c->stream, c->ev_p, 0);
    return check_cuda(c, "gl_step_coupled");
}

gl_status gl_autotune(gl_ctx* c, int32_t* tile_out, int32_t* push_block_out) {
    gl::ApiRange range_("gl_autotune");
    if (!c) return GL_ERR_ARG;
    if (c->pstep != c->step) return fail(c, GL_ERR_STATE, "autotune needs the particles at the fields' time");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto timed = [&](auto&& fn) {
        float acc = 0;
        for (int rep = 0; rep < 4; rep++) {
            cudaEventRecord(e0, c->stream);
            fn();
            cudaEventRecord(e1, c->stream);
            cudaEventSynchronize(e1);
            float m = 0;
            cudaEventElapsedTime(&m, e0, e1);
            if (rep > 0) acc += m;
        }
        return acc / 3;
    };
    // field kernel: writes only the spare time slice and the site fields at
    // the current time, both of which the next coupled step rewrites
    // FP64: tiles 32x4 (1) and 32x2 (2); FP32: strip shapes 0, 1, 2, each with
    // the cost model's segment length, its half and double, and 16 rows
    const int tiles[4] = {0, 1, 2, 3};
    float best = 1e30f;
    for (int k = 0; k < 4; k++) {
        if ((c->prec == GL_FP64 && (k == 0 || k == 3)) || (c->prec != GL_FP64 && k == 3)) {
            c->tune_field_ms[k] = 0;
            continue;
        }
        int cand[4] = {0, 0, 0, 0}, nc = 1;
        if (c->prec != GL_FP64) {
            const int m = strip_model_seg(c->N, tiles[k]);
            const int more[3] = {16, 2 * m, m / 2};
            cand[0] = m;
            for (int j = 0; j < 3; j++) {
                bool dup = more[j] < 4;
                for (int q = 0; q < nc; q++) dup = dup || cand[q] == more[j];
                if (!dup) cand[nc++] = more[j];
            }
        }
        float best_k = 1e30f;
        for (int q = 0; q < nc; q++) {
            const float ms = timed([&] {
                launch_fused_step(c->prec, c->field[c->cur], c->field[1 - c->cur], site_at(c, c->step), c->N,
                                  c->step, c->dt, 0, tiles[k], cand[q], c->stream);
            });
            if (ms < best_k) best_k = ms;
            if (ms < best) { best = ms; c->tile = tiles[k]; c->seg = cand[q]; }
        }
        c->tune_field_ms[k] = best_k;
    }
    // push: on a copy of the particles, at a step where every species is formed
    if (c->np && c->parts_alt) {
        int64_t trial = c->step;
        for (int k = 0; k < c->ns; k++) {
            const int64_t n = (int64_t)ceil(c->t_form[k] / c->dt);
            if (n > trial) trial = n;
        }
        const int blocks[3] = {64, 128, 256};
        best = 1e30f;
        for (int k = 0; k < 3; k++) {
            cudaMemcpyAsync(c->parts_alt, c->parts, particle_bytes(c->prec, c->np), cudaMemcpyDeviceToDevice, c->stream);
            const float ms = timed([&] {
                launch_push(c->prec, site_at(c, c->step), c->field[1 - c->cur], c->parts_alt, c->np, c->N, trial * c->dt, c->dt,
                            active_mask(c, trial), c->spp, c->stream, blocks[k]);
            });
            c->tune_push_ms[k] = ms;
            if (ms < best) { best = ms; c->push_block = blocks[k]; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->site_time[c->step & 1] = -1;  // trial field launches wrote that buffer
    if (tile_out) *tile_out = c->tile;
    if (push_block_out) *push_block_out = c->push_block;
    return check_cuda(c, "gl_autotune");
}

gl_status gl_tuning(const gl_ctx* c, float* field_ms, float* push_ms) {
    if (!c) return GL_ERR_ARG;
    for (int k = 0; k < 4; k++)
        if (field_ms) field_ms[k] = c->tune_field_ms[k];
    for (int k = 0; k < 3; k++)
        if (push_ms) push_ms[k] = c->tune_push_ms[k];
    return GL_OK;
}

// enqueue the observable reductions of a context (no wait)
static void observables_launch(gl_ctx* c, uint32_t what) {
    if (what & GL_OBS_PARTICLES) {
        ObsEvent o;
        ctx_obs_event(c, &o);
        launch_particle_obs(c->prec, o.parts, o.np, o.t, o.mask, o.sp, o.q2ref, o.q3ref, o.partials, o.out, c->stream);
    }
    if (what & GL_OBS_FIELDS) {
        ObsEvent o;
        ctx_obs_event(c, &o);
        launch_field_obs_events(c->prec, o.fo, nullptr, 0, 0, o.fo.nblocks, true, c->stream);
    }
}

// read back the reductions enqueued by observables_launch (waits); the values
// of the parts not in `what` are NaN (counts 0)
static gl_status observables_read(gl_ctx* c, uint32_t what, gl_obs* o) {
    double host[GL_MAX_SPECIES * PO_N + FO_N];
    cudaMemcpyAsync(host, c->obs_dev, sizeof host, cudaMemcpyDeviceToHost, c->stream);
    if (gl_status s = check_cuda(c, "observables")) return s;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return check_cuda(c, "observables sync");
    observables_fill(c, what, host, o);
    return GL_OK;
}

// a gl_obs record from the raw reductions host[GL_MAX_SPECIES * PO_N + FO_N]
static void observables_fill(const gl_ctx* c, uint32_t what, const double* host, gl_obs* o) {
    memset(o, 0, sizeof *o);
    const double u2 = 1.0 / (c->aG * c->aG);  // lattice momentum^2 -> GeV^2
    const bool P = (what & GL_OBS_PARTICLES) != 0, F = (what & GL_OBS_FIELDS) != 0;
    o->step = c->step;
    o->tau_fm = c->pstep * c->dt * c->a_fm;
    o->n_species = c->ns;
    o->what = what & GL_OBS_ALL;
    for (int k = 0; k < c->ns; k++) {
        const double* h = host + k * PO_N;
        o->n_active[k] = P ? (int64_t)llround(h[PO_COUNT]) : 0;
        o->sum_px2[k] = P ? h[PO_PX2] * u2 : NAN;
        o->sum_py2[k] = P ? h[PO_PY2] * u2 : NAN;
        o->sum_pL2[k] = P ? h[PO_PL2] * u2 : NAN;
        o->sum_dpT2[k] = P ? h[PO_DPT2] * u2 : NAN;
        o->casimir2_dev[k] = P ? h[PO_Q2] : NAN;
        o->casimir3_dev[k] = P ? h[PO_Q3] : NAN;
    }
    const double* f = host + GL_MAX_SPECIES * PO_N;
    // the kernels keep the maxima as squared norms
    o->gauss_max = F ? sqrt(f[FO_GMAX]) : NAN;
    o->gauss_rms = F ? sqrt(f[FO_GSUM] / (double)c->Vn) : NAN;
    o->unitarity_max = F ? sqrt(f[FO_UMAX]) : NAN;
    // the means of the squared site fields refer to the last pushed time
    const bool S = F && site_holds(c, c->pstep - 1);
    o->mean_trE_T2 = S ? f[FO_ET2] / (double)c->Vn : NAN;
    o->mean_trE_L2 = S ? f[FO_EL2] / (double)c->Vn : NAN;
    o->mean_trB_T2 = S ? f[FO_BT2] / (double)c->Vn : NAN;
    o->mean_trB_L2 = S ? f[FO_BL2] / (double)c->Vn : NAN;
}

gl_status observables(gl_ctx* c, gl_obs* o) { return gl_observables_ex(c, GL_OBS_ALL, o); }

gl_status gl_jets_observables(gl_ctx* c, double* out3) {
    gl::ApiRange range_("gl_jets_observables");
    if (!c || !out3) return GL_ERR_ARG;
    if (!c->n_jets) return fail(c, GL_ERR_STATE, "the context has no jet-correlator probes");
    double* dout = c->jet_partials + 1024 * 3;
    launch_jets_obs(c->prec, c->jets, c->n_jets, c->jet_partials, dout, c->stream);
    double h[3];
    cudaMemcpyAsync(h, dout, sizeof h, cudaMemcpyDeviceToHost, c->stream);
    if (gl_status s = check_cuda(c, "gl_jets_observables")) return s;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return check_cuda(c, "gl_jets_observables sync");
    const double u2 = 1.0 / (c->aG * c->aG);  // lattice momentum^2 -> GeV^2
    for (int i = 0; i < 3; i++) out3[i] = h[i] * u2;
    return GL_OK;
}

gl_status gl_observables_ex(gl_ctx* c, uint32_t what, gl_obs* o) {
    gl::ApiRange range_("gl_observables_ex");
    if (!c || !o || (what & ~GL_OBS_ALL)) return GL_ERR_ARG;
    observables_launch(c, what);
    return observables_read(c, what, o);
}

}  // extern "C"
