// Internal declarations shared by the translation units of the CUDA library.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/glasma.h"
#include <nvtx3/nvToolsExt.h>

namespace gl {

// a named range on the profiler timeline (NVTX) for the life of a C-ABI call;
// without a profiler attached it costs a pointer test
struct ApiRange {
    explicit ApiRange(const char* name) { nvtxRangePushA(name); }
    ~ApiRange() { nvtxRangePop(); }
    ApiRange(const ApiRange&) = delete;
    ApiRange& operator=(const ApiRange&) = delete;
};


// how a species moves: Wong particles of finite mass, infinitely massive
// static quarks (Sec. 5.1), eikonal light-like partons along +x (Sec. 5.2)
enum { MOTION_WONG = 0, MOTION_STATIC = 1, MOTION_EIKONAL = 2 };

struct SpeciesParams {
    double mass[GL_MAX_SPECIES];   // lattice units; INFINITY = static
    int motion[GL_MAX_SPECIES];
    int n_species;
    int ptau_diag;                 // GL_CFG_PTAU_DIAGNOSTIC
};

// field step n -> n+1 on buffers in/out (FP64 or FP32 two-row layout); the
// same kernel also writes the site E, B at t_n into site (not null).
// FP32: the strip kernel, tile = launch shape 0 (16 warps per SM), 1 (12) or
// 2 (8); its links of row y are re-unitarised in FP64 in the steps n with
// (n + 1 + y) % reunit_every == 0 (0: never).  FP64: tile 2 = 32x2, else 32x4.
// seg: FP32 rows per strip segment (0: the cost model's choice for the shape)
void launch_fused_step(int prec, void* in, void* out, void* site, int N, int64_t n, double dt, int reunit_every,
                       int tile, int seg, cudaStream_t st);
// the cost model's segment length for an N x N lattice and FP32 launch shape `tile`
int strip_model_seg(int N, int tile);
// site E, B at t_n from buffer n (U, phi, e(n-1/2), pi(n-1/2)) and buffer n+1 (e, pi at n+1/2)
void launch_site_fields(int prec, const void* bn, const void* bn1, void* site, int N, double t, cudaStream_t st);
// Euler + CPIC push of all particles active at t_n (bit s of active_mask)
void launch_push(int prec, const void* site, const void* bn1, void* parts, int64_t np, int N, double t, double dt,
                 uint32_t active_mask, const SpeciesParams& sp, cudaStream_t st, int block = 128);
// particle sampling: positions, momenta, Haar charges
void launch_sample(int prec, void* parts, int64_t np, int N, uint64_t seed, const int64_t* offsets, int n_species,
                   const int* rep, const int* mom_mode, const double* p0, const double* p1,
                   const double q0[2][8], cudaStream_t st);
// MV initial condition into field buffer b (FP64 scratch in `scratch`)
int launch_mv_init(int prec, void* b, void* scratch, int N, int Ns, double g2mu_a, double m_a, double Lambda_a,
                   uint64_t seed, int* d_bad, cudaStream_t st);
// canonical FP64 <-> device layout conversions (staging buffer is FP64 canonical)
void launch_parts_convert(int prec, void* parts, int64_t np, double* stg, int to_device, cudaStream_t st);
// species and original indices of a native particle upload checked and
// repaired on the device (*d_bad |= 1 if any was out of range)
void launch_parts_validate(int prec, void* parts, int64_t np, int ns, int* d_bad, cudaStream_t st);
// integrated p^tau of the particles <-> canonical [np] in the caller's order
void launch_ptau_convert(int prec, void* parts, int64_t np, double* stg, int to_device, cudaStream_t st);
size_t init_scratch_bytes(int64_t Vn);
void launch_convert(int prec, int which, int to_device, void* dev, double* staging, int N, int64_t np,
                    cudaStream_t st);
// observables: per-species particle sums and field checks, FP64, fixed-order reductions
// (partials: obs_blocks(np) <= 1024 rows of GL_MAX_SPECIES * PO_N; out: GL_MAX_SPECIES * PO_N)
void launch_particle_obs(int prec, const void* parts, int64_t np, double t, uint32_t active_mask,
                         const SpeciesParams& sp, const double q2ref[GL_MAX_SPECIES],
                         const double q3ref[GL_MAX_SPECIES], double* partials, double* out, cudaStream_t st);
// The FP64 field checks of one event: the fields of the current time, the
// site fields of the last step, N, the event's first block in a launch over
// several events and its number of blocks, the per-block rows
// [blocks][FO_N] and the FO_N results.
struct FieldObsEv {
    const void* fields;
    const void* site;
    int N;
    int block_begin;
    int nblocks;
    double* partials;
    double* out;
};
static constexpr int FIELD_OBS_MAX_BLOCKS = 1024;
// blocks of an N x N event's field checks: one site a thread in blocks of
// 256, at most FIELD_OBS_MAX_BLOCKS (then grid-strided)
inline int field_obs_blocks(int N) {
    const int64_t b = ((int64_t)N * N + 255) / 256;
    return (int)(b < FIELD_OBS_MAX_BLOCKS ? b : FIELD_OBS_MAX_BLOCKS);
}
// The field checks of ne events in one launch of `blocks` blocks (the sum of
// their nblocks), their descriptors `stride` bytes apart from the device
// address evs; or, with ne == 0, of the one event `one` (block_begin 0).  One
// kernel serves both, so an event's results are bitwise the same whether it
// is checked alone or with others.  finalize: also reduce each event's rows
// into its out (one block per event, obs_finalize_block); a caller that
// passes false runs that reduction itself, with the same function.
void launch_field_obs_events(int prec, const FieldObsEv& one, const void* evs, size_t stride, int ne, int blocks,
                             bool finalize, cudaStream_t st);
// one context's particle-observables launch, for the batched reduction
struct ObsEvent {
    void* parts;
    int64_t np;
    double t;
    uint32_t mask;
    SpeciesParams sp;
    double q2ref[GL_MAX_SPECIES], q3ref[GL_MAX_SPECIES];
    double* partials;
    double* out;
    FieldObsEv fo;  // its field checks
};
// energy density per site, tr of the squared site fields (FP64 out[N*N])
void launch_energy(int prec, const void* site, int N, double* out, cudaStream_t st);

// light-like jet-correlator probes (Sec. 5.2), [n][JET_LEN] in the state's
// precision: x0, y0, W (18), X_x, X_y, X_z (8 each)
static constexpr int JET_LEN = 44;
void launch_jets_init(int prec, void* jets, int64_t n, int N, uint64_t seed, cudaStream_t st);
// one step of every probe from t_n = t: site fields at t_n, links at t_{n+1} (bn1)
void launch_jets_step(int prec, const void* site, const void* bn1, void* jets, int64_t n, int N, double t,
                      double dt, cudaStream_t st);
// out[3] = mean over probes of X_i . X_i (FP64, fixed order); partials: 1024 x 3 doubles
void launch_jets_obs(int prec, const void* jets, int64_t n, double* partials, double* out, cudaStream_t st);
// canonical FP64 <-> device probes
void launch_jets_convert(int prec, void* jets, int64_t n, double* stg, int to_device, cudaStream_t st);

// radix sort of the particles by row, motion class and cell from src into dst (same layout)
void launch_sort(int prec, void* src, void* dst, int64_t np, int N, int ns, const int* motion, void* scratch,
                 cudaStream_t st);
// one event of a batched sort; pblk_begin / cblk_begin: its first block in the
// particle-indexed (sort_particle_blocks) and scan-indexed (sort_cell_blocks)
// launches, set by the caller
struct SortEv {
    void* src;
    void* dst;
    int64_t np;
    int N;
    int ng;                      // motion classes present: keys (row, class, cell), ng N^2 of them
    int8_t grp[GL_MAX_SPECIES];  // class of each species
    int nblk;                    // particle blocks of the sort
    int pblk_begin, cblk_begin;  // first particle block and first scan block in a batched launch
    uint32_t* key[2];            // radix pass ping-pong: keys and original indices
    uint32_t* val[2];
    int* hist;                   // [digit][block] counts, scanned in place
    int* bsum;
};
SortEv sort_event(void* src, void* dst, int64_t np, int N, int ns, const int* motion, void* scratch);
int sort_particle_blocks(int64_t np);
int sort_cell_blocks(const SortEv& d);
// digit passes that cover the keys of one event
int sort_passes(const SortEv& d);
// the sort of ne events (descriptors d_ev in device memory) in one launch per
// stage, `passes` digit passes (the largest any of them needs)
void launch_sort_many(int prec, const SortEv* d_ev, int ne, int pblocks, int cblocks, int passes, cudaStream_t st);
size_t sort_scratch_bytes(int64_t Vn, int64_t np, int ns);
bool sort_supported(int64_t Vn, int ns, int64_t np);

size_t particle_bytes(int prec, int64_t np);
size_t site_bytes(int prec, int64_t Vn);
size_t field_bytes(int prec, int64_t Vn);

// context internals the batch reads and drives (capi.cu)
struct CtxView {
    void* field[2];
    void* site[2];
    void* parts;
    int N, prec, cur;
    int64_t step, pstep, np;
    double dt;
    double mass[GL_MAX_SPECIES];
    int motion[GL_MAX_SPECIES];
    double t_form[GL_MAX_SPECIES];
    int ptau_diag;
    int ns;
    void* parts_alt;
    int sort_every;
    void* sort_scratch;
};
void ctx_view(const gl_ctx* c, CtxView* v);
// record that the batch advanced the event by `steps` coupled steps
void ctx_advance(gl_ctx* c, int64_t steps);
// reorder the event's particles (row, motion class, cell) on its stream
void ctx_sort(gl_ctx* c);
// exchange the particle buffer and its spare (after a batched sort into the spare)
void ctx_swap_parts(gl_ctx* c);
void ctx_obs_event(const gl_ctx* c, ObsEvent* o);
size_t ctx_workspace_bytes(const gl_config* cfg, const gl_species* sp, int32_t ns);
// a gl_obs record from a host copy of that row
void ctx_obs_fill(const gl_ctx* c, uint32_t what, const double* row, gl_obs* o);
// gl_upload without its wait: copies, conversions and a particle sort enqueued on st
gl_status ctx_upload_enqueue(gl_ctx* c, gl_buffer which, const double* host, size_t count, cudaStream_t st);
// gl_upload_native's copy alone, enqueued on st (a batch checks the particle
// indices of all its events afterwards, in one launch)
gl_status ctx_upload_native_copy(gl_ctx* c, int part, const void* host, size_t bytes, cudaStream_t st);
// the particle-index check of one event in a launch over several events: its
// particle arrays, count and species, its first block in the launch and its
// number of blocks
struct PartsCheckEv {
    void* parts;
    int64_t np;
    int ns;
    int block_begin;
    int nblocks;
};
PartsCheckEv ctx_parts_check_event(const gl_ctx* c);
int parts_check_blocks(int64_t np);
// the check of ne events (descriptors in device memory) in `blocks` blocks:
// out-of-range species or original indices are repaired and set bad[e]
void launch_parts_validate_events(int prec, const PartsCheckEv* evs, int ne, int blocks, int* bad, cudaStream_t st);

// observable slots
enum { PO_COUNT = 0, PO_PX2, PO_PY2, PO_PL2, PO_DPT2, PO_Q2, PO_Q3, PO_N };
enum { FO_GMAX = 0, FO_GSUM, FO_UMAX, FO_ET2, FO_EL2, FO_BT2, FO_BL2, FO_N };

}  // namespace gl
