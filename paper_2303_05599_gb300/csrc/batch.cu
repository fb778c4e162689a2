// Many independent MV events of uneven N advanced together (the paper
// averages observables over many events, Sec. 7.1).  One coupled step of the
// whole batch is captured once in a CUDA graph and replayed:
//   fused leapfrog + site E/B over the tiles of every event (step s), and
//   concurrently on a second stream the Wong push over the particles of
//   every event (step s - 1: it reads the site fields of t_{s-1} and the
//   links of t_s, neither of which the field step of s writes),
//   then a one-thread tick of the device-resident step counter.
// The kernels read the step index n from device memory, so the captured
// graph is valid for every step.  Each block finds its event in a prefix
// table of tiles or particle chunks (one warp, one round of loads).
//
// Every sort_every steps (per event) the run stops between a push and the next
// field step and the particles of that event are reordered (by row, motion class and cell), as in the
// single-event schedule.  Observables of all events are reduced by one launch
// pair over per-event chunks (obs_body.cuh).
//
// The tile shape of the field kernel and the block size of the push are
// chosen by gl_batch_autotune from timed trial launches that leave the state
// unchanged (the field kernel writes only the spare time slice; the push runs
// on a copy of the particles).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "internal.h"
#include "obs_body.cuh"
#include "push_body.cuh"
#include "strip_body.cuh"

namespace gl {

static constexpr int MAX_EVENTS = 1024;
static constexpr int PUSH_CHUNK = 1024;  // default particles per push block

struct EvDesc {
    void* field[2];
    void* site[2];   // site fields of t_n in site[n & 1]
    void* parts;
    int N;
    int tiles_x;     // FP64: for the chosen tile shape
    int tile_begin;  // FP64: first block of this event in the field launch
    int chunk_begin; // first block of this event in the push launch
    int64_t seg_begin;  // FP32: first segment of this event's strips in the flat segment list
    int64_t np;
    double mass[GL_MAX_SPECIES];
    int motion[GL_MAX_SPECIES];
    double t_form[GL_MAX_SPECIES];
    int ptau_diag;
    int n_species;
    int pad;
};

struct BatchArgs {
    const EvDesc* ev;
    int ne;
    double dt;
    int reunit_every;
    const int64_t* clock;
    int push_chunk;  // particles per push block
    int seg_rows;    // FP32: rows per strip segment
};

// the last event whose first block is <= block (the prefix tables are
// non-decreasing, event 0 starts at 0), found by a whole warp: each lane
// reads one event's entry and a ballot counts those at or before the block,
// 32 events per round, so a block starts after one round of loads instead of
// a chain of dependent ones
__device__ __forceinline__ int find_event_warp(const EvDesc* ev, int ne, int block, bool tiles) {
    const int lane = threadIdx.x & 31;
    int cnt = 0;
    for (int g = 0; g < ne; g += 32) {
        const int k = g + lane;
        const bool le = k < ne && (tiles ? ev[k].tile_begin : ev[k].chunk_begin) <= block;
        const unsigned m = __ballot_sync(0xffffffffu, le);
        cnt += __popc(m);
        if (m != 0xffffffffu) break;
    }
    return cnt > 0 ? cnt - 1 : 0;
}

// the last event whose first segment is <= j, found by a whole warp as in
// find_event_warp
__device__ __forceinline__ int find_event_seg(const EvDesc* ev, int ne, int64_t j) {
    const int lane = threadIdx.x & 31;
    int cnt = 0;
    for (int g = 0; g < ne; g += 32) {
        const int k = g + lane;
        const bool le = k < ne && ev[k].seg_begin <= j;
        const unsigned m = __ballot_sync(0xffffffffu, le);
        cnt += __popc(m);
        if (m != 0xffffffffu) break;
    }
    return cnt > 0 ? cnt - 1 : 0;
}

// FP32 field step of segment j of the batch's flat segment list, by one warp
// in step with its block (j beyond the list: the last segment, no stores)
__device__ __forceinline__ void strip_seg_item(const BatchArgs& b, StripWarpSmem& S, int64_t n, const StripStep& a,
                                               int64_t j, int64_t nseg) {
    const bool real = j < nseg;
    if (!real) j = nseg - 1;
    const EvDesc& d = b.ev[find_event_seg(b.ev, b.ne, j)];
    const int64_t Vn = (int64_t)d.N * d.N;
    strip_run_segment(S, carve_fields<float>(d.field[n & 1], Vn), carve_fields<float>(d.field[(n + 1) & 1], Vn),
                      (float4*)d.site[n & 1], d.N, j - d.seg_begin, real, a, b.seg_rows);
}

// one field tile (block `blk` of the tile prefix table) of step n = clock
template <typename R, int TX, int TY>
__device__ __forceinline__ void field_item(const BatchArgs& b, int blk) {
    // the block's event and step scalars, once per block
    __shared__ int s_e;
    __shared__ int64_t s_n;
    __shared__ StepR<R> s_a;
    if (threadIdx.x < 32) {
        const int64_t n = *b.clock;
        const int e = find_event_warp(b.ev, b.ne, blk, true);
        if (threadIdx.x == 0) {
            const int reunit = b.reunit_every > 0 && (n + 1) % b.reunit_every == 0;
            s_e = e;
            s_n = n;
            s_a = step_r<R>(step_args(b.ev[e].N, b.ev[e].tiles_x, n, b.dt, reunit));
        }
    }
    __syncthreads();
    const EvDesc& d = b.ev[s_e];
    const int64_t n = s_n;
    const int64_t Vn = (int64_t)d.N * d.N;
    fused_tile<R, TX, TY>(carve_fields<R>(d.field[n & 1], Vn), carve_fields<R>(d.field[(n + 1) & 1], Vn),
                                (typename Prec<R>::V*)d.site[n & 1], s_a, blk - d.tile_begin);
}

// one chunk of b.push_chunk particles (block `blk` of the chunk prefix table),
// pushed from t_{clock - lag}
template <typename R>
__device__ __forceinline__ void push_item(const BatchArgs& b, int lag, int blk) {
    // the block's event, time scalars and species table, once per block
    __shared__ int s_e;
    __shared__ int64_t s_n;
    __shared__ uint32_t s_active;
    __shared__ R s_t, s_dt, s_dto;
    __shared__ SpeciesArgs<R> s_sa;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const int64_t n = *b.clock - lag;
        const int e = find_event_warp(b.ev, b.ne, blk, false);
        const EvDesc& d = b.ev[e];
        const double t = n * b.dt;
        // species k on lane k
        bool act = false;
        if (lane < GL_MAX_SPECIES) {
            const int mo = d.motion[lane];
            act = lane < d.n_species && t >= d.t_form[lane];
            s_sa.mass[lane] = (R)(mo == MOTION_WONG ? d.mass[lane] : 0.0);
            s_sa.motion[lane] = mo;
        }
        const uint32_t active = __ballot_sync(0xffffffffu, act);
        if (lane == 0) {
            s_sa.ptau_diag = d.ptau_diag;
            s_e = e;
            s_n = n;
            s_active = active;
            s_t = (R)t;
            s_dt = (R)b.dt;
            s_dto = (R)(t > 0 ? b.dt / t : 0.0);
        }
    }
    __syncthreads();
    const EvDesc& d = b.ev[s_e];
    const int64_t n = s_n;
    const int64_t Vn = (int64_t)d.N * d.N;
    const Parts<R> P = carve_parts<R>(d.parts, d.np);
    const Fields<R> bn1 = carve_fields<R>(d.field[(n + 1) & 1], Vn);
    const int64_t base = (int64_t)(blk - d.chunk_begin) * b.push_chunk;
    const int64_t end = base + b.push_chunk < d.np ? base + b.push_chunk : d.np;
    for (int64_t i = base + threadIdx.x; i < end; i += blockDim.x) {
        // the next particle's state into L2 while this one is pushed
        if (i + blockDim.x < end) P.prefetch_l2(i + blockDim.x);
        push_one<R>((const typename Prec<R>::V*)d.site[n & 1], bn1, P, i, d.N, s_t, s_dt, s_dto, s_active, s_sa);
    }
}

template <typename R, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, (Tile<R, TX, TY>::min_blocks)) batch_field_kernel(BatchArgs b) {
    field_item<R, TX, TY>(b, blockIdx.x);
}

// FP32 field step of the whole batch: blocks of WPB warps take WPB
// consecutive segments of the flat list per item (nseg segments, `items`
// items strided over the grid)
template <int WPB, int MINB>
__global__ void __launch_bounds__(WPB * 32, MINB) batch_strip_kernel(BatchArgs b, int64_t nseg, int items) {
    extern __shared__ __align__(16) unsigned char strip_smem[];
    StripWarpSmem* S = (StripWarpSmem*)strip_smem;
    const int wib = threadIdx.x >> 5;
    const int64_t n = *b.clock;
    const StripStep a = strip_step(n, b.dt, b.reunit_every);
    for (int it = blockIdx.x; it < items; it += gridDim.x)
        strip_seg_item(b, S[wib], n, a, (int64_t)it * WPB + wib, nseg);
}

// at most 64 FP32 registers (B threads, 1024 / B blocks per SM): enough
// warps per SM to keep the particle and site-field loads in flight
template <typename R, int B>
__global__ void __launch_bounds__(B, (sizeof(R) == 4 ? 1024 : 512) / B) batch_push_kernel(BatchArgs b, int lag) {
    push_item<R>(b, lag, blockIdx.x);
}

template <typename R>
static void launch_batch_push(int block, int blocks, const BatchArgs& a, int lag, cudaStream_t st) {
    if (block == 512) batch_push_kernel<R, 512><<<blocks, 512, 0, st>>>(a, lag);
    else if (block == 256) batch_push_kernel<R, 256><<<blocks, 256, 0, st>>>(a, lag);
    else batch_push_kernel<R, 128><<<blocks, 128, 0, st>>>(a, lag);
}

// the same push with a fixed number of resident blocks striding through the
// chunks: launched before the field kernel on the second stream, it keeps a
// share of every SM while the field tiles fill the rest
template <typename R>
__global__ void __launch_bounds__(128) batch_push_persist_kernel(BatchArgs b, int lag, int n_push) {
    for (int blk = blockIdx.x; blk < n_push; blk += gridDim.x) {
        push_item<R>(b, lag, blk);
        __syncthreads();  // the block's shared event data is rewritten by the next chunk
    }
}

// One persistent launch for a whole coupled step: the field tiles of t_s
// (clock) and the push chunks of t_{s - lag}, interleaved evenly in one work
// list that the resident blocks stride through.  The push reads the site
// fields of t_{s-1} and the links and scalar of t_s, which no field tile of
// this launch writes, so the two kinds of work are independent.  Field tiles
// are bound by issue (SU(3) arithmetic), push chunks by memory latency;
// sharing every SM between them keeps both busy.
// The same persistent step with FP32 strips: a field item is 8 consecutive
// segments, one for each of the block's 8 warps.
__global__ void __launch_bounds__(256, 1) batch_fused_strip_kernel(BatchArgs b, int lag, int64_t nseg, int n_field,
                                                                   int n_push) {
    extern __shared__ __align__(16) unsigned char strip_smem[];
    StripWarpSmem* S = (StripWarpSmem*)strip_smem;
    const int wib = threadIdx.x >> 5;
    const int64_t total = (int64_t)n_field + n_push;
    for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
        const int64_t f0 = w * n_field / total, f1 = (w + 1) * n_field / total;
        if (f1 > f0) {
            const int64_t n = *b.clock;
            const StripStep a = strip_step(n, b.dt, b.reunit_every);
            strip_seg_item(b, S[wib], n, a, f0 * 8 + wib, nseg);
        } else {
            push_item<float>(b, lag, (int)(w - f0));
        }
        __syncthreads();  // shared memory is reused by the next item
    }
}

template <typename R, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, (Tile<R, TX, TY>::min_blocks))
    batch_fused_kernel(BatchArgs b, int lag, int n_field, int n_push) {
    const int64_t total = (int64_t)n_field + n_push;
    for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
        const int64_t f0 = w * n_field / total, f1 = (w + 1) * n_field / total;
        if (f1 > f0) field_item<R, TX, TY>(b, (int)f0);
        else push_item<R>(b, lag, (int)(w - f0));
        __syncthreads();  // shared memory is reused by the next item
    }
}

__global__ void tick_kernel(int64_t* clock) { *clock += 1; }

// particle observables of every event: blocks [block_begin, block_begin +
// nblocks) reduce the chunks of event e into its partial rows
struct BObs {
    const void* parts;
    int64_t np;
    double t;
    uint32_t mask;
    int block_begin;
    int nblocks;
    double* partials;
    double* out;
    ObsArgs oa;
    FieldObsEv fo;  // the field checks: the event's blocks of the one launch over all events
};

__device__ __forceinline__ int find_obs_event(const BObs* ev, int ne, int block) {
    int lo = 0, hi = ne - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ev[mid].block_begin <= block) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename R>
__global__ void __launch_bounds__(OBS_THREADS) batch_obs_kernel(const BObs* ev, int ne) {
    __shared__ int s_e;
    if (threadIdx.x == 0) s_e = find_obs_event(ev, ne, blockIdx.x);
    __syncthreads();
    const BObs& d = ev[s_e];
    const int b = blockIdx.x - d.block_begin;
    const int64_t chunk = obs_chunk(d.np);
    const int64_t c0 = (int64_t)b * chunk;
    const int64_t c1 = c0 + chunk < d.np ? c0 + chunk : d.np;
    particle_obs_block<R>(carve_parts<R>((void*)d.parts, d.np), d.t, d.mask, d.oa, c0, c1,
                          d.partials + (size_t)b * GL_MAX_SPECIES * PO_N);
}

// One block per event: the final reductions of the requested parts (the
// particle values, or zeros for an event without particles; the field checks)
// into the event's obs row, by the function the single-event launches use,
// and into all[n_events][OBS_W], so that the host reads every event's row
// with one copy (the parts not requested are not copied: the host does not
// read them).
static constexpr int OBS_W = GL_MAX_SPECIES * PO_N + FO_N;
static_assert(GL_MAX_SPECIES * PO_N <= OBS_FINAL_WARPS * OBS_FINAL_V && FO_N <= OBS_FINAL_WARPS * OBS_FINAL_V,
              "obs_finalize_block takes at most OBS_FINAL_WARPS x OBS_FINAL_V values");
__global__ void __launch_bounds__(OBS_FINAL_WARPS * 32) batch_obs_finish(const BObs* ev, uint32_t what, double* all) {
    const BObs& d = ev[blockIdx.x];
    double* row = all + (size_t)blockIdx.x * OBS_W;
    if (what & GL_OBS_PARTICLES) {
        if (d.nblocks > 0)
            obs_finalize_block(d.partials, d.nblocks, GL_MAX_SPECIES * PO_N, ParticleObsKind(), d.out, row);
        else
            for (int k = threadIdx.x; k < GL_MAX_SPECIES * PO_N; k += blockDim.x) row[k] = 0.0;
    }
    if (what & GL_OBS_FIELDS)
        obs_finalize_block(d.fo.partials, d.fo.nblocks, FO_N, FieldObsKind(), d.fo.out, row + GL_MAX_SPECIES * PO_N);
}

// tile shapes the autotuner chooses from
enum { TILE_32x8 = 0, TILE_32x4 = 1, TILE_32x16 = 2, N_TILES = 3 };
static const int TILE_DIMS[N_TILES][2] = {{32, 8}, {32, 4}, {32, 16}};
static const int PUSH_BLOCKS[3] = {128, 256, 512};
enum { N_CHUNKS = 3 };
static const int PUSH_CHUNKS[N_CHUNKS] = {512, 1024, 2048};  // fused launch
enum { N_SEP_CHUNKS = 4 };
static const int SEP_CHUNKS[N_SEP_CHUNKS] = {128, 256, 512, 1024};  // separate push kernel

template <typename R, int TX, int TY>
static void set_smem_attr() {
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !done[dev]) {
        cudaFuncSetAttribute(batch_field_kernel<R, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Tile<R, TX, TY>::bytes);
        cudaFuncSetAttribute(batch_fused_kernel<R, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Tile<R, TX, TY>::bytes);
        done[dev] = true;
    }
}

// FP32 strip launch shapes the autotuner chooses from (the tile index of an
// FP32 batch), warps per block x blocks per SM: 0 = 8 x 2 (16 warps per SM at
// 128 registers), 1 = 12 x 1 (168 registers), 2 = 8 x 1 (255 registers)

// resident blocks of a strip launch shape on this device (the kernel's own
// occupancy on an idle GPU)
template <int WPB, int MINB>
static int batch_strip_blocks() {
    static int blocks[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!blocks[dev]) {
        const int smem = WPB * (int)sizeof(StripWarpSmem);
        cudaFuncSetAttribute(batch_strip_kernel<WPB, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int per_sm = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_strip_kernel<WPB, MINB>, WPB * 32, smem);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        blocks[dev] = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    }
    return blocks[dev];
}

template <int WPB, int MINB>
static void launch_strip_shape(int64_t nseg, const BatchArgs& b, cudaStream_t st) {
    if (nseg < 1) return;
    const int items = (int)((nseg + WPB - 1) / WPB);
    int grid = batch_strip_blocks<WPB, MINB>();
    if (grid > items) grid = items;
    batch_strip_kernel<WPB, MINB><<<grid, WPB * 32, WPB * sizeof(StripWarpSmem), st>>>(b, nseg, items);
}

// warps per block and resident blocks of FP32 strip launch shape `tile`
static void strip_shape_geometry(int tile, int* wpb, int* blocks) {
    if (tile == 1) { *wpb = 12; *blocks = batch_strip_blocks<12, 1>(); }
    else if (tile == 2) { *wpb = 8; *blocks = batch_strip_blocks<8, 1>(); }
    else { *wpb = 8; *blocks = batch_strip_blocks<8, 2>(); }
}

template <typename R>
static void launch_batch_field(int tile, int blocks, int64_t nseg, const BatchArgs& b, cudaStream_t st) {
    if constexpr (sizeof(R) == 8) {
        // FP64: the 32x4 tile only (shared memory)
        (void)tile;
        (void)nseg;
        set_smem_attr<R, 32, 4>();
        batch_field_kernel<R, 32, 4><<<blocks, 128, Tile<R, 32, 4>::bytes, st>>>(b);
    } else if (tile == 1) {
        launch_strip_shape<12, 1>(nseg, b, st);
    } else if (tile == 2) {
        launch_strip_shape<8, 1>(nseg, b, st);
    } else {
        launch_strip_shape<8, 2>(nseg, b, st);
    }
}

// resident blocks of the fused kernel on the whole GPU (occupancy x SMs)
template <typename R, int TX, int TY>
static int fused_grid() {
    static int grid[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!grid[dev]) {
        set_smem_attr<R, TX, TY>();
        int per_sm = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_fused_kernel<R, TX, TY>, TX * TY,
                                                      Tile<R, TX, TY>::bytes);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid[dev] = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    }
    return grid[dev];
}

template <typename R, int TX, int TY>
static void launch_fused_t(const BatchArgs& b, int lag, int n_field, int n_push, cudaStream_t st) {
    int g = fused_grid<R, TX, TY>();
    const int total = n_field + n_push;
    if (g > total) g = total;
    if (g < 1) return;
    batch_fused_kernel<R, TX, TY><<<g, TX * TY, Tile<R, TX, TY>::bytes, st>>>(b, lag, n_field, n_push);
}

// FP32: the persistent fused launch over strip items and push chunks
static void launch_fused_strip(const BatchArgs& b, int lag, int64_t nseg, int n_push, cudaStream_t st) {
    static int grid[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    const int smem = 8 * (int)sizeof(StripWarpSmem);
    if (!grid[dev]) {
        cudaFuncSetAttribute(batch_fused_strip_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int per_sm = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_fused_strip_kernel, 256, smem);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid[dev] = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    }
    const int n_field = (int)((nseg + 7) / 8);
    int g = grid[dev];
    if (g > n_field + n_push) g = n_field + n_push;
    if (g < 1) return;
    batch_fused_strip_kernel<<<g, 256, smem, st>>>(b, lag, nseg, n_field, n_push);
}

template <typename R>
static void launch_batch_fused(int tile, const BatchArgs& b, int lag, int n_field, int64_t nseg, int n_push,
                               cudaStream_t st) {
    if constexpr (sizeof(R) == 8) {
        (void)tile;
        (void)nseg;
        launch_fused_t<R, 32, 4>(b, lag, n_field, n_push, st);
    } else {
        (void)tile;
        (void)n_field;
        launch_fused_strip(b, lag, nseg, n_push, st);
    }
}

}  // namespace gl

using namespace gl;

struct gl_batch {
    int ne;
    int prec;
    double dt;
    int reunit_every;
    cudaStream_t stream;
    cudaStream_t aux;      // push stream of the overlapped step
    cudaEvent_t ev_a, ev_b;
    gl_ctx** ev;
    EvDesc* h_desc;
    EvDesc* h_prev;        // descriptors last uploaded (valid if desc_valid)
    int desc_valid;
    int64_t clock_host;    // value of the device step counter after the enqueued work
    EvDesc* d_desc;
    int64_t* d_clock;
    BObs* h_obs;
    BObs* d_obs;
    double* d_obs_all;  // [ne][OBS_W], gathered obs rows
    SortEv* h_sort;
    SortEv* d_sort;
    int* sort_every;  // per event (0: no sorting)
    int tile;         // autotuned tile shape
    int push_block;   // autotuned push block size (separate push kernel)
    int push_chunk;   // particles per push block
    int fused;        // 1: one persistent fused launch per step; 0: field and push on two streams
    int push_grid;    // two streams: 0 = one push block per chunk, k > 0 = k resident 128-thread blocks per SM
    int field_blocks;      // FP64: tiles of all events
    int64_t field_segs;    // FP32: segments of all events' strips
    int seg_rows;          // FP32: rows per segment, for the current launch shape
    int seg_tuned[N_TILES];  // FP32: the autotuner's segment length per launch shape (0: the cost model's)
    int push_blocks;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int graph_tile, graph_push_block, graph_push_chunk, graph_fused, graph_push_grid;
    float tune_field_ms[N_TILES];
    float tune_push_ms[3];
    // trial steps: two streams; fused by push chunk; two streams with 1 and 2
    // resident push blocks per SM beside field shapes 0 and 1
    float tune_step_ms[1 + N_CHUNKS + 4];
    int* h_bad;  // pinned [ne]: the index-check flags of a native particle upload (allocated on first use)
    PartsCheckEv* p_pchk;  // pinned [ne]: the index-check descriptors (allocated with h_bad)
    PartsCheckEv* d_pchk;  // [ne] the same on the device, and
    int* d_bad;            // [ne] the index-check flags
    // observables requests: two slots, each with a pinned copy of h_obs for
    // its upload, pinned [ne][OBS_W] for the gathered rows, and an event
    // after its copy back (allocated on first use); obs_count requests are
    // outstanding, the oldest in slot obs_head
    BObs* p_obs[2];
    double* p_rows[2];
    cudaEvent_t obs_done[2];
    uint32_t obs_what[2];
    int obs_head, obs_count;
    char err[256];
};

static size_t a256b(size_t b) { return (b + 255) & ~(size_t)255; }

static gl_status bfail(gl_batch* b, gl_status s, const char* m) {
    if (b) {
        strncpy(b->err, m, sizeof b->err - 1);
        b->err[sizeof b->err - 1] = 0;
    }
    return s;
}

extern "C" {
// the strip segment length of the current launch shape: the one set or
// tuned for it, else the one that spreads all events' strips evenly over its
// resident warps (0: out of host memory)
static int batch_seg_rows(const gl_batch* b) {
    if (b->seg_tuned[b->tile] > 0) return b->seg_tuned[b->tile];
    int wpb = 8, blocks = 1;
    strip_shape_geometry(b->tile, &wpb, &blocks);
    int* Ns = new (std::nothrow) int[b->ne];
    if (!Ns) return 0;
    for (int e = 0; e < b->ne; e++) {
        CtxView v;
        ctx_view(b->ev[e], &v);
        Ns[e] = v.N;
    }
    const int rows = strip_seg_rows(Ns, b->ne, wpb, blocks);
    delete[] Ns;
    return rows;
}

static gl_status sync_desc(gl_batch* b);
}

// descriptors for an autotune trial: the prefix tables of the current tile
// shape and push chunk, the particles pointed at the contexts' spare buffers
static gl_status trial_desc(gl_batch* b) {
    b->desc_valid = 0;
    if (gl_status s = sync_desc(b)) return s;
    for (int e = 0; e < b->ne; e++) {
        CtxView v;
        ctx_view(b->ev[e], &v);
        b->h_desc[e].parts = v.parts_alt;
    }
    cudaMemcpyAsync(b->d_desc, b->h_desc, sizeof(EvDesc) * b->ne, cudaMemcpyHostToDevice, b->stream);
    b->desc_valid = 0;  // the device now holds the trial descriptors
    return GL_OK;
}

// mean duration (ms) of reps - 1 timed repetitions of `launch` after one untimed
template <typename F>
static float time_trial(gl_batch* b, cudaEvent_t e0, cudaEvent_t e1, int reps, F launch) {
    float total = 0;
    for (int rep = 0; rep < reps; rep++) {
        cudaEventRecord(e0, b->stream);
        launch();
        cudaEventRecord(e1, b->stream);
        cudaEventSynchronize(e1);
        float m = 0;
        cudaEventElapsedTime(&m, e0, e1);
        if (rep > 0) total += m;
    }
    return total / (reps - 1);
}

extern "C" {

size_t gl_batch_obs_row_bytes(void) { return sizeof(double) * OBS_W; }

size_t gl_batch_workspace_bytes(const gl_config* cfgs, const gl_species* species, int32_t n_species,
                                int32_t n_events) {
    if (!cfgs || n_events < 1 || n_events > MAX_EVENTS) return 0;
    size_t o = a256b(sizeof(EvDesc) * n_events) + 256 + a256b(sizeof(BObs) * n_events) +
               a256b(sizeof(double) * OBS_W * n_events) + a256b(sizeof(SortEv) * n_events) +
               a256b(sizeof(PartsCheckEv) * n_events) + a256b(sizeof(int) * n_events);
    for (int e = 0; e < n_events; e++) {
        const size_t w = ctx_workspace_bytes(&cfgs[e], species ? species + (size_t)e * n_species : nullptr, n_species);
        if (!w) return 0;
        o += a256b(w);
    }
    return o;
}

gl_status gl_batch_create(const gl_config* cfgs, const gl_species* species, int32_t n_species, int32_t n_events,
                          void* d_workspace, size_t bytes, void* stream, gl_batch** out) {
    if (!out) return GL_ERR_ARG;
    *out = nullptr;
    const size_t need = gl_batch_workspace_bytes(cfgs, species, n_species, n_events);
    if (!need) return GL_ERR_ARG;
    if (bytes < need) return GL_ERR_SIZE;
    if (!d_workspace || ((uintptr_t)d_workspace & 255)) return GL_ERR_ARG;
    for (int e = 0; e < n_events; e++)
        if (cfgs[e].n_jets != 0) return GL_ERR_ARG;  // jet probes: single events only
    for (int e = 1; e < n_events; e++)
        if (cfgs[e].precision != cfgs[0].precision || cfgs[e].dtau_over_a != cfgs[0].dtau_over_a ||
            cfgs[e].reunit_every != cfgs[0].reunit_every)
            return GL_ERR_ARG;  // one precision, time step and re-unitarisation period per batch
    gl_batch* b = new (std::nothrow) gl_batch;
    if (!b) return GL_ERR_ARG;
    memset(b, 0, sizeof *b);
    b->ne = n_events;
    b->prec = cfgs[0].precision;
    b->dt = cfgs[0].dtau_over_a;
    b->reunit_every = cfgs[0].precision == GL_FP32_2ROW ? cfgs[0].reunit_every : 0;
    b->stream = (cudaStream_t)stream;
    b->ev = new (std::nothrow) gl_ctx*[n_events]();
    b->h_desc = new (std::nothrow) EvDesc[n_events]();
    b->h_prev = new (std::nothrow) EvDesc[n_events]();
    b->h_obs = new (std::nothrow) BObs[n_events]();
    b->h_sort = new (std::nothrow) SortEv[n_events]();
    b->sort_every = new (std::nothrow) int[n_events]();
    if (!b->ev || !b->h_desc || !b->h_prev || !b->h_obs || !b->h_sort || !b->sort_every) {
        delete[] b->ev;
        delete[] b->h_desc;
        delete[] b->h_prev;
        delete[] b->h_obs;
        delete[] b->h_sort;
        delete[] b->sort_every;
        delete b;
        return GL_ERR_ARG;
    }
    char* ws = (char*)d_workspace;
    size_t o = 0;
    b->d_desc = (EvDesc*)ws;
    o += a256b(sizeof(EvDesc) * n_events);
    b->d_clock = (int64_t*)(ws + o);
    o += 256;
    b->d_obs = (BObs*)(ws + o);
    o += a256b(sizeof(BObs) * n_events);
    b->d_obs_all = (double*)(ws + o);
    o += a256b(sizeof(double) * OBS_W * n_events);
    b->d_sort = (SortEv*)(ws + o);
    o += a256b(sizeof(SortEv) * n_events);
    b->d_pchk = (PartsCheckEv*)(ws + o);
    o += a256b(sizeof(PartsCheckEv) * n_events);
    b->d_bad = (int*)(ws + o);
    o += a256b(sizeof(int) * n_events);
    for (int e = 0; e < n_events; e++) {
        const gl_species* sp = species ? species + (size_t)e * n_species : nullptr;
        const size_t w = ctx_workspace_bytes(&cfgs[e], sp, n_species);
        gl_status s = gl_create(&cfgs[e], sp, n_species, ws + o, w, stream, &b->ev[e]);
        if (s != GL_OK) {
            for (int k = 0; k < e; k++) gl_destroy(b->ev[k]);
            delete[] b->ev;
            delete[] b->h_desc;
            delete[] b->h_prev;
            delete[] b->h_obs;
            delete[] b->h_sort;
            delete[] b->sort_every;
            delete b;
            return s;
        }
        o += a256b(w);
    }
    b->tile = b->prec == GL_FP64 ? TILE_32x4 : 0;
    b->seg_rows = 16;  // replaced by the first descriptor sync
    b->push_block = 128;
    b->push_chunk = PUSH_CHUNK;
    b->fused = 0;
    b->push_grid = 0;
    b->graph_tile = -1;
    *out = b;
    return GL_OK;
}

gl_status gl_batch_destroy(gl_batch* b) {
    if (!b) return GL_ERR_ARG;
    if (b->aux) {
        cudaStreamSynchronize(b->aux);
        cudaEventDestroy(b->ev_a);
        cudaEventDestroy(b->ev_b);
        cudaStreamDestroy(b->aux);
    }
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->h_bad) cudaFreeHost(b->h_bad);
    if (b->p_pchk) cudaFreeHost(b->p_pchk);
    for (int k = 0; k < 2; k++) {
        if (b->obs_done[k]) {
            cudaEventSynchronize(b->obs_done[k]);  // no copy lands in freed memory
            cudaEventDestroy(b->obs_done[k]);
        }
        if (b->p_obs[k]) cudaFreeHost(b->p_obs[k]);
        if (b->p_rows[k]) cudaFreeHost(b->p_rows[k]);
    }
    for (int e = 0; e < b->ne; e++) gl_destroy(b->ev[e]);
    delete[] b->ev;
    delete[] b->h_desc;
    delete[] b->h_prev;
    delete[] b->h_obs;
    delete[] b->h_sort;
    delete[] b->sort_every;
    delete b;
    return GL_OK;
}

gl_ctx* gl_batch_event(gl_batch* b, int32_t e) { return b && e >= 0 && e < b->ne ? b->ev[e] : nullptr; }

const char* gl_batch_error_string(const gl_batch* b) { return b ? b->err : ""; }

gl_status gl_batch_init(gl_batch* b) {
    gl::ApiRange range_("gl_batch_init");
    if (!b) return GL_ERR_ARG;
    b->desc_valid = 0;
    for (int e = 0; e < b->ne; e++) {
        gl_status s = glasma_init(b->ev[e]);
        if (s == GL_OK) s = wong_init(b->ev[e]);
        if (s != GL_OK) {
            char m[300];
            snprintf(m, sizeof m, "event %d: %s", e, gl_error_string(b->ev[e]));
            return bfail(b, s, m);
        }
    }
    return GL_OK;
}

// refresh the device descriptors from the contexts; all events must be at the
// same step with their particles at that step
static gl_status sync_desc(gl_batch* b) {
    int tb = 0, cb = 0;
    int64_t rb = 0;
    const int TX = TILE_DIMS[b->tile][0], TY = TILE_DIMS[b->tile][1];
    int64_t step0 = -1;
    if (b->prec != GL_FP64) {
        b->seg_rows = batch_seg_rows(b);
        if (b->seg_rows < 1) return bfail(b, GL_ERR_ARG, "out of host memory");
    }
    for (int e = 0; e < b->ne; e++) {
        CtxView v;
        ctx_view(b->ev[e], &v);
        if (step0 < 0) step0 = v.step;
        if (v.step != step0 || v.pstep != v.step || v.cur != (int)(v.step & 1))
            return bfail(b, GL_ERR_STATE, "batch events must be at one common step with their particles");
        EvDesc& d = b->h_desc[e];
        memset(&d, 0, sizeof d);
        d.field[0] = v.field[0];
        d.field[1] = v.field[1];
        d.site[0] = v.site[0];
        d.site[1] = v.site[1];
        d.parts = v.parts;
        d.N = v.N;
        d.tiles_x = (v.N + TX - 1) / TX;
        d.tile_begin = tb;
        tb += d.tiles_x * ((v.N + TY - 1) / TY);
        d.seg_begin = rb;
        rb += b->prec != GL_FP64 ? strip_segments(v.N, b->seg_rows) : 0;
        d.chunk_begin = cb;
        cb += (int)((v.np + b->push_chunk - 1) / b->push_chunk);
        d.np = v.np;
        d.n_species = v.ns;
        d.ptau_diag = v.ptau_diag;
        b->sort_every[e] = v.sort_every;
        for (int k = 0; k < GL_MAX_SPECIES; k++) {
            d.mass[k] = v.mass[k];
            d.motion[k] = v.motion[k];
            d.t_form[k] = v.t_form[k];
        }
    }
    b->field_blocks = tb;
    b->field_segs = rb;
    b->push_blocks = cb;
    // nothing changed since the last upload (the usual case between steps):
    // no copy and no wait
    if (b->desc_valid && b->clock_host == step0 && memcmp(b->h_prev, b->h_desc, sizeof(EvDesc) * b->ne) == 0)
        return GL_OK;
    cudaMemcpyAsync(b->d_desc, b->h_desc, sizeof(EvDesc) * b->ne, cudaMemcpyHostToDevice, b->stream);
    cudaMemcpyAsync(b->d_clock, &step0, sizeof step0, cudaMemcpyHostToDevice, b->stream);
    cudaStreamSynchronize(b->stream);
    if (cudaGetLastError() != cudaSuccess) return bfail(b, GL_ERR_CUDA, "descriptor upload failed");
    memcpy(b->h_prev, b->h_desc, sizeof(EvDesc) * b->ne);
    b->clock_host = step0;
    b->desc_valid = 1;
    return GL_OK;
}

static BatchArgs batch_args(const gl_batch* b, int reunit_every) {
    return BatchArgs{b->d_desc, b->ne, b->dt, reunit_every, b->d_clock, b->push_chunk, b->seg_rows};
}

static void launch_field(gl_batch* b, cudaStream_t st) {
    const BatchArgs a = batch_args(b, b->reunit_every);
    if (b->prec == GL_FP64) launch_batch_field<double>(b->tile, b->field_blocks, b->field_segs, a, st);
    else launch_batch_field<float>(b->tile, b->field_blocks, b->field_segs, a, st);
}

static int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// the separate push kernel: one block per chunk, or push_grid resident blocks per SM
static void launch_push_shape(gl_batch* b, const BatchArgs& a, int lag, int push_block, int push_grid,
                              cudaStream_t st) {
    if (b->push_blocks < 1) return;
    if (push_grid > 0) {
        int g = push_grid * sm_count();
        if (g > b->push_blocks) g = b->push_blocks;
        if (b->prec == GL_FP64) batch_push_persist_kernel<double><<<g, 128, 0, st>>>(a, lag, b->push_blocks);
        else batch_push_persist_kernel<float><<<g, 128, 0, st>>>(a, lag, b->push_blocks);
    } else if (b->prec == GL_FP64) {
        launch_batch_push<double>(push_block, b->push_blocks, a, lag, st);
    } else {
        launch_batch_push<float>(push_block, b->push_blocks, a, lag, st);
    }
}

// a push with nothing beside it: one block per chunk
static void launch_push(gl_batch* b, int lag, cudaStream_t st) {
    launch_push_shape(b, batch_args(b, b->reunit_every), lag, b->push_block, 0, st);
}

static void launch_fused(gl_batch* b, int lag, cudaStream_t st) {
    const BatchArgs a = batch_args(b, b->reunit_every);
    if (b->prec == GL_FP64) launch_batch_fused<double>(b->tile, a, lag, b->field_blocks, b->field_segs, b->push_blocks, st);
    else launch_batch_fused<float>(b->tile, a, lag, b->field_blocks, b->field_segs, b->push_blocks, st);
}

// one steady-state step at clock s, the field step of t_s and the push of the
// particles at t_{s-1}, then the tick: either one fused persistent launch, or
// the two kernels on the main and the second stream
static void enqueue_overlap_step(gl_batch* b) {
    if (b->fused) {
        launch_fused(b, 1, b->stream);
        tick_kernel<<<1, 1, 0, b->stream>>>(b->d_clock);
        return;
    }
    cudaEventRecord(b->ev_a, b->stream);
    cudaStreamWaitEvent(b->aux, b->ev_a, 0);
    launch_push_shape(b, batch_args(b, b->reunit_every), 1, b->push_block, b->push_grid, b->aux);
    cudaEventRecord(b->ev_b, b->aux);
    launch_field(b, b->stream);
    cudaStreamWaitEvent(b->stream, b->ev_b, 0);
    tick_kernel<<<1, 1, 0, b->stream>>>(b->d_clock);
}

static gl_status ensure_aux(gl_batch* b);

gl_status gl_batch_autotune(gl_batch* b, int32_t* tile_out, int32_t* push_block_out) {
    gl::ApiRange range_("gl_batch_autotune");
    if (!b) return GL_ERR_ARG;
    b->desc_valid = 0;  // the trials rewrite the device descriptors and clock
    if (gl_status s = ensure_aux(b)) return s;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int k = 0; k < N_TILES; k++) b->tune_field_ms[k] = 0;
    for (int k = 0; k < 3; k++) b->tune_push_ms[k] = 0;
    for (int k = 0; k < 1 + N_CHUNKS + 4; k++) b->tune_step_ms[k] = 0;
    // field kernel: trial launches write only the spare time slice and the
    // site fields, which the next real step overwrites
    float best_f = 1e30f;
    int bt = b->tile;
    for (int tile = 0; tile < N_TILES; tile++) {
        if (b->prec == GL_FP64 && tile != TILE_32x4) continue;  // FP64 tile must fit shared memory
        b->tile = tile;
        // FP32: the segment lengths tried beside the cost model's choice (its
        // half and double, and 16 rows); the fastest is kept for the shape
        int cand[4] = {0, 0, 0, 0}, nc = 1;
        if (b->prec != GL_FP64) {
            b->seg_tuned[tile] = 0;
            if (gl_status s = sync_desc(b)) return s;
            const int m = b->seg_rows;
            const int more[3] = {16, 2 * m, m / 2};
            cand[0] = m;
            for (int k = 0; k < 3; k++) {
                bool dup = more[k] < 4;
                for (int c = 0; c < nc; c++) dup = dup || cand[c] == more[k];
                if (!dup) cand[nc++] = more[k];
            }
        }
        float best_t = 1e30f;
        int best_seg = 0;
        for (int c = 0; c < nc; c++) {
            if (b->prec != GL_FP64) b->seg_tuned[tile] = cand[c];
            if (gl_status s = sync_desc(b)) return s;
            const BatchArgs a = batch_args(b, 0);
            const float ms = time_trial(b, e0, e1, 4, [&] {
                if (b->prec == GL_FP64) launch_batch_field<double>(tile, b->field_blocks, b->field_segs, a, b->stream);
                else launch_batch_field<float>(tile, b->field_blocks, b->field_segs, a, b->stream);
            });
            if (ms < best_t) { best_t = ms; best_seg = cand[c]; }
        }
        if (b->prec != GL_FP64) b->seg_tuned[tile] = best_seg;
        b->tune_field_ms[tile] = best_t;
        if (best_t < best_f) { best_f = best_t; bt = tile; }
    }
    b->tile = bt;
    if (gl_status s = sync_desc(b)) return s;
    // push and whole-step trials on a copy of the particles (the contexts'
    // spare buffers), at a time where every species is formed
    EvDesc* saved = new EvDesc[b->ne];
    memcpy(saved, b->h_desc, sizeof(EvDesc) * b->ne);
    bool have_copy = b->push_blocks > 0;
    for (int e = 0; e < b->ne && have_copy; e++) {
        CtxView v;
        ctx_view(b->ev[e], &v);
        if (v.np == 0) continue;  // nothing to push or copy
        if (!v.parts_alt) { have_copy = false; break; }
        cudaMemcpyAsync(v.parts_alt, v.parts, particle_bytes(b->prec, v.np), cudaMemcpyDeviceToDevice, b->stream);
        b->h_desc[e].parts = v.parts_alt;
    }
    int bp = b->push_block, bc = b->push_chunk, bf = b->fused;
    if (have_copy) {
        int64_t trial = 0, now = 0;
        for (int e = 0; e < b->ne; e++)
            for (int k = 0; k < b->h_desc[e].n_species; k++) {
                const int64_t n = (int64_t)ceil(b->h_desc[e].t_form[k] / b->dt);
                if (n > trial) trial = n;
            }
        cudaMemcpyAsync(&now, b->d_clock, sizeof now, cudaMemcpyDeviceToHost, b->stream);
        cudaStreamSynchronize(b->stream);
        if (trial < now) trial = now;
        // the push of t_trial runs with the clock at `now` and lag now - trial,
        // so that the field part of a trial step still writes the spare slice
        const int lag = (int)(now - trial);
        cudaMemcpyAsync(b->d_desc, b->h_desc, sizeof(EvDesc) * b->ne, cudaMemcpyHostToDevice, b->stream);
        const BatchArgs a = batch_args(b, 0);
        for (int k = 0; k < 3; k++) {
            const float ms = time_trial(b, e0, e1, 4, [&] {
                if (b->prec == GL_FP64) launch_batch_push<double>(PUSH_BLOCKS[k], b->push_blocks, a, lag, b->stream);
                else launch_batch_push<float>(PUSH_BLOCKS[k], b->push_blocks, a, lag, b->stream);
            });
            b->tune_push_ms[k] = ms;
        }
        // whole steps: field and push on two streams (the push one block per
        // chunk at each chunk and block size, or 1 or 2 resident blocks per SM
        // launched first, beside each field tile shape), or one fused launch
        // by push chunk.  The push block and chunk sizes are chosen here, by
        // the time of the whole overlapped step, not by the push timed alone:
        // beside the field kernel a smaller block often fills the SMs better,
        // and short chunks shorten the tail of blocks of unequal length.
        float best_s = 1e30f;
        int bt2 = b->tile, bg = 0;
        bf = 0;
        bc = b->push_chunk;
        const int tile0 = b->tile;
        for (int g = 0; g <= 2; g++)
            for (int tile = 0; tile < N_TILES; tile++) {
                if (b->prec == GL_FP64 && tile != TILE_32x4) continue;
                // resident push blocks (g > 0) leave no room beside the
                // 512-thread tiles; the plain two-stream step tries every
                // tile shape, since the fastest field kernel alone is not
                // always the fastest beside the push
                if (g > 0 && b->prec == GL_FP64 && tile == TILE_32x16) continue;
                b->tile = tile;
                float best_g = 1e30f;
                const bool per_chunk = g == 0;  // separate push blocks, one per chunk
                for (int kc = 0; kc < (per_chunk ? N_SEP_CHUNKS : 1); kc++) {
                    b->push_chunk = per_chunk ? SEP_CHUNKS[kc] : PUSH_CHUNK;
                    if (gl_status s = trial_desc(b)) return s;
                    const BatchArgs ag = batch_args(b, 0);
                    for (int kb = 0; kb < (per_chunk ? 3 : 1); kb++) {
                        const int blk = per_chunk ? PUSH_BLOCKS[kb] : 128;
                        if (blk > b->push_chunk) continue;  // threads without particles
                        const float ms = time_trial(b, e0, e1, 4, [&] {
                            cudaEventRecord(b->ev_a, b->stream);
                            cudaStreamWaitEvent(b->aux, b->ev_a, 0);
                            launch_push_shape(b, ag, lag, blk, g, b->aux);
                            cudaEventRecord(b->ev_b, b->aux);
                            if (b->prec == GL_FP64)
                                launch_batch_field<double>(tile, b->field_blocks, b->field_segs, ag, b->stream);
                            else launch_batch_field<float>(tile, b->field_blocks, b->field_segs, ag, b->stream);
                            cudaStreamWaitEvent(b->stream, b->ev_b, 0);
                        });
                        if (ms < best_g) best_g = ms;
                        if (ms < best_s) {
                            best_s = ms;
                            bt2 = tile;
                            bg = g;
                            bc = b->push_chunk;
                            if (per_chunk) bp = blk;
                        }
                    }
                }
                float& slot = b->tune_step_ms[g == 0 ? 0 : 1 + N_CHUNKS + 2 * (g - 1) + (tile == TILE_32x4)];
                if (slot == 0 || best_g < slot) slot = best_g;
            }
        b->tile = tile0;
        for (int k = 0; k < N_CHUNKS; k++) {
            b->push_chunk = PUSH_CHUNKS[k];
            if (gl_status s = trial_desc(b)) return s;
            const BatchArgs ak = batch_args(b, 0);
            const float ms = time_trial(b, e0, e1, 4, [&] {
                if (b->prec == GL_FP64)
                    launch_batch_fused<double>(b->tile, ak, lag, b->field_blocks, b->field_segs, b->push_blocks,
                                               b->stream);
                else launch_batch_fused<float>(b->tile, ak, lag, b->field_blocks, b->field_segs, b->push_blocks,
                                               b->stream);
            });
            b->tune_step_ms[1 + k] = ms;
            if (ms < best_s) { best_s = ms; bf = 1; bc = PUSH_CHUNKS[k]; bg = 0; bt2 = tile0; }
        }
        b->push_chunk = bc;
        b->tile = bt2;
        b->push_grid = bg;
    }
    memcpy(b->h_desc, saved, sizeof(EvDesc) * b->ne);
    delete[] saved;
    b->desc_valid = 0;
    b->push_block = bp;
    b->push_chunk = bc;
    b->fused = bf;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (gl_status s = sync_desc(b)) return s;  // real particles, clock and chunk tables
    if (tile_out) *tile_out = b->tile;
    if (push_block_out) *push_block_out = b->push_block;
    return cudaGetLastError() == cudaSuccess ? GL_OK : bfail(b, GL_ERR_CUDA, "autotune launch failed");
}

static gl_status ensure_aux(gl_batch* b) {
    if (b->aux) return GL_OK;
    if (cudaStreamCreateWithFlags(&b->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_a, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_b, cudaEventDisableTiming) != cudaSuccess)
        return bfail(b, GL_ERR_CUDA, "stream creation failed");
    return GL_OK;
}

// steps from the common step `now` to the next sort of any event (at most n)
static int32_t segment_length(const gl_batch* b, int64_t now, int32_t n) {
    int32_t m = n;
    for (int e = 0; e < b->ne; e++) {
        const int se = b->sort_every[e];
        if (se <= 0) continue;
        const int64_t d = se - now % se;
        if (d < m) m = (int32_t)d;
    }
    return m;
}

// after a segment that ended at step `now`: advance the contexts and sort the
// particles of the events whose period divides `now` (between the push and
// the next field step, as the single-event schedule does)
static void end_segment(gl_batch* b, int32_t m, int64_t now) {
    int n = 0, pb = 0, cb = 0, passes = 1;
    for (int e = 0; e < b->ne; e++) {
        ctx_advance(b->ev[e], m);
        if (b->sort_every[e] > 0 && now % b->sort_every[e] == 0) {
            CtxView v;
            ctx_view(b->ev[e], &v);
            if (v.np <= 0) continue;
            SortEv& d = b->h_sort[n++];
            d = sort_event(v.parts, v.parts_alt, v.np, v.N, v.ns, v.motion, v.sort_scratch);
            d.pblk_begin = pb;
            d.cblk_begin = cb;
            pb += sort_particle_blocks(v.np);
            cb += sort_cell_blocks(d);
            if (sort_passes(d) > passes) passes = sort_passes(d);
            ctx_swap_parts(b->ev[e]);
        }
    }
    if (n == 0) return;
    cudaMemcpyAsync(b->d_sort, b->h_sort, sizeof(SortEv) * n, cudaMemcpyHostToDevice, b->stream);
    launch_sort_many(b->prec, b->d_sort, n, pb, cb, passes, b->stream);
}

static int64_t common_step(const gl_batch* b) {
    CtxView v;
    ctx_view(b->ev[0], &v);
    return v.step;
}

// n coupled steps.  Per segment between sorts: the field step of t_s (all
// events) alone, then m - 1 replays of the captured overlapped step, then the
// last push alone.
gl_status gl_batch_step(gl_batch* b, int32_t n_steps) {
    gl::ApiRange range_("gl_batch_step");
    if (!b || n_steps < 0) return GL_ERR_ARG;
    if (n_steps == 0) return GL_OK;
    if (gl_status s = sync_desc(b)) return s;
    if (gl_status s = ensure_aux(b)) return s;
    if (b->prec == GL_FP64) set_smem_attr<double, 32, 4>();
    // (re)capture the overlapped step when the launch shapes changed
    if (!b->exec || b->graph_tile != b->tile || b->graph_push_block != b->push_block ||
        b->graph_push_chunk != b->push_chunk || b->graph_fused != b->fused || b->graph_push_grid != b->push_grid) {
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return bfail(b, GL_ERR_CUDA, "stream capture could not start (the default stream cannot be captured)");
        enqueue_overlap_step(b);
        if (cudaStreamEndCapture(b->stream, &b->graph) != cudaSuccess ||
            cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) {
            cudaGetLastError();
            return bfail(b, GL_ERR_CUDA, "graph capture failed");
        }
        b->graph_tile = b->tile;
        b->graph_push_block = b->push_block;
        b->graph_push_chunk = b->push_chunk;
        b->graph_fused = b->fused;
        b->graph_push_grid = b->push_grid;
    }
    int64_t now = common_step(b);
    for (int32_t left = n_steps; left > 0;) {
        const int32_t m = segment_length(b, now, left);
        launch_field(b, b->stream);
        tick_kernel<<<1, 1, 0, b->stream>>>(b->d_clock);
        for (int k = 1; k < m; k++) cudaGraphLaunch(b->exec, b->stream);
        launch_push(b, 1, b->stream);
        if (cudaGetLastError() != cudaSuccess) return bfail(b, GL_ERR_CUDA, "batch step launch failed");
        now += m;
        left -= m;
        b->clock_host += m;
        end_segment(b, m, now);
        if (left > 0)
            if (gl_status s = sync_desc(b)) return s;
    }
    return GL_OK;
}

// The same steps with the field and push launches of each step run one after
// the other on the batch stream (no overlap), each bracketed by CUDA events:
// returns the summed durations of the field and push kernels (waits).  The
// state evolves exactly as under gl_batch_step.
gl_status gl_batch_step_timed(gl_batch* b, int32_t n_steps, double* field_ms, double* push_ms) {
    gl::ApiRange range_("gl_batch_step_timed");
    if (!b || n_steps < 1) return GL_ERR_ARG;
    if (gl_status s = sync_desc(b)) return s;
    const int ne = 4 * n_steps;
    cudaEvent_t* ev = new (std::nothrow) cudaEvent_t[ne];
    if (!ev) return GL_ERR_ARG;
    for (int k = 0; k < ne; k++) cudaEventCreate(&ev[k]);
    // events 4k, 4k+1 bracket the field launch of step k; 4k+2, 4k+3 its push
    int64_t now = common_step(b);
    gl_status st = GL_OK;
    for (int32_t done = 0; done < n_steps && st == GL_OK;) {
        const int32_t m = segment_length(b, now, n_steps - done);
        for (int32_t k = done; k < done + m; k++) {
            cudaEventRecord(ev[4 * k], b->stream);
            launch_field(b, b->stream);
            cudaEventRecord(ev[4 * k + 1], b->stream);
            tick_kernel<<<1, 1, 0, b->stream>>>(b->d_clock);
            cudaEventRecord(ev[4 * k + 2], b->stream);
            launch_push(b, 1, b->stream);
            cudaEventRecord(ev[4 * k + 3], b->stream);
        }
        now += m;
        done += m;
        b->clock_host += m;
        end_segment(b, m, now);
        if (done < n_steps) st = sync_desc(b);
    }
    cudaStreamSynchronize(b->stream);
    double f = 0, p = 0;
    for (int k = 0; k < n_steps && st == GL_OK; k++) {
        float a = 0, c = 0;
        cudaEventElapsedTime(&a, ev[4 * k], ev[4 * k + 1]);
        cudaEventElapsedTime(&c, ev[4 * k + 2], ev[4 * k + 3]);
        f += a;
        p += c;
    }
    for (int k = 0; k < ne; k++) cudaEventDestroy(ev[k]);
    delete[] ev;
    if (st != GL_OK) return st;
    if (field_ms) *field_ms = f;
    if (push_ms) *push_ms = p;
    if (cudaGetLastError() != cudaSuccess) return bfail(b, GL_ERR_CUDA, "timed batch step failed");
    return GL_OK;
}

static gl_status ensure_aux(gl_batch* b);

// events alternate between the batch stream and the second one (each event has
// its own staging and sort buffers), so that one event's host copy overlaps
// another's conversion and sort
gl_status gl_batch_upload(gl_batch* b, gl_buffer which, const double* const* host, const size_t* count) {
    gl::ApiRange range_("gl_batch_upload");
    if (!b || !host || !count) return GL_ERR_ARG;
    if (gl_status s = ensure_aux(b)) return s;
    cudaEventRecord(b->ev_a, b->stream);
    cudaStreamWaitEvent(b->aux, b->ev_a, 0);
    gl_status st = GL_OK;
    int bad = -1;
    for (int e = 0; e < b->ne && st == GL_OK; e++) {
        st = ctx_upload_enqueue(b->ev[e], which, host[e], count[e], (e & 1) ? b->aux : b->stream);
        if (st != GL_OK) bad = e;
    }
    cudaEventRecord(b->ev_b, b->aux);
    cudaStreamWaitEvent(b->stream, b->ev_b, 0);
    const bool ok = cudaStreamSynchronize(b->stream) == cudaSuccess && cudaGetLastError() == cudaSuccess;
    if (bad >= 0) {
        char m[300];
        snprintf(m, sizeof m, "event %d: %s", bad, gl_error_string(b->ev[bad]));
        return bfail(b, st, m);
    }
    return ok ? GL_OK : bfail(b, GL_ERR_CUDA, "batch upload failed");
}

// as gl_batch_upload: events alternate between the two streams; the index
// checks of native particles land in pinned host flags read after the wait
gl_status gl_batch_upload_native(gl_batch* b, gl_native_part part, const void* const* host, const size_t* bytes) {
    gl::ApiRange range_("gl_batch_upload_native");
    if (!b || !host || !bytes) return GL_ERR_ARG;
    if (gl_status s = ensure_aux(b)) return s;
    const bool parts = part == GL_NATIVE_PARTICLES;
    if (parts && !b->h_bad) {
        if (cudaHostAlloc((void**)&b->h_bad, sizeof(int) * b->ne, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc((void**)&b->p_pchk, sizeof(PartsCheckEv) * b->ne, cudaHostAllocDefault) != cudaSuccess) {
            if (b->h_bad) cudaFreeHost(b->h_bad);
            b->h_bad = nullptr;
            b->p_pchk = nullptr;
            return bfail(b, GL_ERR_CUDA, "pinned host allocation failed");
        }
    }
    // the copies, events alternating between the batch's two streams
    cudaEventRecord(b->ev_a, b->stream);
    cudaStreamWaitEvent(b->aux, b->ev_a, 0);
    gl_status st = GL_OK;
    int bad = -1;
    for (int e = 0; e < b->ne && st == GL_OK; e++) {
        st = ctx_upload_native_copy(b->ev[e], (int)part, host[e], bytes[e], (e & 1) ? b->aux : b->stream);
        if (st != GL_OK) bad = e;
    }
    cudaEventRecord(b->ev_b, b->aux);
    cudaStreamWaitEvent(b->stream, b->ev_b, 0);
    if (bad >= 0) {
        cudaStreamSynchronize(b->stream);
        char m[300];
        snprintf(m, sizeof m, "event %d: %s", bad, gl_error_string(b->ev[bad]));
        return bfail(b, st, m);
    }
    // particles: the index check of every event in one launch, its flags in
    // one copy (events uploaded with no bytes are checked as well: their
    // arrays are unchanged and valid)
    if (parts) {
        int blocks = 0;
        for (int e = 0; e < b->ne; e++) {
            PartsCheckEv d = ctx_parts_check_event(b->ev[e]);
            d.block_begin = blocks;
            blocks += d.nblocks;
            b->p_pchk[e] = d;
        }
        cudaMemcpyAsync(b->d_pchk, b->p_pchk, sizeof(PartsCheckEv) * b->ne, cudaMemcpyHostToDevice, b->stream);
        cudaMemsetAsync(b->d_bad, 0, sizeof(int) * b->ne, b->stream);
        launch_parts_validate_events(b->prec, b->d_pchk, b->ne, blocks, b->d_bad, b->stream);
        cudaMemcpyAsync(b->h_bad, b->d_bad, sizeof(int) * b->ne, cudaMemcpyDeviceToHost, b->stream);
    }
    const bool ok = cudaStreamSynchronize(b->stream) == cudaSuccess && cudaGetLastError() == cudaSuccess;
    if (!ok) return bfail(b, GL_ERR_CUDA, "batch native upload failed");
    if (parts)
        for (int e = 0; e < b->ne; e++)
            if (b->h_bad[e]) {
                char m[300];
                snprintf(m, sizeof m, "event %d: native particles: species or original index out of range (repaired)", e);
                return bfail(b, GL_ERR_ARG, m);
            }
    return GL_OK;
}

gl_status gl_batch_observables(gl_batch* b, gl_obs* out) { return gl_batch_observables_ex(b, GL_OBS_ALL, out); }

// enqueue the observables of every event into slot k: descriptors up, the
// reductions, the gather and the copy back into the slot's pinned rows, then
// the slot's event (no wait)
static gl_status obs_enqueue(gl_batch* b, uint32_t what, int k) {
    // obs rows of all events: out pointers (also for the gather when only the
    // field checks are asked for)
    int blocks = 0, fblocks = 0;
    for (int e = 0; e < b->ne; e++) {
        ObsEvent o;
        ctx_obs_event(b->ev[e], &o);
        b->h_obs[e].out = o.out;
        b->h_obs[e].fo = o.fo;
        b->h_obs[e].fo.block_begin = fblocks;
        fblocks += o.fo.nblocks;
    }
    if (what & GL_OBS_PARTICLES) {
        for (int e = 0; e < b->ne; e++) {
            ObsEvent o;
            ctx_obs_event(b->ev[e], &o);
            BObs& d = b->h_obs[e];
            d.parts = o.parts;
            d.np = o.np;
            d.t = o.t;
            d.mask = o.mask;
            d.block_begin = blocks;
            d.nblocks = obs_blocks(o.np);
            d.partials = o.partials;
            d.out = o.out;
            d.oa.sp = o.sp;
            for (int q = 0; q < GL_MAX_SPECIES; q++) { d.oa.q2ref[q] = o.q2ref[q]; d.oa.q3ref[q] = o.q3ref[q]; }
            blocks += d.nblocks;
            // an event without particles: zero sums, as the single-event path
            if (d.nblocks == 0)
                cudaMemsetAsync(o.out, 0, GL_MAX_SPECIES * PO_N * sizeof(double), b->stream);
        }
    }
    // pinned staging: both copies are plain DMA, without the driver's bounce
    // buffer (the slot's previous copies finished before its wait returned)
    if (!b->p_obs[k]) {
        if (cudaHostAlloc((void**)&b->p_obs[k], sizeof(BObs) * b->ne, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc((void**)&b->p_rows[k], sizeof(double) * OBS_W * b->ne, cudaHostAllocDefault) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->obs_done[k], cudaEventDisableTiming) != cudaSuccess) {
            if (b->p_obs[k]) cudaFreeHost(b->p_obs[k]);
            if (b->p_rows[k]) cudaFreeHost(b->p_rows[k]);
            b->p_obs[k] = nullptr;
            b->p_rows[k] = nullptr;
            b->obs_done[k] = nullptr;
            return bfail(b, GL_ERR_CUDA, "pinned host allocation failed");
        }
    }
    memcpy(b->p_obs[k], b->h_obs, sizeof(BObs) * b->ne);
    cudaMemcpyAsync(b->d_obs, b->p_obs[k], sizeof(BObs) * b->ne, cudaMemcpyHostToDevice, b->stream);
    if (blocks > 0) {
        int ns = 0;
        for (int e = 0; e < b->ne; e++) ns = b->h_obs[e].oa.sp.n_species > ns ? b->h_obs[e].oa.sp.n_species : ns;
        const size_t smem = obs_smem_bytes(ns);
        if (b->prec == GL_FP64) {
            obs_smem_attr(batch_obs_kernel<double>);
            batch_obs_kernel<double><<<blocks, OBS_THREADS, smem, b->stream>>>(b->d_obs, b->ne);
        } else {
            obs_smem_attr(batch_obs_kernel<float>);
            batch_obs_kernel<float><<<blocks, OBS_THREADS, smem, b->stream>>>(b->d_obs, b->ne);
        }
    }
    // the field checks of all events, one launch
    if (what & GL_OBS_FIELDS)
        launch_field_obs_events(b->prec, b->h_obs[0].fo, (const char*)b->d_obs + offsetof(BObs, fo), sizeof(BObs),
                                b->ne, fblocks, false, b->stream);
    batch_obs_finish<<<b->ne, OBS_FINAL_WARPS * 32, 0, b->stream>>>(b->d_obs, what, b->d_obs_all);
    cudaMemcpyAsync(b->p_rows[k], b->d_obs_all, sizeof(double) * OBS_W * b->ne, cudaMemcpyDeviceToHost, b->stream);
    cudaEventRecord(b->obs_done[k], b->stream);
    b->obs_what[k] = what;
    if (cudaGetLastError() != cudaSuccess) return bfail(b, GL_ERR_CUDA, "batch observables launch failed");
    return GL_OK;
}

// wait for slot k's request and fill out[n_events] from its rows
static gl_status obs_finish(gl_batch* b, int k, gl_obs* out) {
    const bool ok = cudaEventSynchronize(b->obs_done[k]) == cudaSuccess && cudaGetLastError() == cudaSuccess;
    if (!ok) return bfail(b, GL_ERR_CUDA, "batch observables failed");
    for (int e = 0; e < b->ne; e++) ctx_obs_fill(b->ev[e], b->obs_what[k], b->p_rows[k] + (size_t)OBS_W * e, &out[e]);
    return GL_OK;
}

gl_status gl_batch_observables_ex(gl_batch* b, uint32_t what, gl_obs* out) {
    gl::ApiRange range_("gl_batch_observables_ex");
    if (!b || !out || (what & ~GL_OBS_ALL)) return GL_ERR_ARG;
    if (b->obs_count > 0) return bfail(b, GL_ERR_STATE, "observables requests outstanding (gl_batch_observables_end)");
    if (gl_status st = obs_enqueue(b, what, b->obs_head)) return st;
    return obs_finish(b, b->obs_head, out);
}

gl_status gl_batch_observables_begin(gl_batch* b, uint32_t what) {
    gl::ApiRange range_("gl_batch_observables_begin");
    if (!b || (what & ~GL_OBS_ALL)) return GL_ERR_ARG;
    if (b->obs_count >= 2) return bfail(b, GL_ERR_STATE, "two observables requests outstanding");
    const int k = (b->obs_head + b->obs_count) & 1;
    if (gl_status st = obs_enqueue(b, what, k)) return st;
    b->obs_count++;
    return GL_OK;
}

gl_status gl_batch_observables_end(gl_batch* b, gl_obs* out) {
    gl::ApiRange range_("gl_batch_observables_end");
    if (!b || !out) return GL_ERR_ARG;
    if (b->obs_count == 0) return bfail(b, GL_ERR_STATE, "no observables request outstanding");
    const int k = b->obs_head;
    b->obs_head ^= 1;
    b->obs_count--;
    return obs_finish(b, k, out);
}

gl_status gl_batch_set_launch(gl_batch* b, int32_t tile, int32_t push_block, int32_t push_chunk, int32_t fused,
                              int32_t push_grid) {
    if (!b || tile < 0 || tile >= N_TILES || (fused != 0 && fused != 1) || push_grid < 0 || push_grid > 2)
        return GL_ERR_ARG;
    if (b->prec == GL_FP64 && tile != TILE_32x4) return GL_ERR_ARG;
    bool ok_b = false, ok_c = false;
    for (int k = 0; k < 3; k++) ok_b = ok_b || PUSH_BLOCKS[k] == push_block;
    for (int k = 0; k < N_CHUNKS; k++) ok_c = ok_c || PUSH_CHUNKS[k] == push_chunk;
    for (int k = 0; k < N_SEP_CHUNKS; k++) ok_c = ok_c || SEP_CHUNKS[k] == push_chunk;
    if (!ok_b || !ok_c) return GL_ERR_ARG;
    b->tile = tile;
    b->push_block = push_block;
    b->push_chunk = push_chunk;
    b->fused = fused;
    b->push_grid = fused ? 0 : push_grid;
    return GL_OK;
}

int32_t gl_batch_segment_rows(const gl_batch* b) {
    if (!b || b->prec == GL_FP64) return 0;
    return b->desc_valid ? b->seg_rows : batch_seg_rows(b);  // the next launch's, also before it
}

gl_status gl_batch_set_segment_rows(gl_batch* b, int32_t rows) {
    if (!b || rows < 0 || rows > 65536) return GL_ERR_ARG;
    if (b->prec == GL_FP64) return rows == 0 ? GL_OK : GL_ERR_ARG;
    b->seg_tuned[b->tile] = rows;  // applied by the next descriptor sync
    b->desc_valid = 0;
    return GL_OK;
}

gl_status gl_batch_get_launch(const gl_batch* b, int32_t* tile, int32_t* push_block, int32_t* push_chunk,
                              int32_t* fused, int32_t* push_grid) {
    if (!b) return GL_ERR_ARG;
    if (tile) *tile = b->tile;
    if (push_block) *push_block = b->push_block;
    if (push_chunk) *push_chunk = b->push_chunk;
    if (fused) *fused = b->fused;
    if (push_grid) *push_grid = b->push_grid;
    return GL_OK;
}

gl_status gl_batch_tuning(const gl_batch* b, float* field_ms, float* push_ms, float* step_ms) {
    if (!b) return GL_ERR_ARG;
    for (int k = 0; k < N_TILES; k++)
        if (field_ms) field_ms[k] = b->tune_field_ms[k];
    for (int k = 0; k < 3; k++)
        if (push_ms) push_ms[k] = b->tune_push_ms[k];
    for (int k = 0; k < 1 + N_CHUNKS + 4; k++)
        if (step_ms) step_ms[k] = b->tune_step_ms[k];
    return GL_OK;
}

}  // extern "C"
