// Counting sort of the particles by lattice row, then by motion class (Wong,
// static, eikonal), then by nearest-grid-point cell: the push reads the site
// fields of neighbouring particles from the same cache lines (a row's fields
// stay in cache while its classes are pushed one after the other), and the 32
// particles of a warp are (but at the edges of a row's class ranges) of one
// class, so they take one branch of the push instead of running every branch
// present with the other lanes idle.  Species of one class stay mixed by cell.
//
//   count:    key[i] = (y ng + g) N + x for particle i of class g (of ng
//             classes present) in cell (x, y), rank[i] = atomic slot within
//             its key
//   scan:     off[k] = number of particles with keys < k (two-level block scan)
//   scatter:  perm[off[key[i]] + rank[i]] = i
//   order:    each key's entries of perm sorted ascending, so the result does
//             not depend on the order the atomics were served in
//   gather:   new[j] = old[perm[j]] for every particle plane
// The original index travels with each particle, so downloads can restore the
// caller's order.  Only the physics-free ordering changes; every particle's
// update is independent of it.
#include <string.h>

#include "internal.h"
#include "parts.cuh"

namespace gl {

static constexpr int SCAN_T = 256, SCAN_PER = 4, SCAN_CHUNK = SCAN_T * SCAN_PER;  // 1024 cells per block
static constexpr int SCAN_MAX_BLOCKS = 32768;                                      // keys <= 32 Mi

// keys of an event: one per (class, cell)
__host__ __device__ inline int64_t sort_keys(int64_t Vn, int ng) { return (int64_t)(ng > 0 ? ng : 1) * Vn; }

// ns (species) bounds the classes present
size_t sort_scratch_bytes(int64_t Vn, int64_t np, int ns) {
    // key, rank, perm (np each), counts/offsets (keys + 1), block sums
    return align256(4 * (size_t)np) * 3 + align256(4 * ((size_t)sort_keys(Vn, ns) + 1)) +
           align256(4 * (size_t)SCAN_MAX_BLOCKS);
}

bool sort_supported(int64_t Vn, int ns) { return sort_keys(Vn, ns) <= (int64_t)SCAN_CHUNK * SCAN_MAX_BLOCKS; }

// Every kernel runs over the particles or the keys of one or many events.
// Particle-indexed launches give each event ceil(np / SORT_PB) blocks of
// SORT_PB particles, key-indexed launches ceil(ng Vn / SCAN_CHUNK) blocks of
// SCAN_CHUNK keys (one scan chunk); a block finds its event by binary search
// in the descriptors, or takes the single descriptor passed by value.
static constexpr int SORT_T = 256, SORT_PB = 1024;

__device__ __forceinline__ int sort_find(const SortEv* ev, int ne, int block, bool cells) {
    int lo = 0, hi = ne - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((cells ? ev[mid].cblk_begin : ev[mid].pblk_begin) <= block) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// the block's event and its block index within the event
struct SortBlock {
    SortEv d;
    int b;
};
__device__ __forceinline__ SortBlock sort_block(const SortEv* ev, int ne, const SortEv& one, bool cells) {
    __shared__ int s_e;
    SortBlock r;
    if (ev) {
        if (threadIdx.x == 0) s_e = sort_find(ev, ne, blockIdx.x, cells);
        __syncthreads();
        r.d = ev[s_e];
    } else {
        r.d = one;
    }
    r.b = blockIdx.x - (cells ? r.d.cblk_begin : r.d.pblk_begin);
    return r;
}

__global__ void __launch_bounds__(SORT_T) zero_counts_kernel(const SortEv* ev, int ne, SortEv one) {
    const SortBlock k = sort_block(ev, ne, one, true);
    const int64_t Vn = sort_keys((int64_t)k.d.N * k.d.N, k.d.ng);
    const int64_t c0 = (int64_t)k.b * SCAN_CHUNK;
    for (int64_t c = c0 + threadIdx.x; c < c0 + SCAN_CHUNK && c < Vn; c += SORT_T) k.d.cnt[c] = 0;
}

template <typename R>
__global__ void __launch_bounds__(SORT_T) cell_count_kernel(const SortEv* ev, int ne, SortEv one) {
    const SortBlock k = sort_block(ev, ne, one, false);
    const Parts<R> P = carve_parts<R>(k.d.src, k.d.np);
    const int N = k.d.N;
    const int64_t i0 = (int64_t)k.b * SORT_PB;
    for (int64_t i = i0 + threadIdx.x; i < i0 + SORT_PB && i < k.d.np; i += SORT_T) {
        const PState<R> p = P.load(i);
        const int ix = wrapi((int)floor(p.x + R(0.5)), N), iy = wrapi((int)floor(p.y + R(0.5)), N);
        const int sp = P.sp[i];
        const int g = (unsigned)sp < (unsigned)GL_MAX_SPECIES ? k.d.grp[sp] : 0;
        const int c = (iy * k.d.ng + g) * N + ix;
        k.d.key[i] = c;
        k.d.rank[i] = atomicAdd(&k.d.cnt[c], 1);
    }
}

// exclusive scan of one chunk of SCAN_CHUNK counts in place; its total to bsum
__global__ void __launch_bounds__(SCAN_T) scan_chunks_kernel(const SortEv* ev, int ne, SortEv one) {
    const SortBlock k = sort_block(ev, ne, one, true);
    __shared__ int warp_tot[SCAN_T / 32];
    int* cnt = k.d.cnt;
    const int64_t n = sort_keys((int64_t)k.d.N * k.d.N, k.d.ng);
    const int64_t base = (int64_t)k.b * SCAN_CHUNK + threadIdx.x * SCAN_PER;
    int v[SCAN_PER], s = 0;
#pragma unroll
    for (int q = 0; q < SCAN_PER; q++) {
        v[q] = base + q < n ? cnt[base + q] : 0;
        s += v[q];
    }
    // inclusive warp scan of the per-thread totals
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    int woff = 0;
    for (int w = 0; w < warp; w++) woff += warp_tot[w];
    int run = woff + inc - s;  // exclusive prefix of this thread
#pragma unroll
    for (int q = 0; q < SCAN_PER; q++) {
        if (base + q < n) cnt[base + q] = run;
        run += v[q];
    }
    if (threadIdx.x == SCAN_T - 1) k.d.bsum[k.b] = run;
}

// one block per event: exclusive scan of the chunk totals, then off[Vn] = total
__global__ void __launch_bounds__(1024) scan_top_kernel(const SortEv* ev, SortEv one) {
    const SortEv d = ev ? ev[blockIdx.x] : one;
    __shared__ int part[1024];
    const int64_t n = sort_keys((int64_t)d.N * d.N, d.ng);
    const int nb = (int)((n + SCAN_CHUNK - 1) / SCAN_CHUNK);
    int* bsum = d.bsum;
    const int per = (nb + 1023) / 1024;
    const int b0 = threadIdx.x * per;
    int s = 0;
    for (int q = 0; q < per; q++)
        if (b0 + q < nb) s += bsum[b0 + q];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int y = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += y;
        __syncthreads();
    }
    int run = part[threadIdx.x] - s;
    for (int q = 0; q < per; q++)
        if (b0 + q < nb) {
            const int v = bsum[b0 + q];
            bsum[b0 + q] = run;
            run += v;
        }
    if (threadIdx.x == 1023) d.cnt[n] = part[1023];
}

__global__ void __launch_bounds__(SORT_T) scan_add_kernel(const SortEv* ev, int ne, SortEv one) {
    const SortBlock k = sort_block(ev, ne, one, true);
    const int64_t Vn = sort_keys((int64_t)k.d.N * k.d.N, k.d.ng);
    const int add = k.d.bsum[k.b];
    const int64_t c0 = (int64_t)k.b * SCAN_CHUNK;
    for (int64_t c = c0 + threadIdx.x; c < c0 + SCAN_CHUNK && c < Vn; c += SORT_T) k.d.cnt[c] += add;
}

__global__ void __launch_bounds__(SORT_T) scatter_kernel(const SortEv* ev, int ne, SortEv one) {
    const SortBlock k = sort_block(ev, ne, one, false);
    const int64_t i0 = (int64_t)k.b * SORT_PB;
    for (int64_t i = i0 + threadIdx.x; i < i0 + SORT_PB && i < k.d.np; i += SORT_T)
        k.d.perm[k.d.cnt[k.d.key[i]] + k.d.rank[i]] = (int)i;
}

// insertion sort of each key's (short) segment of perm
__global__ void __launch_bounds__(SORT_T) cell_order_kernel(const SortEv* ev, int ne, SortEv one) {
    const SortBlock k = sort_block(ev, ne, one, true);
    const int64_t Vn = sort_keys((int64_t)k.d.N * k.d.N, k.d.ng);
    const int* off = k.d.cnt;
    int* perm = k.d.perm;
    const int64_t c0 = (int64_t)k.b * SCAN_CHUNK;
    for (int64_t c = c0 + threadIdx.x; c < c0 + SCAN_CHUNK && c < Vn; c += SORT_T) {
        const int b = off[c], e = off[c + 1];
        for (int i = b + 1; i < e; i++) {
            const int v = perm[i];
            int j = i - 1;
            while (j >= b && perm[j] > v) {
                perm[j + 1] = perm[j];
                j--;
            }
            perm[j + 1] = v;
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(SORT_T) gather_kernel(const SortEv* ev, int ne, SortEv one) {
    const SortBlock k = sort_block(ev, ne, one, false);
    const Parts<R> src = carve_parts<R>(k.d.src, k.d.np), dst = carve_parts<R>(k.d.dst, k.d.np);
    const int64_t j0 = (int64_t)k.b * SORT_PB;
    for (int64_t j = j0 + threadIdx.x; j < j0 + SORT_PB && j < k.d.np; j += SORT_T) {
        const int i = k.d.perm[j];
        dst.store(j, src.load(i));
        dst.sp[j] = src.sp[i];
        dst.pt0[j] = src.pt0[i];
        dst.id[j] = src.id[i];
        dst.ptau[j] = src.ptau[i];
    }
}

SortEv sort_event(void* src, void* dst, int64_t np, int N, int ns, const int* motion, void* scratch) {
    SortEv d;
    memset(&d, 0, sizeof d);
    // classes numbered in order of first appearance among the species
    int code[GL_MAX_SPECIES], ng = 0;
    for (int s = 0; s < ns && s < GL_MAX_SPECIES; s++) {
        int g = 0;
        while (g < ng && code[g] != motion[s]) g++;
        if (g == ng) code[ng++] = motion[s];
        d.grp[s] = (int8_t)g;
    }
    d.ng = ng > 0 ? ng : 1;
    const int64_t keys = sort_keys((int64_t)N * N, d.ng);
    char* c = (char*)scratch;
    d.src = src;
    d.dst = dst;
    d.np = np;
    d.N = N;
    d.key = (int*)c; c += align256(4 * (size_t)np);
    d.rank = (int*)c; c += align256(4 * (size_t)np);
    d.perm = (int*)c; c += align256(4 * (size_t)np);
    d.cnt = (int*)c; c += align256(4 * ((size_t)keys + 1));
    d.bsum = (int*)c;
    return d;
}

int sort_particle_blocks(int64_t np) { return (int)((np + SORT_PB - 1) / SORT_PB); }
int sort_cell_blocks(const SortEv& d) {
    return (int)((sort_keys((int64_t)d.N * d.N, d.ng) + SCAN_CHUNK - 1) / SCAN_CHUNK);
}

// the stages over `pblocks` particle blocks and `cblocks` cell blocks of
// `ne` events (descriptors in device memory), or of the single event `one`
template <typename R>
static void sort_stages(const SortEv* ev, int ne, const SortEv& one, int pblocks, int cblocks, cudaStream_t st) {
    zero_counts_kernel<<<cblocks, SORT_T, 0, st>>>(ev, ne, one);
    cell_count_kernel<R><<<pblocks, SORT_T, 0, st>>>(ev, ne, one);
    scan_chunks_kernel<<<cblocks, SCAN_T, 0, st>>>(ev, ne, one);
    scan_top_kernel<<<ev ? ne : 1, 1024, 0, st>>>(ev, one);
    scan_add_kernel<<<cblocks, SORT_T, 0, st>>>(ev, ne, one);
    scatter_kernel<<<pblocks, SORT_T, 0, st>>>(ev, ne, one);
    cell_order_kernel<<<cblocks, SORT_T, 0, st>>>(ev, ne, one);
    gather_kernel<R><<<pblocks, SORT_T, 0, st>>>(ev, ne, one);
}

void launch_sort(int prec, void* src, void* dst, int64_t np, int N, int ns, const int* motion, void* scratch,
                 cudaStream_t st) {
    if (np <= 0) return;
    const SortEv one = sort_event(src, dst, np, N, ns, motion, scratch);
    const int pb = sort_particle_blocks(np), cb = sort_cell_blocks(one);
    if (prec == 0) sort_stages<double>(nullptr, 1, one, pb, cb, st);
    else sort_stages<float>(nullptr, 1, one, pb, cb, st);
}

void launch_sort_many(int prec, const SortEv* d_ev, int ne, int pblocks, int cblocks, cudaStream_t st) {
    if (ne <= 0 || pblocks <= 0) return;
    SortEv none;
    memset(&none, 0, sizeof none);
    if (prec == 0) sort_stages<double>(d_ev, ne, none, pblocks, cblocks, st);
    else sort_stages<float>(d_ev, ne, none, pblocks, cblocks, st);
}

}  // namespace gl
