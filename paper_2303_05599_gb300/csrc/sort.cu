// Sort of the particles by lattice row, then by motion class (Wong, static,
// eikonal), then by nearest-grid-point cell: the push reads the site fields
// of neighbouring particles from the same cache lines (a row's fields stay in
// cache while its classes are pushed one after the other), and the 32
// particles of a warp are (but at the edges of a row's class ranges) of one
// class, so they take one branch of the push instead of running every branch
// present with the other lanes idle.  Species of one class stay mixed by cell.
//
// The key of particle i of class g (of ng classes present) in cell (x, y) is
// (y ng + g) N + x.  Particles are ordered by key and, among equal keys, by
// their index before the sort: an LSD radix sort of (key, index) pairs with
// 8-bit digits, stable in every pass, so the result is unique whatever the
// distribution of the keys (all particles in one cell included) and takes
// O(np) work per pass:
//   keys:     key[i], val[i] = i
//   per pass (digit p of the key):
//     hist:    per block of SORT_PB pairs, the count of each digit value,
//              stored digit-major: hist[digit][block]
//     scan:    exclusive prefix sum of hist (two-level block scan), so that
//              hist[digit][block] is where that block's first pair of that
//              digit goes
//     scatter: each pair to hist[digit][block] + its rank among the block's
//              pairs of the same digit in their current order
//   gather:   new[j] = old[val[j]] for every particle plane
// The original index travels with each particle, so downloads can restore the
// caller's order.  Only the physics-free ordering changes; every particle's
// update is independent of it.
#include <string.h>

#include "internal.h"
#include "parts.cuh"

namespace gl {

static constexpr int SCAN_T = 256, SCAN_PER = 4, SCAN_CHUNK = SCAN_T * SCAN_PER;  // 1024 entries per block
static constexpr int SCAN_MAX_BLOCKS = 32768;                                      // entries <= 32 Mi
static constexpr int RADIX_BITS = 8, RADIX = 1 << RADIX_BITS;

// Particle-indexed launches give each event ceil(np / SORT_PB) blocks of
// SORT_PB particles (SORT_T threads, SORT_PB / SORT_T rounds), scan-indexed
// launches ceil(RADIX nblk / SCAN_CHUNK) blocks of SCAN_CHUNK histogram
// entries; a block finds its event by binary search in the descriptors, or
// takes the single descriptor passed by value.
static constexpr int SORT_T = 256, SORT_PB = 1024, SORT_ROUNDS = SORT_PB / SORT_T;
static_assert(SORT_T == RADIX, "one thread per digit value");

static inline int64_t sort_nblk(int64_t np) { return (np + SORT_PB - 1) / SORT_PB; }

// ns (species) bounds the classes present
size_t sort_scratch_bytes(int64_t Vn, int64_t np, int ns) {
    (void)Vn;
    (void)ns;
    // keys and values twice (ping-pong), the histogram and the scan's block sums
    return align256(4 * (size_t)np) * 4 + align256(4 * ((size_t)RADIX * sort_nblk(np) + 1)) +
           align256(4 * (size_t)SCAN_MAX_BLOCKS);
}

// keys fit 31 bits; the histogram fits the scan
bool sort_supported(int64_t Vn, int ns, int64_t np) {
    const int64_t keys = (int64_t)(ns > 0 ? ns : 1) * Vn;
    return keys <= 0x7fffffff && RADIX * sort_nblk(np) <= (int64_t)SCAN_CHUNK * SCAN_MAX_BLOCKS;
}

__device__ __forceinline__ int sort_find(const SortEv* ev, int ne, int block, bool scan) {
    int lo = 0, hi = ne - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((scan ? ev[mid].cblk_begin : ev[mid].pblk_begin) <= block) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// the block's event and its block index within the event
struct SortBlock {
    SortEv d;
    int b;
};
__device__ __forceinline__ SortBlock sort_block(const SortEv* ev, int ne, const SortEv& one, bool scan) {
    __shared__ int s_e;
    SortBlock r;
    if (ev) {
        if (threadIdx.x == 0) s_e = sort_find(ev, ne, blockIdx.x, scan);
        __syncthreads();
        r.d = ev[s_e];
    } else {
        r.d = one;
    }
    r.b = blockIdx.x - (scan ? r.d.cblk_begin : r.d.pblk_begin);
    return r;
}

template <typename R>
__global__ void __launch_bounds__(SORT_T) key_kernel(const SortEv* ev, int ne, SortEv one) {
    const SortBlock k = sort_block(ev, ne, one, false);
    const Parts<R> P = carve_parts<R>(k.d.src, k.d.np);
    const int N = k.d.N;
    const int64_t i0 = (int64_t)k.b * SORT_PB;
    for (int64_t i = i0 + threadIdx.x; i < i0 + SORT_PB && i < k.d.np; i += SORT_T) {
        const PState<R> p = P.load(i);
        // wrapi keeps the cell inside the lattice for any position (a
        // non-finite coordinate converts to 0)
        const int ix = wrapi((int)floor(p.x + R(0.5)), N), iy = wrapi((int)floor(p.y + R(0.5)), N);
        const int sp = P.sp[i];
        const int g = (unsigned)sp < (unsigned)GL_MAX_SPECIES ? k.d.grp[sp] : 0;
        k.d.key[0][i] = (uint32_t)((iy * k.d.ng + g) * N + ix);
        k.d.val[0][i] = (uint32_t)i;
    }
}

// digit counts of one block of pairs, digit-major
__global__ void __launch_bounds__(SORT_T) hist_kernel(const SortEv* ev, int ne, SortEv one, int pass) {
    const SortBlock k = sort_block(ev, ne, one, false);
    __shared__ int h[RADIX];
    const uint32_t* key = k.d.key[pass & 1];
    const int shift = pass * RADIX_BITS;
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t i0 = (int64_t)k.b * SORT_PB;
    for (int64_t i = i0 + threadIdx.x; i < i0 + SORT_PB && i < k.d.np; i += SORT_T)
        atomicAdd(&h[(key[i] >> shift) & (RADIX - 1)], 1);
    __syncthreads();
    k.d.hist[(int64_t)threadIdx.x * k.d.nblk + k.b] = h[threadIdx.x];
}

// exclusive scan of one chunk of SCAN_CHUNK histogram entries in place; its
// total to bsum
__global__ void __launch_bounds__(SCAN_T) scan_chunks_kernel(const SortEv* ev, int ne, SortEv one) {
    const SortBlock k = sort_block(ev, ne, one, true);
    __shared__ int warp_tot[SCAN_T / 32];
    int* cnt = k.d.hist;
    const int64_t n = (int64_t)RADIX * k.d.nblk;
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

// one block per event: exclusive scan of the chunk totals, then hist[n] = total
__global__ void __launch_bounds__(1024) scan_top_kernel(const SortEv* ev, SortEv one) {
    const SortEv d = ev ? ev[blockIdx.x] : one;
    __shared__ int part[1024];
    const int64_t n = (int64_t)RADIX * d.nblk;
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
    if (threadIdx.x == 1023) d.hist[n] = part[1023];
}

__global__ void __launch_bounds__(SORT_T) scan_add_kernel(const SortEv* ev, int ne, SortEv one) {
    const SortBlock k = sort_block(ev, ne, one, true);
    const int64_t n = (int64_t)RADIX * k.d.nblk;
    const int add = k.d.bsum[k.b];
    const int64_t c0 = (int64_t)k.b * SCAN_CHUNK;
    for (int64_t c = c0 + threadIdx.x; c < c0 + SCAN_CHUNK && c < n; c += SORT_T) k.d.hist[c] += add;
}

// stable scatter of one block of pairs by digit `pass`: the block's pairs go
// in SORT_ROUNDS rounds of SORT_T (round r: pairs r SORT_T .. r SORT_T + 255,
// so rounds, warps and lanes follow the pairs' order); a pair's rank among the
// block's pairs of its digit is the count of that digit in earlier rounds,
// earlier warps of its round and earlier lanes of its warp
__global__ void __launch_bounds__(SORT_T) radix_scatter_kernel(const SortEv* ev, int ne, SortEv one, int pass) {
    const SortBlock k = sort_block(ev, ne, one, false);
    __shared__ int base[RADIX];               // destination of the block's first pair of each digit
    __shared__ int wcnt[SORT_T / 32][RADIX];  // this round's pairs of each digit, per warp
    const uint32_t* kin = k.d.key[pass & 1];
    const uint32_t* vin = k.d.val[pass & 1];
    uint32_t* kout = k.d.key[(pass + 1) & 1];
    uint32_t* vout = k.d.val[(pass + 1) & 1];
    const int shift = pass * RADIX_BITS;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    base[tid] = k.d.hist[(int64_t)tid * k.d.nblk + k.b];
    const int64_t i0 = (int64_t)k.b * SORT_PB;
    for (int r = 0; r < SORT_ROUNDS; r++) {
#pragma unroll
        for (int q = 0; q < SORT_T / 32; q++) wcnt[q][tid] = 0;
        __syncthreads();
        const int64_t i = i0 + (int64_t)r * SORT_T + tid;
        const bool ok = i < k.d.np;
        uint32_t key = 0, val = 0;
        int dig = -1;  // lanes without a pair form a group of their own
        if (ok) {
            key = kin[i];
            val = vin[i];
            dig = (int)((key >> shift) & (RADIX - 1));
        }
        const unsigned m = __match_any_sync(0xffffffffu, dig);
        const int lrank = __popc(m & ((1u << lane) - 1u));
        if (ok && lrank == 0) wcnt[w][dig] = __popc(m);
        __syncthreads();
        if (ok) {
            int pos = base[dig] + lrank;
            for (int q = 0; q < w; q++) pos += wcnt[q][dig];
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        // the round's pairs of digit tid advance its destination
        int tot = 0;
#pragma unroll
        for (int q = 0; q < SORT_T / 32; q++) tot += wcnt[q][tid];
        base[tid] += tot;
    }
}

template <typename R>
__global__ void __launch_bounds__(SORT_T) gather_kernel(const SortEv* ev, int ne, SortEv one, int passes) {
    const SortBlock k = sort_block(ev, ne, one, false);
    const Parts<R> src = carve_parts<R>(k.d.src, k.d.np), dst = carve_parts<R>(k.d.dst, k.d.np);
    const uint32_t* perm = k.d.val[passes & 1];
    const int64_t j0 = (int64_t)k.b * SORT_PB;
    for (int64_t j = j0 + threadIdx.x; j < j0 + SORT_PB && j < k.d.np; j += SORT_T) {
        const int64_t i = perm[j];
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
    char* c = (char*)scratch;
    d.src = src;
    d.dst = dst;
    d.np = np;
    d.N = N;
    d.nblk = (int)sort_nblk(np);
    for (int h = 0; h < 2; h++) { d.key[h] = (uint32_t*)c; c += align256(4 * (size_t)np); }
    for (int h = 0; h < 2; h++) { d.val[h] = (uint32_t*)c; c += align256(4 * (size_t)np); }
    d.hist = (int*)c; c += align256(4 * ((size_t)RADIX * d.nblk + 1));
    d.bsum = (int*)c;
    return d;
}

int sort_particle_blocks(int64_t np) { return (int)sort_nblk(np); }
int sort_cell_blocks(const SortEv& d) {
    return (int)(((int64_t)RADIX * d.nblk + SCAN_CHUNK - 1) / SCAN_CHUNK);
}

// digit passes that cover every key of an event
int sort_passes(const SortEv& d) {
    const uint64_t top = (uint64_t)d.ng * d.N * d.N - 1;
    int bits = 1;
    while (bits < 32 && (top >> bits) != 0) bits++;
    return (bits + RADIX_BITS - 1) / RADIX_BITS;
}

// the stages over `pblocks` particle blocks and `cblocks` scan blocks of `ne`
// events (descriptors in device memory), or of the single event `one`
template <typename R>
static void sort_stages(const SortEv* ev, int ne, const SortEv& one, int pblocks, int cblocks, int passes,
                        cudaStream_t st) {
    key_kernel<R><<<pblocks, SORT_T, 0, st>>>(ev, ne, one);
    for (int p = 0; p < passes; p++) {
        hist_kernel<<<pblocks, SORT_T, 0, st>>>(ev, ne, one, p);
        scan_chunks_kernel<<<cblocks, SCAN_T, 0, st>>>(ev, ne, one);
        scan_top_kernel<<<ev ? ne : 1, 1024, 0, st>>>(ev, one);
        scan_add_kernel<<<cblocks, SORT_T, 0, st>>>(ev, ne, one);
        radix_scatter_kernel<<<pblocks, SORT_T, 0, st>>>(ev, ne, one, p);
    }
    gather_kernel<R><<<pblocks, SORT_T, 0, st>>>(ev, ne, one, passes);
}

void launch_sort(int prec, void* src, void* dst, int64_t np, int N, int ns, const int* motion, void* scratch,
                 cudaStream_t st) {
    if (np <= 0) return;
    const SortEv one = sort_event(src, dst, np, N, ns, motion, scratch);
    const int pb = sort_particle_blocks(np), cb = sort_cell_blocks(one), passes = sort_passes(one);
    if (prec == 0) sort_stages<double>(nullptr, 1, one, pb, cb, passes, st);
    else sort_stages<float>(nullptr, 1, one, pb, cb, passes, st);
}

void launch_sort_many(int prec, const SortEv* d_ev, int ne, int pblocks, int cblocks, int passes, cudaStream_t st) {
    if (ne <= 0 || pblocks <= 0) return;
    SortEv none;
    memset(&none, 0, sizeof none);
    if (prec == 0) sort_stages<double>(d_ev, ne, none, pblocks, cblocks, passes, st);
    else sort_stages<float>(d_ev, ne, none, pblocks, cblocks, passes, st);
}

}  // namespace gl
