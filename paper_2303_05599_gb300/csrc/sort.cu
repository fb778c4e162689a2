// Counting sort of the particles by nearest-grid-point cell, so that the push
// reads the site fields of neighbouring particles from the same cache lines.
//
//   count:    key[i] = cell of particle i, rank[i] = atomic slot within its cell
//   scan:     off[c] = number of particles in cells < c (two-level block scan)
//   scatter:  perm[off[key[i]] + rank[i]] = i
//   order:    each cell's entries of perm sorted ascending, so the result does
//             not depend on the order the atomics were served in
//   gather:   new[j] = old[perm[j]] for every particle plane
// The original index travels with each particle, so downloads can restore the
// caller's order.  Only the physics-free ordering changes; every particle's
// update is independent of it.
#include "internal.h"
#include "parts.cuh"

namespace gl {

static constexpr int SCAN_T = 256, SCAN_PER = 4, SCAN_CHUNK = SCAN_T * SCAN_PER;  // 1024 cells per block
static constexpr int SCAN_MAX_BLOCKS = 4096;                                       // cells <= 4 Mi

size_t sort_scratch_bytes(int64_t Vn, int64_t np) {
    // key, rank, perm (np each), counts/offsets (Vn + 1), block sums
    return align256(4 * (size_t)np) * 3 + align256(4 * ((size_t)Vn + 1)) + align256(4 * (size_t)SCAN_MAX_BLOCKS);
}

bool sort_supported(int64_t Vn) { return Vn <= (int64_t)SCAN_CHUNK * SCAN_MAX_BLOCKS; }

template <typename R>
__global__ void cell_count_kernel(Parts<R> P, int N, int* cnt, int* key, int* rank) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.np; i += (int64_t)gridDim.x * blockDim.x) {
        const PState<R> p = P.load(i);
        const int ix = wrapi((int)floor(p.x + R(0.5)), N), iy = wrapi((int)floor(p.y + R(0.5)), N);
        const int c = iy * N + ix;
        key[i] = c;
        rank[i] = atomicAdd(&cnt[c], 1);
    }
}

// exclusive scan of cnt[0, n) in place, per chunk of SCAN_CHUNK; chunk totals to bsum
__global__ void __launch_bounds__(SCAN_T) scan_chunks_kernel(int* cnt, int64_t n, int* bsum) {
    __shared__ int warp_tot[SCAN_T / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + threadIdx.x * SCAN_PER;
    int v[SCAN_PER], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER; k++) {
        v[k] = base + k < n ? cnt[base + k] : 0;
        s += v[k];
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
    for (int k = 0; k < SCAN_PER; k++) {
        if (base + k < n) cnt[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == SCAN_T - 1) bsum[blockIdx.x] = run;
}

// exclusive scan of the chunk totals (one block), then off[n] = total
__global__ void __launch_bounds__(1024) scan_top_kernel(int* bsum, int nb, int* off, int64_t n) {
    __shared__ int part[1024];
    const int per = (nb + 1023) / 1024;
    const int b0 = threadIdx.x * per;
    int s = 0;
    for (int k = 0; k < per; k++)
        if (b0 + k < nb) s += bsum[b0 + k];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int y = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += y;
        __syncthreads();
    }
    int run = part[threadIdx.x] - s;
    for (int k = 0; k < per; k++)
        if (b0 + k < nb) {
            const int v = bsum[b0 + k];
            bsum[b0 + k] = run;
            run += v;
        }
    if (threadIdx.x == 1023) off[n] = part[1023];
}

__global__ void scan_add_kernel(int* cnt, int64_t n, const int* bsum) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        cnt[i] += bsum[i / SCAN_CHUNK];
}

__global__ void scatter_kernel(int64_t np, const int* key, const int* rank, const int* off, int* perm) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x)
        perm[off[key[i]] + rank[i]] = (int)i;
}

// insertion sort of each cell's (short) segment of perm
__global__ void cell_order_kernel(int64_t Vn, const int* off, int* perm) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < Vn; c += (int64_t)gridDim.x * blockDim.x) {
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
__global__ void gather_kernel(Parts<R> src, Parts<R> dst, const int* perm) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < src.np; j += (int64_t)gridDim.x * blockDim.x) {
        const int i = perm[j];
        dst.store(j, src.load(i));
        dst.sp[j] = src.sp[i];
        dst.pt0[j] = src.pt0[i];
        dst.id[j] = src.id[i];
    }
}

static unsigned grid(int64_t n, int t) {
    int64_t b = (n + t - 1) / t;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)(b < 1 ? 1 : b);
}

template <typename R>
static void sort_t(void* src, void* dst, int64_t np, int N, void* scratch, cudaStream_t st) {
    const int64_t Vn = (int64_t)N * N;
    char* c = (char*)scratch;
    int* key = (int*)c; c += align256(4 * (size_t)np);
    int* rank = (int*)c; c += align256(4 * (size_t)np);
    int* perm = (int*)c; c += align256(4 * (size_t)np);
    int* cnt = (int*)c; c += align256(4 * ((size_t)Vn + 1));
    int* bsum = (int*)c;
    const int nb = (int)((Vn + SCAN_CHUNK - 1) / SCAN_CHUNK);
    Parts<R> ps = carve_parts<R>(src, np), pd = carve_parts<R>(dst, np);
    cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)Vn, st);
    cell_count_kernel<R><<<grid(np, 256), 256, 0, st>>>(ps, N, cnt, key, rank);
    scan_chunks_kernel<<<nb, SCAN_T, 0, st>>>(cnt, Vn, bsum);
    scan_top_kernel<<<1, 1024, 0, st>>>(bsum, nb, cnt, Vn);
    scan_add_kernel<<<grid(Vn, 256), 256, 0, st>>>(cnt, Vn, bsum);
    scatter_kernel<<<grid(np, 256), 256, 0, st>>>(np, key, rank, cnt, perm);
    cell_order_kernel<<<grid(Vn, 128), 128, 0, st>>>(Vn, cnt, perm);
    gather_kernel<R><<<grid(np, 128), 128, 0, st>>>(ps, pd, perm);
}

void launch_sort(int prec, void* src, void* dst, int64_t np, int N, void* scratch, cudaStream_t st) {
    if (np <= 0) return;
    if (prec == 0) sort_t<double>(src, dst, np, N, scratch, st);
    else sort_t<float>(src, dst, np, N, scratch, st);
}

}  // namespace gl
