// Ensemble sums without any device allocation.
//
// Some callers cannot allocate device memory at all: code embedded in a host
// that owns every device allocation itself (another framework's memory pool,
// a pre-reserved arena), or a process that must not grow its device
// footprint after start-up.  For them this file provides one entry point,
// gl_ensemble_sums_noalloc, that computes the per-species momentum sums of the
// observables() call from particle records the caller already holds on the
// device, with its scratch space in a fixed array compiled into the library.
//
// The scratch array below is a file-scope __device__ array: every GPU that
// loads the library holds its 917,504 bytes until the process exits.  In host
// code its name is only a host-side stand-in, so the host looks up its device
// address once per device with cudaGetSymbolAddress and passes that address to
// the kernels.
#include <mutex>

#include "internal.h"
#include "layout.cuh"

namespace gl {

static constexpr int NA_THREADS = 256;
static constexpr int NA_PER_THREAD = 4;
static constexpr int NA_PER_BLOCK = NA_THREADS * NA_PER_THREAD;  // 1024 particles per block
static constexpr int NA_MAX_BLOCKS = GL_NOALLOC_MAX_PARTICLES / NA_PER_BLOCK;
static constexpr int NA_WIDTH = GL_MAX_SPECIES * PO_N;

static_assert(GL_NOALLOC_MAX_PARTICLES % NA_PER_BLOCK == 0, "block size must divide the maximum");

// one slot of NA_WIDTH partial results per block; each block writes its whole
// slot before the finishing kernel reads it, so nothing needs clearing
static __device__ __align__(256) double na_scratch[NA_MAX_BLOCKS * NA_WIDTH];

struct NaArgs {
    double mass[GL_MAX_SPECIES];
    int accumulated[GL_MAX_SPECIES];  // static or eikonal: p_L is the accumulated P_eta slot
    double q2ref[GL_MAX_SPECIES], q3ref[GL_MAX_SPECIES];
    int n_species;
};

__device__ __forceinline__ bool na_is_max(int k) { return k == PO_Q2 || k == PO_Q3; }

// per-block sums over canonical FP64 particle records [np][16]
__global__ void __launch_bounds__(NA_THREADS) na_sums_kernel(const double* __restrict__ rec, int64_t np, double t,
                                                             uint32_t active, NaArgs a, double* partials) {
    __shared__ double wacc[NA_THREADS / 32][NA_WIDTH];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = lane; k < NA_WIDTH; k += 32) wacc[warp][k] = 0.0;
    __syncwarp();
    for (int r = 0; r < NA_PER_THREAD; r++) {
        const int64_t i = (int64_t)blockIdx.x * NA_PER_BLOCK + (int64_t)r * NA_THREADS + threadIdx.x;
        int s = -1;
        double v[PO_N] = {0, 0, 0, 0, 0, 0, 0};
        if (i < np) {
            const double* p = rec + i * 16;
            s = (int)p[15];
            if (s < 0 || s >= a.n_species || !((active >> s) & 1u)) s = -1;
            if (s >= 0) {
                const double px = p[3], py = p[4], Pe = p[5], eta = p[2];
                double pl;
                if (a.accumulated[s]) {
                    pl = Pe;
                } else {
                    const double w = t > 0 ? Pe / t : 0.0;
                    const double ptau = sqrt(px * px + py * py + w * w + a.mass[s] * a.mass[s]);
                    pl = ptau * sinh(eta) + w * cosh(eta);
                }
                A8<double> q;
                for (int c = 0; c < 8; c++) q.v[c] = p[6 + c];
                const M3<double> Q = alg_to_mat(q);
                const M3<double> Q2 = mul(Q, Q);
                double tr3 = 0;
                for (int x = 0; x < 3; x++)
                    for (int y = 0; y < 3; y++) tr3 += Q2.re[x][y] * Q.re[y][x] - Q2.im[x][y] * Q.im[y][x];
                v[PO_COUNT] = 1.0;
                v[PO_PX2] = px * px;
                v[PO_PY2] = py * py;
                v[PO_PL2] = pl * pl;
                v[PO_DPT2] = px * px + py * py - p[14];
                v[PO_Q2] = fabs(a_dot(q, q) - a.q2ref[s]);
                v[PO_Q3] = fabs(4.0 * tr3 - a.q3ref[s]);
            }
        }
        for (int sp = 0; sp < a.n_species; sp++) {
            const bool mine = s == sp;
            if (!__any_sync(0xffffffffu, mine)) continue;
            double x[PO_N];
#pragma unroll
            for (int k = 0; k < PO_N; k++) x[k] = mine ? v[k] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int k = 0; k < PO_N; k++) {
                    const double y = __shfl_down_sync(0xffffffffu, x[k], o);
                    x[k] = na_is_max(k) ? nanmax(x[k], y) : x[k] + y;
                }
            if (lane == 0)
                for (int k = 0; k < PO_N; k++) {
                    double* d = &wacc[warp][sp * PO_N + k];
                    *d = na_is_max(k) ? nanmax(*d, x[k]) : *d + x[k];
                }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NA_WIDTH; k += NA_THREADS) {
        double acc = 0.0;
        for (int w = 0; w < NA_THREADS / 32; w++)
            acc = na_is_max(k % PO_N) ? nanmax(acc, wacc[w][k]) : acc + wacc[w][k];
        partials[(size_t)blockIdx.x * NA_WIDTH + k] = acc;
    }
}

__global__ void na_finish_kernel(const double* partials, int nblocks, int n_species, double* out) {
    for (int k = threadIdx.x; k < n_species * PO_N; k += blockDim.x) {
        double acc = 0.0;
        for (int b = 0; b < nblocks; b++) {
            const double x = partials[(size_t)b * NA_WIDTH + k];
            acc = na_is_max(k % PO_N) ? nanmax(acc, x) : acc + x;
        }
        out[k] = acc;
    }
}

static std::mutex na_mutex;
static void* na_ptr[256];  // device address of na_scratch, per device ordinal

}  // namespace gl

using namespace gl;

extern "C" gl_status gl_ensemble_sums_noalloc(const double* d_particles, int64_t np, int32_t n_species,
                                              const double* mass, const int32_t* rep, const int32_t* kind,
                                              uint32_t active_mask, double t, double* d_out, void* stream) {
    if (np < 0 || n_species < 1 || n_species > GL_MAX_SPECIES || !mass || !rep || !kind || !d_out ||
        (np > 0 && !d_particles))
        return GL_ERR_ARG;
    for (int k = 0; k < n_species; k++)
        if (kind[k] < MOTION_WONG || kind[k] > MOTION_EIKONAL || (rep[k] != 0 && rep[k] != 1)) return GL_ERR_ARG;
    if (np > GL_NOALLOC_MAX_PARTICLES) return GL_ERR_SIZE;  // more particles than the static scratch covers
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return GL_ERR_CUDA;
    void* scratch = nullptr;
    {
        // set-up, once per device, with that device current: the device address
        // of the static array (its host-side name is not a device address)
        std::lock_guard<std::mutex> lock(na_mutex);
        if (!na_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, na_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return GL_ERR_CUDA;
            }
            na_ptr[dev] = p;
        }
        scratch = na_ptr[dev];
    }
    NaArgs a;
    a.n_species = n_species;
    for (int k = 0; k < GL_MAX_SPECIES; k++) {
        const bool on = k < n_species;
        a.accumulated[k] = on && kind[k] != MOTION_WONG;
        a.mass[k] = on && !a.accumulated[k] ? mass[k] : 0.0;
        a.q2ref[k] = on && rep[k] == 1 ? 24.0 : 4.0;
        a.q3ref[k] = on && rep[k] == 1 ? 0.0 : 10.0 / 3.0;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int blocks = (int)((np + NA_PER_BLOCK - 1) / NA_PER_BLOCK);
    if (blocks < 1) blocks = 1;
    na_sums_kernel<<<blocks, NA_THREADS, 0, st>>>(d_particles, np, t, active_mask, a, (double*)scratch);
    na_finish_kernel<<<1, 64, 0, st>>>((const double*)scratch, blocks, n_species, d_out);
    return cudaGetLastError() == cudaSuccess ? GL_OK : GL_ERR_CUDA;
}
