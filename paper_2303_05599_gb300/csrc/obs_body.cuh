// Per-species particle observables (Sec. 3.1: momentum broadening <p_T^2>,
// <p_L^2>, <p_T^2(tau) - p_T^2(tau_form)>; Casimir drifts of the colour
// charges) as one block's partial sums over a fixed chunk of particles.
//
// The particles of an event are cut into chunks of obs_chunk(np) particles,
// one block each, and every block writes GL_MAX_SPECIES x PO_N partial values
// (sums, or maxima for the Casimir drifts).  A second pass reduces the partials
// of an event in a fixed order.  The chunking depends only on the event's
// particle count, so an event gives bitwise the same observables whether it is
// reduced on its own or inside a batch.
//
// Per-particle quantities are evaluated in the state's precision; every
// accumulation is FP64.  Within a block each thread accumulates its own
// particles (c0 + tid, c0 + tid + OBS_THREADS, ...) into its own column of
// shared memory, then one fixed-order tree combines the columns: one FP64
// add per particle and value, instead of a warp-wide shuffle tree per group
// of 32 particles (FP64 issue is the scarce resource of this reduction).
#pragma once
#include "internal.h"
#include "layout.cuh"
#include "parts.cuh"
#include "su3.cuh"

namespace gl {

static constexpr int OBS_THREADS = 256;
static constexpr int OBS_MAX_BLOCKS = 1024;

// particles per observables block: at least 1024, at most OBS_MAX_BLOCKS blocks
__host__ __device__ inline int64_t obs_chunk(int64_t np) {
    int64_t c = (np + OBS_MAX_BLOCKS - 1) / OBS_MAX_BLOCKS;
    c = (c + OBS_THREADS - 1) / OBS_THREADS * OBS_THREADS;
    return c < 1024 ? 1024 : c;
}
__host__ __device__ inline int obs_blocks(int64_t np) {
    return np > 0 ? (int)((np + obs_chunk(np) - 1) / obs_chunk(np)) : 0;
}

struct ObsArgs {
    SpeciesParams sp;
    double q2ref[GL_MAX_SPECIES], q3ref[GL_MAX_SPECIES];
};

__device__ __forceinline__ bool po_is_max(int k) { return k == PO_Q2 || k == PO_Q3; }

// p_L = p^tau sinh(eta) + w cosh(eta) with w = P_eta / t (static quarks and
// eikonal partons: the accumulated P_eta slot), in the precision of the state
template <typename R>
__device__ __forceinline__ R particle_pl(const PState<R>& p, R t, R mass, bool accumulated) {
    if (accumulated) return p.Pe;
    const R w = t > R(0) ? p.Pe / t : R(0);
    const R ptau = sqrt(p.px * p.px + p.py * p.py + w * w + mass * mass);
    return ptau * sinh(p.eta) + w * cosh(p.eta);
}

// dynamic shared memory of particle_obs_block for ns species:
// [ns * PO_N][OBS_THREADS] doubles
__host__ __device__ inline size_t obs_smem_bytes(int ns) {
    return (size_t)ns * PO_N * OBS_THREADS * sizeof(double);
}

// partial observables of particles [c0, c1) into out[GL_MAX_SPECIES * PO_N];
// blockDim.x == OBS_THREADS, obs_smem_bytes(oa.sp.n_species) of dynamic
// shared memory at least
template <typename R>
__device__ __forceinline__ void particle_obs_block(const Parts<R>& P, double t, uint32_t active, const ObsArgs& oa,
                                                   int64_t c0, int64_t c1, double* out) {
    extern __shared__ double obs_acc[];
    const int ns = oa.sp.n_species, rows = ns * PO_N, tid = threadIdx.x;
    for (int r = 0; r < rows; r++) obs_acc[r * OBS_THREADS + tid] = 0.0;
    for (int64_t i = c0 + tid; i < c1; i += OBS_THREADS) {
        const int s = P.sp[i];
        if ((unsigned)s >= (unsigned)ns || !((active >> s) & 1u)) continue;
        const PState<R> p = P.load(i);
        const R pl = particle_pl<R>(p, (R)t, (R)oa.sp.mass[s], oa.sp.motion[s] != MOTION_WONG);
        const double px = p.px, py = p.py;
        double v[PO_N];
        v[PO_COUNT] = 1.0;
        v[PO_PX2] = px * px;
        v[PO_PY2] = py * py;
        v[PO_PL2] = (double)pl * (double)pl;
        v[PO_DPT2] = px * px + py * py - P.pt0[i];
        v[PO_Q2] = fabs((double)a_dot(p.q, p.q) - oa.q2ref[s]);
        v[PO_Q3] = fabs((double)casimir3(p.q) - oa.q3ref[s]);
        double* a = obs_acc + (size_t)s * PO_N * OBS_THREADS + tid;
#pragma unroll
        for (int k = 0; k < PO_N; k++)
            a[k * OBS_THREADS] = po_is_max(k) ? nanmax(a[k * OBS_THREADS], v[k]) : a[k * OBS_THREADS] + v[k];
    }
    // level o folds column c + o into column c (c < o) of every row
    for (int o = OBS_THREADS / 2; o > 0; o >>= 1) {
        __syncthreads();
        for (int w = tid; w < rows * o; w += OBS_THREADS) {
            const int r = w / o, c = w - r * o;
            double* a = obs_acc + r * OBS_THREADS;
            a[c] = po_is_max(r % PO_N) ? nanmax(a[c], a[c + o]) : a[c] + a[c + o];
        }
    }
    __syncthreads();
    for (int k = tid; k < GL_MAX_SPECIES * PO_N; k += OBS_THREADS) out[k] = k < rows ? obs_acc[k * OBS_THREADS] : 0.0;
}

// allow the largest dynamic shared memory of particle_obs_block on kernel f
template <typename K>
inline void obs_smem_attr(K f) {
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)obs_smem_bytes(GL_MAX_SPECIES));
}

// value k of GL_MAX_SPECIES * PO_N from nblocks partial rows: strided partial
// results, then a fixed-order tree; blockDim.x == 256
__device__ __forceinline__ void particle_obs_reduce(const double* partials, int nblocks, int k, double* out) {
    __shared__ double red[256];
    const int width = GL_MAX_SPECIES * PO_N;
    const bool mx = po_is_max(k % PO_N);
    double a = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        const double v = partials[(size_t)b * width + k];
        a = mx ? nanmax(a, v) : a + v;
    }
    red[threadIdx.x] = a;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = mx ? nanmax(red[threadIdx.x], red[threadIdx.x + o]) : red[threadIdx.x] + red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = red[0];
}

}  // namespace gl
