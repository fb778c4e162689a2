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
// shared memory, then one fixed-order tree combines the columns.  FP64 issue
// is the scarce resource of this reduction, so a particle costs four FP64
// fused adds (p_x^2, p_y^2, p_L^2, p_T^2(tau_form)) and its conversions: the
// count is an integer and the Casimir deviations are taken at the extremes.
#pragma once
#include "internal.h"
#include "layout.cuh"
#include "parts.cuh"
#include "su3.cuh"

namespace gl {

static constexpr int OBS_THREADS = 256;
static constexpr int OBS_MAX_BLOCKS = 1024;

// particles per observables block: at least 4096 (16 a thread, so that the
// block's final tree is a small share of its FP64 work), at most
// OBS_MAX_BLOCKS blocks
__host__ __device__ inline int64_t obs_chunk(int64_t np) {
    int64_t c = (np + OBS_MAX_BLOCKS - 1) / OBS_MAX_BLOCKS;
    c = (c + OBS_THREADS - 1) / OBS_THREADS * OBS_THREADS;
    return c < 4096 ? 4096 : c;
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

// Casimir deviations |q - ref| of one thread's particles.  FP32 state: the
// thread keeps the smallest and largest q (exact in any precision: no
// rounding) in the 8-byte slot of its column and takes |q - ref| in FP64 at
// the two extremes only, where the largest deviation lies; bitwise the
// maximum of the per-particle FP64 deviations.  FP64 state: the deviation per
// particle.  A NaN q propagates.
__device__ __forceinline__ float nanmin_f(float a, float b) { return (a < b || a != a) ? a : b; }
__device__ __forceinline__ float nanmax_f(float a, float b) { return (a > b || a != a) ? a : b; }

template <typename R>
struct CasimirSlot;
// (smallest, largest) packed into the 8 bytes of a double slot (low, high word)
__device__ __forceinline__ double pack_minmax(float mn, float mx) {
    return __hiloint2double(__float_as_int(mx), __float_as_int(mn));
}
__device__ __forceinline__ float unpack_min(double d) { return __int_as_float(__double2loint(d)); }
__device__ __forceinline__ float unpack_max(double d) { return __int_as_float(__double2hiint(d)); }

template <>
struct CasimirSlot<float> {
    static __device__ __forceinline__ void init(double* slot) { *slot = pack_minmax(INFINITY, -INFINITY); }
    static __device__ __forceinline__ void add(double* slot, float q, double) {
        *slot = pack_minmax(nanmin_f(unpack_min(*slot), q), nanmax_f(unpack_max(*slot), q));
    }
    static __device__ __forceinline__ double finish(const double* slot, double ref, long long n) {
        if (n == 0) return 0.0;
        return nanmax(fabs((double)unpack_min(*slot) - ref), fabs((double)unpack_max(*slot) - ref));
    }
};
template <>
struct CasimirSlot<double> {
    static __device__ __forceinline__ void init(double* slot) { *slot = 0.0; }
    static __device__ __forceinline__ void add(double* slot, double q, double ref) {
        *slot = nanmax(*slot, fabs(q - ref));
    }
    static __device__ __forceinline__ double finish(const double* slot, double, long long) { return *slot; }
};

// partial observables of particles [c0, c1) into out[GL_MAX_SPECIES * PO_N];
// blockDim.x == OBS_THREADS, obs_smem_bytes(oa.sp.n_species) of dynamic
// shared memory at least.  Per thread and species, in its column: the count
// (an integer in the PO_COUNT slot until the end), sums of p_x^2, p_y^2, p_L^2
// (the products of the state's values, exact in FP64) and of p_T^2(tau_form)
// in the PO_DPT2 slot (<dp_T^2> = sum p_x^2 + sum p_y^2 - sum p_T^2(tau_form)),
// and the Casimir slots; then one fixed-order tree over the columns.
template <typename R>
__device__ __forceinline__ void particle_obs_block(const Parts<R>& P, double t, uint32_t active, const ObsArgs& oa,
                                                   int64_t c0, int64_t c1, double* out) {
    extern __shared__ double obs_acc[];
    const int ns = oa.sp.n_species, rows = ns * PO_N, tid = threadIdx.x;
    for (int s = 0; s < ns; s++) {
        double* a = obs_acc + (size_t)s * PO_N * OBS_THREADS + tid;
        a[PO_COUNT * OBS_THREADS] = __longlong_as_double(0);
        a[PO_PX2 * OBS_THREADS] = 0.0;
        a[PO_PY2 * OBS_THREADS] = 0.0;
        a[PO_PL2 * OBS_THREADS] = 0.0;
        a[PO_DPT2 * OBS_THREADS] = 0.0;
        CasimirSlot<R>::init(a + PO_Q2 * OBS_THREADS);
        CasimirSlot<R>::init(a + PO_Q3 * OBS_THREADS);
    }
    // two particles per iteration, both loaded before either is accumulated
    // (in order: the first, then the second), so their loads overlap
    auto accumulate = [&](int64_t i, int s, const PState<R>& p, double pt0) {
        const R pl = particle_pl<R>(p, (R)t, (R)oa.sp.mass[s], oa.sp.motion[s] != MOTION_WONG);
        const double px = p.px, py = p.py, dpl = pl;
        double* a = obs_acc + (size_t)s * PO_N * OBS_THREADS + tid;
        a[PO_COUNT * OBS_THREADS] = __longlong_as_double(__double_as_longlong(a[PO_COUNT * OBS_THREADS]) + 1);
        a[PO_PX2 * OBS_THREADS] = fma(px, px, a[PO_PX2 * OBS_THREADS]);
        a[PO_PY2 * OBS_THREADS] = fma(py, py, a[PO_PY2 * OBS_THREADS]);
        a[PO_PL2 * OBS_THREADS] = fma(dpl, dpl, a[PO_PL2 * OBS_THREADS]);
        a[PO_DPT2 * OBS_THREADS] += pt0;
        CasimirSlot<R>::add(a + PO_Q2 * OBS_THREADS, a_dot(p.q, p.q), oa.q2ref[s]);
        CasimirSlot<R>::add(a + PO_Q3 * OBS_THREADS, casimir3(p.q), oa.q3ref[s]);
    };
    for (int64_t i = c0 + tid; i < c1; i += 2 * OBS_THREADS) {
        const int64_t j = i + OBS_THREADS;
        const int si = P.sp[i];
        const int sj = j < c1 ? P.sp[j] : -1;
        const bool oki = (unsigned)si < (unsigned)ns && ((active >> si) & 1u);
        const bool okj = (unsigned)sj < (unsigned)ns && ((active >> sj) & 1u);
        PState<R> pi_, pj;
        double ti = 0.0, tj = 0.0;
        if (oki) { pi_ = P.load(i); ti = P.pt0[i]; }
        if (okj) { pj = P.load(j); tj = P.pt0[j]; }
        if (oki) accumulate(i, si, pi_, ti);
        if (okj) accumulate(j, sj, pj, tj);
    }
    // the thread's partial values in place, in its own column
    for (int s = 0; s < ns; s++) {
        double* a = obs_acc + (size_t)s * PO_N * OBS_THREADS + tid;
        const long long n = __double_as_longlong(a[PO_COUNT * OBS_THREADS]);
        a[PO_COUNT * OBS_THREADS] = (double)n;
        a[PO_DPT2 * OBS_THREADS] = a[PO_PX2 * OBS_THREADS] + a[PO_PY2 * OBS_THREADS] - a[PO_DPT2 * OBS_THREADS];
        a[PO_Q2 * OBS_THREADS] = CasimirSlot<R>::finish(a + PO_Q2 * OBS_THREADS, oa.q2ref[s], n);
        a[PO_Q3 * OBS_THREADS] = CasimirSlot<R>::finish(a + PO_Q3 * OBS_THREADS, oa.q3ref[s], n);
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
