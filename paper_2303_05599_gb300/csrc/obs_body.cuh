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
// Per-particle quantities are evaluated in the state's precision.  Within a
// block each thread accumulates its own particles (c0 + tid, c0 + tid +
// OBS_THREADS, ...) into its own column of shared memory, then a fixed-order
// reduction combines the columns (per row: each lane over eight columns, then a
// shuffle tree).  FP64 issue is the scarce
// resource of this reduction (GB300 runs FP64 at 1/64 of the FP32 rate), so a
// particle of an FP32 state costs one FP64 add (p_T^2(tau_form), stored in
// FP64): its squares p_x^2, p_y^2, p_L^2 are summed as exact float pairs (see
// SquareSum), the count is an integer and the Casimir deviations are taken at
// the extremes.  An FP64 state sums its squares with FP64 fused adds.
#pragma once
#include "internal.h"
#include "layout.cuh"
#include "parts.cuh"
#include "su3.cuh"

namespace gl {

static constexpr int OBS_THREADS = 256;
static constexpr int OBS_MAX_BLOCKS = 1024;

// particles per observables block: an eighth of the event's particles, kept
// within [1024, 4096] (at least 4 a thread, so that the block's reductions of
// its columns stay a small share of its work; small events still spread over
// 8 blocks, large ones take 16 a thread), and at most OBS_MAX_BLOCKS blocks;
// a multiple of OBS_THREADS.  A function of the event's particle count only.
__host__ __device__ inline int64_t obs_chunk(int64_t np) {
    int64_t t = (np + 7) / 8;
    t = t < 1024 ? 1024 : t > 4096 ? 4096 : t;
    int64_t c = (np + OBS_MAX_BLOCKS - 1) / OBS_MAX_BLOCKS;
    if (c < t) c = t;
    return (c + OBS_THREADS - 1) / OBS_THREADS * OBS_THREADS;
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

// Casimir drifts max |q - ref|.  FP32 state: the smallest and largest q
// (exact in any precision: no rounding) are kept in the 8-byte slot, through
// the block's tree as well, and |q - ref| is taken in FP64 once per block at
// the two extremes, where the largest deviation lies.  The rounded |q - ref|
// is monotonic on either side of ref, so this is bitwise the maximum of the
// per-particle FP64 deviations.  FP64 state: the deviation per particle.  A
// NaN q propagates.
__device__ __forceinline__ float nanmin_f(float a, float b) { return (a < b || a != a) ? a : b; }
__device__ __forceinline__ float nanmax_f(float a, float b) { return (a > b || a != a) ? a : b; }

// two floats in the 8 bytes of a double slot (low word, high word)
__device__ __forceinline__ double pack_f2(float lo_word, float hi_word) {
    return __hiloint2double(__float_as_int(hi_word), __float_as_int(lo_word));
}
__device__ __forceinline__ float f2_lo(double d) { return __int_as_float(__double2loint(d)); }
__device__ __forceinline__ float f2_hi(double d) { return __int_as_float(__double2hiint(d)); }

template <typename R>
struct CasimirSlot;
template <>
struct CasimirSlot<float> {
    // (smallest, largest) in the (low, high) word
    static __device__ __forceinline__ double init() { return pack_f2(INFINITY, -INFINITY); }
    static __device__ __forceinline__ double add(double v, float q, double) {
        return pack_f2(nanmin_f(f2_lo(v), q), nanmax_f(f2_hi(v), q));
    }
    static __device__ __forceinline__ double combine(double a, double b) {
        return pack_f2(nanmin_f(f2_lo(a), f2_lo(b)), nanmax_f(f2_hi(a), f2_hi(b)));
    }
    static __device__ __forceinline__ double finish(double v, double ref, long long n) {
        if (n == 0) return 0.0;
        return nanmax(fabs((double)f2_lo(v) - ref), fabs((double)f2_hi(v) - ref));
    }
};
template <>
struct CasimirSlot<double> {
    static __device__ __forceinline__ double init() { return 0.0; }
    static __device__ __forceinline__ double add(double v, double q, double ref) { return nanmax(v, fabs(q - ref)); }
    static __device__ __forceinline__ double combine(double a, double b) { return nanmax(a, b); }
    static __device__ __forceinline__ double finish(double v, double, long long) { return v; }
};

// Sums of squares x^2.  FP32 state: the square of a float is exact as a pair
// of floats, hi = x*x rounded and lo = fma(x, x, -hi) its rounding error
// (Dekker's product with a fused multiply-add).  A sum is kept as an
// unevaluated pair (S, s) in the 8-byte slot, through the block's tree as
// well: hi parts (and, in the tree, the other S) enter S through Knuth's
// error-free two-sum, and the two-sum errors and lo parts are added up in s.
// Every step but the additions into s is exact, so a sum of k squares carries
// a relative error of about k 2^-48 (an FP64 sum: k 2^-53), on FP32 issue
// only; the pair becomes one FP64 value once per block.  The operations are
// the round-to-nearest intrinsics, which the compiler neither contracts into
// fused multiply-adds nor reorders.  A square beyond the FP32 range (|x| >
// 1.8e19) makes the sum NaN.  FP64 state: FP64 fused adds.
__device__ __forceinline__ void two_sum_f(float a, float b, float& t, float& err) {
    t = __fadd_rn(a, b);
    const float bv = __fsub_rn(t, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(t, bv)), __fsub_rn(b, bv));
}
template <typename R>
struct SquareSum;
template <>
struct SquareSum<float> {
    // (S, s) in the (low, high) word
    static __device__ __forceinline__ double init() { return pack_f2(0.0f, 0.0f); }
    static __device__ __forceinline__ double add(double v, float x) {
        const float hi = __fmul_rn(x, x), lo = __fmaf_rn(x, x, -hi);
        float t, err;
        two_sum_f(f2_lo(v), hi, t, err);
        return pack_f2(t, __fadd_rn(f2_hi(v), __fadd_rn(err, lo)));
    }
    static __device__ __forceinline__ double combine(double a, double b) {
        float t, err;
        two_sum_f(f2_lo(a), f2_lo(b), t, err);
        return pack_f2(t, __fadd_rn(__fadd_rn(f2_hi(a), f2_hi(b)), err));
    }
    static __device__ __forceinline__ double finish(double v) { return (double)f2_lo(v) + (double)f2_hi(v); }
};
template <>
struct SquareSum<double> {
    static __device__ __forceinline__ double init() { return 0.0; }
    static __device__ __forceinline__ double add(double v, double x) { return fma(x, x, v); }
    static __device__ __forceinline__ double combine(double a, double b) { return a + b; }
    static __device__ __forceinline__ double finish(double v) { return v; }
};

// the particle count, a 64-bit integer in the slot's bits
__device__ __forceinline__ double count_add(double v, long long k) {
    return __longlong_as_double(__double_as_longlong(v) + k);
}

// the tree's combination of two slots of kind k (PO_*)
template <typename R>
__device__ __forceinline__ double obs_combine(int k, double a, double b) {
    switch (k) {
    case PO_COUNT: return count_add(a, __double_as_longlong(b));
    case PO_PX2:
    case PO_PY2:
    case PO_PL2: return SquareSum<R>::combine(a, b);
    case PO_DPT2: return a + b;
    default: return CasimirSlot<R>::combine(a, b);
    }
}

// partial observables of particles [c0, c1) into out[GL_MAX_SPECIES * PO_N];
// blockDim.x == OBS_THREADS, obs_smem_bytes(oa.sp.n_species) of dynamic
// shared memory at least.  Per thread and species, in its column: the count,
// the sums of p_x^2, p_y^2, p_L^2 (SquareSum) and of p_T^2(tau_form) (FP64,
// in the PO_DPT2 slot) and the Casimir slots; then one fixed-order reduction
// of each row's columns, and one thread per species turns the block's slots
// into FP64 values (<dp_T^2> = sum p_x^2 + sum p_y^2 - sum p_T^2(tau_form)).
template <typename R>
__device__ __forceinline__ void particle_obs_block(const Parts<R>& P, double t, uint32_t active, const ObsArgs& oa,
                                                   int64_t c0, int64_t c1, double* out) {
    extern __shared__ double obs_acc[];
    __shared__ R obs_mass[GL_MAX_SPECIES];
    const int ns = oa.sp.n_species, rows = ns * PO_N, tid = threadIdx.x;
    for (int s = 0; s < ns; s++) {
        double* a = obs_acc + (size_t)s * PO_N * OBS_THREADS + tid;
        a[PO_COUNT * OBS_THREADS] = __longlong_as_double(0);
        a[PO_PX2 * OBS_THREADS] = SquareSum<R>::init();
        a[PO_PY2 * OBS_THREADS] = SquareSum<R>::init();
        a[PO_PL2 * OBS_THREADS] = SquareSum<R>::init();
        a[PO_DPT2 * OBS_THREADS] = 0.0;
        a[PO_Q2 * OBS_THREADS] = CasimirSlot<R>::init();
        a[PO_Q3 * OBS_THREADS] = CasimirSlot<R>::init();
    }
    // the masses in the state's precision, converted once per block
    if (tid < ns) obs_mass[tid] = (R)oa.sp.mass[tid];
    __syncthreads();
    const R tr = (R)t;
    // two particles per iteration, both loaded before either is accumulated
    // (in order: the first, then the second), so their loads overlap
    auto accumulate = [&](int s, const PState<R>& p, double pt0) {
        const R pl = particle_pl<R>(p, tr, obs_mass[s], oa.sp.motion[s] != MOTION_WONG);
        double* a = obs_acc + (size_t)s * PO_N * OBS_THREADS + tid;
        a[PO_COUNT * OBS_THREADS] = count_add(a[PO_COUNT * OBS_THREADS], 1);
        a[PO_PX2 * OBS_THREADS] = SquareSum<R>::add(a[PO_PX2 * OBS_THREADS], p.px);
        a[PO_PY2 * OBS_THREADS] = SquareSum<R>::add(a[PO_PY2 * OBS_THREADS], p.py);
        a[PO_PL2 * OBS_THREADS] = SquareSum<R>::add(a[PO_PL2 * OBS_THREADS], pl);
        a[PO_DPT2 * OBS_THREADS] += pt0;
        a[PO_Q2 * OBS_THREADS] = CasimirSlot<R>::add(a[PO_Q2 * OBS_THREADS], a_dot(p.q, p.q), oa.q2ref[s]);
        a[PO_Q3 * OBS_THREADS] = CasimirSlot<R>::add(a[PO_Q3 * OBS_THREADS], casimir3(p.q), oa.q3ref[s]);
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
        if (oki) accumulate(si, pi_, ti);
        if (okj) accumulate(sj, pj, tj);
    }
    // each row's columns: warp w takes rows w, w + 8, ...; lane l combines
    // columns l, l + 32, ... in order, then the warp's fixed shuffle tree, and
    // lane 0 leaves the row's total in column 0
    __syncthreads();
    const int lane = tid & 31;
    for (int r = tid >> 5; r < rows; r += OBS_THREADS / 32) {
        double* a = obs_acc + r * OBS_THREADS;
        const int kind = r % PO_N;
        double x = a[lane];
        for (int c = lane + 32; c < OBS_THREADS; c += 32) x = obs_combine<R>(kind, x, a[c]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = obs_combine<R>(kind, x, __shfl_down_sync(0xffffffffu, x, o));
        if (lane == 0) a[0] = x;
    }
    __syncthreads();
    if (tid < ns) {
        const double* a = obs_acc + (size_t)tid * PO_N * OBS_THREADS;  // column 0
        double* o = out + tid * PO_N;
        const long long n = __double_as_longlong(a[PO_COUNT * OBS_THREADS]);
        const double px2 = SquareSum<R>::finish(a[PO_PX2 * OBS_THREADS]);
        const double py2 = SquareSum<R>::finish(a[PO_PY2 * OBS_THREADS]);
        o[PO_COUNT] = (double)n;
        o[PO_PX2] = px2;
        o[PO_PY2] = py2;
        o[PO_PL2] = SquareSum<R>::finish(a[PO_PL2 * OBS_THREADS]);
        o[PO_DPT2] = px2 + py2 - a[PO_DPT2 * OBS_THREADS];
        o[PO_Q2] = CasimirSlot<R>::finish(a[PO_Q2 * OBS_THREADS], oa.q2ref[tid], n);
        o[PO_Q3] = CasimirSlot<R>::finish(a[PO_Q3 * OBS_THREADS], oa.q3ref[tid], n);
    }
    for (int k = rows + tid; k < GL_MAX_SPECIES * PO_N; k += OBS_THREADS) out[k] = 0.0;
}

// allow the largest dynamic shared memory of particle_obs_block on kernel f
template <typename K>
inline void obs_smem_attr(K f) {
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)obs_smem_bytes(GL_MAX_SPECIES));
}

// The final reduction of per-block partial rows [nblocks][width] (sums, or
// NaN-propagating maxima where is_max(k)) into out[0, width) and, when copy
// is not null, into copy[0, width) as well, by one block of 8 warps: warp w
// takes values w, w + 8, ... (at most OBS_FINAL_V of them); for each, lane l
// combines rows l, l + 32, ... in order, then the warp's fixed shuffle tree.
// A lane loads its row's values of all the warp's values at once, so a
// reduction over at most 32 rows waits on one load.  The order depends only
// on nblocks, so every launch that reduces the same rows (one event, or one
// block per event of a batch) gives bitwise the same values.
static constexpr int OBS_FINAL_WARPS = 8, OBS_FINAL_V = 8;
template <typename IsMax>
__device__ __forceinline__ void obs_finalize_block(const double* partials, int nblocks, int width, IsMax is_max,
                                                   double* out, double* copy = nullptr) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double acc[OBS_FINAL_V];
#pragma unroll
    for (int j = 0; j < OBS_FINAL_V; j++) acc[j] = 0.0;
    for (int b = lane; b < nblocks; b += 32) {
        const double* row = partials + (size_t)b * width;
        double v[OBS_FINAL_V];
#pragma unroll
        for (int j = 0; j < OBS_FINAL_V; j++) {
            const int k = w + j * OBS_FINAL_WARPS;
            v[j] = k < width ? row[k] : 0.0;
        }
#pragma unroll
        for (int j = 0; j < OBS_FINAL_V; j++) {
            const int k = w + j * OBS_FINAL_WARPS;
            acc[j] = (k < width && is_max(k)) ? nanmax(acc[j], v[j]) : acc[j] + v[j];
        }
    }
#pragma unroll
    for (int j = 0; j < OBS_FINAL_V; j++) {
        const int k = w + j * OBS_FINAL_WARPS;
        const bool mx = k < width && is_max(k);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double oth = __shfl_down_sync(0xffffffffu, acc[j], o);
            acc[j] = mx ? nanmax(acc[j], oth) : acc[j] + oth;
        }
        if (lane == 0 && k < width) {
            out[k] = acc[j];
            if (copy) copy[k] = acc[j];
        }
    }
}

// the kinds of the particle values (GL_MAX_SPECIES x PO_N) and of the field
// checks (FO_N)
struct ParticleObsKind {
    __device__ bool operator()(int k) const { return po_is_max(k % PO_N); }
};
struct FieldObsKind {
    __device__ bool operator()(int k) const { return k == FO_GMAX || k == FO_UMAX; }
};

}  // namespace gl
