// Device data layout.  Every per-site or per-particle quantity is stored as
// planes of 16-byte vectors (double2 for the FP64 path, float4 for the FP32
// path), one plane per group of components, so a warp reading one plane reads
// 512 contiguous bytes.
//
//   links   U   [dir][LP][V]  FP64: 9 double2 = 3x3 complex, row-major
//                             FP32: 3 float4 = rows 0 and 1 only
//                             (u00,u01) (u02,u10) (u11,u12); row 2 is rebuilt
//                             as conj(row0 x row1) on every load
//   algebra     [AP][V]       8 components X^a: FP64 4 double2, FP32 2 float4
//   particles   see particles.cu
#pragma once
#include <stdint.h>
#include "su3.cuh"

namespace gl {

template <typename R>
struct Prec;
template <>
struct Prec<double> {
    using V = double2;
    static constexpr int LP = 9;
    static constexpr int AP = 4;
};
template <>
struct Prec<float> {
    using V = float4;
    static constexpr int LP = 3;
    static constexpr int AP = 2;
};

// one time slice of the fields: U(n), phi(n), e(n-1/2), pi(n-1/2)
template <typename R>
struct Fields {
    using V = typename Prec<R>::V;
    V* U;    // [2][LP][Vn]
    V* phi;  // [AP][Vn]
    V* e;    // [2][AP][Vn]
    V* pi;   // [AP][Vn]
};

template <typename R>
__host__ __device__ inline size_t fields_vectors(int64_t Vn) {
    return (size_t)Vn * (2 * Prec<R>::LP + 4 * Prec<R>::AP);
}

template <typename R>
__host__ __device__ inline Fields<R> carve_fields(void* base, int64_t Vn) {
    using V = typename Prec<R>::V;
    Fields<R> f;
    V* p = (V*)base;
    f.U = p; p += (size_t)2 * Prec<R>::LP * Vn;
    f.phi = p; p += (size_t)Prec<R>::AP * Vn;
    f.e = p; p += (size_t)2 * Prec<R>::AP * Vn;
    f.pi = p;
    return f;
}

__device__ __forceinline__ M3<double> load_link(const double2* __restrict__ U, int d, int64_t s, int64_t Vn) {
    const double2* b = U + (size_t)d * 9 * Vn + s;
    M3<double> m;
#pragma unroll
    for (int k = 0; k < 9; k++) {
        double2 v = __ldg(b + (size_t)k * Vn);
        m.re[k / 3][k % 3] = v.x;
        m.im[k / 3][k % 3] = v.y;
    }
    return m;
}

__device__ __forceinline__ M3<float> load_link(const float4* __restrict__ U, int d, int64_t s, int64_t Vn) {
    const float4* b = U + (size_t)d * 3 * Vn + s;
    float4 a = __ldg(b), c = __ldg(b + Vn), e = __ldg(b + 2 * Vn);
    M3<float> m;
    m.re[0][0] = a.x; m.im[0][0] = a.y; m.re[0][1] = a.z; m.im[0][1] = a.w;
    m.re[0][2] = c.x; m.im[0][2] = c.y; m.re[1][0] = c.z; m.im[1][0] = c.w;
    m.re[1][1] = e.x; m.im[1][1] = e.y; m.re[1][2] = e.z; m.im[1][2] = e.w;
    rebuild_row2(m);
    return m;
}

__device__ __forceinline__ void store_link(double2* U, int d, int64_t s, int64_t Vn, const M3<double>& m) {
    double2* b = U + (size_t)d * 9 * Vn + s;
#pragma unroll
    for (int k = 0; k < 9; k++) b[(size_t)k * Vn] = make_double2(m.re[k / 3][k % 3], m.im[k / 3][k % 3]);
}

__device__ __forceinline__ void store_link(float4* U, int d, int64_t s, int64_t Vn, const M3<float>& m) {
    float4* b = U + (size_t)d * 3 * Vn + s;
    b[0] = make_float4(m.re[0][0], m.im[0][0], m.re[0][1], m.im[0][1]);
    b[Vn] = make_float4(m.re[0][2], m.im[0][2], m.re[1][0], m.im[1][0]);
    b[2 * Vn] = make_float4(m.re[1][1], m.im[1][1], m.re[1][2], m.im[1][2]);
}

__device__ __forceinline__ A8<double> load_alg(const double2* __restrict__ A, int64_t s, int64_t Vn) {
    A8<double> x;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        double2 v = __ldg(A + (size_t)k * Vn + s);
        x.v[2 * k] = v.x;
        x.v[2 * k + 1] = v.y;
    }
    return x;
}

__device__ __forceinline__ A8<float> load_alg(const float4* __restrict__ A, int64_t s, int64_t Vn) {
    A8<float> x;
    float4 a = __ldg(A + s), b = __ldg(A + Vn + s);
    x.v[0] = a.x; x.v[1] = a.y; x.v[2] = a.z; x.v[3] = a.w;
    x.v[4] = b.x; x.v[5] = b.y; x.v[6] = b.z; x.v[7] = b.w;
    return x;
}

__device__ __forceinline__ void store_alg(double2* A, int64_t s, int64_t Vn, const A8<double>& x) {
#pragma unroll
    for (int k = 0; k < 4; k++) A[(size_t)k * Vn + s] = make_double2(x.v[2 * k], x.v[2 * k + 1]);
}

__device__ __forceinline__ void store_alg(float4* A, int64_t s, int64_t Vn, const A8<float>& x) {
    A[s] = make_float4(x.v[0], x.v[1], x.v[2], x.v[3]);
    A[Vn + s] = make_float4(x.v[4], x.v[5], x.v[6], x.v[7]);
}

// the same stores with the streaming (evict-first) cache hint: for values the
// next launch reads long after they have left L2, so that they do not push
// out lines that are still to be read
__device__ __forceinline__ void store_link_cs(double2* U, int d, int64_t s, int64_t Vn, const M3<double>& m) {
    double2* b = U + (size_t)d * 9 * Vn + s;
#pragma unroll
    for (int k = 0; k < 9; k++) __stcs(b + (size_t)k * Vn, make_double2(m.re[k / 3][k % 3], m.im[k / 3][k % 3]));
}
__device__ __forceinline__ void store_link_cs(float4* U, int d, int64_t s, int64_t Vn, const M3<float>& m) {
    float4* b = U + (size_t)d * 3 * Vn + s;
    __stcs(b, make_float4(m.re[0][0], m.im[0][0], m.re[0][1], m.im[0][1]));
    __stcs(b + Vn, make_float4(m.re[0][2], m.im[0][2], m.re[1][0], m.im[1][0]));
    __stcs(b + 2 * Vn, make_float4(m.re[1][1], m.im[1][1], m.re[1][2], m.im[1][2]));
}
__device__ __forceinline__ void store_alg_cs(double2* A, int64_t s, int64_t Vn, const A8<double>& x) {
#pragma unroll
    for (int k = 0; k < 4; k++) __stcs(A + (size_t)k * Vn + s, make_double2(x.v[2 * k], x.v[2 * k + 1]));
}
__device__ __forceinline__ void store_alg_cs(float4* A, int64_t s, int64_t Vn, const A8<float>& x) {
    __stcs(A + s, make_float4(x.v[0], x.v[1], x.v[2], x.v[3]));
    __stcs(A + Vn + s, make_float4(x.v[4], x.v[5], x.v[6], x.v[7]));
}

// components of i[A, B] for Hermitian A, B: -f_abc A^a B^b T^c, with the nine
// independent structure constants of SU(3)
template <typename R>
__device__ __forceinline__ A8<R> icomm(const A8<R>& A, const A8<R>& B) {
    A8<R> o = a_zero<R>();
    const R h = R(0.5), s = R(0.86602540378443864676);
#define GL_F(a, b, c, F)                                              \
    {                                                                 \
        o.v[c] -= (F) * (A.v[a] * B.v[b] - A.v[b] * B.v[a]);         \
        o.v[a] -= (F) * (A.v[b] * B.v[c] - A.v[c] * B.v[b]);         \
        o.v[b] -= (F) * (A.v[c] * B.v[a] - A.v[a] * B.v[c]);         \
    }
    GL_F(0, 1, 2, R(1));
    GL_F(0, 3, 6, h);
    GL_F(0, 4, 5, -h);
    GL_F(1, 3, 5, h);
    GL_F(1, 4, 6, h);
    GL_F(2, 3, 4, h);
    GL_F(2, 5, 6, -h);
    GL_F(3, 4, 7, s);
    GL_F(5, 6, 7, s);
#undef GL_F
    return o;
}

// maximum that propagates NaN (fmax drops it), so that a non-finite value
// anywhere shows in the reported maxima
__device__ __forceinline__ double nanmax(double a, double b) { return (a > b || a != a) ? a : b; }

// i mod n in [0, n) for n > 0; indices within one period of the lattice
// (tile halos, particle cells) take a compare and an add instead of a
// division by the runtime n
__device__ __forceinline__ int wrapi(int i, int n) {
    if (i >= -n && i < 2 * n) return i < 0 ? i + n : (i >= n ? i - n : i);
    i %= n;
    return i < 0 ? i + n : i;
}

}  // namespace gl
