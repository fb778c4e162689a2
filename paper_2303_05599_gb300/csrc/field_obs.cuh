// The FP64 field checks of one site (Gauss constraint of Sec. 2, unitarity of
// the links, the squared site fields whose lattice means give the energy
// density) and the block reduction of their accumulators, shared by the
// single-event launch (obs.cu) and the one launch over all events of a batch.
// The maxima leave the kernels as squared norms; the host takes their roots.
#pragma once
#include "internal.h"
#include "layout.cuh"
#include "obs_body.cuh"

namespace gl {

template <typename R>
__device__ __forceinline__ A8<double> to_d(const A8<R>& a) {
    A8<double> o;
#pragma unroll
    for (int k = 0; k < 8; k++) o.v[k] = (double)a.v[k];
    return o;
}
template <typename R>
__device__ __forceinline__ M3<double> to_d(const M3<R>& a) {
    M3<double> o;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) { o.re[i][j] = a.re[i][j]; o.im[i][j] = a.im[i][j]; }
    return o;
}

// Site s = (x, y) into the accumulators v[FO_N]:
//   G(x) = sum_i [e_i(x) - U_i(x-i)^+ e_i(x-i) U_i(x-i)] + i[phi(x), pi(x)]
// (with the full transport: for a link that is not unitary, which is what the
// check is for, U^+ e U has a trace) and ||U U^+ - 1||_F of both links at s,
// in FP64; the maxima are kept as squared norms (the root, monotonic, is taken
// once of the maximum).  The sums of squares of the six site fields, whose
// halves are tr X^2 = X^a X^a / 2, go into SquareSum<R> slots: an FP32
// state's squares are exact as float pairs, so its sums cost no FP64 issue
// (field_obs_finish turns the slots into FP64 values).
template <typename R>
__device__ __forceinline__ void field_obs_site(const Fields<R>& f, const typename Prec<R>::V* __restrict__ site,
                                               int N, int64_t Vn, int64_t s, double* v) {
    constexpr int AP = Prec<R>::AP;
    const int x = (int)(s % N), y = (int)(s / N);
    const int64_t sb[2] = {(int64_t)y * N + (x == 0 ? N - 1 : x - 1), (int64_t)(y == 0 ? N - 1 : y - 1) * N + x};
    A8<double> G = icomm(to_d(load_alg(f.phi, s, Vn)), to_d(load_alg(f.pi, s, Vn)));
#pragma unroll
    for (int d = 0; d < 2; d++) {
        const typename Prec<R>::V* e = f.e + (size_t)d * AP * Vn;
        const A8<double> eh = to_d(load_alg(e, s, Vn));
        const A8<double> eb = conj_dn(to_d(load_link(f.U, d, sb[d], Vn)), to_d(load_alg(e, sb[d], Vn)));
        for (int a = 0; a < 8; a++) G.v[a] += eh.v[a] - eb.v[a];
        // unitarity of the link at (d, s): ||U U^+ - 1||_F^2 from the Gram
        // matrix of the rows (Hermitian: upper triangle, off-diagonal twice;
        // the diagonal is real)
        const M3<double> u = to_d(load_link(f.U, d, s, Vn));
        double n2 = 0;
        for (int i = 0; i < 3; i++)
            for (int j = i; j < 3; j++) {
                double gr = 0, gi = 0;
                for (int k = 0; k < 3; k++) {
                    gr = fma(u.re[i][k], u.re[j][k], gr);
                    gr = fma(u.im[i][k], u.im[j][k], gr);
                    if (i != j) {
                        gi = fma(u.im[i][k], u.re[j][k], gi);
                        gi = fma(-u.re[i][k], u.im[j][k], gi);
                    }
                }
                const double r = gr - (i == j ? 1.0 : 0.0);
                n2 += (i == j ? 1.0 : 2.0) * (r * r + gi * gi);
            }
        v[FO_UMAX] = nanmax(v[FO_UMAX], n2);
    }
    const double g2 = a_dot(G, G);
    v[FO_GMAX] = nanmax(v[FO_GMAX], g2);
    v[FO_GSUM] += g2;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const A8<R> X = load_alg(site + (size_t)k * AP * Vn, s, Vn);
        const int slot = k < 2 ? FO_ET2 : k == 2 ? FO_EL2 : k < 5 ? FO_BT2 : FO_BL2;
#pragma unroll
        for (int a = 0; a < 8; a++) v[slot] = SquareSum<R>::add(v[slot], X.v[a]);
    }
}

// the thread's accumulators before its first site
template <typename R>
__device__ __forceinline__ void field_obs_init(double* v) {
    v[FO_GMAX] = v[FO_GSUM] = v[FO_UMAX] = 0.0;
#pragma unroll
    for (int k = FO_ET2; k <= FO_BL2; k++) v[k] = SquareSum<R>::init();
}

// after its last site: the sums of squares as FP64 halves (tr X^2)
template <typename R>
__device__ __forceinline__ void field_obs_finish(double* v) {
#pragma unroll
    for (int k = FO_ET2; k <= FO_BL2; k++) v[k] = 0.5 * SquareSum<R>::finish(v[k]);
}

// the block's accumulators (maxima and sums, fixed order) into row[FO_N];
// every thread of the block calls it
__device__ __forceinline__ void field_obs_block_reduce(double* v, double* row) {
    __shared__ double wacc[32][FO_N];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < FO_N; k++) {
            const double oth = __shfl_down_sync(0xffffffffu, v[k], o);
            v[k] = (k == FO_GMAX || k == FO_UMAX) ? nanmax(v[k], oth) : v[k] + oth;
        }
    if (lane == 0)
        for (int k = 0; k < FO_N; k++) wacc[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x < FO_N) {
        const int k = threadIdx.x;
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++)
            a = (k == FO_GMAX || k == FO_UMAX) ? nanmax(a, wacc[w][k]) : a + wacc[w][k];
        row[k] = a;
    }
}

}  // namespace gl
