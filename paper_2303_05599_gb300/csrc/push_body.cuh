// Particle push body shared by the single-event and batched kernels.
#pragma once
#include "parts.cuh"

namespace gl {

template <typename R>
struct SpeciesArgs {
    R mass[GL_MAX_SPECIES];
    int motion[GL_MAX_SPECIES];  // MOTION_*
    int ptau_diag;               // integrate p^tau beside the mass shell
};

template <typename R>
__device__ __forceinline__ R floor_r(R v);
template <>
__device__ __forceinline__ double floor_r<double>(double v) { return floor(v); }
template <>
__device__ __forceinline__ float floor_r<float>(float v) { return floorf(v); }

template <typename R>
__device__ __forceinline__ R fmod_r(R a, R b);
template <>
__device__ __forceinline__ double fmod_r<double>(double a, double b) { return fmod(a, b); }
template <>
__device__ __forceinline__ float fmod_r<float>(float a, float b) { return fmodf(a, b); }

// temporal constraint (Sec. 3.1): one Euler step of p^tau from its own
// equation of motion, started at the mass shell at the particle's first push
// (NaN before).  Kept out of line, so that the arithmetic of the push itself
// is compiled the same way in every kernel that inlines it.
template <typename R>
__device__ __noinline__ R ptau_step(R pt, R shell, R w, R t, R dt, R work) {
    if (pt != pt) pt = shell;
    const R drift = (t > R(0) && shell > R(0)) ? w * w / (t * shell) : R(0);
    return pt + dt * (work - drift);
}

// Euler + CPIC update of particle i (Sec. 3.1 and 3.2); site: site fields at
// t_n, bn1: links and scalar at t_{n+1}
template <typename R>
__device__ __forceinline__ void push_one(const typename Prec<R>::V* __restrict__ site, const Fields<R>& bn1,
                                         const Parts<R>& P, int64_t i, int N, R t, R dt, R dt_over_t,
                                         uint32_t active, const SpeciesArgs<R>& sa) {
    constexpr int AP = Prec<R>::AP;
    const int64_t Vn = (int64_t)N * N;
    const int s = P.sp[i];
    if (!((active >> s) & 1u)) return;
    PState<R> p = P.load_cs(i);
    const int ixu = (int)floor_r<R>(p.x + R(0.5)), iyu = (int)floor_r<R>(p.y + R(0.5));
    // wrap keeps every index inside the lattice even for a non-finite position
    // (float-to-int conversion maps NaN to 0 and saturates out-of-range values)
    const int ix = wrapi(ixu, N), iy = wrapi(iyu, N);
    const int64_t cell = (int64_t)iy * N + ix;
    const R qEx = a_dot(p.q, load_alg(site, cell, Vn));
    const R qEy = a_dot(p.q, load_alg(site + (size_t)1 * AP * Vn, cell, Vn));
    const R qEe = a_dot(p.q, load_alg(site + (size_t)2 * AP * Vn, cell, Vn));
    if (sa.motion[s] == MOTION_STATIC) {
        // infinitely massive: no motion and no colour rotation (temporal gauge)
        p.px += dt * qEx;
        p.py += dt * qEy;
        p.Pe += dt * qEe;
        P.store_momenta_cs(i, p);
        return;
    }
    if (sa.motion[s] == MOTION_EIKONAL) {
        // light-like parton along +x at eta = 0 (Sec. 5.2): fixed path
        // x = x0 + t; the kicks of the Lorentz force (E_x, E_y - B_z, E_z + B_y)
        // accumulate in p^x, p^y and the P_eta slot (lab p_z); Q is carried
        // along by the crossed x link
        const R qBy = a_dot(p.q, load_alg(site + (size_t)4 * AP * Vn, cell, Vn));
        const R qBe = a_dot(p.q, load_alg(site + (size_t)5 * AP * Vn, cell, Vn));
        p.px += dt * qEx;
        p.py += dt * (qEy - qBe);
        p.Pe += dt * (qEe + qBy);
        R xn = p.x + dt;
        const int jxu = (int)floor_r<R>(xn + R(0.5));
        xn = fmod_r<R>(xn, (R)N);
        if (xn < R(0)) xn += (R)N;
        p.x = xn;
        if (jxu != ixu) p.q = conj_dn(load_link(bn1.U, 0, cell, Vn), p.q);
        P.store_cs(i, p);
        return;
    }
    const R qBx = a_dot(p.q, load_alg(site + (size_t)3 * AP * Vn, cell, Vn));
    const R qBy = a_dot(p.q, load_alg(site + (size_t)4 * AP * Vn, cell, Vn));
    const R qBe = a_dot(p.q, load_alg(site + (size_t)5 * AP * Vn, cell, Vn));
    const R m = sa.mass[s];
    const R w = t > R(0) ? p.Pe / t : R(0);  // tau p^eta
    const R ptau = sqrt(p.px * p.px + p.py * p.py + w * w + m * m);
    const R inv_pt = ptau > R(0) ? R(1) / ptau : R(0);
    const R vx = p.px * inv_pt, vy = p.py * inv_pt, vw = w * inv_pt;
    if (sa.ptau_diag) P.ptau[i] = ptau_step<R>(P.ptau[i], ptau, w, t, dt, qEe * vw + qEx * vx + qEy * vy);
    // Wong's equations in Milne coordinates (Sec. 3.1), forward Euler
    const R dpx = qEx + qBe * vy - qBy * vw;
    const R dpy = qEy - qBe * vx + qBx * vw;
    const R dPe = t * (qEe - qBx * vy + qBy * vx);
    const R deta = dt_over_t * vw;
    R xn = p.x + dt * vx, yn = p.y + dt * vy;
    p.eta += deta;
    p.px += dt * dpx;
    p.py += dt * dpy;
    p.Pe += dt * dPe;
    const int jxu = (int)floor_r<R>(xn + R(0.5)), jyu = (int)floor_r<R>(yn + R(0.5));
    xn = fmod_r<R>(xn, (R)N);
    if (xn < R(0)) xn += (R)N;
    yn = fmod_r<R>(yn, (R)N);
    if (yn < R(0)) yn += (R)N;
    p.x = xn;
    p.y = yn;
    // CPIC: rotate with the crossed links at t_{n+1}, x first, then y.  A step
    // up takes U^+ Q U with the link of the old cell, a step down U Q U^+ =
    // (U^+)^+ Q U^+ with the link of the new cell.  Each lane has up to two
    // transports to make (bit 0: x, bit 1: y); one loop body serves both axes,
    // with the link and U or U^+ chosen per lane, so that a warp runs as many
    // transports as its busiest lane needs (crossings are rare, but some lane
    // of a warp crosses almost every step).  The traceless transport: a link is
    // unitary to rounding
    const int dxc = jxu - ixu, dyc = jyu - iyu;
    const int jx = wrapi(jxu, N), jy = wrapi(jyu, N);
    // cell indices of an event fit in 32 bits (N <= 32768)
    const int ix_link = dxc == 1 ? (int)cell : iy * N + jx;
    const int iy_link = dyc == 1 ? iy * N + jx : jy * N + jx;
    int todo = ((dxc == 1 || dxc == -1) ? 1 : 0) | ((dyc == 1 || dyc == -1) ? 2 : 0);
#pragma unroll 1
    while (todo) {
        const bool on_x = todo & 1;
        const M3<R> U = load_link(bn1.U, on_x ? 0 : 1, on_x ? ix_link : iy_link, Vn);
        p.q = conj_dn_t((on_x ? dxc : dyc) == 1 ? U : dag(U), p.q);
        todo &= todo - 1;
    }
    // rapidity Wilson line at the new cell: Q <- e^{-i deta phi} Q e^{+i deta phi}
    if (deta != R(0)) {
        const A8<R> ph = load_alg(bn1.phi, (int64_t)jy * N + jx, Vn);
        p.q = conj_up_t(exp_i_alg<R, (sizeof(R) == 8 ? 20 : 6)>(ph, -deta), p.q);
    }
    P.store_cs(i, p);
}

}  // namespace gl
