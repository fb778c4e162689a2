// Fused Glasma leapfrog step and site E/B interpolation (Sec. 2.1 and 3.2 of
// arXiv:2303.05599) on shared-memory tiles.
//
// One CTA owns a TX x TY tile of sites (TX = 32: one warp per tile row).  Per
// step it computes, from U(n), phi(n), e(n-1/2), pi(n-1/2):
//   the momenta e(n+1/2), pi(n+1/2), the links U(n+1) and the scalar phi(n+1),
//   and the site fields E, B at t_n that the particle push gathers.
// Every cell plaquette is formed once per tile and shared.  With
//   A(c)  = components of i[P(c)]_ah,  P(c) = Ux(c) Uy(c+x) Ux(c+y)^+ Uy(c)^+,
//   Dn(s) = Uy(s-y)^+ A(s-y) Uy(s-y),   Lf(s) = Ux(s-x)^+ A(s-x) Ux(s-x),
// the plaquette forces and the clover are
//   F_x = t (A - Dn),  F_y = t (Lf - A),
//   B_eta = (A + Lf + Dn + Uy(s-y)^+ Lf(s-y) Uy(s-y)) / 4.
// E_x(s) needs e_x(n+1/2) at s - x and E_y(s) needs e_y(n+1/2) at s - y, so
// the tile also advances e_x on one halo column (x0 - 1) and e_y (with Lf) on
// one halo row (y0 - 1); nothing else of the halo is needed.
//
// The tile's inputs are copied to shared memory with cp.async in the storage
// layout of global memory (16-byte vectors; FP32 links as two rows, the third
// rebuilt when a link is read).  Regions, in tile coordinates:
//   links, phi:                   x in [-1, TX],   y in [-1, TY]    (LW x LH)
//   plaquettes A, momenta, Lf:    x in [-1, TX-1], y in [-1, TY-1]  (EW x EH)
// pi(n-1/2) is read by each site's thread straight from global memory.
//
// Every site does each computation at the same point of the code (own and
// halo momenta share one loop body), so the results do not depend on the tile
// shape.  The links arrive in their own group of copies, so the plaquettes
// start while phi and e(n-1/2) are still in flight.
#pragma once
#include "internal.h"
#include "layout.cuh"

namespace gl {

template <typename R>
struct ExpN;
template <>
struct ExpN<double> { static constexpr int n = 20; };
template <>
struct ExpN<float> { static constexpr int n = 6; };

template <typename R, int TX, int TY>
struct Tile {
    using V = typename Prec<R>::V;
    static constexpr int LP = Prec<R>::LP, AP = Prec<R>::AP;
    static constexpr int LW = TX + 2, LH = TY + 2, LN = LW * LH;
    static constexpr int EW = TX + 1, EH = TY + 1, EN = EW * EH;
    static constexpr int NT = TX * TY;
    static constexpr int NH = TX + TY;  // halo momenta: left column (e_x), bottom row (e_y, Lf)
    static_assert(NH <= NT, "halo momenta are one per thread");
    // vectors: links 2 LP LN, phi AP LN, A AP EN, e sums 2 AP EN, Lf AP EN
    static constexpr size_t vecs = (size_t)2 * LP * LN + (size_t)AP * LN + (size_t)4 * AP * EN;
    // FP32 two-row links: the third rows, rebuilt once per staged link,
    // [2][3][LN] float2 after the vectors
    static constexpr size_t row2_bytes = sizeof(R) == 4 ? (size_t)2 * 3 * LN * 8 : 0;
    static constexpr size_t bytes = vecs * sizeof(V) + row2_bytes;
    // CTAs per SM the launch bounds ask for: FP32 kernels are capped at 128
    // registers a thread so that 16 warps fit an SM (the shared memory of
    // 32x4: 4 CTAs, 32x8: 2, 32x16: 1); FP64 tiles take one CTA
    static constexpr int min_blocks = sizeof(R) == 8 ? 1 : (NT >= 512 ? 1 : 512 / NT);
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// link (d) of shared-memory site li, planes of LN vectors
__device__ __forceinline__ M3<double> s_link(const double2* sU, int d, int li, int LN) {
    const double2* b = sU + (size_t)d * 9 * LN + li;
    M3<double> m;
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const double2 v = b[k * LN];
        m.re[k / 3][k % 3] = v.x;
        m.im[k / 3][k % 3] = v.y;
    }
    return m;
}
__device__ __forceinline__ M3<float> s_link(const float4* sU, int d, int li, int LN) {
    const float4* b = sU + (size_t)d * 3 * LN + li;
    const float4 a = b[0], c = b[LN], e = b[2 * LN];
    M3<float> m;
    m.re[0][0] = a.x; m.im[0][0] = a.y; m.re[0][1] = a.z; m.im[0][1] = a.w;
    m.re[0][2] = c.x; m.im[0][2] = c.y; m.re[1][0] = c.z; m.im[1][0] = c.w;
    m.re[1][1] = e.x; m.im[1][1] = e.y; m.re[1][2] = e.z; m.im[1][2] = e.w;
    rebuild_row2(m);
    return m;
}

// links of the tile in shared memory; FP32 links come with their third rows
// stored beside them (rebuilt once when staged)
template <typename R>
struct SLinks;
template <>
struct SLinks<double> {
    const double2* u;
    int LN;
    __device__ __forceinline__ M3<double> operator()(int d, int li) const { return s_link(u, d, li, LN); }
};
template <>
struct SLinks<float> {
    const float4* u;
    const float2* r2;
    int LN;
    __device__ __forceinline__ M3<float> operator()(int d, int li) const {
        const float4* b = u + (size_t)d * 3 * LN + li;
        const float4 a = b[0], c = b[LN], e = b[2 * LN];
        const float2* t = r2 + (size_t)d * 3 * LN + li;
        const float2 f0 = t[0], f1 = t[LN], f2 = t[2 * LN];
        M3<float> m;
        m.re[0][0] = a.x; m.im[0][0] = a.y; m.re[0][1] = a.z; m.im[0][1] = a.w;
        m.re[0][2] = c.x; m.im[0][2] = c.y; m.re[1][0] = c.z; m.im[1][0] = c.w;
        m.re[1][1] = e.x; m.im[1][1] = e.y; m.re[1][2] = e.z; m.im[1][2] = e.w;
        m.re[2][0] = f0.x; m.im[2][0] = f0.y; m.re[2][1] = f1.x; m.im[2][1] = f1.y;
        m.re[2][2] = f2.x; m.im[2][2] = f2.y;
        return m;
    }
};

__device__ __forceinline__ A8<double> s_alg(const double2* s, int i, int n) {
    A8<double> x;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const double2 v = s[k * n + i];
        x.v[2 * k] = v.x;
        x.v[2 * k + 1] = v.y;
    }
    return x;
}
__device__ __forceinline__ A8<float> s_alg(const float4* s, int i, int n) {
    const float4 a = s[i], b = s[n + i];
    A8<float> x;
    x.v[0] = a.x; x.v[1] = a.y; x.v[2] = a.z; x.v[3] = a.w;
    x.v[4] = b.x; x.v[5] = b.y; x.v[6] = b.z; x.v[7] = b.w;
    return x;
}
__device__ __forceinline__ void s_alg_put(double2* s, int i, int n, const A8<double>& x) {
#pragma unroll
    for (int k = 0; k < 4; k++) s[k * n + i] = make_double2(x.v[2 * k], x.v[2 * k + 1]);
}
__device__ __forceinline__ void s_alg_put(float4* s, int i, int n, const A8<float>& x) {
    s[i] = make_float4(x.v[0], x.v[1], x.v[2], x.v[3]);
    s[n + i] = make_float4(x.v[4], x.v[5], x.v[6], x.v[7]);
}

// FP64 Gram-Schmidt of rows 0 and 1 (FP32 links are stored as two rows)
__device__ __forceinline__ void reunit(M3<float>& u) {
    double r0r[3], r0i[3], r1r[3], r1i[3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        r0r[j] = u.re[0][j]; r0i[j] = u.im[0][j];
        r1r[j] = u.re[1][j]; r1i[j] = u.im[1][j];
    }
    double n0 = 0;
#pragma unroll
    for (int j = 0; j < 3; j++) n0 += r0r[j] * r0r[j] + r0i[j] * r0i[j];
    n0 = 1.0 / sqrt(n0);
#pragma unroll
    for (int j = 0; j < 3; j++) { r0r[j] *= n0; r0i[j] *= n0; }
    double cr = 0, ci = 0;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        cr += r0r[j] * r1r[j] + r0i[j] * r1i[j];
        ci += r0r[j] * r1i[j] - r0i[j] * r1r[j];
    }
#pragma unroll
    for (int j = 0; j < 3; j++) {
        r1r[j] -= cr * r0r[j] - ci * r0i[j];
        r1i[j] -= cr * r0i[j] + ci * r0r[j];
    }
    double n1 = 0;
#pragma unroll
    for (int j = 0; j < 3; j++) n1 += r1r[j] * r1r[j] + r1i[j] * r1i[j];
    n1 = 1.0 / sqrt(n1);
#pragma unroll
    for (int j = 0; j < 3; j++) {
        u.re[0][j] = (float)r0r[j]; u.im[0][j] = (float)r0i[j];
        u.re[1][j] = (float)(r1r[j] * n1); u.im[1][j] = (float)(r1i[j] * n1);
    }
}
__device__ __forceinline__ void reunit(M3<double>&) {}

struct StepArgs {
    int N;
    int tiles_x;
    double t, dt, inv_t, dt_over_th, dt_th;
    int reunit;
};

// the step scalars in the kernel's precision (converted once per launch or
// block: double arithmetic costs far more than single on GPUs with slow FP64)
template <typename R>
struct StepR {
    int N, tiles_x, reunit;
    R t, dt, inv_t, dt_over_th, dt_th;
};
template <typename R>
__host__ __device__ inline StepR<R> step_r(const StepArgs& a) {
    StepR<R> r;
    r.N = a.N;
    r.tiles_x = a.tiles_x;
    r.reunit = a.reunit;
    r.t = (R)a.t;
    r.dt = (R)a.dt;
    r.inv_t = (R)a.inv_t;
    r.dt_over_th = (R)a.dt_over_th;
    r.dt_th = (R)a.dt_th;
    return r;
}

// one tile (index `tile` of a lattice with tiles_x tiles per row); the caller
// provides the dynamic shared memory of Tile<R, TX, TY>::bytes
template <typename R, int TX, int TY>
__device__ __forceinline__ void fused_tile(const Fields<R>& in, const Fields<R>& out, typename Prec<R>::V* site,
                                           const StepR<R>& a, int tile) {
    using T = Tile<R, TX, TY>;
    using Vec = typename Prec<R>::V;
    constexpr int LP = T::LP, AP = T::AP;
    constexpr int LW = T::LW, LN = T::LN, EW = T::EW, EN = T::EN, NT = T::NT, NH = T::NH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Vec* sU = (Vec*)smem_raw;          // [2][LP][LN]
    Vec* sPhi = sU + 2 * LP * LN;      // [AP][LN]
    Vec* sA = sPhi + AP * LN;          // [AP][EN]
    Vec* sEs = sA + AP * EN;           // [2][AP][EN]: e(n-1/2), then e(n-1/2) + e(n+1/2)
    Vec* sLf = sEs + 2 * AP * EN;      // [AP][EN]
    float2* sU2 = (float2*)(smem_raw + T::vecs * sizeof(Vec));  // FP32: [2][3][LN] third rows
    SLinks<R> lk;
    if constexpr (sizeof(R) == 4) lk = SLinks<R>{(const float4*)sU, sU2, LN};
    else lk = SLinks<R>{(const double2*)sU, LN};

    const int N = a.N;
    const int64_t Vn = (int64_t)N * N;
    const int x0 = (tile % a.tiles_x) * TX, y0 = (tile / a.tiles_x) * TY;
    const int tid = threadIdx.x;
    const R t = a.t, dt = a.dt, inv_t = a.inv_t;
    // this thread's site in tile coordinates and its shared-memory indices
    const int ix = tid % TX, iy = tid / TX;
    const int ls = (iy + 1) * LW + (ix + 1), es = (iy + 1) * EW + (ix + 1);

    // ---- phase 1: asynchronous copies of the tile's inputs, in two groups:
    // the links (all phase 2 needs), then phi and e(n-1/2)
    for (int i = tid; i < LN; i += NT) {
        const int gx = wrapi(x0 + i % LW - 1, N), gy = wrapi(y0 + i / LW - 1, N);
        const int64_t g = (int64_t)gy * N + gx;
#pragma unroll
        for (int k = 0; k < 2 * LP; k++) cp_async16(sU + (size_t)k * LN + i, in.U + (size_t)k * Vn + g);
    }
    cp_async_commit();
    for (int i = tid; i < LN; i += NT) {
        const int gx = wrapi(x0 + i % LW - 1, N), gy = wrapi(y0 + i / LW - 1, N);
        const int64_t g = (int64_t)gy * N + gx;
#pragma unroll
        for (int k = 0; k < AP; k++) cp_async16(sPhi + (size_t)k * LN + i, in.phi + (size_t)k * Vn + g);
    }
    for (int i = tid; i < EN; i += NT) {
        const int gx = wrapi(x0 + i % EW - 1, N), gy = wrapi(y0 + i / EW - 1, N);
        const int64_t g = (int64_t)gy * N + gx;
#pragma unroll
        for (int k = 0; k < 2 * AP; k++) cp_async16(sEs + (size_t)k * EN + i, in.e + (size_t)k * Vn + g);
    }
    cp_async_commit();
    cp_async_wait_group<1>();
    if constexpr (sizeof(R) == 4) {
        // third rows of the links this thread copied (its own copies are
        // complete after the wait), once per staged link
        for (int i = tid; i < LN; i += NT)
#pragma unroll
            for (int d = 0; d < 2; d++) {
                const M3<float> m = s_link((const float4*)sU, d, i, LN);
#pragma unroll
                for (int k = 0; k < 3; k++)
                    sU2[(size_t)(d * 3 + k) * LN + i] = make_float2(m.re[2][k], m.im[2][k]);
            }
    }
    __syncthreads();

    // ---- phase 2: plaquettes of the cells x in [-1, TX-1], y in [-1, TY-1]
    for (int i = tid; i < EN; i += NT) {
        const int l = (i / EW) * LW + (i % EW);  // cell (i % EW - 1, i / EW - 1)
        const M3<R> C = mul(lk(0, l), lk(1, l + 1));
        s_alg_put(sA, i, EN, iah_of_mul_nd(mul_nd(C, lk(0, l + LW)), lk(1, l)));
    }
    cp_async_wait_group<0>();
    __syncthreads();

    // ---- phase 3: momenta at n+1/2 of the tile site (kept in registers for
    // phase 4) and of the halo.  Item 0 is the thread's own site (both components); item 1, for the first
    // NH threads, a halo site: left column (-1, h) needs e_x only, bottom row
    // (h, -1) e_y and Lf only.  One loop body (not unrolled) computes both, so
    // a momentum is computed by the same code whether the site is a tile's
    // own or another tile's halo.
    A8<R> my_ex, my_ey, my_tx, my_ty, my_b;
    const int gx = x0 + ix, gy = y0 + iy;
    const bool valid = gx < N && gy < N;
    const int64_t g = (int64_t)gy * N + gx;
    const int n_items = tid < NH ? 2 : 1;
#pragma unroll 1
    for (int it = 0; it < n_items; it++) {
        int e = es, l = ls;
        bool wx = true, wy = true;
        if (it == 1) {
            if (tid < TY) {
                e = (tid + 1) * EW;
                l = (tid + 1) * LW;
                wy = false;
            } else {
                e = tid - TY + 1;
                l = tid - TY + 1;
                wx = false;
            }
        }
        const A8<R> A0 = s_alg(sA, e, EN);
        const A8<R> ph = s_alg(sPhi, l, LN);
        if (wx) {
            const A8<R> Dn = conj_dn_t(lk(1, l - LW), s_alg(sA, e - EW, EN));
            const A8<R> tx = conj_up_t(lk(0, l), s_alg(sPhi, l + 1, LN));
            const A8<R> cx = icomm(tx, ph);
            const A8<R> eox = s_alg(sEs, e, EN);
            A8<R> ex_n, sx;
#pragma unroll
            for (int c = 0; c < 8; c++) {
                ex_n.v[c] = eox.v[c] + dt * (t * (A0.v[c] - Dn.v[c]) + inv_t * cx.v[c]);
                sx.v[c] = eox.v[c] + ex_n.v[c];
            }
            // only this thread reads site e of sEs before the barrier
            s_alg_put(sEs, e, EN, sx);
            if (it == 0) {
                my_ex = ex_n;
                my_tx = tx;
                my_b = Dn;
            }
        }
        if (wy) {
            const A8<R> Lf = conj_dn_t(lk(0, l - 1), s_alg(sA, e - 1, EN));
            const A8<R> ty = conj_up_t(lk(1, l), s_alg(sPhi, l + LW, LN));
            const A8<R> cy = icomm(ty, ph);
            const A8<R> eoy = s_alg(sEs + AP * EN, e, EN);
            A8<R> ey_n, sy;
#pragma unroll
            for (int c = 0; c < 8; c++) {
                ey_n.v[c] = eoy.v[c] + dt * (t * (Lf.v[c] - A0.v[c]) + inv_t * cy.v[c]);
                sy.v[c] = eoy.v[c] + ey_n.v[c];
            }
            s_alg_put(sEs + AP * EN, e, EN, sy);
            s_alg_put(sLf, e, EN, Lf);
            if (it == 0) {
                my_ey = ey_n;
                my_ty = ty;
#pragma unroll
                for (int c = 0; c < 8; c++) my_b.v[c] = A0.v[c] + Lf.v[c] + my_b.v[c];
            }
        }
    }
    __syncthreads();

    // ---- phase 4: the tile sites
    // sites of a ragged tile beyond the lattice do nothing (no early return:
    // persistent callers reach further barriers)
    if (valid) {
        const A8<R> p_old = load_alg(in.pi, g, Vn);
        const A8<R> ph = s_alg(sPhi, ls, LN);
        const M3<R> Ux_m = lk(0, ls - 1);
        const M3<R> Uy_m = lk(1, ls - LW);
        const A8<R> bx = conj_dn_t(Ux_m, s_alg(sPhi, ls - 1, LN));
        const A8<R> by = conj_dn_t(Uy_m, s_alg(sPhi, ls - LW, LN));
        A8<R> p_new, ph_new;
#pragma unroll
        for (int c = 0; c < 8; c++) {
            const R lap = my_tx.v[c] + my_ty.v[c] + bx.v[c] + by.v[c] - R(4) * ph.v[c];
            p_new.v[c] = p_old.v[c] + dt * inv_t * lap;
            ph_new.v[c] = ph.v[c] + a.dt_th * p_new.v[c];
        }
        // the site fields of t_n, written by every field step (one code path for
        // every caller, so the fields evolve bitwise alike whether or not the
        // site fields are used)
        // E_i = (1/4t){e_i(s) + U_i(s-i)^+ e_i(s-i) U_i(s-i)}, e summed over n -+ 1/2
        const A8<R> sx = conj_dn_t(Ux_m, s_alg(sEs, es - 1, EN));
        const A8<R> sy = conj_dn_t(Uy_m, s_alg(sEs + AP * EN, es - EW, EN));
        const A8<R> hx = s_alg(sEs, es, EN), hy = s_alg(sEs + AP * EN, es, EN);
        const A8<R> cr = conj_dn_t(Uy_m, s_alg(sLf, es - EW, EN));
        A8<R> Ex, Ey, Ee, Bx, By, Be;
        const R q = R(0.25) * inv_t, hf = R(0.5) * inv_t;
#pragma unroll
        for (int c = 0; c < 8; c++) {
            Ex.v[c] = q * (hx.v[c] + sx.v[c]);
            Ey.v[c] = q * (hy.v[c] + sy.v[c]);
            Ee.v[c] = R(0.5) * (p_old.v[c] + p_new.v[c]);
            Bx.v[c] = -hf * (my_ty.v[c] - by.v[c]);
            By.v[c] = hf * (my_tx.v[c] - bx.v[c]);
            Be.v[c] = R(0.25) * (my_b.v[c] + cr.v[c]);
        }
        store_alg(site, g, Vn, Ex);
        store_alg(site + (size_t)1 * AP * Vn, g, Vn, Ey);
        store_alg(site + (size_t)2 * AP * Vn, g, Vn, Ee);
        store_alg(site + (size_t)3 * AP * Vn, g, Vn, Bx);
        store_alg(site + (size_t)4 * AP * Vn, g, Vn, By);
        store_alg(site + (size_t)5 * AP * Vn, g, Vn, Be);
        store_alg_cs(out.e, g, Vn, my_ex);
        store_alg_cs(out.e + (size_t)AP * Vn, g, Vn, my_ey);
        store_alg_cs(out.pi, g, Vn, p_new);
        store_alg_cs(out.phi, g, Vn, ph_new);
        M3<R> nx = mul(exp_i_alg<R, ExpN<R>::n>(my_ex, a.dt_over_th), lk(0, ls));
        if (a.reunit) reunit(nx);
        store_link_cs(out.U, 0, g, Vn, nx);
        M3<R> ny = mul(exp_i_alg<R, ExpN<R>::n>(my_ey, a.dt_over_th), lk(1, ls));
        if (a.reunit) reunit(ny);
        store_link_cs(out.U, 1, g, Vn, ny);
    }
}

// step scalars of t_n = n dt, computed the same way on the host and the device
__host__ __device__ inline StepArgs step_args(int N, int tiles_x, int64_t n, double dt, int reunit) {
    StepArgs a;
    a.N = N;
    a.tiles_x = tiles_x;
    const double t = n * dt, th = t + 0.5 * dt;
    a.t = t;
    a.dt = dt;
    a.inv_t = t > 0 ? 1.0 / t : 0.0;
    a.dt_over_th = dt / th;
    a.dt_th = dt * th;
    a.reunit = reunit;
    return a;
}

}  // namespace gl
