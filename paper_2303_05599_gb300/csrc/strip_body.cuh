// FP32 Glasma leapfrog step and site E/B interpolation (Sec. 2.1 and 3.2 of
// arXiv:2303.05599) on column strips, one warp per strip segment.
//
// A warp owns a strip of 32 columns (lane l has x = x0 + l, x0 a multiple of
// 32) and walks up a range of its rows.  For row y it computes, from U(n),
// phi(n), e(n-1/2), pi(n-1/2):
//   the momenta e(n+1/2), pi(n+1/2), the links U(n+1), the scalar phi(n+1),
//   and the site fields E, B at t_n,
// with the plaquette A(s) = i[Ux(s) Uy(s+x) Ux(s+y)^+ Uy(s)^+]_ah formed once
// per site.  The neighbours a site needs come from three places:
//   x + 1 (Uy, phi):       the next lane, by shuffle (the last valid lane of
//                          the strip loads its right neighbour itself);
//   x - 1 (transports by the left link of A, phi and the summed e_x):
//                          the previous lane computes them as transports by
//                          its own Ux and hands them over by shuffle; lane 0
//                          takes them from the halo pass (below);
//   y - 1 (transports by the lower Uy of A, phi, the summed e_y and Lf):
//                          carried in registers from the previous row;
//   y + 1 (Ux, phi):       the next row, already staged in shared memory.
// So every site does its nine adjoint transports, one plaquette, two
// exponential link updates, and no work is repeated for halo sites, except
// the left column once per 23 rows (the halo pass) and one row per segment
// start (the carries of the row below, a "dry" row whose stores are off).
//
// Inputs of a row (the two links as two float4 rows each, phi) are copied by
// each lane into its own slots of a two-row ring in shared memory with
// cp.async: row r + 2 goes into the slot of row r as soon as row r has read
// it into registers, near the start of row r, so each copy has about a row to
// land.  e and pi go to a one-row slot that is refilled for the next row as
// soon as this row has read them.  Each lane copies and reads only its own
// slots, so the only waits are per-thread cp.async waits, one __syncwarp per
// halo block and the block barriers that keep the warps in step.
//
// Results do not depend on how rows are split among warps: the carries of a
// segment's first row come from the same loop body (dry), and the values of
// the column left of a strip always come from the halo pass, whose code does
// not depend on where its block starts.
#pragma once
#include "fused_body.cuh"
#include "internal.h"
#include "layout.cuh"

namespace gl {

constexpr int STRIP_W = 32;  // columns per strip = lanes per warp
constexpr int HALO_B = 23;   // rows per halo block (at most 31: one lane computes the row below)
constexpr int RING_V = 8;    // float4 per lane per row: Ux (3), Uy (3), phi (2)
constexpr int RING_X = 5;    // the last lane's right neighbour: Uy (3), phi (2)
constexpr int MOM_V = 6;     // float4 per lane per row: e_x (2), e_y (2), pi (2)
constexpr int STRIP_SYNC = 2;  // rows between the block barriers that keep a block's warps in step

// One warp's staging area, 13,632 bytes: 16 warps fit an SM.  (A second
// momentum slot, so that the next row's momenta could be issued a whole row
// ahead, takes the shared memory of 12 warps to 200 KB; the L1 left beside it
// is too small and both the field step and the push beside it run slower.)
struct StripWarpSmem {
    float4 ring[2][RING_V][STRIP_W];
    float4 mom[MOM_V][STRIP_W];
    float4 extra[2][RING_X];
    float4 halo[HALO_B][6];  // Lf source, bx source, sx source at (x0 - 1, y): 2 float4 each
};

// step scalars of t_n in single precision, the step index and the
// re-unitarisation period: the links of row y are re-unitarised in the step
// n with (n + 1 + y) % every == 0, so each link once every `every` steps and
// the FP64 work spread evenly over the steps (every = 0: never)
struct StripStep {
    float t, dt, inv_t, dt_over_th, dt_th;
    int every;
    int64_t n;
};

__host__ __device__ inline StripStep strip_step(int64_t n, double dt, int every) {
    const StepArgs a = step_args(0, 0, n, dt, 0);
    StripStep s;
    s.t = (float)a.t;
    s.dt = (float)a.dt;
    s.inv_t = (float)a.inv_t;
    s.dt_over_th = (float)a.dt_over_th;
    s.dt_th = (float)a.dt_th;
    s.every = every;
    s.n = n;
    return s;
}

// Gram-Schmidt of rows 0 and 1 of a two-row link with the sums in FP64: the
// squared norms and the inner product are accumulated in FP64 from the FP32
// entries (each product exact) and the reciprocal square roots taken by the
// FP64 rsqrt; the rows are scaled and corrected in FP32, the precision they
// are stored in.  Right after it a link is unitary to FP32 rounding.
__device__ __forceinline__ void reunit_rows(M3<float>& u) {
    double n0 = 0;
#pragma unroll
    for (int j = 0; j < 3; j++)
        n0 = fma((double)u.re[0][j], (double)u.re[0][j], fma((double)u.im[0][j], (double)u.im[0][j], n0));
    const float s0 = (float)rsqrt(n0);
#pragma unroll
    for (int j = 0; j < 3; j++) { u.re[0][j] *= s0; u.im[0][j] *= s0; }
    double cr = 0, ci = 0;  // <r0, r1>
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const double ar = u.re[0][j], ai = u.im[0][j], br = u.re[1][j], bi = u.im[1][j];
        cr = fma(ar, br, fma(ai, bi, cr));
        ci = fma(ar, bi, fma(-ai, br, ci));
    }
    const float fr = (float)cr, fi = (float)ci;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const float ar = u.re[0][j], ai = u.im[0][j];
        u.re[1][j] -= fr * ar - fi * ai;
        u.im[1][j] -= fr * ai + fi * ar;
    }
    double n1 = 0;
#pragma unroll
    for (int j = 0; j < 3; j++)
        n1 = fma((double)u.re[1][j], (double)u.re[1][j], fma((double)u.im[1][j], (double)u.im[1][j], n1));
    const float s1 = (float)rsqrt(n1);
#pragma unroll
    for (int j = 0; j < 3; j++) { u.re[1][j] *= s1; u.im[1][j] *= s1; }
}

__device__ __forceinline__ M3<float> link_of(const float4 a, const float4 c, const float4 e) {
    M3<float> m;
    m.re[0][0] = a.x; m.im[0][0] = a.y; m.re[0][1] = a.z; m.im[0][1] = a.w;
    m.re[0][2] = c.x; m.im[0][2] = c.y; m.re[1][0] = c.z; m.im[1][0] = c.w;
    m.re[1][1] = e.x; m.im[1][1] = e.y; m.re[1][2] = e.z; m.im[1][2] = e.w;
    rebuild_row2(m);
    return m;
}
__device__ __forceinline__ A8<float> alg_of(const float4 a, const float4 b) {
    A8<float> x;
    x.v[0] = a.x; x.v[1] = a.y; x.v[2] = a.z; x.v[3] = a.w;
    x.v[4] = b.x; x.v[5] = b.y; x.v[6] = b.z; x.v[7] = b.w;
    return x;
}

// Products of SU(3) matrices with rows 0 and 1 multiplied out and row 2 the
// conjugate cross product of the two, as for a stored link: c = a b and
// c = a b^+.
__device__ __forceinline__ M3<float> mul_su3(const M3<float>& a, const M3<float>& b) {
    M3<float> c;
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            float sr = 0.f, si = 0.f;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                sr = fmaf(a.re[i][k], b.re[k][j], sr);
                sr = fmaf(-a.im[i][k], b.im[k][j], sr);
                si = fmaf(a.re[i][k], b.im[k][j], si);
                si = fmaf(a.im[i][k], b.re[k][j], si);
            }
            c.re[i][j] = sr;
            c.im[i][j] = si;
        }
    rebuild_row2(c);
    return c;
}
__device__ __forceinline__ M3<float> mul_nd_su3(const M3<float>& a, const M3<float>& b) {
    M3<float> c;
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            float sr = 0.f, si = 0.f;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                sr = fmaf(a.re[i][k], b.re[j][k], sr);
                sr = fmaf(a.im[i][k], b.im[j][k], sr);
                si = fmaf(a.im[i][k], b.re[j][k], si);
                si = fmaf(-a.re[i][k], b.im[j][k], si);
            }
            c.re[i][j] = sr;
            c.im[i][j] = si;
        }
    rebuild_row2(c);
    return c;
}

// Component-wise updates of algebra elements on packed pairs of FP32
// components (2i, 2i + 1), one f32x2 instruction per pair.
__device__ __forceinline__ float2 pr(const A8<float>& x, int i) { return make_float2(x.v[2 * i], x.v[2 * i + 1]); }
__device__ __forceinline__ void put(A8<float>& x, int i, float2 p) {
    x.v[2 * i] = p.x;
    x.v[2 * i + 1] = p.y;
}
__device__ __forceinline__ float2 bc(float s) { return make_float2(s, s); }

// The momentum update of one link direction, e(n+1/2) = e(n-1/2) + dt (t (P - Q)
// + c / t), with P - Q the plaquette difference and c the scalar current; es
// = e(n-1/2) + e(n+1/2), the sum the site field E averages.
__device__ __forceinline__ void e_update(const A8<float>& e, const A8<float>& P, const A8<float>& Q,
                                         const A8<float>& c, float t, float dt, float inv_t, A8<float>& en,
                                         A8<float>& es) {
#pragma unroll
    for (int i = 0; i < 4; i++) {
        float2 u = __fmul2_rn(bc(-t), pr(Q, i));
        u = __ffma2_rn(bc(t), pr(P, i), u);
        u = __ffma2_rn(bc(inv_t), pr(c, i), u);
        const float2 n = __ffma2_rn(bc(dt), u, pr(e, i));
        put(en, i, n);
        put(es, i, __fadd2_rn(pr(e, i), n));
    }
}

__device__ __forceinline__ A8<float> shfl_up_a8(const A8<float>& x) {
    A8<float> o;
#pragma unroll
    for (int c = 0; c < 8; c++) o.v[c] = __shfl_up_sync(0xffffffffu, x.v[c], 1);
    return o;
}
__device__ __forceinline__ A8<float> shfl_down_a8(const A8<float>& x) {
    A8<float> o;
#pragma unroll
    for (int c = 0; c < 8; c++) o.v[c] = __shfl_down_sync(0xffffffffu, x.v[c], 1);
    return o;
}
__device__ __forceinline__ M3<float> shfl_down_m3(const M3<float>& m) {
    M3<float> o;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            o.re[i][j] = __shfl_down_sync(0xffffffffu, m.re[i][j], 1);
            o.im[i][j] = __shfl_down_sync(0xffffffffu, m.im[i][j], 1);
        }
    return o;
}


// the lane's column geometry within its strip
struct StripLane {
    int lane;
    int x;      // own column (wrapped onto the lattice for lanes beyond it)
    int xr;     // right neighbour of the last valid lane
    int xl;     // column left of the strip
    bool valid; // x0 + lane < N
    bool last;  // the last valid lane of the strip
};

__device__ __forceinline__ StripLane strip_lane(int N, int x0) {
    StripLane L;
    L.lane = threadIdx.x & 31;
    const int w = N - x0 < STRIP_W ? N - x0 : STRIP_W;  // valid lanes
    L.valid = L.lane < w;
    L.last = L.lane == w - 1;
    L.x = L.valid ? x0 + L.lane : x0;  // lanes beyond the lattice read a valid column, store nothing
    L.xr = wrapi(x0 + w, N);
    L.xl = wrapi(x0 - 1, N);
    return L;
}

// row y's links and scalar of this lane (and the last lane's right
// neighbour) into ring slot k: one cp.async group
__device__ __forceinline__ void strip_issue_row(StripWarpSmem& S, int k, const Fields<float>& in, int64_t Vn, int N,
                                                const StripLane& L, int y) {
    const int64_t g = (int64_t)wrapi(y, N) * N;
#pragma unroll
    for (int p = 0; p < 6; p++) cp_async16(&S.ring[k][p][L.lane], in.U + (size_t)p * Vn + g + L.x);
#pragma unroll
    for (int p = 0; p < 2; p++) cp_async16(&S.ring[k][6 + p][L.lane], in.phi + (size_t)p * Vn + g + L.x);
    if (L.last) {
#pragma unroll
        for (int p = 0; p < 3; p++) cp_async16(&S.extra[k][p], in.U + (size_t)(3 + p) * Vn + g + L.xr);
#pragma unroll
        for (int p = 0; p < 2; p++) cp_async16(&S.extra[k][3 + p], in.phi + (size_t)p * Vn + g + L.xr);
    }
    cp_async_commit();
}

// row y's momenta e_x, e_y, pi of this lane into the momentum slot: one
// cp.async group
__device__ __forceinline__ void strip_issue_mom(StripWarpSmem& S, const Fields<float>& in, int64_t Vn, int N,
                                                const StripLane& L, int y) {
    const int64_t g = (int64_t)wrapi(y, N) * N + L.x;
#pragma unroll
    for (int p = 0; p < 4; p++) cp_async16(&S.mom[p][L.lane], in.e + (size_t)p * Vn + g);
#pragma unroll
    for (int p = 0; p < 2; p++) cp_async16(&S.mom[4 + p][L.lane], in.pi + (size_t)p * Vn + g);
    cp_async_commit();
}

// Halo pass: the transports by Ux(x0 - 1, y) of A, phi and the summed e_x at
// the column left of the strip, for rows y0 .. y0 + nb - 1 (nb <= HALO_B), into
// S.halo[y - y0].  Lane j works on row y0 - 1 + j; it needs the transported
// plaquette of the row below, which lane j - 1 supplies.
__device__ __forceinline__ void strip_halo(StripWarpSmem& S, const Fields<float>& in, int64_t Vn, int N, int x0,
                                           const StripLane& L, int y0, int nb, const StripStep& a) {
    const int yh = wrapi(y0 - 1 + L.lane, N);
    const int yu = wrapi(y0 + L.lane, N);
    const int64_t gl = (int64_t)yh * N + L.xl, g0 = (int64_t)yh * N + x0;
    // lanes 0 .. nb work on the rows handed on; lane nb + 1 only supplies its
    // Ux (the link of the row above lane nb's); the lanes beyond load nothing
    // and work on zeros
    M3<float> Ux = m_zero<float>(), Uy = m_zero<float>(), UyR = m_zero<float>();
    A8<float> ph = a_zero<float>(), phR = a_zero<float>(), ex = a_zero<float>();
    if (L.lane <= nb + 1) Ux = load_link(in.U, 0, gl, Vn);
    if (L.lane <= nb) {
        Uy = load_link(in.U, 1, gl, Vn);
        UyR = load_link(in.U, 1, g0, Vn);
        ph = load_alg(in.phi, gl, Vn);
        phR = load_alg(in.phi, g0, Vn);
        ex = load_alg(in.e, gl, Vn);
    }
    // Ux of the row above: the next lane's link, the last lane loads it
    M3<float> UxU = shfl_down_m3(Ux);
    if (L.lane == 31 && L.lane <= nb) UxU = load_link(in.U, 0, (int64_t)yu * N + L.xl, Vn);
    const A8<float> A = iah_of_mul_nd(mul_nd_su3(mul_su3(Ux, UyR), UxU), Uy);
    const A8<float> Dn = shfl_up_a8(conj_dn_t(Uy, A));
    const A8<float> tx = conj_up_t(Ux, phR);
    const A8<float> cx = icomm(tx, ph);
    A8<float> en, es;
    e_update(ex, A, Dn, cx, a.t, a.dt, a.inv_t, en, es);
    const A8<float> lf = conj_dn_t(Ux, A);
    const A8<float> bx = conj_dn_t(Ux, ph);
    const A8<float> sx = conj_dn_t(Ux, es);
    if (L.lane >= 1 && L.lane <= nb) {
        float4* h = S.halo[L.lane - 1];
        h[0] = make_float4(lf.v[0], lf.v[1], lf.v[2], lf.v[3]);
        h[1] = make_float4(lf.v[4], lf.v[5], lf.v[6], lf.v[7]);
        h[2] = make_float4(bx.v[0], bx.v[1], bx.v[2], bx.v[3]);
        h[3] = make_float4(bx.v[4], bx.v[5], bx.v[6], bx.v[7]);
        h[4] = make_float4(sx.v[0], sx.v[1], sx.v[2], sx.v[3]);
        h[5] = make_float4(sx.v[4], sx.v[5], sx.v[6], sx.v[7]);
    }
    __syncwarp();
}

// the transports carried from row y - 1 to row y (all by Uy(x, y - 1))
struct StripCarry {
    A8<float> dn;  // plaquette below: Uy^+ A Uy
    A8<float> by;  // scalar below: Uy^+ phi Uy
    A8<float> sy;  // summed e_y below: Uy^+ (e_y(n-1/2) + e_y(n+1/2)) Uy
    A8<float> cr;  // Lf below: Uy^+ Lf Uy (the fourth clover leaf)
};

// Rows y_begin .. y_end - 1 of the strip at x0 (y_end - y_begin <= N) for
// the fields of step n in `in`: step n + 1 into `out`, the site fields of t_n
// into `site`.  Rows at or beyond y_stop store nothing (dummy rows, which keep
// the warps of a block in step; y_stop <= y_end).  With `sync`, every second
// row starts at a block barrier (often enough to keep the warps on the same
// instructions), so all warps of the block must call this with the same
// y_end - y_begin.
__device__ __forceinline__ void strip_segment(StripWarpSmem& S, const Fields<float>& in, const Fields<float>& out,
                                              float4* site, int N, int x0, int y_begin, int y_end, int y_stop,
                                              const StripStep& a, bool sync) {
    const int64_t Vn = (int64_t)N * N;
    const StripLane L = strip_lane(N, x0);
    const float t = a.t, dt = a.dt, inv_t = a.inv_t, c_link = a.dt_over_th, dt_th = a.dt_th;
    const float q = 0.25f * inv_t, hf = 0.5f * inv_t;

    StripCarry C;
    C.dn = C.by = C.sy = C.cr = a_zero<float>();
    // rows r = y_begin - 1 (dry: only its carries are formed) .. y_end - 1
    const int r_first = y_begin - 1;
    strip_issue_row(S, 0, in, Vn, N, L, r_first);
    strip_issue_row(S, 1, in, Vn, N, L, r_first + 1);
    strip_issue_mom(S, in, Vn, N, L, r_first);
    int halo_end = r_first;  // rows below halo_end have halo values in S.halo
    int halo_base = r_first;
    // the bounds the row body tests, as values the compiler cannot relate to
    // the loop's first and last rows: one copy of the row body serves the dry
    // row and the rows near the end (no peeled iterations to fetch)
    int yb = y_begin, ye = y_end;
    asm volatile("" : "+r"(yb), "+r"(ye), "+r"(halo_end));
    // (n + 1 + r) mod every, the re-unitarisation phase of row r (the rows
    // that store have y = r): one 64-bit remainder per segment, then a step
    // of one per row
    int ru = a.every > 0 ? (int)((a.n + 1 + r_first) % a.every) : 1;
#pragma unroll 1
    for (int r = r_first; r < y_end; r++) {
        if (sync && (r - r_first) % STRIP_SYNC == 0) __syncthreads();
        if (r == halo_end) {
            const int nb = y_end - r < HALO_B ? y_end - r : HALO_B;
            strip_halo(S, in, Vn, N, x0, L, r, nb, a);
            halo_base = r;
            halo_end = r + nb;
        }
        const bool dry = r < yb;
        const bool st = !dry && L.valid && r < y_stop;
        const int k = (r - r_first) & 1, k1 = k ^ 1;
        const int y = wrapi(r, N);
        const int64_t g = (int64_t)y * N + L.x;
        // rows r and r + 1 are in the ring (r + 1 was issued a row ago).  Each
        // row commits two cp.async groups, ring row r + 2 after the plaquette
        // and the momenta of row r + 1 at its end (empty groups where there is
        // nothing to copy), so all but the newest group (row r's momenta)
        // are complete here, and all but the newest (ring row r + 2) before
        // the momenta are read: their copy has the plaquette's time as well
        cp_async_wait_group<1>();
        const M3<float> Ux = link_of(S.ring[k][0][L.lane], S.ring[k][1][L.lane], S.ring[k][2][L.lane]);
        const M3<float> Uy = link_of(S.ring[k][3][L.lane], S.ring[k][4][L.lane], S.ring[k][5][L.lane]);
        const A8<float> ph = alg_of(S.ring[k][6][L.lane], S.ring[k][7][L.lane]);
        M3<float> UyR = shfl_down_m3(Uy);
        if (L.last) UyR = link_of(S.extra[k][0], S.extra[k][1], S.extra[k][2]);
        A8<float> phR = shfl_down_a8(ph);
        if (L.last) phR = alg_of(S.extra[k][3], S.extra[k][4]);
        const M3<float> UxN = link_of(S.ring[k1][0][L.lane], S.ring[k1][1][L.lane], S.ring[k1][2][L.lane]);
        const A8<float> phN = alg_of(S.ring[k1][6][L.lane], S.ring[k1][7][L.lane]);

        // Each value is used as soon as it is known and the outputs stored as
        // they are formed, so that few values live at once.  The dry row forms
        // only what the carries need (A, Lf, the e_y update).
        const A8<float> A = iah_of_mul_nd(mul_nd_su3(mul_su3(Ux, UyR), UxN), Uy);   // plaquette at (x, y)
        // ring slot k (Ux, Uy, phi and the right neighbour's Uy, phi of row r)
        // has been read into registers above: row r + 2 goes there
        if (r + 2 <= ye) strip_issue_row(S, k, in, Vn, N, L, r + 2);
        else cp_async_commit();
        const float4* h = S.halo[r - halo_base];
        // clover: A, its transports from x - 1 (Lf, by the left lane's Ux) and
        // from y - 1, and the fourth leaf carried from the row below
        A8<float> Lf = shfl_up_a8(conj_dn_t(Ux, A));
        if (L.lane == 0) Lf = alg_of(h[0], h[1]);
        A8<float> lap = a_zero<float>();  // the covariant Laplacian of phi, x part first
        if (!dry) {
            A8<float> Be;
#pragma unroll
            for (int c = 0; c < 8; c++) Be.v[c] = 0.25f * (((A.v[c] + Lf.v[c]) + C.dn.v[c]) + C.cr.v[c]);
            if (st) store_alg(site + (size_t)10 * Vn, g, Vn, Be);
            // x direction: D_x phi, the e_x update, E_x, the x link
            A8<float> bx = shfl_up_a8(conj_dn_t(Ux, ph));
            if (L.lane == 0) bx = alg_of(h[2], h[3]);
            const A8<float> tx = conj_up_t(Ux, phR);
            const A8<float> cx = icomm(tx, ph);
            A8<float> By;
#pragma unroll
            for (int c = 0; c < 8; c++) {
                By.v[c] = hf * (tx.v[c] - bx.v[c]);
                lap.v[c] = tx.v[c] + bx.v[c];
            }
            if (st) store_alg(site + (size_t)8 * Vn, g, Vn, By);
            cp_async_wait_group<1>();
            const A8<float> ex = alg_of(S.mom[0][L.lane], S.mom[1][L.lane]);
            A8<float> exn, exs;
            e_update(ex, A, C.dn, cx, t, dt, inv_t, exn, exs);
            A8<float> sx = shfl_up_a8(conj_dn_t(Ux, exs));
            if (L.lane == 0) sx = alg_of(h[4], h[5]);
            A8<float> Ex;
#pragma unroll
            for (int c = 0; c < 8; c++) Ex.v[c] = q * (exs.v[c] + sx.v[c]);
            if (st) {
                store_alg(site, g, Vn, Ex);
                store_alg_cs(out.e, g, Vn, exn);
                M3<float> nx = mul(exp_i_alg<float, ExpN<float>::n>(exn, c_link), Ux);
                if (ru == 0) reunit_rows(nx);
                store_link_cs(out.U, 0, g, Vn, nx);
            }
        }
        const A8<float> ty = conj_up_t(Uy, phN);
        const A8<float> cy = icomm(ty, ph);
        // y direction: D_y phi, the e_y update, E_y, the scalar and pi
        cp_async_wait_group<1>();
        const A8<float> ey = alg_of(S.mom[2][L.lane], S.mom[3][L.lane]);
        A8<float> eyn, eys;
        e_update(ey, Lf, A, cy, t, dt, inv_t, eyn, eys);
        if (!dry) {
            const A8<float> po = alg_of(S.mom[4][L.lane], S.mom[5][L.lane]);
            A8<float> Ey, Ee, Bx, pn, phn;
#pragma unroll
            for (int c = 0; c < 8; c++) {
                Ey.v[c] = q * (eys.v[c] + C.sy.v[c]);
                Bx.v[c] = -hf * (ty.v[c] - C.by.v[c]);
                pn.v[c] = po.v[c] + dt * inv_t * ((lap.v[c] + (ty.v[c] + C.by.v[c])) - 4.0f * ph.v[c]);
                phn.v[c] = ph.v[c] + dt_th * pn.v[c];
                Ee.v[c] = 0.5f * (po.v[c] + pn.v[c]);
            }
            if (st) {
                store_alg(site + (size_t)2 * Vn, g, Vn, Ey);
                store_alg(site + (size_t)4 * Vn, g, Vn, Ee);
                store_alg(site + (size_t)6 * Vn, g, Vn, Bx);
                store_alg_cs(out.e + (size_t)2 * Vn, g, Vn, eyn);
                store_alg_cs(out.pi, g, Vn, pn);
                store_alg_cs(out.phi, g, Vn, phn);
            }
        }
        // the momentum slot's values are all read now: the next row's go there
        if (r + 1 < ye) strip_issue_mom(S, in, Vn, N, L, r + 1);
        else cp_async_commit();
        if (st) {
            M3<float> ny = mul(exp_i_alg<float, ExpN<float>::n>(eyn, c_link), Uy);
            if (ru == 0) reunit_rows(ny);
            store_link_cs(out.U, 1, g, Vn, ny);
        }
        if (a.every > 0 && ++ru == a.every) ru = 0;
        // the carries for row r + 1, by this row's Uy
        C.dn = conj_dn_t(Uy, A);
        C.by = conj_dn_t(Uy, ph);
        C.sy = conj_dn_t(Uy, eys);
        C.cr = conj_dn_t(Uy, Lf);
    }
    cp_async_wait_group<0>();
}

// Work split: the strips of an event are cut into segments of `seg` rows (the
// last one shorter when seg does not divide N); segment j of the event is
// strip j % nstrips, rows from (j / nstrips) seg: neighbouring strips over the
// same rows are consecutive, so the W warps of a block, which take W
// consecutive segments of the flat list and run them in step (a barrier every
// second row), read and write the same rows of each plane at the same time.
// Warps beyond the list repeat its last segment without storing.  The segment
// length is chosen per launch (below) so that the segments fill the resident
// warps evenly.
__host__ __device__ inline int64_t strip_segments(int N, int seg) {
    return (int64_t)((N + STRIP_W - 1) / STRIP_W) * ((N + seg - 1) / seg);
}

struct StripSeg {
    int x0, y0, len;
};

__device__ __forceinline__ StripSeg strip_seg_of(int N, int64_t j, int seg) {
    const int nstrips = (N + STRIP_W - 1) / STRIP_W;
    const int blk = (int)(j / nstrips), strip = (int)(j - (int64_t)blk * nstrips);
    StripSeg g;
    g.x0 = strip * STRIP_W;
    g.y0 = blk * seg;
    g.len = N - g.y0 < seg ? N - g.y0 : seg;
    return g;
}

// one segment of an event in step with the block (real: store its rows)
__device__ __forceinline__ void strip_run_segment(StripWarpSmem& S, const Fields<float>& in, const Fields<float>& out,
                                                  float4* site, int N, int64_t j, bool real, const StripStep& a,
                                                  int seg) {
    const StripSeg g = strip_seg_of(N, j, seg);
    strip_segment(S, in, out, site, N, g.x0, g.y0, g.y0 + seg, real ? g.y0 + g.len : g.y0, a, true);
}

// Segment length for lattices Ns[0..n) on `blocks` resident blocks of `wpb`
// warps: the length S >= 4 that minimises the modelled time, rounds x (S rows
// + the dry row + the halo passes), where rounds = the items of wpb segments
// per resident block, rounded up.  The dry row costs about 0.6 of a row and a
// halo pass (up to HALO_B rows of the left column) about 0.45.  Long segments
// cost fewer dry rows and halo passes; short ones fill the last round.
inline int strip_seg_rows(const int* Ns, int n, int wpb, int blocks) {
    int nmax = 1;
    for (int e = 0; e < n; e++) nmax = Ns[e] > nmax ? Ns[e] : nmax;
    int best = nmax < 4 ? nmax : 4;
    double best_cost = 1e300;
    for (int S = 4; S <= (nmax > 4 ? nmax : 4); S++) {
        int64_t nseg = 0;
        for (int e = 0; e < n; e++) nseg += strip_segments(Ns[e], S);
        const int64_t items = (nseg + wpb - 1) / wpb;
        const int64_t rounds = (items + blocks - 1) / (blocks > 0 ? blocks : 1);
        const double cost = (double)rounds * (S + 0.6 + 0.45 * ((S + 1 + HALO_B - 1) / HALO_B));
        if (cost < best_cost - 1e-9) { best_cost = cost; best = S; }
    }
    return best;
}

}  // namespace gl
