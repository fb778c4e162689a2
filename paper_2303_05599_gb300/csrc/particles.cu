// Test particles (Sec. 3 of arXiv:2303.05599): site interpolation of E and B,
// Euler integration of Wong's equations in Milne coordinates, CPIC colour
// rotation, and the sampling of positions, momenta and Haar-random charges.
//
// Particle layout (structure of arrays, np entries per plane):
//   FP64: double2 xy, pxy, (eta, P_eta), q[4]    (7 planes, 112 B per particle)
//   FP32: float4 (x, y, p^x, p^y), float2 (eta, P_eta), float4 q[2]  (56 B)
//   both: int32 species, double p_T^2 at formation, int32 original index
// P_eta = tau^2 p^eta is evolved instead of p^eta so that the step is regular
// at tau = 0; for an infinitely massive species its slot accumulates p_L.
#include "internal.h"
#include "layout.cuh"
#include "parts.cuh"
#include "philox.cuh"
#include "push_body.cuh"
#include "obs_body.cuh"

namespace gl {

size_t particle_bytes(int prec, int64_t np) {
    if (prec == 0) return align256(16 * np) * 3 + align256(64 * np) + align256(4 * np) * 2 + align256(8 * np) * 2;
    return align256(16 * np) + align256(8 * np) + align256(32 * np) + align256(4 * np) * 3 + align256(8 * np);
}

size_t site_bytes(int prec, int64_t Vn) { return (size_t)6 * 8 * Vn * (prec == 0 ? 8 : 4); }

size_t field_bytes(int prec, int64_t Vn) {
    return prec == 0 ? fields_vectors<double>(Vn) * 16 : fields_vectors<float>(Vn) * 16;
}

// ------------------------------------------------------------ site fields
// Sec. 3.2 interpolation at t_n:
//   E_i   = (1/4t) { e_i(x) + U_i(x-i)^+ e_i(x-i) U_i(x-i) }, e summed over n +- 1/2
//   E_eta = (pi(n+1/2) + pi(n-1/2)) / 2
//   B_x   = -(1/t) D_y phi,  B_y = +(1/t) D_x phi   (central covariant differences;
//           the components follow B_i = eps_ij F_eta_j / tau and Wong's equations)
//   B_eta = (i/4) [U_xy + U_y,-x + U_-x,-y + U_-y,x]_ah   (clover of the four plaquettes)
template <typename R>
__global__ void __launch_bounds__(128) site_fields_kernel(Fields<R> bn, Fields<R> bn1,
                                                          typename Prec<R>::V* site, int N, R inv_t) {
    constexpr int AP = Prec<R>::AP;
    const int64_t Vn = (int64_t)N * N;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < Vn; s += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(s % N), y = (int)(s / N);
        const int xp = x + 1 == N ? 0 : x + 1, xm = x == 0 ? N - 1 : x - 1;
        const int yp = y + 1 == N ? 0 : y + 1, ym = y == 0 ? N - 1 : y - 1;
        const int64_t s_xp = (int64_t)y * N + xp, s_xm = (int64_t)y * N + xm;
        const int64_t s_yp = (int64_t)yp * N + x, s_ym = (int64_t)ym * N + x;
        const M3<R> Ux = load_link(bn.U, 0, s, Vn), Uy = load_link(bn.U, 1, s, Vn);
        const M3<R> Ux_xm = load_link(bn.U, 0, s_xm, Vn), Uy_ym = load_link(bn.U, 1, s_ym, Vn);
        // electric
        for (int d = 0; d < 2; d++) {
            const int64_t sb = d == 0 ? s_xm : s_ym;
            const typename Prec<R>::V* eo = bn.e + (size_t)d * AP * Vn;
            const typename Prec<R>::V* en = bn1.e + (size_t)d * AP * Vn;
            A8<R> h = load_alg(eo, s, Vn), hn = load_alg(en, s, Vn);
            A8<R> b = load_alg(eo, sb, Vn), bnn = load_alg(en, sb, Vn);
#pragma unroll
            for (int a = 0; a < 8; a++) { h.v[a] += hn.v[a]; b.v[a] += bnn.v[a]; }
            const A8<R> bt = adj_dag(d == 0 ? Ux_xm : Uy_ym, b);
            A8<R> E;
#pragma unroll
            for (int a = 0; a < 8; a++) E.v[a] = R(0.25) * inv_t * (h.v[a] + bt.v[a]);
            store_alg(site + (size_t)d * AP * Vn, s, Vn, E);
        }
        {
            A8<R> p = load_alg(bn.pi, s, Vn), pn = load_alg(bn1.pi, s, Vn);
#pragma unroll
            for (int a = 0; a < 8; a++) p.v[a] = R(0.5) * (p.v[a] + pn.v[a]);
            store_alg(site + (size_t)2 * AP * Vn, s, Vn, p);
        }
        // magnetic, longitudinal components from the scalar
        {
            const A8<R> fx = adj(Ux, load_alg(bn.phi, s_xp, Vn));
            const A8<R> bx = adj_dag(Ux_xm, load_alg(bn.phi, s_xm, Vn));
            const A8<R> fy = adj(Uy, load_alg(bn.phi, s_yp, Vn));
            const A8<R> by = adj_dag(Uy_ym, load_alg(bn.phi, s_ym, Vn));
            A8<R> Bx, By;
#pragma unroll
            for (int a = 0; a < 8; a++) {
                Bx.v[a] = -R(0.5) * inv_t * (fy.v[a] - by.v[a]);
                By.v[a] = R(0.5) * inv_t * (fx.v[a] - bx.v[a]);
            }
            store_alg(site + (size_t)3 * AP * Vn, s, Vn, Bx);
            store_alg(site + (size_t)4 * AP * Vn, s, Vn, By);
        }
        // B_eta from the clover
        {
            const int64_t s_xm_yp = (int64_t)yp * N + xm, s_xm_ym = (int64_t)ym * N + xm;
            const int64_t s_xp_ym = (int64_t)ym * N + xp;
            // U_xy(x) = Ux(x) Uy(x+x) Ux(x+y)^+ Uy(x)^+
            M3<R> c = mul_nd(mul_nd(mul(Ux, load_link(bn.U, 1, s_xp, Vn)), load_link(bn.U, 0, s_yp, Vn)), Uy);
            // U_y,-x(x) = Uy(x) Ux(x-x+y)^+ Uy(x-x)^+ Ux(x-x)
            const M3<R> Uy_xm = load_link(bn.U, 1, s_xm, Vn);
            c = add(c, mul(mul_nd(mul_nd(Uy, load_link(bn.U, 0, s_xm_yp, Vn)), Uy_xm), Ux_xm));
            // U_-x,-y(x) = Ux(x-x)^+ Uy(x-x-y)^+ Ux(x-x-y) Uy(x-y)
            c = add(c, mul(mul(mul_dn(Ux_xm, dag(load_link(bn.U, 1, s_xm_ym, Vn))), load_link(bn.U, 0, s_xm_ym, Vn)),
                           Uy_ym));
            // U_-y,x(x) = Uy(x-y)^+ Ux(x-y) Uy(x+x-y) Ux(x)^+
            c = add(c, mul_nd(mul(mul_dn(Uy_ym, load_link(bn.U, 0, s_ym, Vn)), load_link(bn.U, 1, s_xp_ym, Vn)), Ux));
            A8<R> Be = iah_to_alg(c);
#pragma unroll
            for (int a = 0; a < 8; a++) Be.v[a] *= R(0.25);
            store_alg(site + (size_t)5 * AP * Vn, s, Vn, Be);
        }
    }
}

template <typename R>
static void site_fields_t(const void* bn, const void* bn1, void* site, int N, double t, cudaStream_t st) {
    const int64_t Vn = (int64_t)N * N;
    const int threads = 128;
    int64_t blocks = (Vn + threads - 1) / threads;
    if (blocks > 152 * 64) blocks = 152 * 64;
    site_fields_kernel<R><<<(unsigned)blocks, threads, 0, st>>>(
        carve_fields<R>((void*)bn, Vn), carve_fields<R>((void*)bn1, Vn), (typename Prec<R>::V*)site, N,
        (R)(t > 0 ? 1.0 / t : 0.0));
}

void launch_site_fields(int prec, const void* bn, const void* bn1, void* site, int N, double t, cudaStream_t st) {
    if (prec == 0) site_fields_t<double>(bn, bn1, site, N, t, st);
    else site_fields_t<float>(bn, bn1, site, N, t, st);
}

// ------------------------------------------------------------ push
template <typename R, int B>
__global__ void __launch_bounds__(B, (sizeof(R) == 4 ? 1024 : 512) / B) push_kernel(const typename Prec<R>::V* __restrict__ site,
                                                           Fields<R> bn1, Parts<R> P, int N, R t, R dt, R dt_over_t,
                                                           uint32_t active, SpeciesArgs<R> sa) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.np; i += stride) {
        // the next particle's state into L2 while this one is pushed
        if (i + stride < P.np) P.prefetch_l2(i + stride);
        push_one<R>(site, bn1, P, i, N, t, dt, dt_over_t, active, sa);
    }
}

template <typename R>
static void push_t(const void* site, const void* bn1, void* parts, int64_t np, int N, double t, double dt,
                   uint32_t active, const SpeciesParams& sp, cudaStream_t st, int block) {
    const int64_t Vn = (int64_t)N * N;
    SpeciesArgs<R> sa;
    for (int k = 0; k < GL_MAX_SPECIES; k++) {
        sa.mass[k] = (R)(k < sp.n_species && sp.motion[k] == MOTION_WONG ? sp.mass[k] : 0.0);
        sa.motion[k] = k < sp.n_species ? sp.motion[k] : MOTION_WONG;
    }
    sa.ptau_diag = sp.ptau_diag;
    const int threads = block == 64 || block == 256 ? block : 128;
    int64_t blocks = (np + threads - 1) / threads;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) return;
    const Fields<R> f = carve_fields<R>((void*)bn1, Vn);
    const Parts<R> P = carve_parts<R>(parts, np);
    const R tr = (R)t, dtr = (R)dt, dto = (R)(t > 0 ? dt / t : 0.0);
    if (threads == 64)
        push_kernel<R, 64><<<(unsigned)blocks, 64, 0, st>>>((const typename Prec<R>::V*)site, f, P, N, tr, dtr, dto, active, sa);
    else if (threads == 256)
        push_kernel<R, 256><<<(unsigned)blocks, 256, 0, st>>>((const typename Prec<R>::V*)site, f, P, N, tr, dtr, dto, active, sa);
    else
        push_kernel<R, 128><<<(unsigned)blocks, 128, 0, st>>>((const typename Prec<R>::V*)site, f, P, N, tr, dtr, dto, active, sa);
}

void launch_push(int prec, const void* site, const void* bn1, void* parts, int64_t np, int N, double t, double dt,
                 uint32_t active_mask, const SpeciesParams& sp, cudaStream_t st, int block) {
    if (prec == 0) push_t<double>(site, bn1, parts, np, N, t, dt, active_mask, sp, st, block);
    else push_t<float>(site, bn1, parts, np, N, t, dt, active_mask, sp, st, block);
}

// ------------------------------------------------------------ sampling
struct SampleArgs {
    int64_t off[GL_MAX_SPECIES + 1];
    int rep[GL_MAX_SPECIES], mode[GL_MAX_SPECIES];
    double p0[GL_MAX_SPECIES], p1[GL_MAX_SPECIES];
    double q0[2][8];
    int n_species;
};

// Haar-random U(3) from the QR decomposition of a complex Ginibre matrix
// (Gram-Schmidt on the columns, R's diagonal positive), then Q = U Q0 U^+.
__device__ A8<double> haar_charge(const double* g, const double* q0) {
    double zr[3][3], zi[3][3];
    const double is2 = 0.70710678118654752440;
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) { zr[r][c] = g[2 * (3 * r + c)] * is2; zi[r][c] = g[2 * (3 * r + c) + 1] * is2; }
    M3<double> u;
    for (int c = 0; c < 3; c++) {
        double vr[3], vi[3];
        for (int r = 0; r < 3; r++) { vr[r] = zr[r][c]; vi[r] = zi[r][c]; }
        for (int pass = 0; pass < 2; pass++)
            for (int k = 0; k < c; k++) {
                double dr = 0, di = 0;  // sum conj(u_rk) v_r
                for (int r = 0; r < 3; r++) {
                    dr += u.re[r][k] * vr[r] + u.im[r][k] * vi[r];
                    di += u.re[r][k] * vi[r] - u.im[r][k] * vr[r];
                }
                for (int r = 0; r < 3; r++) {
                    vr[r] -= dr * u.re[r][k] - di * u.im[r][k];
                    vi[r] -= dr * u.im[r][k] + di * u.re[r][k];
                }
            }
        double n = 0;
        for (int r = 0; r < 3; r++) n += vr[r] * vr[r] + vi[r] * vi[r];
        n = 1.0 / sqrt(n);
        for (int r = 0; r < 3; r++) { u.re[r][c] = vr[r] * n; u.im[r][c] = vi[r] * n; }
    }
    A8<double> Q0;
    for (int a = 0; a < 8; a++) Q0.v[a] = q0[a];
    return adj(u, Q0);
}

template <typename R>
__global__ void sample_kernel(Parts<R> P, int N, uint32_t k0, uint32_t k1, SampleArgs sa) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.np; i += (int64_t)gridDim.x * blockDim.x) {
        int s = 0;
        while (s + 1 < sa.n_species && i >= sa.off[s + 1]) s++;
        const uint32_t idx = (uint32_t)(i - sa.off[s]);
        U4 w = philox4x32_10(U4{idx, (uint32_t)s, 2u, 0u}, k0, k1);
        const double x = N * u01(w.x), y = N * u01(w.y);
        const double psi = 2.0 * 3.14159265358979323846 * u01(w.z);
        const double pt = sa.mode[s] == 1 ? sa.p0[s] + (sa.p1[s] - sa.p0[s]) * u01(w.w) : sa.p0[s];
        double px = pt * cos(psi), py = pt * sin(psi);
        if (sa.mode[s] == 2) { px = sa.p0[s]; py = 0.0; }
        if (sa.mode[s] == 3) { px = 0.0; py = 0.0; }  // eikonal: only the kicks are recorded
        double g[20];
        for (int j = 0; j < 5; j++) {
            U4 v = philox4x32_10(U4{idx, (uint32_t)s, 3u, (uint32_t)j}, k0, k1);
            box_muller(u01(v.x), u01(v.y), g[4 * j], g[4 * j + 1]);
            box_muller(u01(v.z), u01(v.w), g[4 * j + 2], g[4 * j + 3]);
        }
        const A8<double> q = haar_charge(g, sa.q0[sa.rep[s]]);
        PState<R> p;
        p.x = (R)x; p.y = (R)y; p.eta = R(0); p.px = (R)px; p.py = (R)py; p.Pe = R(0);
        for (int a = 0; a < 8; a++) p.q.v[a] = (R)q.v[a];
        P.store(i, p);
        P.sp[i] = s;
        P.pt0[i] = (double)p.px * (double)p.px + (double)p.py * (double)p.py;
        P.id[i] = (int32_t)i;
        P.ptau[i] = R(NAN);
    }
}

template <typename R>
static void sample_t(void* parts, int64_t np, int N, uint64_t seed, const SampleArgs& sa, cudaStream_t st) {
    const int threads = 128;
    int64_t blocks = (np + threads - 1) / threads;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) return;
    sample_kernel<R><<<(unsigned)blocks, threads, 0, st>>>(carve_parts<R>(parts, np), N, (uint32_t)seed,
                                                           (uint32_t)(seed >> 32), sa);
}

void launch_sample(int prec, void* parts, int64_t np, int N, uint64_t seed, const int64_t* offsets, int n_species,
                   const int* rep, const int* mom_mode, const double* p0, const double* p1,
                   const double q0[2][8], cudaStream_t st) {
    SampleArgs sa;
    sa.n_species = n_species;
    for (int k = 0; k <= GL_MAX_SPECIES; k++) sa.off[k] = k <= n_species ? offsets[k] : np;
    for (int k = 0; k < GL_MAX_SPECIES; k++) {
        sa.rep[k] = k < n_species ? rep[k] : 0;
        sa.mode[k] = k < n_species ? mom_mode[k] : 0;
        sa.p0[k] = k < n_species ? p0[k] : 0;
        sa.p1[k] = k < n_species ? p1[k] : 0;
    }
    for (int r = 0; r < 2; r++)
        for (int a = 0; a < 8; a++) sa.q0[r][a] = q0[r][a];
    if (prec == 0) sample_t<double>(parts, np, N, seed, sa, st);
    else sample_t<float>(parts, np, N, seed, sa, st);
}

// ------------------------------------------------------------ canonical conversion of particles
template <typename R>
__global__ void parts_convert_kernel(Parts<R> P, double* stg, int to_device) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.np; i += (int64_t)gridDim.x * blockDim.x) {
        double* r = stg + i * 16;
        if (to_device) {
            PState<R> p;
            p.x = (R)r[0]; p.y = (R)r[1]; p.eta = (R)r[2]; p.px = (R)r[3]; p.py = (R)r[4]; p.Pe = (R)r[5];
            for (int a = 0; a < 8; a++) p.q.v[a] = (R)r[6 + a];
            P.store(i, p);
            P.pt0[i] = r[14];
            P.sp[i] = (int32_t)r[15];
            P.id[i] = (int32_t)i;
            P.ptau[i] = R(NAN);  // fresh particles: the p^tau integration restarts
        } else {
            // records go back to the caller's order (the device order may be sorted)
            r = stg + (int64_t)P.id[i] * 16;
            PState<R> p = P.load(i);
            r[0] = p.x; r[1] = p.y; r[2] = p.eta; r[3] = p.px; r[4] = p.py; r[5] = p.Pe;
            for (int a = 0; a < 8; a++) r[6 + a] = p.q.v[a];
            r[14] = P.pt0[i];
            r[15] = (double)P.sp[i];
        }
    }
}

// indices of a particle array copied in from a native snapshot: a species
// index outside [0, ns) becomes 0 and an original index outside [0, np) the
// particle's own position, and *bad is set, so that no later kernel indexes
// outside its arrays with them
template <typename R>
__global__ void parts_validate_kernel(Parts<R> P, int ns, int* bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.np; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = P.sp[i], id = P.id[i];
        if (s < 0 || s >= ns) {
            P.sp[i] = 0;
            atomicOr(bad, 1);
        }
        if (id < 0 || (int64_t)id >= P.np) {
            P.id[i] = (int32_t)i;
            atomicOr(bad, 1);
        }
    }
}

void launch_parts_validate(int prec, void* parts, int64_t np, int ns, int* d_bad, cudaStream_t st) {
    const int threads = 256;
    int64_t blocks = (np + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) return;
    if (prec == 0) parts_validate_kernel<double><<<(unsigned)blocks, threads, 0, st>>>(carve_parts<double>(parts, np), ns, d_bad);
    else parts_validate_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(carve_parts<float>(parts, np), ns, d_bad);
}

int parts_check_blocks(int64_t np) { return (int)((np + 255) / 256 < 1024 ? (np + 255) / 256 : 1024); }

// block b is block b - block_begin of its event, grid-strided over that
// event's particles
template <typename R>
__global__ void __launch_bounds__(256) parts_validate_events_kernel(const PartsCheckEv* ev, int ne, int* bad) {
    int lo = 0, hi = ne - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ev[mid].block_begin <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const PartsCheckEv& d = ev[lo];
    const Parts<R> P = carve_parts<R>(d.parts, d.np);
    const int blk = blockIdx.x - d.block_begin;
    for (int64_t i = (int64_t)blk * blockDim.x + threadIdx.x; i < P.np; i += (int64_t)d.nblocks * blockDim.x) {
        const int32_t s = P.sp[i], id = P.id[i];
        if (s < 0 || s >= d.ns) {
            P.sp[i] = 0;
            atomicOr(bad + lo, 1);
        }
        if (id < 0 || (int64_t)id >= P.np) {
            P.id[i] = (int32_t)i;
            atomicOr(bad + lo, 1);
        }
    }
}

void launch_parts_validate_events(int prec, const PartsCheckEv* evs, int ne, int blocks, int* bad, cudaStream_t st) {
    if (blocks < 1 || ne < 1) return;
    if (prec == 0) parts_validate_events_kernel<double><<<blocks, 256, 0, st>>>(evs, ne, bad);
    else parts_validate_events_kernel<float><<<blocks, 256, 0, st>>>(evs, ne, bad);
}

void launch_parts_convert(int prec, void* parts, int64_t np, double* stg, int to_device, cudaStream_t st) {
    const int threads = 128;
    int64_t blocks = (np + threads - 1) / threads;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) return;
    if (prec == 0) parts_convert_kernel<double><<<(unsigned)blocks, threads, 0, st>>>(carve_parts<double>(parts, np), stg, to_device);
    else parts_convert_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(carve_parts<float>(parts, np), stg, to_device);
}

// ------------------------------------------------------------ particle observables
// one block per chunk of obs_chunk(np) particles, then one block for the final reduction
template <typename R>
__global__ void __launch_bounds__(OBS_THREADS) particle_obs_kernel(Parts<R> P, double t, uint32_t active, ObsArgs oa,
                                                                   double* partials) {
    const int64_t chunk = obs_chunk(P.np);
    const int64_t c0 = (int64_t)blockIdx.x * chunk;
    const int64_t c1 = c0 + chunk < P.np ? c0 + chunk : P.np;
    particle_obs_block<R>(P, t, active, oa, c0, c1, partials + (size_t)blockIdx.x * GL_MAX_SPECIES * PO_N);
}

__global__ void __launch_bounds__(OBS_FINAL_WARPS * 32) particle_obs_finalize(const double* partials, int nblocks, double* out) {
    obs_finalize_block(partials, nblocks, GL_MAX_SPECIES * PO_N, ParticleObsKind(), out);
}

void launch_particle_obs(int prec, const void* parts, int64_t np, double t, uint32_t active_mask,
                         const SpeciesParams& sp, const double q2ref[GL_MAX_SPECIES],
                         const double q3ref[GL_MAX_SPECIES], double* partials, double* out, cudaStream_t st) {
    ObsArgs oa;
    oa.sp = sp;
    for (int k = 0; k < GL_MAX_SPECIES; k++) { oa.q2ref[k] = q2ref[k]; oa.q3ref[k] = q3ref[k]; }
    const int blocks = obs_blocks(np);
    if (blocks < 1) {
        cudaMemsetAsync(out, 0, GL_MAX_SPECIES * PO_N * sizeof(double), st);
        return;
    }
    const size_t smem = obs_smem_bytes(sp.n_species);
    if (prec == 0) {
        obs_smem_attr(particle_obs_kernel<double>);
        particle_obs_kernel<double><<<blocks, OBS_THREADS, smem, st>>>(carve_parts<double>((void*)parts, np), t,
                                                                       active_mask, oa, partials);
    } else {
        obs_smem_attr(particle_obs_kernel<float>);
        particle_obs_kernel<float><<<blocks, OBS_THREADS, smem, st>>>(carve_parts<float>((void*)parts, np), t,
                                                                      active_mask, oa, partials);
    }
    particle_obs_finalize<<<1, OBS_FINAL_WARPS * 32, 0, st>>>(partials, blocks, out);
}

}  // namespace gl

namespace gl {
// integrated p^tau <-> canonical [np] in the caller's particle order
template <typename R>
__global__ void ptau_convert_kernel(Parts<R> P, double* stg, int to_device) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.np; i += (int64_t)gridDim.x * blockDim.x) {
        if (to_device) P.ptau[i] = (R)stg[P.id[i]];
        else stg[P.id[i]] = (double)P.ptau[i];
    }
}

void launch_ptau_convert(int prec, void* parts, int64_t np, double* stg, int to_device, cudaStream_t st) {
    const int threads = 256;
    int64_t blocks = (np + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) return;
    if (prec == 0) ptau_convert_kernel<double><<<(unsigned)blocks, threads, 0, st>>>(carve_parts<double>(parts, np), stg, to_device);
    else ptau_convert_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(carve_parts<float>(parts, np), stg, to_device);
}
}  // namespace gl
