// Boost-invariant SU(3) Glasma leapfrog (Sec. 2.1 of arXiv:2303.05599), one
// fused kernel per time step: momentum update from plaquettes/staples and the
// transported scalar, then the link and scalar update, ping-pong buffers.
//
// Lattice units (a = 1), e_i = g a P^i, pi = g a^2 P^eta, phi = g A_eta:
//   e_i(n+1/2) = e_i(n-1/2) + dt [ t_n i[U_ij + U_i,-j]_ah + (1/t_n) i[phi~_i, phi] ]
//   pi(n+1/2)  = pi(n-1/2)  + dt (1/t_n) sum_i (phi~_i + phi^_i - 2 phi)
//   U_i(n+1)   = exp(i dt/t_{n+1/2} e_i(n+1/2)) U_i(n)
//   phi(n+1)   = phi(n) + dt t_{n+1/2} pi(n+1/2)
// phi~_i(x) = U_i(x) phi(x+i) U_i(x)^+ and phi^_i(x) = U_i(x-i)^+ phi(x-i) U_i(x-i).
// The paper's P^i force is printed without the factor i that makes it
// Hermitian; the form above follows from the lattice Hamiltonian.
#include "internal.h"
#include "layout.cuh"

namespace gl {

template <typename R>
struct ExpTerms;
template <>
struct ExpTerms<double> { static constexpr int n = 20; };
template <>
struct ExpTerms<float> { static constexpr int n = 12; };

// FP64 Gram-Schmidt of rows 0 and 1 (FP32 links are stored as two rows)
__device__ __forceinline__ void reunitarise(M3<float>& u) {
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
    // c = <r0, r1> = sum conj(r0_j) r1_j
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
__device__ __forceinline__ void reunitarise(M3<double>&) {}

template <typename R>
__global__ void __launch_bounds__(128) field_step_kernel(Fields<R> in, Fields<R> out, int N, R t, R dt,
                                                         R inv_t, R dt_over_th, R dt_th, int reunit) {
    const int64_t Vn = (int64_t)N * N;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < Vn; s += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(s % N), y = (int)(s / N);
        const int xp = x + 1 == N ? 0 : x + 1, xm = x == 0 ? N - 1 : x - 1;
        const int yp = y + 1 == N ? 0 : y + 1, ym = y == 0 ? N - 1 : y - 1;
        const int64_t s_xp = (int64_t)y * N + xp, s_xm = (int64_t)y * N + xm;
        const int64_t s_yp = (int64_t)yp * N + x, s_ym = (int64_t)ym * N + x;
        const int64_t s_xp_ym = (int64_t)ym * N + xp, s_xm_yp = (int64_t)yp * N + xm;

        const M3<R> Ux = load_link(in.U, 0, s, Vn);
        const M3<R> Uy = load_link(in.U, 1, s, Vn);
        A8<R> fx, fy;
        {
            // P(x) = Ux(x) Uy(x+x) Ux(x+y)^+ Uy(x)^+ = C Uy(x)^+, C = Ux(x) A, A = Uy(x+x) Ux(x+y)^+
            const M3<R> A = mul_nd(load_link(in.U, 1, s_xp, Vn), load_link(in.U, 0, s_yp, Vn));
            const M3<R> C = mul(Ux, A);
            const M3<R> P = mul_nd(C, Uy);
            // lower staple of the x link: Uy(x+x-y)^+ Ux(x-y)^+ Uy(x-y) = B^+ Uy(x-y)
            const M3<R> Uy_ym = load_link(in.U, 1, s_ym, Vn);
            const M3<R> B = mul(load_link(in.U, 0, s_ym, Vn), load_link(in.U, 1, s_xp_ym, Vn));
            const M3<R> Mx = add(P, mul(Ux, mul_dn(B, Uy_ym)));
            // left staple of the y link: Ux(x-x+y)^+ Uy(x-x)^+ Ux(x-x) = D^+ Ux(x-x)
            const M3<R> Ux_xm = load_link(in.U, 0, s_xm, Vn);
            const M3<R> D = mul(load_link(in.U, 1, s_xm, Vn), load_link(in.U, 0, s_xm_yp, Vn));
            const M3<R> My = add(dag(P), mul(Uy, mul_dn(D, Ux_xm)));
            fx = iah_to_alg(Mx);
            fy = iah_to_alg(My);
        }
        const A8<R> ph = load_alg(in.phi, s, Vn);
        A8<R> lap;
#pragma unroll
        for (int a = 0; a < 8; a++) lap.v[a] = R(-4) * ph.v[a];
        {
            const A8<R> tx = adj(Ux, load_alg(in.phi, s_xp, Vn));
            const A8<R> ty = adj(Uy, load_alg(in.phi, s_yp, Vn));
            const A8<R> bx = adj_dag(load_link(in.U, 0, s_xm, Vn), load_alg(in.phi, s_xm, Vn));
            const A8<R> by = adj_dag(load_link(in.U, 1, s_ym, Vn), load_alg(in.phi, s_ym, Vn));
            const A8<R> cx = icomm(tx, ph), cy = icomm(ty, ph);
#pragma unroll
            for (int a = 0; a < 8; a++) {
                lap.v[a] += tx.v[a] + ty.v[a] + bx.v[a] + by.v[a];
                fx.v[a] = t * fx.v[a] + inv_t * cx.v[a];
                fy.v[a] = t * fy.v[a] + inv_t * cy.v[a];
            }
        }
        // momenta at n+1/2
        A8<R> ex = load_alg(in.e, s, Vn), ey = load_alg(in.e + (size_t)Prec<R>::AP * Vn, s, Vn);
        A8<R> p = load_alg(in.pi, s, Vn), phn;
#pragma unroll
        for (int a = 0; a < 8; a++) {
            ex.v[a] += dt * fx.v[a];
            ey.v[a] += dt * fy.v[a];
            p.v[a] += dt * inv_t * lap.v[a];
            phn.v[a] = ph.v[a] + dt_th * p.v[a];
        }
        store_alg(out.e, s, Vn, ex);
        store_alg(out.e + (size_t)Prec<R>::AP * Vn, s, Vn, ey);
        store_alg(out.pi, s, Vn, p);
        store_alg(out.phi, s, Vn, phn);
        // links at n+1
        M3<R> nx = mul(exp_i_alg<R, ExpTerms<R>::n>(ex, dt_over_th), Ux);
        M3<R> ny = mul(exp_i_alg<R, ExpTerms<R>::n>(ey, dt_over_th), Uy);
        if (reunit) { reunitarise(nx); reunitarise(ny); }
        store_link(out.U, 0, s, Vn, nx);
        store_link(out.U, 1, s, Vn, ny);
    }
}

template <typename R>
static void launch_field_step_t(void* in, void* out, int N, double t, double dt, int reunit, cudaStream_t st) {
    const int64_t Vn = (int64_t)N * N;
    Fields<R> fi = carve_fields<R>(in, Vn), fo = carve_fields<R>(out, Vn);
    const double th = t + 0.5 * dt;
    const double inv_t = t > 0 ? 1.0 / t : 0.0;
    int threads = 128;
    int64_t blocks = (Vn + threads - 1) / threads;
    if (blocks > 152 * 64) blocks = 152 * 64;
    field_step_kernel<R><<<(unsigned)blocks, threads, 0, st>>>(fi, fo, N, (R)t, (R)dt, (R)inv_t, (R)(dt / th),
                                                                (R)(dt * th), reunit);
}

void launch_field_step(int prec, void* in, void* out, int N, double t, double dt, int reunit, cudaStream_t st) {
    if (prec == 0) launch_field_step_t<double>(in, out, N, t, dt, 0, st);
    else launch_field_step_t<float>(in, out, N, t, dt, reunit, st);
}

}  // namespace gl
