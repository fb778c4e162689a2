// Field checks in FP64 (Gauss constraint of Sec. 2, unitarity of the links,
// lattice means of the squared site fields) and the conversions between the
// canonical FP64 host layout and the device layouts.
#include "internal.h"
#include "layout.cuh"

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

// G(x) = sum_i [e_i(x) - U_i(x-i)^+ e_i(x-i) U_i(x-i)] + i[phi(x), pi(x)]
template <typename R>
__global__ void __launch_bounds__(256) field_obs_kernel(Fields<R> f, const typename Prec<R>::V* __restrict__ site,
                                                        int N, double* partials) {
    constexpr int AP = Prec<R>::AP;
    __shared__ double wacc[8][FO_N];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double v[FO_N] = {0, 0, 0, 0, 0, 0, 0};
    const int64_t Vn = (int64_t)N * N;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < Vn; s += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(s % N), y = (int)(s / N);
        const int64_t sb[2] = {(int64_t)y * N + (x == 0 ? N - 1 : x - 1), (int64_t)(y == 0 ? N - 1 : y - 1) * N + x};
        A8<double> G = icomm(to_d(load_alg(f.phi, s, Vn)), to_d(load_alg(f.pi, s, Vn)));
        for (int d = 0; d < 2; d++) {
            const typename Prec<R>::V* e = f.e + (size_t)d * AP * Vn;
            const A8<double> eh = to_d(load_alg(e, s, Vn));
            const A8<double> eb = conj_dn(to_d(load_link(f.U, d, sb[d], Vn)), to_d(load_alg(e, sb[d], Vn)));
            for (int a = 0; a < 8; a++) G.v[a] += eh.v[a] - eb.v[a];
            // unitarity of the link at (d, s): ||U U^+ - 1||_F from the Gram
            // matrix of the rows (Hermitian: upper triangle, off-diagonal twice)
            const M3<double> u = to_d(load_link(f.U, d, s, Vn));
            double n2 = 0;
            for (int i = 0; i < 3; i++)
                for (int j = i; j < 3; j++) {
                    double gr = 0, gi = 0;
                    for (int k = 0; k < 3; k++) {
                        gr += u.re[i][k] * u.re[j][k] + u.im[i][k] * u.im[j][k];
                        gi += u.im[i][k] * u.re[j][k] - u.re[i][k] * u.im[j][k];
                    }
                    const double r = gr - (i == j ? 1.0 : 0.0);
                    n2 += (i == j ? 1.0 : 2.0) * (r * r + gi * gi);
                }
            v[FO_UMAX] = nanmax(v[FO_UMAX], sqrt(n2));
        }
        const double g2 = a_dot(G, G);
        v[FO_GMAX] = nanmax(v[FO_GMAX], sqrt(g2));
        v[FO_GSUM] += g2;
        // tr X^2 = X^a X^a / 2
        double tr[6];
        for (int k = 0; k < 6; k++) {
            const A8<double> X = to_d(load_alg(site + (size_t)k * AP * Vn, s, Vn));
            tr[k] = 0.5 * a_dot(X, X);
        }
        v[FO_ET2] += tr[0] + tr[1];
        v[FO_EL2] += tr[2];
        v[FO_BT2] += tr[3] + tr[4];
        v[FO_BL2] += tr[5];
    }
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
        partials[(size_t)blockIdx.x * FO_N + k] = a;
    }
}

// one block per output value: strided partial results, then a fixed-order tree
__global__ void __launch_bounds__(256) field_obs_finalize(const double* partials, int nblocks, double* out) {
    __shared__ double red[256];
    const int k = blockIdx.x;
    const bool mx = k == FO_GMAX || k == FO_UMAX;
    double a = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        const double v = partials[(size_t)b * FO_N + k];
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

void launch_field_obs(int prec, const void* b, const void* site, int N, double* partials, int max_blocks,
                      double* out, cudaStream_t st) {
    const int64_t Vn = (int64_t)N * N;
    const int threads = 256;
    int64_t blocks = (Vn + threads - 1) / threads;
    if (blocks > max_blocks) blocks = max_blocks;
    if (prec == 0)
        field_obs_kernel<double><<<(unsigned)blocks, threads, 0, st>>>(carve_fields<double>((void*)b, Vn),
                                                                       (const double2*)site, N, partials);
    else
        field_obs_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(carve_fields<float>((void*)b, Vn),
                                                                      (const float4*)site, N, partials);
    field_obs_finalize<<<FO_N, 256, 0, st>>>(partials, (int)blocks, out);
}

// ------------------------------------------------------------ canonical <-> device
template <typename R>
__device__ __forceinline__ void alg_io(typename Prec<R>::V* plane, int64_t s, int64_t Vn, double* c, int to_dev) {
    if (to_dev) {
        A8<R> x;
        for (int a = 0; a < 8; a++) x.v[a] = (R)c[a];
        store_alg(plane, s, Vn, x);
    } else {
        const A8<R> x = load_alg(plane, s, Vn);
        for (int a = 0; a < 8; a++) c[a] = x.v[a];
    }
}

__device__ __forceinline__ M3<float> link_in(const M3<double>& m, float) {
    M3<float> o;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) { o.re[i][j] = (float)m.re[i][j]; o.im[i][j] = (float)m.im[i][j]; }
    return o;
}
__device__ __forceinline__ M3<double> link_in(const M3<double>& m, double) { return m; }

template <typename R>
__global__ void convert_kernel(int which, int to_dev, Fields<R> f, typename Prec<R>::V* site, double* stg, int N) {
    constexpr int AP = Prec<R>::AP;
    const int64_t Vn = (int64_t)N * N;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < Vn; s += (int64_t)gridDim.x * blockDim.x) {
        switch (which) {
            case GL_BUF_LINKS:
                for (int d = 0; d < 2; d++) {
                    double* c = stg + ((size_t)d * Vn + s) * 18;
                    if (to_dev) {
                        M3<double> m;
                        for (int k = 0; k < 9; k++) { m.re[k / 3][k % 3] = c[2 * k]; m.im[k / 3][k % 3] = c[2 * k + 1]; }
                        store_link(f.U, d, s, Vn, link_in(m, R(0)));
                    } else {
                        const M3<R> m = load_link(f.U, d, s, Vn);
                        for (int k = 0; k < 9; k++) { c[2 * k] = m.re[k / 3][k % 3]; c[2 * k + 1] = m.im[k / 3][k % 3]; }
                    }
                }
                break;
            case GL_BUF_PHI: alg_io<R>(f.phi, s, Vn, stg + s * 8, to_dev); break;
            case GL_BUF_PI: alg_io<R>(f.pi, s, Vn, stg + s * 8, to_dev); break;
            case GL_BUF_E:
                for (int d = 0; d < 2; d++) alg_io<R>(f.e + (size_t)d * AP * Vn, s, Vn, stg + ((size_t)d * Vn + s) * 8, to_dev);
                break;
            case GL_BUF_SITE:
                for (int k = 0; k < 6; k++) alg_io<R>(site + (size_t)k * AP * Vn, s, Vn, stg + ((size_t)k * Vn + s) * 8, to_dev);
                break;
        }
    }
}

// energy density per site: sum over the six site fields of tr X^2 = X^a X^a / 2
template <typename R>
__global__ void energy_kernel(const typename Prec<R>::V* __restrict__ site, int N, double* out) {
    constexpr int AP = Prec<R>::AP;
    const int64_t Vn = (int64_t)N * N;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < Vn; s += (int64_t)gridDim.x * blockDim.x) {
        double e = 0.0;
        for (int k = 0; k < 6; k++) {
            const A8<double> X = to_d(load_alg(site + (size_t)k * AP * Vn, s, Vn));
            e += 0.5 * a_dot(X, X);
        }
        out[s] = e;
    }
}

void launch_energy(int prec, const void* site, int N, double* out, cudaStream_t st) {
    const int64_t Vn = (int64_t)N * N;
    int64_t blocks = (Vn + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (prec == 0) energy_kernel<double><<<(unsigned)blocks, 256, 0, st>>>((const double2*)site, N, out);
    else energy_kernel<float><<<(unsigned)blocks, 256, 0, st>>>((const float4*)site, N, out);
}

void launch_convert(int prec, int which, int to_device, void* dev, double* staging, int N, int64_t np,
                    cudaStream_t st) {
    (void)np;
    const int64_t Vn = (int64_t)N * N;
    const int threads = 128;
    int64_t blocks = (Vn + threads - 1) / threads;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (prec == 0) {
        Fields<double> f = carve_fields<double>(dev, Vn);
        convert_kernel<double><<<(unsigned)blocks, threads, 0, st>>>(which, to_device, f, (double2*)dev, staging, N);
    } else {
        Fields<float> f = carve_fields<float>(dev, Vn);
        convert_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(which, to_device, f, (float4*)dev, staging, N);
    }
}

}  // namespace gl
