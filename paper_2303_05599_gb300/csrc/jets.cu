// Light-like jet correlator (Sec. 5.2, light-like jets).
//
// A probe starts at (x0, y0) at tau = 0 and moves along +x at the speed of
// light: at t_n it sits at x = x0 + t_n.  It carries the Wilson line W of the
// x links it has crossed (W <- W U_x at each crossing, links at t_{n+1}) and
// the integrals of the transported Lorentz-force components
//   X_i += dt W f_i W^+,   f = (E_x, E_y - B_eta, E_eta + B_y)
// of the site fields at its cell at t_n.  A parton of charge Q0 on the same
// path receives the kicks Q0 . X_i; averaged over charges of Casimir q2 the
// momentum broadening is (q2 / 8) X_i . X_i.
//
// Probe records are [n][JET_LEN] in the state's precision: x0, y0, W (3x3
// complex, row-major re/im), X_x, X_y, X_z (8 components each).
#include "internal.h"
#include "layout.cuh"
#include "philox.cuh"

namespace gl {

template <typename R>
__device__ __forceinline__ M3<R> jet_w(const R* r) {
    M3<R> w;
#pragma unroll
    for (int k = 0; k < 9; k++) { w.re[k / 3][k % 3] = r[2 + 2 * k]; w.im[k / 3][k % 3] = r[3 + 2 * k]; }
    return w;
}

template <typename R>
__global__ void jets_init_kernel(R* jets, int64_t n, int N, uint32_t k0, uint32_t k1) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        R* r = jets + j * JET_LEN;
        const U4 w = philox4x32_10(U4{(uint32_t)j, 0u, 4u, 0u}, k0, k1);
        r[0] = (R)(N * u01(w.x));
        r[1] = (R)(N * u01(w.y));
        for (int k = 2; k < JET_LEN; k++) r[k] = R(0);
        for (int i = 0; i < 3; i++) r[2 + 2 * (3 * i + i)] = R(1);
    }
}

template <typename R>
__global__ void jets_step_kernel(const typename Prec<R>::V* __restrict__ site, Fields<R> bn1, R* jets, int64_t n,
                                 int N, R t, R dt) {
    constexpr int AP = Prec<R>::AP;
    const int64_t Vn = (int64_t)N * N;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        R* r = jets + j * JET_LEN;
        const R x = r[0] + t;
        const int ixu = (int)floor(x + R(0.5)), iyu = (int)floor(r[1] + R(0.5));
        const int64_t cell = (int64_t)wrapi(iyu, N) * N + wrapi(ixu, N);
        const A8<R> Ex = load_alg(site, cell, Vn);
        const A8<R> Ey = load_alg(site + (size_t)1 * AP * Vn, cell, Vn);
        const A8<R> Ee = load_alg(site + (size_t)2 * AP * Vn, cell, Vn);
        const A8<R> By = load_alg(site + (size_t)4 * AP * Vn, cell, Vn);
        const A8<R> Be = load_alg(site + (size_t)5 * AP * Vn, cell, Vn);
        A8<R> f[3];
#pragma unroll
        for (int a = 0; a < 8; a++) {
            f[0].v[a] = Ex.v[a];
            f[1].v[a] = Ey.v[a] - Be.v[a];
            f[2].v[a] = Ee.v[a] + By.v[a];
        }
        M3<R> W = jet_w(r);
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const A8<R> g = conj_up(W, f[i]);  // W f_i W^+
#pragma unroll
            for (int a = 0; a < 8; a++) r[20 + 8 * i + a] += dt * g.v[a];
        }
        if ((int)floor(x + dt + R(0.5)) != ixu) {
            W = mul(W, load_link(bn1.U, 0, cell, Vn));
#pragma unroll
            for (int k = 0; k < 9; k++) { r[2 + 2 * k] = W.re[k / 3][k % 3]; r[3 + 2 * k] = W.im[k / 3][k % 3]; }
        }
    }
}

// block partials of sum_j X_i . X_i over a fixed chunk of probes, then one
// block combines the partials in a fixed order and divides by n
static constexpr int JET_OBS_THREADS = 256, JET_OBS_BLOCKS = 1024;

template <typename R>
__global__ void __launch_bounds__(JET_OBS_THREADS) jets_obs_kernel(const R* jets, int64_t n, int64_t chunk,
                                                                  double* partials) {
    __shared__ double red[3][JET_OBS_THREADS];
    const int64_t j0 = blockIdx.x * chunk, j1 = j0 + chunk < n ? j0 + chunk : n;
    double s[3] = {0, 0, 0};
    for (int64_t j = j0 + threadIdx.x; j < j1; j += JET_OBS_THREADS)
        for (int i = 0; i < 3; i++)
            for (int a = 0; a < 8; a++) {
                const double v = jets[j * JET_LEN + 20 + 8 * i + a];
                s[i] += v * v;
            }
    for (int i = 0; i < 3; i++) red[i][threadIdx.x] = s[i];
    __syncthreads();
    for (int o = JET_OBS_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int i = 0; i < 3; i++) red[i][threadIdx.x] += red[i][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 3) partials[(size_t)blockIdx.x * 3 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(JET_OBS_THREADS) jets_obs_finalize(const double* partials, int nblocks, int64_t n,
                                                                     double* out) {
    __shared__ double red[3][JET_OBS_THREADS];
    double s[3] = {0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += JET_OBS_THREADS)
        for (int i = 0; i < 3; i++) s[i] += partials[(size_t)b * 3 + i];
    for (int i = 0; i < 3; i++) red[i][threadIdx.x] = s[i];
    __syncthreads();
    for (int o = JET_OBS_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int i = 0; i < 3; i++) red[i][threadIdx.x] += red[i][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 3) out[threadIdx.x] = n > 0 ? red[threadIdx.x][0] / (double)n : 0.0;
}

template <typename R>
__global__ void jets_convert_kernel(R* jets, int64_t n, double* stg, int to_device) {
    const int64_t total = n * JET_LEN;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        if (to_device) jets[k] = (R)stg[k];
        else stg[k] = (double)jets[k];
    }
}

static unsigned jet_grid(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

void launch_jets_init(int prec, void* jets, int64_t n, int N, uint64_t seed, cudaStream_t st) {
    if (n <= 0) return;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    if (prec == 0) jets_init_kernel<double><<<jet_grid(n, 128), 128, 0, st>>>((double*)jets, n, N, k0, k1);
    else jets_init_kernel<float><<<jet_grid(n, 128), 128, 0, st>>>((float*)jets, n, N, k0, k1);
}

void launch_jets_step(int prec, const void* site, const void* bn1, void* jets, int64_t n, int N, double t, double dt,
                      cudaStream_t st) {
    if (n <= 0) return;
    const int64_t Vn = (int64_t)N * N;
    if (prec == 0)
        jets_step_kernel<double><<<jet_grid(n, 128), 128, 0, st>>>(
            (const double2*)site, carve_fields<double>((void*)bn1, Vn), (double*)jets, n, N, t, dt);
    else
        jets_step_kernel<float><<<jet_grid(n, 128), 128, 0, st>>>(
            (const float4*)site, carve_fields<float>((void*)bn1, Vn), (float*)jets, n, N, (float)t, (float)dt);
}

void launch_jets_obs(int prec, const void* jets, int64_t n, double* partials, double* out, cudaStream_t st) {
    int64_t chunk = (n + JET_OBS_BLOCKS - 1) / JET_OBS_BLOCKS;
    if (chunk < JET_OBS_THREADS) chunk = JET_OBS_THREADS;
    const int blocks = n > 0 ? (int)((n + chunk - 1) / chunk) : 1;
    if (prec == 0) jets_obs_kernel<double><<<blocks, JET_OBS_THREADS, 0, st>>>((const double*)jets, n, chunk, partials);
    else jets_obs_kernel<float><<<blocks, JET_OBS_THREADS, 0, st>>>((const float*)jets, n, chunk, partials);
    jets_obs_finalize<<<1, JET_OBS_THREADS, 0, st>>>(partials, blocks, n, out);
}

void launch_jets_convert(int prec, void* jets, int64_t n, double* stg, int to_device, cudaStream_t st) {
    if (n <= 0) return;
    if (prec == 0) jets_convert_kernel<double><<<jet_grid(n * JET_LEN, 256), 256, 0, st>>>((double*)jets, n, stg, to_device);
    else jets_convert_kernel<float><<<jet_grid(n * JET_LEN, 256), 256, 0, st>>>((float*)jets, n, stg, to_device);
}

}  // namespace gl
