// Field checks in FP64 (Gauss constraint of Sec. 2, unitarity of the links,
// lattice means of the squared site fields) and the conversions between the
// canonical FP64 host layout and the device layouts.
#include "field_obs.cuh"
#include "internal.h"
#include "layout.cuh"

namespace gl {

// event e's descriptor (ne > 0) or the one passed by value
__device__ __forceinline__ FieldObsEv field_obs_event(const FieldObsEv& one, const char* evs, size_t stride, int e) {
    return evs ? *(const FieldObsEv*)(evs + (size_t)e * stride) : one;
}

// Block b is block b - block_begin of its event, grid-strided over that
// event's sites; one row of partial results per block.
template <typename R>
__global__ void __launch_bounds__(256) field_obs_kernel(FieldObsEv one, const char* evs, size_t stride, int ne) {
    int e = 0;
    if (ne > 0) {
        int lo = 0, hi = ne - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (((const FieldObsEv*)(evs + (size_t)mid * stride))->block_begin <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        e = lo;
    }
    const FieldObsEv d = field_obs_event(one, ne > 0 ? evs : nullptr, stride, e);
    const int blk = blockIdx.x - d.block_begin;
    const int64_t Vn = (int64_t)d.N * d.N;
    const Fields<R> f = carve_fields<R>((void*)d.fields, Vn);
    const typename Prec<R>::V* site = (const typename Prec<R>::V*)d.site;
    double v[FO_N];
    field_obs_init<R>(v);
    for (int64_t s = (int64_t)blk * blockDim.x + threadIdx.x; s < Vn; s += (int64_t)d.nblocks * blockDim.x)
        field_obs_site<R>(f, site, d.N, Vn, s, v);
    field_obs_finish<R>(v);
    field_obs_block_reduce(v, d.partials + (size_t)blk * FO_N);
}

// the FO_N values of event e in block e
__global__ void __launch_bounds__(OBS_FINAL_WARPS * 32) field_obs_finalize(FieldObsEv one, const char* evs, size_t stride, int ne) {
    const FieldObsEv d = field_obs_event(one, ne > 0 ? evs : nullptr, stride, blockIdx.x);
    obs_finalize_block(d.partials, d.nblocks, FO_N, FieldObsKind(), d.out);
}

void launch_field_obs_events(int prec, const FieldObsEv& one, const void* evs, size_t stride, int ne, int blocks,
                             bool finalize, cudaStream_t st) {
    if (blocks < 1) return;
    const char* p = (const char*)evs;
    if (prec == 0) field_obs_kernel<double><<<blocks, 256, 0, st>>>(one, p, stride, ne);
    else field_obs_kernel<float><<<blocks, 256, 0, st>>>(one, p, stride, ne);
    if (finalize) field_obs_finalize<<<ne > 0 ? ne : 1, OBS_FINAL_WARPS * 32, 0, st>>>(one, p, stride, ne);
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
