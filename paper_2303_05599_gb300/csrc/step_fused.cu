// Single-event launch of the fused leapfrog + site E/B kernel (fused_body.cuh).
#include "fused_body.cuh"

namespace gl {

template <typename R, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, (Tile<R, TX, TY>::min_blocks)) fused_step_kernel(Fields<R> in, Fields<R> out,
                                                             typename Prec<R>::V* site, StepR<R> a) {
    fused_tile<R, TX, TY>(in, out, site, a, blockIdx.x);
}

template <typename R, int TX, int TY>
static void launch_t(void* in, void* out, void* site, int N, int64_t n, double dt, int reunit, cudaStream_t st) {
    using T = Tile<R, TX, TY>;
    // the dynamic shared-memory limit is a per-device function attribute
    static bool attr[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr[dev]) {
        cudaFuncSetAttribute(fused_step_kernel<R, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)T::bytes);
        attr[dev] = true;
    }
    const int64_t Vn = (int64_t)N * N;
    StepArgs a = step_args(N, (N + TX - 1) / TX, n, dt, reunit);
    const int tiles_y = (N + TY - 1) / TY;
    fused_step_kernel<R, TX, TY><<<a.tiles_x * tiles_y, TX * TY, T::bytes, st>>>(
        carve_fields<R>(in, Vn), carve_fields<R>(out, Vn), (typename Prec<R>::V*)site, step_r<R>(a));
}

void launch_fused_step(int prec, void* in, void* out, void* site, int N, int64_t n, double dt, int reunit, int tile,
                       cudaStream_t st) {
    if (prec == 0) {
        // FP64 tiles: 32x4 (139 KB of shared memory) or 32x2
        if (tile == 2) launch_t<double, 32, 2>(in, out, site, N, n, dt, 0, st);
        else launch_t<double, 32, 4>(in, out, site, N, n, dt, 0, st);
    } else if (tile == 1) {
        launch_t<float, 32, 4>(in, out, site, N, n, dt, reunit, st);
    } else if (tile == 2) {
        launch_t<float, 32, 2>(in, out, site, N, n, dt, reunit, st);
    } else if (tile == 3) {
        launch_t<float, 32, 16>(in, out, site, N, n, dt, reunit, st);
    } else {
        launch_t<float, 32, 8>(in, out, site, N, n, dt, reunit, st);
    }
}

}  // namespace gl
