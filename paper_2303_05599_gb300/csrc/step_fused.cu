// Single-event launch of the field step: the FP32 strip kernel
// (strip_body.cuh) or the FP64 tile kernel (fused_body.cuh), both writing the
// site E, B of t_n beside the fields of step n + 1.
#include "strip_body.cuh"

namespace gl {

template <typename R, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, (Tile<R, TX, TY>::min_blocks)) fused_step_kernel(Fields<R> in, Fields<R> out,
                                                             typename Prec<R>::V* site, StepR<R> a) {
    fused_tile<R, TX, TY>(in, out, site, a, blockIdx.x);
}

template <typename R, int TX, int TY>
static void launch_t(void* in, void* out, void* site, int N, int64_t n, double dt, cudaStream_t st) {
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
    StepArgs a = step_args(N, (N + TX - 1) / TX, n, dt, 0);
    const int tiles_y = (N + TY - 1) / TY;
    fused_step_kernel<R, TX, TY><<<a.tiles_x * tiles_y, TX * TY, T::bytes, st>>>(
        carve_fields<R>(in, Vn), carve_fields<R>(out, Vn), (typename Prec<R>::V*)site, step_r<R>(a));
}

// FP32: blocks of WPB warps take WPB consecutive segments of the event's
// strips per item and run them in step; `items` items strided over the grid
template <int WPB, int MINB>
__global__ void __launch_bounds__(WPB * 32, MINB) strip_step_kernel(Fields<float> in, Fields<float> out, float4* site,
                                                                     int N, StripStep a, int items, int seg) {
    extern __shared__ __align__(16) unsigned char strip_smem[];
    StripWarpSmem* S = (StripWarpSmem*)strip_smem;
    const int wib = threadIdx.x >> 5;
    const int64_t nseg = strip_segments(N, seg);
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int64_t j = (int64_t)it * WPB + wib;
        strip_run_segment(S[wib], in, out, site, N, j < nseg ? j : nseg - 1, j < nseg, a, seg);
    }
}

// resident blocks of a strip launch shape on this device
template <int WPB, int MINB>
static int strip_blocks() {
    static int blocks[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!blocks[dev]) {
        const int smem = WPB * (int)sizeof(StripWarpSmem);
        cudaFuncSetAttribute(strip_step_kernel<WPB, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int per_sm = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, strip_step_kernel<WPB, MINB>, WPB * 32, smem);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        blocks[dev] = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    }
    return blocks[dev];
}

template <int WPB, int MINB>
static void launch_strip(void* in, void* out, void* site, int N, int64_t n, double dt, int every, int seg,
                         cudaStream_t st) {
    const int64_t Vn = (int64_t)N * N;
    int grid = strip_blocks<WPB, MINB>();
    if (seg <= 0) seg = strip_seg_rows(&N, 1, WPB, grid);
    const int items = (int)((strip_segments(N, seg) + WPB - 1) / WPB);
    if (grid > items) grid = items;
    strip_step_kernel<WPB, MINB><<<grid, WPB * 32, WPB * sizeof(StripWarpSmem), st>>>(
        carve_fields<float>(in, Vn), carve_fields<float>(out, Vn), (float4*)site, N, strip_step(n, dt, every), items,
        seg);
}

void launch_fused_step(int prec, void* in, void* out, void* site, int N, int64_t n, double dt, int reunit_every,
                       int tile, int seg, cudaStream_t st) {
    if (prec == 0) {
        // FP64 tiles: 32x4 (139 KB of shared memory) or 32x2
        if (tile == 2) launch_t<double, 32, 2>(in, out, site, N, n, dt, st);
        else launch_t<double, 32, 4>(in, out, site, N, n, dt, st);
    } else if (tile == 1) {
        launch_strip<12, 1>(in, out, site, N, n, dt, reunit_every, seg, st);
    } else if (tile == 2) {
        launch_strip<8, 1>(in, out, site, N, n, dt, reunit_every, seg, st);
    } else {
        launch_strip<8, 2>(in, out, site, N, n, dt, reunit_every, seg, st);
    }
}

int strip_model_seg(int N, int tile) {
    if (tile == 1) return strip_seg_rows(&N, 1, 12, strip_blocks<12, 1>());
    if (tile == 2) return strip_seg_rows(&N, 1, 8, strip_blocks<8, 1>());
    return strip_seg_rows(&N, 1, 8, strip_blocks<8, 2>());
}

}  // namespace gl
