// Internal declarations shared by the translation units of the CUDA library.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/glasma.h"

namespace gl {

struct SpeciesParams {
    double mass[GL_MAX_SPECIES];   // lattice units; INFINITY = static
    int is_static[GL_MAX_SPECIES];
    int n_species;
};

// field step n -> n+1 on buffers in/out (FP64 or FP32 two-row layout); when
// site is not null the same kernel also writes the site E, B at t_n
// tile: 0 = 32x8, 1 = 32x4, 2 = 32x2, 3 = 32x16 (FP64: 32x4 for 0, 1 and 3)
void launch_fused_step(int prec, void* in, void* out, void* site, int N, int64_t n, double dt, int reunit, int tile,
                       cudaStream_t st);
// site E, B at t_n from buffer n (U, phi, e(n-1/2), pi(n-1/2)) and buffer n+1 (e, pi at n+1/2)
void launch_site_fields(int prec, const void* bn, const void* bn1, void* site, int N, double t, cudaStream_t st);
// Euler + CPIC push of all particles active at t_n (bit s of active_mask)
void launch_push(int prec, const void* site, const void* bn1, void* parts, int64_t np, int N, double t, double dt,
                 uint32_t active_mask, const SpeciesParams& sp, cudaStream_t st, int block = 128);
// particle sampling: positions, momenta, Haar charges
void launch_sample(int prec, void* parts, int64_t np, int N, uint64_t seed, const int64_t* offsets, int n_species,
                   const int* rep, const int* mom_mode, const double* p0, const double* p1,
                   const double q0[2][8], cudaStream_t st);
// MV initial condition into field buffer b (FP64 scratch in `scratch`)
int launch_mv_init(int prec, void* b, void* scratch, int N, int Ns, double g2mu_a, double m_a, double Lambda_a,
                   uint64_t seed, int* d_bad, cudaStream_t st);
// canonical FP64 <-> device layout conversions (staging buffer is FP64 canonical)
void launch_parts_convert(int prec, void* parts, int64_t np, double* stg, int to_device, cudaStream_t st);
size_t init_scratch_bytes(int64_t Vn);
void launch_convert(int prec, int which, int to_device, void* dev, double* staging, int N, int64_t np,
                    cudaStream_t st);
// observables: per-species particle sums and field checks, FP64, fixed-order reductions
void launch_particle_obs(int prec, const void* parts, int64_t np, double t, uint32_t active_mask,
                         const SpeciesParams& sp, const double q2ref[GL_MAX_SPECIES],
                         const double q3ref[GL_MAX_SPECIES], double* partials, int max_blocks, double* out,
                         cudaStream_t st);
void launch_field_obs(int prec, const void* b, const void* site, int N, double* partials, int max_blocks,
                      double* out, cudaStream_t st);

// counting sort of the particles by cell from src into dst (same layout)
void launch_sort(int prec, void* src, void* dst, int64_t np, int N, void* scratch, cudaStream_t st);
size_t sort_scratch_bytes(int64_t Vn, int64_t np);
bool sort_supported(int64_t Vn);

size_t particle_bytes(int prec, int64_t np);
size_t site_bytes(int prec, int64_t Vn);
size_t field_bytes(int prec, int64_t Vn);

// observable slots
enum { PO_COUNT = 0, PO_PX2, PO_PY2, PO_PL2, PO_DPT2, PO_Q2, PO_Q3, PO_N };
enum { FO_GMAX = 0, FO_GSUM, FO_UMAX, FO_ET2, FO_EL2, FO_BT2, FO_BL2, FO_N };

}  // namespace gl
