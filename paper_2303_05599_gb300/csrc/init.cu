// McLerran-Venugopalan initial conditions on the GPU (Sec. 2.1 of
// arXiv:2303.05599), all in FP64:
//   rho^a_n(x) ~ N(0, (g^2 mu a)^2 / Ns) per sheet n, colour a, site x
//   alpha_n = rho_n / (k^2 + m^2) in Fourier space (lattice k^2, zero mode
//             removed, modes with k > Lambda removed), radix-2 FFTs in shared memory
//   V^+(x) = prod_n exp(-i alpha_n(x)), sheet 1 leftmost
//   U^{A,B}_i(x) = V(x) V^+(x+i)
//   Glasma link U_i: tr T^a [(U^A + U^B)(1 + U^+) - h.c.] = 0, Newton iteration
//   E_eta(0) = -i [alpha_A^i, alpha_B^i] from the link algebra elements -i[U]_ah,
//              forward and backward links averaged (the backward one
//              transported with the Glasma link)
// The paper states only that the continuum conditions are discretised; the
// matching condition is the standard one of the boost-invariant Glasma
// literature it builds on.
#include "internal.h"
#include "layout.cuh"
#include "philox.cuh"

namespace gl {

// scratch layout (bytes): [rho | U64] overlapped, then VdA, VdB
//   rho: 8 planes of Vn double2;  U64: 2 dirs x 9 planes of Vn double2
//   VdA, VdB: 9 planes of Vn double2 each
static size_t init_region0(int64_t Vn) { return (size_t)18 * Vn * sizeof(double2); }

size_t init_scratch_bytes(int64_t Vn) { return init_region0(Vn) + (size_t)18 * Vn * sizeof(double2); }

__global__ void set_identity_kernel(double2* Vd, int64_t Vn) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < Vn; s += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < 9; k++) Vd[(size_t)k * Vn + s] = make_double2(k % 4 == 0 ? 1.0 : 0.0, 0.0);
}

__global__ void rho_kernel(double2* rho, int64_t Vn, int Ns, int nucleus, int sheet, double sigma, uint32_t k0,
                           uint32_t k1) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < Vn; s += (int64_t)gridDim.x * blockDim.x) {
        double z[8];
        for (int j = 0; j < 2; j++) {
            U4 w = philox4x32_10(U4{(uint32_t)s, (uint32_t)((nucleus * Ns + sheet) * 2 + j), 1u, 0u}, k0, k1);
            box_muller(u01(w.x), u01(w.y), z[4 * j], z[4 * j + 1]);
            box_muller(u01(w.z), u01(w.w), z[4 * j + 2], z[4 * j + 3]);
        }
        for (int a = 0; a < 8; a++) rho[(size_t)a * Vn + s] = make_double2(sigma * z[a], 0.0);
    }
}

// one line (row or column) of one plane per block, radix 2 in shared memory
__global__ void fft_pow2_kernel(double2* data, int N, int log2N, int sign, int rows, int64_t Vn) {
    extern __shared__ double2 sh[];
    double2* base = data + (size_t)blockIdx.y * Vn;
    const int line = blockIdx.x;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const int64_t idx = rows ? (int64_t)line * N + k : (int64_t)k * N + line;
        const int rev = (int)(__brev((unsigned)k) >> (32 - log2N));
        sh[rev] = base[idx];
    }
    __syncthreads();
    for (int len = 2; len <= N; len <<= 1) {
        const int half = len >> 1;
        for (int b = threadIdx.x; b < N / 2; b += blockDim.x) {
            const int grp = b / half, k = b % half;
            const int i0 = grp * len + k, i1 = i0 + half;
            double sn, cs;
            sincospi(sign * 2.0 * (double)k / (double)len, &sn, &cs);
            const double2 u = sh[i0], v = sh[i1];
            const double2 vw = make_double2(v.x * cs - v.y * sn, v.x * sn + v.y * cs);
            sh[i0] = make_double2(u.x + vw.x, u.y + vw.y);
            sh[i1] = make_double2(u.x - vw.x, u.y - vw.y);
        }
        __syncthreads();
    }
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const int64_t idx = rows ? (int64_t)line * N + k : (int64_t)k * N + line;
        base[idx] = sh[k];
    }
}

// direct DFT of one line (any N), used when N is not a power of two
__global__ void dft_kernel(double2* data, int N, int sign, int rows, int64_t Vn) {
    extern __shared__ double2 sh[];
    double2* base = data + (size_t)blockIdx.y * Vn;
    const int line = blockIdx.x;
    for (int k = threadIdx.x; k < N; k += blockDim.x)
        sh[k] = base[rows ? (int64_t)line * N + k : (int64_t)k * N + line];
    __syncthreads();
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        double re = 0, im = 0;
        for (int j = 0; j < N; j++) {
            double sn, cs;
            sincospi(sign * 2.0 * (double)((int64_t)j * k % N) / (double)N, &sn, &cs);
            re += sh[j].x * cs - sh[j].y * sn;
            im += sh[j].x * sn + sh[j].y * cs;
        }
        base[rows ? (int64_t)line * N + k : (int64_t)k * N + line] = make_double2(re, im);
    }
}

static void fft2(double2* data, int planes, int N, int sign, cudaStream_t st) {
    const int64_t Vn = (int64_t)N * N;
    int log2N = 0;
    while ((1 << log2N) < N) log2N++;
    const bool pow2 = (1 << log2N) == N;
    const size_t shm = (size_t)N * sizeof(double2);
    dim3 grid(N, planes);
    const int threads = N >= 512 ? 256 : 128;
    for (int rows = 1; rows >= 0; rows--) {
        if (pow2) fft_pow2_kernel<<<grid, threads, shm, st>>>(data, N, log2N, sign, rows, Vn);
        else dft_kernel<<<grid, threads, shm, st>>>(data, N, sign, rows, Vn);
    }
}

__global__ void green_kernel(double2* rho, int N, double m2, double lam2, double invV) {
    const int64_t Vn = (int64_t)N * N;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < Vn; s += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(s % N), ky = (int)(s / N);
        const double sx = sinpi((double)kx / N), sy = sinpi((double)ky / N);
        const double k2 = 4.0 * (sx * sx + sy * sy);
        double g = 1.0 / (k2 + m2);
        if (kx == 0 && ky == 0) g = 0.0;
        if (lam2 > 0 && k2 > lam2) g = 0.0;
        g *= invV;
        for (int a = 0; a < 8; a++) {
            double2 v = rho[(size_t)a * Vn + s];
            rho[(size_t)a * Vn + s] = make_double2(v.x * g, v.y * g);
        }
    }
}

__global__ void wilson_accum_kernel(double2* Vd, const double2* rho, int64_t Vn) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < Vn; s += (int64_t)gridDim.x * blockDim.x) {
        A8<double> al;
        for (int a = 0; a < 8; a++) al.v[a] = -rho[(size_t)a * Vn + s].x;
        const M3<double> e = exp_i_alg<double, 20>(al, 1.0);
        const M3<double> v = load_link(Vd, 0, s, Vn);
        store_link(Vd, 0, s, Vn, mul(v, e));
    }
}

// tr(T^a M) for the eight generators, complex
__device__ void tr_T(const M3<double>& M, double* re, double* im) {
    const double h = 0.5, s3 = 0.5 * inv_sqrt3<double>();
    re[0] = h * (M.re[1][0] + M.re[0][1]);             im[0] = h * (M.im[1][0] + M.im[0][1]);
    re[1] = h * (M.im[1][0] - M.im[0][1]);             im[1] = h * (-M.re[1][0] + M.re[0][1]);
    re[2] = h * (M.re[0][0] - M.re[1][1]);             im[2] = h * (M.im[0][0] - M.im[1][1]);
    re[3] = h * (M.re[2][0] + M.re[0][2]);             im[3] = h * (M.im[2][0] + M.im[0][2]);
    re[4] = h * (M.im[2][0] - M.im[0][2]);             im[4] = h * (-M.re[2][0] + M.re[0][2]);
    re[5] = h * (M.re[2][1] + M.re[1][2]);             im[5] = h * (M.im[2][1] + M.im[1][2]);
    re[6] = h * (M.im[2][1] - M.im[1][2]);             im[6] = h * (-M.re[2][1] + M.re[1][2]);
    re[7] = s3 * (M.re[0][0] + M.re[1][1] - 2 * M.re[2][2]);
    im[7] = s3 * (M.im[0][0] + M.im[1][1] - 2 * M.im[2][2]);
}

__device__ double match_residual(const M3<double>& W, const M3<double>& U, double* F) {
    M3<double> one_ud = dag(U);
    one_ud.re[0][0] += 1; one_ud.re[1][1] += 1; one_ud.re[2][2] += 1;
    const M3<double> M = mul(W, one_ud);
    double re[8];
    tr_T(M, re, F);
    double r = 0;
    for (int a = 0; a < 8; a++) r = fmax(r, fabs(F[a]));
    return r;
}

__device__ int solve8(double J[8][8], double* b) {
    for (int c = 0; c < 8; c++) {
        int p = c;
        for (int r = c + 1; r < 8; r++) if (fabs(J[r][c]) > fabs(J[p][c])) p = r;
        if (fabs(J[p][c]) < 1e-300) return 1;
        if (p != c) {
            for (int k = 0; k < 8; k++) { double t = J[c][k]; J[c][k] = J[p][k]; J[p][k] = t; }
            double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int r = c + 1; r < 8; r++) {
            const double f = J[r][c] / J[c][c];
            for (int k = c; k < 8; k++) J[r][k] -= f * J[c][k];
            b[r] -= f * b[c];
        }
    }
    for (int c = 7; c >= 0; c--) {
        for (int k = c + 1; k < 8; k++) b[c] -= J[c][k] * b[k];
        b[c] /= J[c][c];
    }
    return 0;
}

// Newton solve for the Glasma link from the pure-gauge links of both nuclei
__device__ int solve_link(const M3<double>& UA, const M3<double>& UB, M3<double>& U) {
    const M3<double> W = add(UA, UB);
    U = mul(UA, UB);
    double F[8];
    double r = match_residual(W, U, F);
    for (int it = 0; it < 100 && r > 1e-14; it++) {
        // dF^a/dx^b for U -> exp(i x.T) U:  -Re tr(T^a W U^+ T^b)
        const M3<double> K = mul_nd(W, U);
        double J[8][8];
        for (int b = 0; b < 8; b++) {
            A8<double> eb = a_zero<double>();
            eb.v[b] = 1.0;
            const M3<double> KT = mul(K, alg_to_mat(eb));
            double re[8], im[8];
            tr_T(KT, re, im);
            for (int a = 0; a < 8; a++) J[a][b] = -re[a];
        }
        double dx[8];
        for (int a = 0; a < 8; a++) dx[a] = -F[a];
        if (solve8(J, dx)) break;
        double lam = 1.0;
        for (int k = 0; k < 30; k++) {
            A8<double> st;
            for (int a = 0; a < 8; a++) st.v[a] = lam * dx[a];
            const M3<double> Un = mul(exp_i_alg<double, 20>(st, 1.0), U);
            double Fn[8];
            const double rn = match_residual(W, Un, Fn);
            if (rn < r || k == 29) {
                U = Un;
                r = rn;
                for (int a = 0; a < 8; a++) F[a] = Fn[a];
                break;
            }
            lam *= 0.5;
        }
    }
    return r > 1e-12;
}

__device__ __forceinline__ M3<double> nucleus_link(const double2* Vd, int d, int64_t s, int N, int64_t Vn) {
    const int x = (int)(s % N), y = (int)(s / N);
    const int64_t sn = d == 0 ? (int64_t)y * N + (x + 1 == N ? 0 : x + 1) : (int64_t)(y + 1 == N ? 0 : y + 1) * N + x;
    return mul_dn(load_link(Vd, 0, s, Vn), load_link(Vd, 0, sn, Vn));
}

__global__ void glasma_link_kernel(const double2* VdA, const double2* VdB, double2* U64, int N, int* bad) {
    const int64_t Vn = (int64_t)N * N;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < 2 * Vn; l += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(l / Vn);
        const int64_t s = l % Vn;
        M3<double> U;
        const int b = solve_link(nucleus_link(VdA, d, s, N, Vn), nucleus_link(VdB, d, s, N, Vn), U);
        if (b) atomicAdd(bad, 1);
        store_link(U64, d, s, Vn, U);
    }
}

template <typename R>
__device__ __forceinline__ M3<R> to_r(const M3<double>& m) {
    M3<R> o;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) { o.re[i][j] = (R)m.re[i][j]; o.im[i][j] = (R)m.im[i][j]; }
    return o;
}

template <typename R>
__global__ void initial_fields_kernel(const double2* VdA, const double2* VdB, const double2* U64, Fields<R> f,
                                      int N) {
    const int64_t Vn = (int64_t)N * N;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < Vn; s += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(s % N), y = (int)(s / N);
        A8<double> pi = a_zero<double>();
        for (int d = 0; d < 2; d++) {
            const int64_t sb = d == 0 ? (int64_t)y * N + (x == 0 ? N - 1 : x - 1)
                                      : (int64_t)(y == 0 ? N - 1 : y - 1) * N + x;
            for (int k = 0; k < 2; k++) {
                const int64_t sl = k == 0 ? s : sb;
                A8<double> a = iah_to_alg(nucleus_link(VdA, d, sl, N, Vn));
                A8<double> b = iah_to_alg(nucleus_link(VdB, d, sl, N, Vn));
                for (int c = 0; c < 8; c++) { a.v[c] = -a.v[c]; b.v[c] = -b.v[c]; }  // -i[U]_ah
                A8<double> c = icomm(a, b);                                          // i[a, b]
                if (k == 1) c = adj_dag(load_link(U64, d, sb, Vn), c);
                for (int q = 0; q < 8; q++) pi.v[q] -= 0.5 * c.v[q];
            }
        }
        A8<R> pr, z;
        for (int a = 0; a < 8; a++) { pr.v[a] = (R)pi.v[a]; z.v[a] = R(0); }
        store_alg(f.pi, s, Vn, pr);
        store_alg(f.phi, s, Vn, z);
        store_alg(f.e, s, Vn, z);
        store_alg(f.e + (size_t)Prec<R>::AP * Vn, s, Vn, z);
        for (int d = 0; d < 2; d++) store_link(f.U, d, s, Vn, to_r<R>(load_link(U64, d, s, Vn)));
    }
}

static unsigned grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)(b < 1 ? 1 : b);
}

int launch_mv_init(int prec, void* buf, void* scratch, int N, int Ns, double g2mu_a, double m_a, double Lambda_a,
                   uint64_t seed, int* d_bad, cudaStream_t st) {
    const int64_t Vn = (int64_t)N * N;
    char* sc = (char*)scratch;
    double2* rho = (double2*)sc;
    double2* U64 = (double2*)sc;  // reused after the Wilson lines are complete
    double2* VdA = (double2*)(sc + init_region0(Vn));
    double2* VdB = VdA + (size_t)9 * Vn;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const double sigma = g2mu_a / sqrt((double)Ns);
    const int T = 128;
    for (int nucleus = 0; nucleus < 2; nucleus++) {
        double2* Vd = nucleus == 0 ? VdA : VdB;
        set_identity_kernel<<<grid_for(Vn, T), T, 0, st>>>(Vd, Vn);
        for (int sheet = 0; sheet < Ns; sheet++) {
            rho_kernel<<<grid_for(Vn, T), T, 0, st>>>(rho, Vn, Ns, nucleus, sheet, sigma, k0, k1);
            fft2(rho, 8, N, -1, st);
            green_kernel<<<grid_for(Vn, T), T, 0, st>>>(rho, N, m_a * m_a, Lambda_a > 0 ? Lambda_a * Lambda_a : 0.0,
                                                          1.0 / (double)Vn);
            fft2(rho, 8, N, +1, st);
            wilson_accum_kernel<<<grid_for(Vn, T), T, 0, st>>>(Vd, rho, Vn);
        }
    }
    cudaMemsetAsync(d_bad, 0, sizeof(int), st);
    glasma_link_kernel<<<grid_for(2 * Vn, 64), 64, 0, st>>>(VdA, VdB, U64, N, d_bad);
    if (prec == 0)
        initial_fields_kernel<double><<<grid_for(Vn, T), T, 0, st>>>(VdA, VdB, U64, carve_fields<double>(buf, Vn), N);
    else
        initial_fields_kernel<float><<<grid_for(Vn, T), T, 0, st>>>(VdA, VdB, U64, carve_fields<float>(buf, Vn), N);
    return 0;
}

}  // namespace gl
