/*
 * McLerran-Venugopalan initial conditions for the FP64 oracle (test
 * infrastructure; see oracle.h).  Sec. 2.1: Gaussian colour charges on Ns
 * sheets (eq. for the regularised charge correlator), Poisson solve by FFT
 * with IR regulator m and UV cutoff Lambda, path-ordered Wilson lines
 * V^+ = prod_n exp(-i alpha_n), pure-gauge links of each nucleus, and the
 * tau = 0 Glasma fields of Sec. 2 (the paper only says these are discretised;
 * the lattice matching condition used here is the standard one of the
 * boost-invariant Glasma literature it cites).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle_internal.h"

static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

void or_fft(double* data, int n, int sign) {
    double complex* a = (double complex*)data;
    if (!is_pow2(n)) {
        double complex* out = malloc(sizeof(double complex) * n);
        for (int k = 0; k < n; k++) {
            double complex s = 0;
            for (int j = 0; j < n; j++) s += a[j] * cexp(sign * 2.0 * M_PI * I * ((double)((int64_t)j * k % n)) / n);
            out[k] = s;
        }
        memcpy(a, out, sizeof(double complex) * n);
        free(out);
        return;
    }
    /* iterative Cooley-Tukey: bit reversal, then butterflies */
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { double complex t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (int len = 2; len <= n; len <<= 1) {
        for (int i = 0; i < n; i += len)
            for (int k = 0; k < len / 2; k++) {
                double complex w = cexp(sign * 2.0 * M_PI * I * (double)k / len);
                double complex u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
    }
}

static void fft2(double complex* f, int N, int sign) {
    double complex* col = malloc(sizeof(double complex) * N);
    for (int y = 0; y < N; y++) or_fft((double*)(f + (int64_t)y * N), N, sign);
    for (int x = 0; x < N; x++) {
        for (int y = 0; y < N; y++) col[y] = f[(int64_t)y * N + x];
        or_fft((double*)col, N, sign);
        for (int y = 0; y < N; y++) f[(int64_t)y * N + x] = col[y];
    }
    free(col);
}

void or_wilson_lines(int N, int Ns, double g2mu_a, double m_a, double Lambda_a,
                     uint64_t seed, int nucleus, double* vdag) {
    const int64_t V = (int64_t)N * N;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    double complex* rho = malloc(sizeof(double complex) * V * 8);
    double* kern = malloc(sizeof(double) * V);
    /* lattice Green function of -Laplacian + m^2 */
    for (int ky = 0; ky < N; ky++)
        for (int kx = 0; kx < N; kx++) {
            double sx = sin(M_PI * kx / N), sy = sin(M_PI * ky / N);
            double k2 = 4.0 * (sx * sx + sy * sy);
            double g = 1.0 / (k2 + m_a * m_a);
            if (kx == 0 && ky == 0) g = 0.0;
            if (Lambda_a > 0 && k2 > Lambda_a * Lambda_a) g = 0.0;
            kern[(int64_t)ky * N + kx] = g;
        }
    for (int64_t s = 0; s < V; s++) m_store(m_id(), vdag + s * 18);
    const double sigma = g2mu_a / sqrt((double)Ns);
    for (int sheet = 0; sheet < Ns; sheet++) {
#pragma omp parallel for schedule(static)
        for (int64_t s = 0; s < V; s++) {
            double z[8];
            for (int j = 0; j < 2; j++) {
                uint32_t ctr[4] = {(uint32_t)s, (uint32_t)((nucleus * Ns + sheet) * 2 + j), PURPOSE_MV, 0}, w[4];
                or_philox4x32_10(ctr, key, w);
                box_muller(u01(w[0]), u01(w[1]), &z[4 * j], &z[4 * j + 1]);
                box_muller(u01(w[2]), u01(w[3]), &z[4 * j + 2], &z[4 * j + 3]);
            }
            for (int a = 0; a < 8; a++) rho[a * V + s] = sigma * z[a];
        }
#pragma omp parallel for schedule(static)
        for (int a = 0; a < 8; a++) {
            double complex* f = rho + a * V;
            fft2(f, N, -1);
            for (int64_t s = 0; s < V; s++) f[s] *= kern[s];
            fft2(f, N, +1);
            for (int64_t s = 0; s < V; s++) f[s] /= (double)V;
        }
        /* V^+ <- V^+ exp(-i alpha_n): sheet 1 leftmost */
#pragma omp parallel for schedule(static)
        for (int64_t s = 0; s < V; s++) {
            double al[8];
            for (int a = 0; a < 8; a++) al[a] = -creal(rho[a * V + s]);
            mat3 e = m_exp(m_scale(alg_to_mat(al), I));
            m_store(m_mul(m_load(vdag + s * 18), e), vdag + s * 18);
        }
    }
    free(rho);
    free(kern);
}

/* Solve J dx = -F (8x8, Gaussian elimination with partial pivoting). */
static int solve8(double J[8][8], double* b) {
    for (int c = 0; c < 8; c++) {
        int p = c;
        for (int r = c + 1; r < 8; r++) if (fabs(J[r][c]) > fabs(J[p][c])) p = r;
        if (fabs(J[p][c]) < 1e-300) return 1;
        if (p != c) {
            for (int k = 0; k < 8; k++) { double t = J[c][k]; J[c][k] = J[p][k]; J[p][k] = t; }
            double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int r = c + 1; r < 8; r++) {
            double f = J[r][c] / J[c][c];
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

/* F^a(U) = Im tr(T^a (U^A + U^B)(1 + U^+)); zero for the Glasma link. */
static double residual(mat3 W, mat3 U, double* F) {
    mat3 M = m_mul(W, m_add(m_id(), m_dag(U)));
    double mx = 0;
    for (int a = 0; a < 8; a++) {
        F[a] = cimag(m_tr(m_mul(gen(a), M)));
        if (fabs(F[a]) > mx) mx = fabs(F[a]);
    }
    return mx;
}

int or_solve_link(const double* ua18, const double* ub18, double* u18) {
    mat3 UA = m_load(ua18), UB = m_load(ub18);
    mat3 W = m_add(UA, UB);
    mat3 U = m_mul(UA, UB);
    double F[8];
    double r = residual(W, U, F);
    for (int it = 0; it < 100 && r > 1e-14; it++) {
        /* dF^a/dx^b for U -> exp(i x.T) U:  -Re tr(T^a W U^+ T^b) */
        double J[8][8];
        mat3 WU = m_mul(W, m_dag(U));
        for (int a = 0; a < 8; a++)
            for (int b = 0; b < 8; b++)
                J[a][b] = -creal(m_tr(m_mul(m_mul(gen(a), WU), gen(b))));
        double dx[8];
        for (int a = 0; a < 8; a++) dx[a] = -F[a];
        if (solve8(J, dx)) break;
        /* backtracking: halve the step until the residual decreases */
        double lam = 1.0;
        for (int k = 0; k < 30; k++) {
            double st[8];
            for (int a = 0; a < 8; a++) st[a] = lam * dx[a];
            mat3 Un = m_mul(m_exp(m_scale(alg_to_mat(st), I)), U);
            double Fn[8];
            double rn = residual(W, Un, Fn);
            if (rn < r || k == 29) {
                U = Un; r = rn; memcpy(F, Fn, sizeof F);
                break;
            }
            lam *= 0.5;
        }
    }
    m_store(U, u18);
    return r > 1e-12;
}

int or_mv_init(int N, int Ns, double g2mu_a, double m_a, double Lambda_a, uint64_t seed,
               double* U, double* pi) {
    const int64_t V = (int64_t)N * N;
    double* vA = malloc(sizeof(double) * V * 18);
    double* vB = malloc(sizeof(double) * V * 18);
    or_wilson_lines(N, Ns, g2mu_a, m_a, Lambda_a, seed, 0, vA);
    or_wilson_lines(N, Ns, g2mu_a, m_a, Lambda_a, seed, 1, vB);
    /* pure-gauge links U^{A,B}_i(x) = V(x) V^+(x+i) */
    double* uA = malloc(sizeof(double) * 2 * V * 18);
    double* uB = malloc(sizeof(double) * 2 * V * 18);
    for (int d = 0; d < 2; d++)
        for (int64_t s = 0; s < V; s++) {
            int x = (int)(s % N), y = (int)(s / N);
            int64_t sn = site_index(N, x + (d == 0), y + (d == 1));
            mat3 a = m_mul(m_dag(m_load(vA + s * 18)), m_load(vA + sn * 18));
            mat3 b = m_mul(m_dag(m_load(vB + s * 18)), m_load(vB + sn * 18));
            m_store(a, uA + (d * V + s) * 18);
            m_store(b, uB + (d * V + s) * 18);
        }
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t l = 0; l < 2 * V; l++)
        bad += or_solve_link(uA + l * 18, uB + l * 18, U + l * 18);
    /* E_eta(0) = -i [alpha_A^i, alpha_B^i] (g = 1 units), with the link
     * algebra elements a = -i [U]_ah and the commutators of the forward and
     * backward links averaged at the site (backward one transported by the
     * Glasma link). */
    for (int64_t s = 0; s < V; s++) {
        int x = (int)(s % N), y = (int)(s / N);
        mat3 acc = m_zero();
        for (int d = 0; d < 2; d++) {
            int64_t sb = site_index(N, x - (d == 0), y - (d == 1));
            for (int k = 0; k < 2; k++) {
                int64_t l = d * V + (k == 0 ? s : sb);
                mat3 a = m_scale(m_ah(m_load(uA + l * 18)), -I);
                mat3 b = m_scale(m_ah(m_load(uB + l * 18)), -I);
                mat3 c = m_sub(m_mul(a, b), m_mul(b, a));
                if (k == 1) {
                    mat3 ub = m_load(U + l * 18);
                    c = m_mul(m_mul(m_dag(ub), c), ub);
                }
                acc = m_add(acc, c);
            }
        }
        mat_to_alg(m_scale(acc, -0.5 * I), pi + s * 8);
    }
    free(vA); free(vB); free(uA); free(uB);
    return bad;
}
