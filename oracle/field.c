/*
 * Boost-invariant SU(3) Glasma leapfrog for the FP64 oracle (test
 * infrastructure; see oracle.h).  Sec. 2.1 of the paper: links and A_eta at
 * integer steps, conjugate momenta at half steps.
 *
 * Lattice-unit equations (obtained from the boost-invariant lattice Hamiltonian
 *   H = sum_x [ (1/t) sum_i tr e_i^2 + t tr pi^2 + 2t Re tr(1 - U_xy)
 *               + (1/t) sum_i tr(phi~_i - phi)^2 ]
 * by Hamilton's equations; the paper's P^i force carries a missing factor i,
 * read here so that the momenta stay Hermitian):
 *   e_i(n+1/2)  = e_i(n-1/2) + dt [ i t_n sum_j [U_ij + U_i,-j]_ah
 *                                   + (i/t_n) [phi~_i, phi] ]
 *   pi(n+1/2)   = pi(n-1/2) + dt (1/t_n) sum_i [phi~_i + phi^_i - 2 phi]
 *   U_i(n+1)    = exp(i dt/t_{n+1/2} e_i(n+1/2)) U_i(n)
 *   phi(n+1)    = phi(n) + dt t_{n+1/2} pi(n+1/2)
 * with phi~_i(x) = U_i(x) phi(x+i) U_i(x)^+ (the paper's transported scalar)
 * and  phi^_i(x) = U_i(x-i)^+ phi(x-i) U_i(x-i).
 */
#include <complex.h>
#include <math.h>
#include <string.h>
#include <stdlib.h>
#include "oracle_internal.h"

#define LINK(U, N, d, x, y) m_load((U) + ((int64_t)(d) * (N) * (N) + site_index(N, x, y)) * 18)
#define ALG(A, N, x, y) ((A) + site_index(N, x, y) * 8)

static const int DX[2] = {1, 0}, DY[2] = {0, 1};

/* plaquette U_ij(x) with i, j in {+x, +y, -x, -y}: (dir, sign) pairs */
static mat3 hop(const double* U, int N, int x, int y, int d, int s) {
    /* U_{s*d}(x): forward link or dagger of the backward link */
    if (s > 0) return LINK(U, N, d, x, y);
    return m_dag(LINK(U, N, d, x - DX[d], y - DY[d]));
}
static mat3 plaq(const double* U, int N, int x, int y, int di, int si, int dj, int sj) {
    /* U_ij(x) = U_i(x) U_j(x+i) U_-i(x+i+j) U_-j(x+j)  (Sec. 2.1) */
    int xi = x + si * DX[di], yi = y + si * DY[di];
    int xij = xi + sj * DX[dj], yij = yi + sj * DY[dj];
    int xj = x + sj * DX[dj], yj = y + sj * DY[dj];
    mat3 r = hop(U, N, x, y, di, si);
    r = m_mul(r, hop(U, N, xi, yi, dj, sj));
    r = m_mul(r, hop(U, N, xij, yij, di, -si));
    r = m_mul(r, hop(U, N, xj, yj, dj, -sj));
    return r;
}

void or_field_step(int N, double t, double dt,
                   const double* U, const double* phi, const double* e, const double* pi,
                   double* U1, double* phi1, double* e1, double* pi1) {
    const int64_t V = (int64_t)N * N;
    const double inv_t = t > 0 ? 1.0 / t : 0.0;
    const double th = t + 0.5 * dt;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < V; s++) {
        int x = (int)(s % N), y = (int)(s / N);
        mat3 ph = alg_to_mat(ALG(phi, N, x, y));
        mat3 lap = m_scale(ph, -4.0);
        for (int d = 0; d < 2; d++) {
            int dj = 1 - d;
            mat3 Ui = LINK(U, N, d, x, y);
            /* magnetic force: i t [U_ij + U_i,-j]_ah */
            mat3 p1 = plaq(U, N, x, y, d, +1, dj, +1);
            mat3 p2 = plaq(U, N, x, y, d, +1, dj, -1);
            mat3 fm = m_scale(m_ah(m_add(p1, p2)), I * t);
            /* scalar force: (i/t) [phi~_i, phi] */
            mat3 pt = m_mul(m_mul(Ui, alg_to_mat(ALG(phi, N, x + DX[d], y + DY[d]))), m_dag(Ui));
            mat3 comm = m_sub(m_mul(pt, ph), m_mul(ph, pt));
            mat3 fs = m_scale(comm, I * inv_t);
            double f[8];
            mat_to_alg(m_add(fm, fs), f);
            const double* eo = e + ((int64_t)d * V + s) * 8;
            double* en = e1 + ((int64_t)d * V + s) * 8;
            for (int a = 0; a < 8; a++) en[a] = eo[a] + dt * f[a];
            /* backward transported scalar for the covariant Laplacian */
            mat3 Ub = LINK(U, N, d, x - DX[d], y - DY[d]);
            mat3 pb = m_mul(m_mul(m_dag(Ub), alg_to_mat(ALG(phi, N, x - DX[d], y - DY[d]))), Ub);
            lap = m_add(lap, m_add(pt, pb));
            /* link update with the new momentum */
            double arg[8];
            for (int a = 0; a < 8; a++) arg[a] = dt / th * en[a];
            mat3 Ex = m_exp(m_scale(alg_to_mat(arg), I));
            m_store(m_mul(Ex, Ui), U1 + ((int64_t)d * V + s) * 18);
        }
        double l[8];
        mat_to_alg(lap, l);
        for (int a = 0; a < 8; a++) {
            pi1[s * 8 + a] = pi[s * 8 + a] + dt * inv_t * l[a];
            phi1[s * 8 + a] = phi[s * 8 + a] + dt * th * pi1[s * 8 + a];
        }
    }
}

void or_gauss(int N, const double* U, const double* phi, const double* e, const double* pi,
              double* g) {
    const int64_t V = (int64_t)N * N;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < V; s++) {
        int x = (int)(s % N), y = (int)(s / N);
        mat3 G = m_zero();
        for (int d = 0; d < 2; d++) {
            G = m_add(G, alg_to_mat(e + ((int64_t)d * V + s) * 8));
            int xb = x - DX[d], yb = y - DY[d];
            mat3 Ub = LINK(U, N, d, xb, yb);
            mat3 eb = alg_to_mat(e + ((int64_t)d * V + site_index(N, xb, yb)) * 8);
            G = m_sub(G, m_mul(m_mul(m_dag(Ub), eb), Ub));
        }
        mat3 ph = alg_to_mat(phi + s * 8), p = alg_to_mat(pi + s * 8);
        G = m_add(G, m_scale(m_sub(m_mul(ph, p), m_mul(p, ph)), I));
        mat_to_alg(G, g + s * 8);
    }
}

void or_site_fields(int N, double t, const double* U, const double* phi,
                    const double* e_old, const double* e_new,
                    const double* pi_old, const double* pi_new, double* out) {
    const int64_t V = (int64_t)N * N;
    const double inv_t = t > 0 ? 1.0 / t : 0.0;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < V; s++) {
        int x = (int)(s % N), y = (int)(s / N);
        /* E_i = (1/4t) { e(x) + e(x) + U_i(x-i)^+ [e(x-i) + e(x-i)] U_i(x-i) }, both times */
        for (int d = 0; d < 2; d++) {
            int xb = x - DX[d], yb = y - DY[d];
            int64_t sb = site_index(N, xb, yb);
            double here[8], back[8];
            for (int a = 0; a < 8; a++) {
                here[a] = e_new[((int64_t)d * V + s) * 8 + a] + e_old[((int64_t)d * V + s) * 8 + a];
                back[a] = e_new[((int64_t)d * V + sb) * 8 + a] + e_old[((int64_t)d * V + sb) * 8 + a];
            }
            mat3 Ub = LINK(U, N, d, xb, yb);
            mat3 m = m_add(alg_to_mat(here), m_mul(m_mul(m_dag(Ub), alg_to_mat(back)), Ub));
            mat_to_alg(m_scale(m, 0.25 * inv_t), out + ((int64_t)d * V + s) * 8);
        }
        /* E_eta = (pi(n+1/2) + pi(n-1/2)) / 2 */
        for (int a = 0; a < 8; a++)
            out[(2 * V + s) * 8 + a] = 0.5 * (pi_new[s * 8 + a] + pi_old[s * 8 + a]);
        /* central covariant differences of phi along each direction:
         * D_i phi ~ (phi~_i - phi^_i)/2;  B_x = -(1/t) D_y phi,  B_y = +(1/t) D_x phi */
        mat3 dphi[2];
        for (int d = 0; d < 2; d++) {
            mat3 Uf = LINK(U, N, d, x, y);
            mat3 Ub = LINK(U, N, d, x - DX[d], y - DY[d]);
            mat3 pf = m_mul(m_mul(Uf, alg_to_mat(ALG(phi, N, x + DX[d], y + DY[d]))), m_dag(Uf));
            mat3 pb = m_mul(m_mul(m_dag(Ub), alg_to_mat(ALG(phi, N, x - DX[d], y - DY[d]))), Ub);
            dphi[d] = m_scale(m_sub(pf, pb), 0.5 * inv_t);
        }
        mat_to_alg(m_scale(dphi[1], -1.0), out + (3 * V + s) * 8);
        mat_to_alg(dphi[0], out + (4 * V + s) * 8);
        /* B_eta = (i/4) [U_xy + U_y,-x + U_-x,-y + U_-y,x]_ah  (clover average) */
        mat3 c = plaq(U, N, x, y, 0, +1, 1, +1);
        c = m_add(c, plaq(U, N, x, y, 1, +1, 0, -1));
        c = m_add(c, plaq(U, N, x, y, 0, -1, 1, -1));
        c = m_add(c, plaq(U, N, x, y, 1, -1, 0, +1));
        mat_to_alg(m_scale(m_ah(c), 0.25 * I), out + (5 * V + s) * 8);
    }
}

void or_unitarity(int N, const double* U, double* max_unit, double* max_det) {
    const int64_t L = 2 * (int64_t)N * N;
    double mu = 0, md = 0;
    for (int64_t l = 0; l < L; l++) {
        mat3 u = m_load(U + l * 18);
        double a = m_norm(m_sub(m_mul(u, m_dag(u)), m_id()));
        double b = cabs(m_det(u) - 1.0);
        if (a > mu) mu = a;
        if (b > md) md = b;
    }
    *max_unit = mu;
    *max_det = md;
}

int or_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
