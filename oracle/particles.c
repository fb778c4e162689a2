/*
 * Test particles for the FP64 oracle (test infrastructure; see oracle.h):
 * classical SU(3) charges sampled over the Haar measure (Sec. 4.2, App. C),
 * Wong's equations in Milne coordinates integrated with Euler's method
 * (Sec. 3.1 and 3.2, App. A), and CPIC colour rotation with nearest-grid-point links
 * (Sec. 3.2, eq. for the short Wilson line U(tau_{n-1}, tau_n)).
 */
#include <complex.h>
#include <math.h>
#include <string.h>
#include "oracle_internal.h"

/* Q0 with the Casimirs q2, q3 of the fundamental (4, 10/3) or adjoint (24, 0)
 * classical charge (App. B).  Fundamental: only Q^5 and Q^8 nonzero, so
 * q2 = Q5^2 + Q8^2 and q3 = 3 d_558 Q5^2 Q8 + d_888 Q8^3, i.e. Q8 = s solves
 * s^3 - 12 s - 20/sqrt(3) = 0 (root near -1.06209), Q5 = -sqrt(4 - s^2). */
void or_q0(int rep, double* q) {
    memset(q, 0, 8 * sizeof(double));
    if (rep == 1) { q[0] = sqrt(24.0); return; }
    double s = -1.06;
    for (int it = 0; it < 60; it++) {
        double f = s * s * s - 12.0 * s - 20.0 / sqrt(3.0);
        double df = 3.0 * s * s - 12.0;
        s -= f / df;
    }
    q[7] = s;
    q[4] = -sqrt(4.0 - s * s);
}

void or_casimirs(const double* q, double* q2, double* q3) {
    double a = 0, b = 0;
    for (int i = 0; i < 8; i++) a += q[i] * q[i];
    for (int i = 0; i < 8; i++)
        for (int j = 0; j < 8; j++)
            for (int k = 0; k < 8; k++) b += or_d(i, j, k) * q[i] * q[j] * q[k];
    *q2 = a;
    *q3 = b;
}

/* Gram-Schmidt QR of the Ginibre matrix Z: the Q factor with R's diagonal
 * real positive is Haar distributed on U(3) (Mezzadri 2007). */
void or_haar_from_normals(const double* g, double* out18) {
    double complex Z[3][3], Qm[3][3];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++)
            Z[r][c] = (g[2 * (3 * r + c)] + I * g[2 * (3 * r + c) + 1]) / sqrt(2.0);
    for (int c = 0; c < 3; c++) {
        double complex v[3] = {Z[0][c], Z[1][c], Z[2][c]};
        /* modified Gram-Schmidt, two passes (keeps Q unitary to rounding
         * for ill-conditioned draws); R's diagonal is the final norm */
        for (int pass = 0; pass < 2; pass++)
            for (int k = 0; k < c; k++) {
                double complex dot = 0;
                for (int r = 0; r < 3; r++) dot += conj(Qm[r][k]) * v[r];
                for (int r = 0; r < 3; r++) v[r] -= dot * Qm[r][k];
            }
        double nrm = sqrt(creal(v[0] * conj(v[0]) + v[1] * conj(v[1]) + v[2] * conj(v[2])));
        for (int r = 0; r < 3; r++) Qm[r][c] = v[r] / nrm;
    }
    mat3 u;
    for (int r = 0; r < 3; r++) for (int c = 0; c < 3; c++) u.m[r][c] = Qm[r][c];
    m_store(u, out18);
}

static void key_of(uint64_t seed, uint32_t key[2]) {
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
}

void or_sample_species(int N, uint64_t seed, int species, int rep, int mom_mode,
                       double p0, double p1, int64_t n, double* out) {
    uint32_t key[2];
    key_of(seed, key);
    double q0[8];
    or_q0(rep, q0);
    mat3 Q0 = alg_to_mat(q0);
    for (int64_t p = 0; p < n; p++) {
        double* r = out + p * 16;
        uint32_t ctr[4] = {(uint32_t)p, (uint32_t)species, PURPOSE_KIN, 0}, w[4];
        or_philox4x32_10(ctr, key, w);
        double x = N * u01(w[0]), y = N * u01(w[1]);
        double psi = 2.0 * M_PI * u01(w[2]);
        double pt = mom_mode == 1 ? p0 + (p1 - p0) * u01(w[3]) : p0;
        double px = pt * cos(psi), py = pt * sin(psi);
        if (mom_mode == 2) { px = p0; py = 0.0; }
        if (mom_mode == 3) { px = 0.0; py = 0.0; }  /* eikonal: only the kicks are recorded */
        /* 18 normals from 5 Philox blocks (Box-Muller on pairs of uniforms) */
        double g[20];
        for (int j = 0; j < 5; j++) {
            uint32_t c2[4] = {(uint32_t)p, (uint32_t)species, PURPOSE_HAAR, (uint32_t)j}, v[4];
            or_philox4x32_10(c2, key, v);
            box_muller(u01(v[0]), u01(v[1]), &g[4 * j], &g[4 * j + 1]);
            box_muller(u01(v[2]), u01(v[3]), &g[4 * j + 2], &g[4 * j + 3]);
        }
        double u18[18];
        or_haar_from_normals(g, u18);
        mat3 u = m_load(u18);
        mat3 Q = m_mul(m_mul(u, Q0), m_dag(u));
        r[0] = x; r[1] = y; r[2] = 0.0;
        r[3] = px; r[4] = py; r[5] = 0.0;
        mat_to_alg(Q, r + 6);
        r[14] = px * px + py * py;
        r[15] = (double)species;
    }
}

/* Q.X = Q^a X^a (the g/T_R tr(Q F) of Wong's equations with both in the
 * fundamental basis) */
static double qdot(const double* q, const double* x) {
    double s = 0;
    for (int a = 0; a < 8; a++) s += q[a] * x[a];
    return s;
}

static void rotate(double* q, mat3 W) {
    /* Q <- W Q W^+ */
    mat3 Q = alg_to_mat(q);
    mat_to_alg(m_mul(m_mul(W, Q), m_dag(W)), q);
}

void or_push_kinds(int N, double t, double dt, const double* site, const double* U1,
                   const double* phi1, int64_t n, double* part, const double* mass,
                   const int* kind, const int* active) {
    const int64_t V = (int64_t)N * N;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; p++) {
        double* r = part + p * 16;
        int s = (int)r[15];
        if (!active[s]) continue;
        double m = mass[s];
        /* nearest grid point of the position at t_n */
        int ixu = (int)floor(r[0] + 0.5), iyu = (int)floor(r[1] + 0.5);
        int64_t cell = site_index(N, ixu, iyu);
        const double* Ex = site + (0 * V + cell) * 8;
        const double* Ey = site + (1 * V + cell) * 8;
        const double* Ee = site + (2 * V + cell) * 8;
        const double* Bx = site + (3 * V + cell) * 8;
        const double* By = site + (4 * V + cell) * 8;
        const double* Be = site + (5 * V + cell) * 8;
        double* q = r + 6;
        double qEx = qdot(q, Ex), qEy = qdot(q, Ey), qEe = qdot(q, Ee);
        double qBx = qdot(q, Bx), qBy = qdot(q, By), qBe = qdot(q, Be);
        if (kind[s] == OR_KIND_STATIC) {
            /* infinitely massive: no motion, no colour rotation (temporal
             * gauge), momentum kicks from the electric field only */
            r[3] += dt * qEx;
            r[4] += dt * qEy;
            r[5] += dt * qEe;
            continue;
        }
        if (kind[s] == OR_KIND_EIKONAL) {
            /* light-like parton along +x at eta = 0 (Sec. 5.2): the path is
             * x = x0 + t, the kicks of the Lorentz force (E_x, E_y - B_z,
             * E_z + B_y) accumulate in p^x, p^y and the P_eta slot (lab p_z),
             * and Q is carried along by the crossed x links */
            r[3] += dt * qEx;
            r[4] += dt * (qEy - qBe);
            r[5] += dt * (qEe + qBy);
            double xn = r[0] + dt;
            int jxu = (int)floor(xn + 0.5);
            xn = fmod(xn, (double)N); if (xn < 0) xn += N;
            r[0] = xn;
            if (jxu != ixu) {
                mat3 u = m_load(U1 + (0 * V + site_index(N, ixu, iyu)) * 18);
                rotate(q, m_dag(u));
            }
            continue;
        }
        double px = r[3], py = r[4], Pe = r[5];
        double w = t > 0 ? Pe / t : 0.0;                  /* tau p^eta in lattice units */
        double ptau = sqrt(px * px + py * py + w * w + m * m);
        double vx = ptau > 0 ? px / ptau : 0.0;
        double vy = ptau > 0 ? py / ptau : 0.0;
        double vw = ptau > 0 ? w / ptau : 0.0;
        double dpx = qEx + qBe * vy - qBy * vw;
        double dpy = qEy - qBe * vx + qBx * vw;
        double dPe = t * (qEe - qBx * vy + qBy * vx);
        double deta = t > 0 ? dt * vw / t : 0.0;
        double xn = r[0] + dt * vx, yn = r[1] + dt * vy;
        r[2] += deta;
        r[3] = px + dt * dpx;
        r[4] = py + dt * dpy;
        r[5] = Pe + dt * dPe;
        int jxu = (int)floor(xn + 0.5), jyu = (int)floor(yn + 0.5);
        xn = fmod(xn, (double)N); if (xn < 0) xn += N;
        yn = fmod(yn, (double)N); if (yn < 0) yn += N;
        r[0] = xn; r[1] = yn;
        /* CPIC: rotate with the crossed links at t_{n+1}; x first, then y */
        int dxc = jxu - ixu, dyc = jyu - iyu;
        if (dxc == 1) {
            mat3 u = m_load(U1 + (0 * V + site_index(N, ixu, iyu)) * 18);
            rotate(q, m_dag(u));
        } else if (dxc == -1) {
            mat3 u = m_load(U1 + (0 * V + site_index(N, jxu, iyu)) * 18);
            rotate(q, u);
        }
        if (dyc == 1) {
            mat3 u = m_load(U1 + (1 * V + site_index(N, jxu, iyu)) * 18);
            rotate(q, m_dag(u));
        } else if (dyc == -1) {
            mat3 u = m_load(U1 + (1 * V + site_index(N, jxu, jyu)) * 18);
            rotate(q, u);
        }
        /* rapidity Wilson line at the new cell: Q <- e^{-i deta phi} Q e^{+i deta phi} */
        if (deta != 0.0) {
            const double* ph = phi1 + site_index(N, jxu, jyu) * 8;
            double arg[8];
            for (int a = 0; a < 8; a++) arg[a] = -deta * ph[a];
            rotate(q, m_exp(m_scale(alg_to_mat(arg), I)));
        }
    }
}

void or_push(int N, double t, double dt, const double* site, const double* U1,
             const double* phi1, int64_t n, double* part, const double* mass,
             const int* active) {
    int kind[OR_MAX_SPECIES];
    for (int s = 0; s < OR_MAX_SPECIES; s++) kind[s] = OR_KIND_WONG;
    for (int64_t p = 0; p < n; p++) {
        int s = (int)part[p * 16 + 15];
        if (s >= 0 && s < OR_MAX_SPECIES && isinf(mass[s])) kind[s] = OR_KIND_STATIC;
    }
    or_push_kinds(N, t, dt, site, U1, phi1, n, part, mass, kind, active);
}

double or_pL_kind(const double* r, double t, double m, int kind) {
    if (kind != OR_KIND_WONG) return r[5];
    double w = t > 0 ? r[5] / t : 0.0;
    double ptau = sqrt(r[3] * r[3] + r[4] * r[4] + w * w + m * m);
    return ptau * sinh(r[2]) + w * cosh(r[2]);
}

double or_pL(const double* r, double t, double m) {
    if (isinf(m)) return r[5];
    double w = t > 0 ? r[5] / t : 0.0;
    double ptau = sqrt(r[3] * r[3] + r[4] * r[4] + w * w + m * m);
    return ptau * sinh(r[2]) + w * cosh(r[2]);
}

void or_particle_obs(int64_t n, const double* part, double t, const double* mass,
                     const int* kind, const int* active, const int* rep, int n_species, double* out) {
    memset(out, 0, (size_t)n_species * 8 * sizeof(double));
    double q2r[2], q3r[2];
    for (int k = 0; k < 2; k++) {
        double q0[8];
        or_q0(k, q0);
        or_casimirs(q0, &q2r[k], &q3r[k]);
    }
    for (int64_t p = 0; p < n; p++) {
        const double* r = part + p * 16;
        int s = (int)r[15];
        if (!active[s]) continue;
        double* o = out + s * 8;
        double pl = or_pL_kind(r, t, mass[s], kind[s]);
        double q2, q3;
        or_casimirs(r + 6, &q2, &q3);
        o[0] += 1;
        o[1] += r[3] * r[3];
        o[2] += r[4] * r[4];
        o[3] += pl * pl;
        o[4] += r[3] * r[3] + r[4] * r[4] - r[14];
        double d2 = fabs(q2 - q2r[rep[s]]), d3 = fabs(q3 - q3r[rep[s]]);
        if (d2 > o[5]) o[5] = d2;
        if (d3 > o[6]) o[6] = d3;
    }
}

/* ---- light-like jet correlator (Sec. 5.2, light-like jets) ------------- */
/* A probe starts at (x0, y0) at tau = 0 and moves along +x at the speed of
 * light (x = x0 + t in lattice units).  It carries the Wilson line W of the x
 * links it has crossed (W <- W U_x on each crossing, links at t_{n+1}) and
 * the integrals X_i = sum_n dt W f_i W^+ of the Lorentz-force components
 * f = (E_x, E_y - B_z, E_z + B_y) at its cell, so that a parton of charge Q0
 * would have received the kicks Q0 . X_i.  Record: x0, y0, W (18), X (3 x 8). */
void or_jets_init(int N, uint64_t seed, int64_t n, double* jets) {
    uint32_t key[2];
    key_of(seed, key);
    for (int64_t j = 0; j < n; j++) {
        double* r = jets + j * OR_JET_LEN;
        memset(r, 0, OR_JET_LEN * sizeof(double));
        uint32_t ctr[4] = {(uint32_t)j, 0u, PURPOSE_JET, 0u}, w[4];
        or_philox4x32_10(ctr, key, w);
        r[0] = N * u01(w[0]);
        r[1] = N * u01(w[1]);
        for (int i = 0; i < 3; i++) r[2 + 2 * (3 * i + i)] = 1.0;  /* W = 1 */
    }
}

void or_jets_step(int N, double t, double dt, const double* site, const double* U1, int64_t n, double* jets) {
    const int64_t V = (int64_t)N * N;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++) {
        double* r = jets + j * OR_JET_LEN;
        const double x = r[0] + t;
        const int ixu = (int)floor(x + 0.5), iyu = (int)floor(r[1] + 0.5);
        const int64_t cell = site_index(N, ixu, iyu);
        const double* Ex = site + (0 * V + cell) * 8;
        const double* Ey = site + (1 * V + cell) * 8;
        const double* Ee = site + (2 * V + cell) * 8;
        const double* By = site + (4 * V + cell) * 8;
        const double* Be = site + (5 * V + cell) * 8;
        double f[3][8];
        for (int a = 0; a < 8; a++) {
            f[0][a] = Ex[a];
            f[1][a] = Ey[a] - Be[a];
            f[2][a] = Ee[a] + By[a];
        }
        mat3 W = m_load(r + 2);
        for (int i = 0; i < 3; i++) {
            double g[8];
            mat_to_alg(m_mul(m_mul(W, alg_to_mat(f[i])), m_dag(W)), g);
            for (int a = 0; a < 8; a++) r[20 + 8 * i + a] += dt * g[a];
        }
        if ((int)floor(x + dt + 0.5) != ixu) {
            W = m_mul(W, m_load(U1 + (0 * V + cell) * 18));
            m_store(W, r + 2);
        }
    }
}

void or_jets_obs(int64_t n, const double* jets, double* out3) {
    out3[0] = out3[1] = out3[2] = 0.0;
    for (int64_t j = 0; j < n; j++)
        for (int i = 0; i < 3; i++)
            for (int a = 0; a < 8; a++) {
                const double v = jets[j * OR_JET_LEN + 20 + 8 * i + a];
                out3[i] += v * v;
            }
    if (n > 0)
        for (int i = 0; i < 3; i++) out3[i] /= (double)n;
}

/* ---- temporal constraint (Sec. 3.1 equation for p^tau; the diagnostic of
 * the temporal-constraint section) --------------------------------------- */
/* One forward-Euler step of p^tau from its own equation of motion,
 *   dp^tau/dtau = -(tau p^eta) p^eta / p^tau
 *                 + Q.E_eta (tau p^eta / p^tau) + Q.E_x p^x/p^tau + Q.E_y p^y/p^tau,
 * in lattice units with w = tau p^eta = P_eta / t and the mass-shell p^tau
 * in the velocities, evaluated with the state at t_n (before the push).  A
 * NaN entry is first set to the mass-shell value: the integration starts at
 * the particle's first push.  Only active Wong particles are stepped. */
void or_ptau_step(int N, double t, double dt, const double* site, int64_t n, const double* part,
                  const double* mass, const int* kind, const int* active, double* ptau) {
    const int64_t V = (int64_t)N * N;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; p++) {
        const double* r = part + p * 16;
        int s = (int)r[15];
        if (!active[s] || kind[s] != OR_KIND_WONG) continue;
        double m = mass[s];
        int ixu = (int)floor(r[0] + 0.5), iyu = (int)floor(r[1] + 0.5);
        int64_t cell = site_index(N, ixu, iyu);
        const double* q = r + 6;
        double qEx = qdot(q, site + (0 * V + cell) * 8);
        double qEy = qdot(q, site + (1 * V + cell) * 8);
        double qEe = qdot(q, site + (2 * V + cell) * 8);
        double px = r[3], py = r[4];
        double w = t > 0 ? r[5] / t : 0.0;
        double pt = sqrt(px * px + py * py + w * w + m * m);
        if (isnan(ptau[p])) ptau[p] = pt;
        double vx = pt > 0 ? px / pt : 0.0, vy = pt > 0 ? py / pt : 0.0, vw = pt > 0 ? w / pt : 0.0;
        double drift = (t > 0 && pt > 0) ? w * w / (t * pt) : 0.0;
        ptau[p] += dt * (qEe * vw + qEx * vx + qEy * vy - drift);
    }
}
