/*
 * SU(3) algebra for the FP64 oracle (test infrastructure; see oracle.h).
 * Generators T^a = lambda^a/2 with the Gell-Mann matrices (App. B, generators
 * normalised as tr(T^a T^b) = delta/2); f_abc and d_abc are obtained from
 * traces of the generators, Tables I and II of the paper list the values.
 */
#include <complex.h>
#include <math.h>
#include <string.h>
#include "oracle_internal.h"

mat3 m_zero(void) { mat3 r; memset(&r, 0, sizeof r); return r; }
mat3 m_id(void) { mat3 r = m_zero(); r.m[0][0] = r.m[1][1] = r.m[2][2] = 1.0; return r; }

mat3 m_mul(mat3 a, mat3 b) {
    mat3 r;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double complex s = 0;
            for (int k = 0; k < 3; k++) s += a.m[i][k] * b.m[k][j];
            r.m[i][j] = s;
        }
    return r;
}
mat3 m_dag(mat3 a) {
    mat3 r;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) r.m[i][j] = conj(a.m[j][i]);
    return r;
}
mat3 m_add(mat3 a, mat3 b) {
    for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) a.m[i][j] += b.m[i][j];
    return a;
}
mat3 m_sub(mat3 a, mat3 b) {
    for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) a.m[i][j] -= b.m[i][j];
    return a;
}
mat3 m_scale(mat3 a, double complex s) {
    for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) a.m[i][j] *= s;
    return a;
}
double complex m_tr(mat3 a) { return a.m[0][0] + a.m[1][1] + a.m[2][2]; }

double complex m_det(mat3 a) {
    return a.m[0][0] * (a.m[1][1] * a.m[2][2] - a.m[1][2] * a.m[2][1])
         - a.m[0][1] * (a.m[1][0] * a.m[2][2] - a.m[1][2] * a.m[2][0])
         + a.m[0][2] * (a.m[1][0] * a.m[2][1] - a.m[1][1] * a.m[2][0]);
}

/* [M]_ah = (M - M^+)/2 - tr(M - M^+)/6 * 1  (traceless anti-Hermitian part). */
mat3 m_ah(mat3 a) {
    mat3 r = m_scale(m_sub(a, m_dag(a)), 0.5);
    double complex t = m_tr(r) / 3.0;
    for (int i = 0; i < 3; i++) r.m[i][i] -= t;
    return r;
}

double m_norm(mat3 a) {
    double s = 0;
    for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) {
        double x = cabs(a.m[i][j]);
        s += x * x;
    }
    return sqrt(s);
}

mat3 m_load(const double* p) { mat3 r; memcpy(&r, p, sizeof r); return r; }
void m_store(mat3 a, double* p) { memcpy(p, &a, sizeof a); }

/* Gell-Mann matrices lambda^1..lambda^8, halved. */
static mat3 gen_table[8];
static int gen_ready = 0;
static void gen_init(void) {
    if (gen_ready) return;
    for (int a = 0; a < 8; a++) gen_table[a] = m_zero();
    gen_table[0].m[0][1] = 1;  gen_table[0].m[1][0] = 1;
    gen_table[1].m[0][1] = -I; gen_table[1].m[1][0] = I;
    gen_table[2].m[0][0] = 1;  gen_table[2].m[1][1] = -1;
    gen_table[3].m[0][2] = 1;  gen_table[3].m[2][0] = 1;
    gen_table[4].m[0][2] = -I; gen_table[4].m[2][0] = I;
    gen_table[5].m[1][2] = 1;  gen_table[5].m[2][1] = 1;
    gen_table[6].m[1][2] = -I; gen_table[6].m[2][1] = I;
    gen_table[7].m[0][0] = 1.0 / sqrt(3.0);
    gen_table[7].m[1][1] = 1.0 / sqrt(3.0);
    gen_table[7].m[2][2] = -2.0 / sqrt(3.0);
    for (int a = 0; a < 8; a++) gen_table[a] = m_scale(gen_table[a], 0.5);
    gen_ready = 1;
}
mat3 gen(int a) { gen_init(); return gen_table[a]; }

void or_generator(int a, double* out18) { m_store(gen(a), out18); }

/* X = sum_a x^a T^a */
mat3 alg_to_mat(const double* x) {
    mat3 r = m_zero();
    for (int a = 0; a < 8; a++) r = m_add(r, m_scale(gen(a), x[a]));
    return r;
}
/* x^a = 2 Re tr(X T^a) (X Hermitian). */
void mat_to_alg(mat3 X, double* x) {
    for (int a = 0; a < 8; a++) x[a] = 2.0 * creal(m_tr(m_mul(X, gen(a))));
}

double or_f(int a, int b, int c) {
    mat3 ta = gen(a), tb = gen(b), tc = gen(c);
    mat3 comm = m_sub(m_mul(ta, tb), m_mul(tb, ta));
    return creal(-2.0 * I * m_tr(m_mul(comm, tc)));
}
static double d_direct(int a, int b, int c) {
    mat3 ta = gen(a), tb = gen(b), tc = gen(c);
    mat3 acomm = m_add(m_mul(ta, tb), m_mul(tb, ta));
    return creal(2.0 * m_tr(m_mul(acomm, tc)));
}
/* d_abc evaluated once from the traces and kept (the Casimir q3 sums it 512 times) */
static double d_table[512];
static int d_ready = 0;
double or_d(int a, int b, int c) {
    if (!d_ready) {
        for (int i = 0; i < 512; i++) d_table[i] = d_direct(i / 64, (i / 8) % 8, i % 8);
        d_ready = 1;
    }
    return d_table[a * 64 + b * 8 + c];
}

/* exp(A) by scaling and squaring of the Taylor series, summed until the
 * terms stop changing the sum in double precision. */
mat3 m_exp(mat3 A) {
    double nrm = m_norm(A);
    int s = 0;
    while (nrm > 0.25) { nrm *= 0.5; s++; }
    mat3 B = m_scale(A, ldexp(1.0, -s));
    mat3 sum = m_id(), term = m_id();
    for (int k = 1; k < 40; k++) {
        term = m_scale(m_mul(term, B), 1.0 / k);
        sum = m_add(sum, term);
        if (m_norm(term) < 1e-18) break;
    }
    for (int i = 0; i < s; i++) sum = m_mul(sum, sum);
    return sum;
}

void or_expm(const double* m18, double* out18) { m_store(m_exp(m_load(m18)), out18); }

void or_exp_i_alg(const double* x8, double* out18) {
    m_store(m_exp(m_scale(alg_to_mat(x8), I)), out18);
}

/* Fill the generator and d_abc tables when the library is loaded, so that
 * no OpenMP worker ever races on their first use. */
__attribute__((constructor)) static void tables_at_load(void) {
    gen_init();
    (void)or_d(0, 0, 0);
}
