/* Private helpers of the FP64 oracle (test infrastructure; see oracle.h). */
#ifndef ORACLE_INTERNAL_H
#define ORACLE_INTERNAL_H
#include <complex.h>
#include <stdint.h>
#include "oracle.h"

typedef struct { double complex m[3][3]; } mat3;

mat3 m_zero(void);
mat3 m_id(void);
mat3 m_mul(mat3 a, mat3 b);
mat3 m_dag(mat3 a);
mat3 m_add(mat3 a, mat3 b);
mat3 m_sub(mat3 a, mat3 b);
mat3 m_scale(mat3 a, double complex s);
double complex m_tr(mat3 a);
double complex m_det(mat3 a);
mat3 m_ah(mat3 a);
double m_norm(mat3 a);
mat3 m_load(const double* p);
void m_store(mat3 a, double* p);
mat3 gen(int a);
mat3 alg_to_mat(const double* x);
void mat_to_alg(mat3 X, double* x);
mat3 m_exp(mat3 A);

/* uniform in (0,1) from a 32-bit word: (r + 1/2) 2^-32 */
double u01(uint32_t r);
/* two standard normals from two uniforms (Box-Muller) */
void box_muller(double u1, double u2, double* z0, double* z1);
/* Philox counter purposes */
enum { PURPOSE_MV = 1, PURPOSE_KIN = 2, PURPOSE_HAAR = 3, PURPOSE_JET = 4 };

static inline int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }
static inline int64_t site_index(int N, int x, int y) { return (int64_t)wrap(y, N) * N + wrap(x, N); }

#endif
