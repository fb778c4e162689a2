// SU(3) algebra on the device, templated on the real type (double for the
// plain FP64 path, float for the FP32 path).
//
// Matrices are held as separate real and imaginary 3x3 arrays so that every
// element lives in a register after unrolling.  The Lie algebra is spanned by
// T^a = lambda^a / 2 (Gell-Mann); an element is stored as its 8 real
// components X^a = 2 tr(X T^a) (App. B of arXiv:2303.05599).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace gl {

template <typename R>
struct M3 {
    R re[3][3];
    R im[3][3];
};

template <typename R>
struct A8 {
    R v[8];
};

template <typename R>
__host__ __device__ __forceinline__ R inv_sqrt3() { return R(0.57735026918962576451); }

template <typename R>
__device__ __forceinline__ M3<R> m_zero() {
    M3<R> m;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) { m.re[i][j] = R(0); m.im[i][j] = R(0); }
    return m;
}

template <typename R>
__device__ __forceinline__ M3<R> m_id() {
    M3<R> m = m_zero<R>();
    m.re[0][0] = m.re[1][1] = m.re[2][2] = R(1);
    return m;
}

// c = a b
template <typename R>
__device__ __forceinline__ M3<R> mul(const M3<R>& a, const M3<R>& b) {
    M3<R> c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            R sr = R(0), si = R(0);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                sr = fma(a.re[i][k], b.re[k][j], sr);
                sr = fma(-a.im[i][k], b.im[k][j], sr);
                si = fma(a.re[i][k], b.im[k][j], si);
                si = fma(a.im[i][k], b.re[k][j], si);
            }
            c.re[i][j] = sr;
            c.im[i][j] = si;
        }
    return c;
}

// c = a b^+
template <typename R>
__device__ __forceinline__ M3<R> mul_nd(const M3<R>& a, const M3<R>& b) {
    M3<R> c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            R sr = R(0), si = R(0);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                // a_ik conj(b_jk)
                sr = fma(a.re[i][k], b.re[j][k], sr);
                sr = fma(a.im[i][k], b.im[j][k], sr);
                si = fma(a.im[i][k], b.re[j][k], si);
                si = fma(-a.re[i][k], b.im[j][k], si);
            }
            c.re[i][j] = sr;
            c.im[i][j] = si;
        }
    return c;
}

// c = a^+ b
template <typename R>
__device__ __forceinline__ M3<R> mul_dn(const M3<R>& a, const M3<R>& b) {
    M3<R> c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            R sr = R(0), si = R(0);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                // conj(a_ki) b_kj
                sr = fma(a.re[k][i], b.re[k][j], sr);
                sr = fma(a.im[k][i], b.im[k][j], sr);
                si = fma(a.re[k][i], b.im[k][j], si);
                si = fma(-a.im[k][i], b.re[k][j], si);
            }
            c.re[i][j] = sr;
            c.im[i][j] = si;
        }
    return c;
}

template <typename R>
__device__ __forceinline__ M3<R> dag(const M3<R>& a) {
    M3<R> c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) { c.re[i][j] = a.re[j][i]; c.im[i][j] = -a.im[j][i]; }
    return c;
}

template <typename R>
__device__ __forceinline__ M3<R> add(const M3<R>& a, const M3<R>& b) {
    M3<R> c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) { c.re[i][j] = a.re[i][j] + b.re[i][j]; c.im[i][j] = a.im[i][j] + b.im[i][j]; }
    return c;
}

template <typename R>
__device__ __forceinline__ M3<R> sub(const M3<R>& a, const M3<R>& b) {
    M3<R> c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) { c.re[i][j] = a.re[i][j] - b.re[i][j]; c.im[i][j] = a.im[i][j] - b.im[i][j]; }
    return c;
}

// Hermitian matrix X = sum_a x^a T^a
template <typename R>
__device__ __forceinline__ M3<R> alg_to_mat(const A8<R>& x) {
    const R h = R(0.5), s3 = inv_sqrt3<R>();
    M3<R> m;
    m.re[0][0] = h * (x.v[2] + x.v[7] * s3); m.im[0][0] = R(0);
    m.re[1][1] = h * (-x.v[2] + x.v[7] * s3); m.im[1][1] = R(0);
    m.re[2][2] = -x.v[7] * s3; m.im[2][2] = R(0);
    m.re[0][1] = h * x.v[0]; m.im[0][1] = -h * x.v[1];
    m.re[1][0] = h * x.v[0]; m.im[1][0] = h * x.v[1];
    m.re[0][2] = h * x.v[3]; m.im[0][2] = -h * x.v[4];
    m.re[2][0] = h * x.v[3]; m.im[2][0] = h * x.v[4];
    m.re[1][2] = h * x.v[5]; m.im[1][2] = -h * x.v[6];
    m.re[2][1] = h * x.v[5]; m.im[2][1] = h * x.v[6];
    return m;
}

// components x^a = 2 Re tr(X T^a) of the traceless part of a Hermitian X
template <typename R>
__device__ __forceinline__ A8<R> herm_to_alg(const M3<R>& X) {
    A8<R> x;
    x.v[0] = X.re[0][1] + X.re[1][0];
    x.v[1] = X.im[1][0] - X.im[0][1];
    x.v[2] = X.re[0][0] - X.re[1][1];
    x.v[3] = X.re[0][2] + X.re[2][0];
    x.v[4] = X.im[2][0] - X.im[0][2];
    x.v[5] = X.re[1][2] + X.re[2][1];
    x.v[6] = X.im[2][1] - X.im[1][2];
    x.v[7] = (X.re[0][0] + X.re[1][1] - R(2) * X.re[2][2]) * inv_sqrt3<R>();
    return x;
}

// components of the Hermitian traceless matrix i [M]_ah, with
// [M]_ah = (M - M^+)/2 - tr(M - M^+)/6  (anti-Hermitian traceless part)
template <typename R>
__device__ __forceinline__ A8<R> iah_to_alg(const M3<R>& M) {
    A8<R> x;
    x.v[0] = -(M.im[0][1] + M.im[1][0]);
    x.v[1] = M.re[1][0] - M.re[0][1];
    x.v[2] = M.im[1][1] - M.im[0][0];
    x.v[3] = -(M.im[0][2] + M.im[2][0]);
    x.v[4] = M.re[2][0] - M.re[0][2];
    x.v[5] = -(M.im[1][2] + M.im[2][1]);
    x.v[6] = M.re[2][1] - M.re[1][2];
    x.v[7] = (R(2) * M.im[2][2] - M.im[0][0] - M.im[1][1]) * inv_sqrt3<R>();
    return x;
}

template <typename R>
__device__ __forceinline__ void cmul(R ar, R ai, R br, R bi, R& cr, R& ci) {
    cr = ar * br - ai * bi;
    ci = ar * bi + ai * br;
}

template <typename R>
__device__ __forceinline__ A8<R> a_zero() {
    A8<R> x;
#pragma unroll
    for (int a = 0; a < 8; a++) x.v[a] = R(0);
    return x;
}

template <typename R>
__device__ __forceinline__ R a_dot(const A8<R>& p, const A8<R>& q) {
    R s = R(0);
#pragma unroll
    for (int a = 0; a < 8; a++) s = fma(p.v[a], q.v[a], s);
    return s;
}

// U X U^+ for Hermitian X, as algebra components
template <typename R>
__device__ __forceinline__ A8<R> adj(const M3<R>& U, const A8<R>& x) {
    return herm_to_alg(mul_nd(mul(U, alg_to_mat(x)), U));
}

// U^+ X U for Hermitian X, as algebra components
template <typename R>
__device__ __forceinline__ A8<R> adj_dag(const M3<R>& U, const A8<R>& x) {
    return herm_to_alg(mul(mul_dn(U, alg_to_mat(x)), U));
}

// 2 X for X = sum_a x^a T^a: the off-diagonal entries are the components
// themselves (no factor 1/2)
template <typename R>
__device__ __forceinline__ M3<R> alg_to_mat2(const A8<R>& x) {
    const R s3 = inv_sqrt3<R>();
    M3<R> m;
    m.re[0][0] = x.v[2] + x.v[7] * s3; m.im[0][0] = R(0);
    m.re[1][1] = -x.v[2] + x.v[7] * s3; m.im[1][1] = R(0);
    m.re[2][2] = R(-2) * (x.v[7] * s3); m.im[2][2] = R(0);
    m.re[0][1] = x.v[0]; m.im[0][1] = -x.v[1];
    m.re[1][0] = x.v[0]; m.im[1][0] = x.v[1];
    m.re[0][2] = x.v[3]; m.im[0][2] = -x.v[4];
    m.re[2][0] = x.v[3]; m.im[2][0] = x.v[4];
    m.re[1][2] = x.v[5]; m.im[1][2] = -x.v[6];
    m.re[2][1] = x.v[5]; m.im[2][1] = x.v[6];
    return m;
}

// components of V^+ X V for Hermitian X (only the upper triangle of the
// Hermitian result is formed).  The product is taken of 2 X, so that the
// off-diagonal components need no factor 2 and the diagonal ones a factor
// 1/2; scaling by powers of 2 is exact, so the result is bitwise that of X.
template <typename R>
__device__ __forceinline__ A8<R> conj_dn(const M3<R>& V, const A8<R>& x) {
    const M3<R> X = alg_to_mat2(x);
    M3<R> Y;  // X V, with X's diagonal real
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            R sr = X.re[i][i] * V.re[i][j], si = X.re[i][i] * V.im[i][j];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (k == i) continue;
                sr = fma(X.re[i][k], V.re[k][j], sr);
                sr = fma(-X.im[i][k], V.im[k][j], sr);
                si = fma(X.re[i][k], V.im[k][j], si);
                si = fma(X.im[i][k], V.re[k][j], si);
            }
            Y.re[i][j] = sr;
            Y.im[i][j] = si;
        }
    R zr[3][3], zi[3][3];  // V^+ Y, upper triangle
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = i; j < 3; j++) {
            R sr = R(0), si = R(0);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                sr = fma(V.re[k][i], Y.re[k][j], sr);
                sr = fma(V.im[k][i], Y.im[k][j], sr);
                if (i != j) {
                    si = fma(V.re[k][i], Y.im[k][j], si);
                    si = fma(-V.im[k][i], Y.re[k][j], si);
                }
            }
            zr[i][j] = sr;
            zi[i][j] = si;
        }
    A8<R> o;
    o.v[0] = zr[0][1];
    o.v[1] = -zi[0][1];
    o.v[2] = R(0.5) * (zr[0][0] - zr[1][1]);
    o.v[3] = zr[0][2];
    o.v[4] = -zi[0][2];
    o.v[5] = zr[1][2];
    o.v[6] = -zi[1][2];
    o.v[7] = (zr[0][0] + zr[1][1] - R(2) * zr[2][2]) * (R(0.5) * inv_sqrt3<R>());
    return o;
}

// conj_dn for the field step, where the transports are the bulk of the
// arithmetic.  V^+ X V is traceless like X, so the (2, 2) entry is not formed:
// the eighth component follows from the first two diagonal entries (the same
// value up to rounding).  Rows 0 and 1 of the result, all that is left to
// form, are rows 0 and 1 of W = V^+ (2X) times V, so the product is
// associated that way and only two rows of W are formed: six entries instead
// of the nine of (2X) V, about 108 multiply-adds instead of 138.
template <typename R>
__device__ __forceinline__ A8<R> conj_dn_t(const M3<R>& V, const A8<R>& x) {
    const M3<R> X = alg_to_mat2(x);
    R wr[2][3], wi[2][3];  // W = V^+ X, rows 0 and 1, with X's diagonal real
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            // conj(V_ji) X_jj, then conj(V_ki) X_kj for k != j
            R sr = V.re[j][i] * X.re[j][j], si = -(V.im[j][i] * X.re[j][j]);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (k == j) continue;
                sr = fma(V.re[k][i], X.re[k][j], sr);
                sr = fma(V.im[k][i], X.im[k][j], sr);
                si = fma(V.re[k][i], X.im[k][j], si);
                si = fma(-V.im[k][i], X.re[k][j], si);
            }
            wr[i][j] = sr;
            wi[i][j] = si;
        }
    R zr[2][3], zi[2][3];  // Z = W V, upper triangle of rows 0 and 1
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = i; j < 3; j++) {
            R sr = R(0), si = R(0);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                sr = fma(wr[i][k], V.re[k][j], sr);
                sr = fma(-wi[i][k], V.im[k][j], sr);
                if (i != j) {
                    si = fma(wr[i][k], V.im[k][j], si);
                    si = fma(wi[i][k], V.re[k][j], si);
                }
            }
            zr[i][j] = sr;
            zi[i][j] = si;
        }
    A8<R> o;
    o.v[0] = zr[0][1];
    o.v[1] = -zi[0][1];
    o.v[2] = R(0.5) * (zr[0][0] - zr[1][1]);
    o.v[3] = zr[0][2];
    o.v[4] = -zi[0][2];
    o.v[5] = zr[1][2];
    o.v[6] = -zi[1][2];
    // (Z00 + Z11 - 2 Z22) / sqrt 3 with Z22 = -(Z00 + Z11), halved for 2X
    o.v[7] = (zr[0][0] + zr[1][1]) * R(0.86602540378443864676);
    return o;
}

// components of V X V^+ for Hermitian X
template <typename R>
__device__ __forceinline__ A8<R> conj_up(const M3<R>& V, const A8<R>& x) {
    return conj_dn(dag(V), x);
}
template <typename R>
__device__ __forceinline__ A8<R> conj_up_t(const M3<R>& V, const A8<R>& x) {
    return conj_dn_t(dag(V), x);
}

// X^2 for Hermitian X: the upper triangle is formed, the lower one mirrored
template <typename R>
__device__ __forceinline__ M3<R> sq_herm(const M3<R>& X) {
    M3<R> Z;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = i; j < 3; j++) {
            R sr = R(0), si = R(0);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                sr = fma(X.re[i][k], X.re[k][j], sr);
                sr = fma(-X.im[i][k], X.im[k][j], sr);
                if (i != j) {
                    si = fma(X.re[i][k], X.im[k][j], si);
                    si = fma(X.im[i][k], X.re[k][j], si);
                }
            }
            Z.re[i][j] = sr;
            Z.im[i][j] = si;
            Z.re[j][i] = sr;
            Z.im[j][i] = -si;
        }
#pragma unroll
    for (int i = 0; i < 3; i++) Z.im[i][i] = R(0);
    return Z;
}

// components of i[A B^+]_ah without forming the whole product: only the
// imaginary parts of the diagonal and both triangles are needed
template <typename R>
__device__ __forceinline__ A8<R> iah_of_mul_nd(const M3<R>& A, const M3<R>& B) {
    R dr[3][3], di[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            R sr = R(0), si = R(0);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                // A_ik conj(B_jk)
                if (i != j) {
                    sr = fma(A.re[i][k], B.re[j][k], sr);
                    sr = fma(A.im[i][k], B.im[j][k], sr);
                }
                si = fma(A.im[i][k], B.re[j][k], si);
                si = fma(-A.re[i][k], B.im[j][k], si);
            }
            dr[i][j] = sr;
            di[i][j] = si;
        }
    A8<R> x;
    x.v[0] = -(di[0][1] + di[1][0]);
    x.v[1] = dr[1][0] - dr[0][1];
    x.v[2] = di[1][1] - di[0][0];
    x.v[3] = -(di[0][2] + di[2][0]);
    x.v[4] = dr[2][0] - dr[0][2];
    x.v[5] = -(di[1][2] + di[2][1]);
    x.v[6] = dr[2][1] - dr[1][2];
    x.v[7] = (R(2) * di[2][2] - di[0][0] - di[1][1]) * inv_sqrt3<R>();
    return x;
}

// cubic Casimir q3 = d_abc Q^a Q^b Q^c from the 16 independent nonzero
// symmetric structure constants of SU(3) (Table II), each weighted by the
// number of distinct index orderings
template <typename R>
__device__ __forceinline__ R casimir3(const A8<R>& q) {
    const R s3 = inv_sqrt3<R>();  // 1/sqrt(3)
    const R* Q = q.v;             // Q[0] = Q^1 ... Q[7] = Q^8
    const R h = R(0.5);
    R r = R(3) * s3 * (Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2]) * Q[7]    // d118, d228, d338
        + R(6) * h * (Q[0] * Q[3] * Q[5] + Q[0] * Q[4] * Q[6]             // d146, d157
                      - Q[1] * Q[3] * Q[6] + Q[1] * Q[4] * Q[5])          // d247, d256
        + R(3) * h * Q[2] * (Q[3] * Q[3] + Q[4] * Q[4] - Q[5] * Q[5] - Q[6] * Q[6])  // d344 d355 d366 d377
        - R(3) * h * s3 * (Q[3] * Q[3] + Q[4] * Q[4] + Q[5] * Q[5] + Q[6] * Q[6]) * Q[7]  // d448..d778
        - s3 * Q[7] * Q[7] * Q[7];                                           // d888
    return r;
}

// exp(i s X) for Hermitian traceless X = x^a T^a.  Cayley-Hamilton gives
// X^3 = c1 X + c0 with c1 = tr(X^2)/2 and c0 = det X, so every power of iX
// is a combination of 1, X, X^2; the exponential series is summed on those
// three scalar coefficients (scaling and squaring when |sX| > 1).
template <typename R, int TERMS>
__device__ __forceinline__ M3<R> exp_i_alg(const A8<R>& x, R s) {
    // s X: 2 X from the components, times s / 2 (exact: a power of 2), one
    // product per distinct entry
    M3<R> X = alg_to_mat2(x);
    const R hs = R(0.5) * s;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        X.re[i][i] *= hs;
#pragma unroll
        for (int j = i + 1; j < 3; j++) {
            X.re[i][j] *= hs;
            X.im[i][j] *= hs;
            X.re[j][i] = X.re[i][j];
            X.im[j][i] = -X.im[i][j];
        }
    }
    M3<R> X2 = sq_herm(X);
    R c1 = R(0.5) * (X2.re[0][0] + X2.re[1][1] + X2.re[2][2]);
    int nsq = 0;
    R scl = R(1);
    // Frobenius norm^2 of X is 2 c1; scale until the truncated series is
    // accurate: |X| <= 1 with 12 or more terms, |X| <= 0.5 with 8 to 11,
    // |X| <= 0.2 with fewer (truncation error below 1e-8 in each case)
    const R lim = TERMS >= 12 ? R(1) : (TERMS >= 8 ? R(0.25) : R(0.04));
    R nrm2 = R(2) * c1;
    while (nrm2 > lim && nsq < 30) { nrm2 *= R(0.25); scl *= R(0.5); nsq++; }
    if (nsq) {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                X.re[i][j] *= scl; X.im[i][j] *= scl;
                X2.re[i][j] *= scl * scl; X2.im[i][j] *= scl * scl;
            }
        c1 *= scl * scl;
    }
    // det X of Hermitian X (real diagonal, X_ji = conj X_ij): x00 x11 x22
    // + 2 Re(x01 x12 conj x02) - x00 |x12|^2 - x11 |x02|^2 - x22 |x01|^2
    const R pr = X.re[0][1] * X.re[1][2] - X.im[0][1] * X.im[1][2];
    const R pi_ = X.re[0][1] * X.im[1][2] + X.im[0][1] * X.re[1][2];
    const R n01 = X.re[0][1] * X.re[0][1] + X.im[0][1] * X.im[0][1];
    const R n02 = X.re[0][2] * X.re[0][2] + X.im[0][2] * X.im[0][2];
    const R n12 = X.re[1][2] * X.re[1][2] + X.im[1][2] * X.im[1][2];
    const R c0 = X.re[0][0] * (X.re[1][1] * X.re[2][2] - n12) - X.re[1][1] * n02 - X.re[2][2] * n01 +
                 R(2) * (pr * X.re[0][2] + pi_ * X.im[0][2]);
    // (iX)^k / k! = i^k (a_k + b_k X + g_k X^2) with real a, b, g: from
    // X^3 = c1 X + c0, a_{k+1} = c0 g_k / (k+1), b_{k+1} = (a_k + c1 g_k) /
    // (k+1), g_{k+1} = b_k / (k+1).  The factor i^k only decides, at compile
    // time, which part of the complex sums f0, f1, f2 a term enters, and with
    // which sign.
    R a = R(1), b = R(0), g = R(0);
    R f0r = R(1), f0i = R(0), f1r = R(0), f1i = R(0), f2r = R(0), f2i = R(0);
#pragma unroll
    for (int k = 1; k <= TERMS; k++) {
        const R inv = R(1) / R(k);
        const R na = c0 * g * inv, nb = (a + c1 * g) * inv, ng = b * inv;
        a = na; b = nb; g = ng;
        if ((k & 3) == 1) { f0i += a; f1i += b; f2i += g; }
        else if ((k & 3) == 2) { f0r -= a; f1r -= b; f2r -= g; }
        else if ((k & 3) == 3) { f0i -= a; f1i -= b; f2i -= g; }
        else { f0r += a; f1r += b; f2r += g; }
    }
    M3<R> U;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const R d = (i == j) ? R(1) : R(0);
            // (f0 + f1 X + f2 X2)_ij, complex coefficients
            U.re[i][j] = f0r * d + f1r * X.re[i][j] - f1i * X.im[i][j] + f2r * X2.re[i][j] - f2i * X2.im[i][j];
            U.im[i][j] = f0i * d + f1r * X.im[i][j] + f1i * X.re[i][j] + f2r * X2.im[i][j] + f2i * X2.re[i][j];
        }
    for (int k = 0; k < nsq; k++) U = mul(U, U);
    return U;
}

// third row of an SU(3) matrix from the first two: u_2 = conj(u_0 x u_1)
template <typename R>
__device__ __forceinline__ void rebuild_row2(M3<R>& u) {
#define GL_CX(ar, ai, br, bi, cr, ci, dr, di) ((ar) * (br) - (ai) * (bi) - ((cr) * (dr) - (ci) * (di)))
#define GL_CY(ar, ai, br, bi, cr, ci, dr, di) ((ar) * (bi) + (ai) * (br) - ((cr) * (di) + (ci) * (dr)))
    // u20 = conj(u01 u12 - u02 u11)
    u.re[2][0] = GL_CX(u.re[0][1], u.im[0][1], u.re[1][2], u.im[1][2], u.re[0][2], u.im[0][2], u.re[1][1], u.im[1][1]);
    u.im[2][0] = -GL_CY(u.re[0][1], u.im[0][1], u.re[1][2], u.im[1][2], u.re[0][2], u.im[0][2], u.re[1][1], u.im[1][1]);
    // u21 = conj(u02 u10 - u00 u12)
    u.re[2][1] = GL_CX(u.re[0][2], u.im[0][2], u.re[1][0], u.im[1][0], u.re[0][0], u.im[0][0], u.re[1][2], u.im[1][2]);
    u.im[2][1] = -GL_CY(u.re[0][2], u.im[0][2], u.re[1][0], u.im[1][0], u.re[0][0], u.im[0][0], u.re[1][2], u.im[1][2]);
    // u22 = conj(u00 u11 - u01 u10)
    u.re[2][2] = GL_CX(u.re[0][0], u.im[0][0], u.re[1][1], u.im[1][1], u.re[0][1], u.im[0][1], u.re[1][0], u.im[1][0]);
    u.im[2][2] = -GL_CY(u.re[0][0], u.im[0][0], u.re[1][1], u.im[1][1], u.re[0][1], u.im[0][1], u.re[1][0], u.im[1][0]);
#undef GL_CX
#undef GL_CY
}

}  // namespace gl
