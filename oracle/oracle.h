/*
 * FP64 CPU oracle for the colored particle-in-cell (CPIC) Glasma + Wong method
 * (arXiv:2303.05599).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no source, header,
 * table or helper with the CUDA library; neither includes the other.
 *
 * Everything is in lattice units (a = 1):
 *   t = tau/a, dt = dtau/a,
 *   phi = g A_eta                    (Hermitian, 8 algebra components)
 *   pi  = g a^2 P^eta                (Hermitian, at half steps)
 *   e_i = g a P^i                    (Hermitian, on link (x, x+i), at half steps)
 *   site fields  E^ = g a^2 E,  B^ = g a^2 B   (Hermitian, 8 components each)
 *   momenta p^ = p a, mass m^ = m a, P_eta = tau^2 p^eta (dimensionless).
 *
 * Canonical host layouts (all double):
 *   links  U   [2][N*N][18]  direction (x=0, y=1), site s = y*N + x,
 *                            3x3 row-major complex, (re, im) interleaved
 *   phi, pi    [N*N][8]      algebra components X^a = 2 tr(X T^a), T^a = lambda^a/2
 *   e          [2][N*N][8]
 *   site       [6][N*N][8]   E_x, E_y, E_eta, B_x, B_y, B_eta at integer time t_n
 *   particle   [n][16]       x, y, eta, p^x, p^y, P_eta, Q^1..Q^8, pT0^2, species
 *                            (x, y in lattice units in [0, N); static species keep
 *                            the accumulated longitudinal momentum in the P_eta slot)
 *
 * Parity unpinned: none of the functions below.  Each is pinned by a CPU test
 * (tests/test_oracle_algebra.py, test_oracle_field.py, test_oracle_particles.py)
 * against what the paper or the mathematics fixes: closed forms, limiting
 * cases, conservation laws, brute force and printed values.
 */
#ifndef ORACLE_GLASMA_H
#define ORACLE_GLASMA_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- SU(3) algebra (su3.c) -------------------------------------------- */
/* Generators T^a = lambda^a / 2 (Gell-Mann), a = 0..7, as 3x3 complex. */
void or_generator(int a, double* out18);
/* f_abc = -2i tr([T^a,T^b] T^c), d_abc = 2 tr({T^a,T^b} T^c), 0-based. */
double or_f(int a, int b, int c);
double or_d(int a, int b, int c);
/* exp(i X) for Hermitian X given by 8 algebra components; Taylor series with
 * scaling and squaring, summed to machine precision. */
void or_exp_i_alg(const double* x8, double* out18);
/* exp(M) for a general 3x3 complex matrix (same method). */
void or_expm(const double* m18, double* out18);

/* ---- RNG (rng.c) ------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* ---- fields (field.c) -------------------------------------------------- */
/* One leapfrog step n -> n+1 (Eqs. for P^eta, P^i and the link/scalar update
 * of Sec. 2.1).  In: U(n), phi(n), e(n-1/2), pi(n-1/2) at t = t_n.
 * Out: U(n+1), phi(n+1), e(n+1/2), pi(n+1/2).  The 1/t terms are taken as 0
 * at t = 0 (the fields they multiply vanish there). */
void or_field_step(int N, double t, double dt,
                   const double* U, const double* phi, const double* e, const double* pi,
                   double* U1, double* phi1, double* e1, double* pi1);
/* Lattice Gauss residual per site, G(x) = sum_i [e_i(x) - U_i(x-i)^+ e_i(x-i) U_i(x-i)]
 * + i[phi(x), pi(x)], as 8 components -> g[N*N][8]. */
void or_gauss(int N, const double* U, const double* phi, const double* e, const double* pi,
              double* g);
/* Site E and B at t_n (Sec. 3.2 interpolation formulas), out [6][N*N][8]. */
void or_site_fields(int N, double t, const double* U, const double* phi,
                    const double* e_old, const double* e_new,
                    const double* pi_old, const double* pi_new, double* out);
/* Max over links of ||U U^+ - 1||_F and of |det U - 1|. */
void or_unitarity(int N, const double* U, double* max_unit, double* max_det);

/* ---- particles (particles.c) ------------------------------------------ */
/* Initial colour vectors Q0 for the fundamental (rep 0) and adjoint (rep 1)
 * classical charges with q2 = 4, q3 = 10/3 and q2 = 24, q3 = 0. */
void or_q0(int rep, double* q8);
/* q2 = Q^a Q^a, q3 = d_abc Q^a Q^b Q^c. */
void or_casimirs(const double* q8, double* q2, double* q3);
/* Haar-random U(3) from the QR decomposition of a complex Ginibre matrix with
 * the phase fix; g18 = 18 standard normals (real/imag, row-major). */
void or_haar_from_normals(const double* g18, double* out18);
/* Sample n particles of one species (positions, momenta, Haar charges).
 * mom_mode: 0 fixed |pT| = p0 with uniform azimuth; 1 |pT| ~ U[p0, p1] with
 * uniform azimuth; 2 p^x = p0, p^y = 0; 3 zero (eikonal partons record only
 * their kicks).  Momenta in lattice units. */
void or_sample_species(int N, uint64_t seed, int species, int rep, int mom_mode,
                       double p0, double p1, int64_t n, double* out16);
/* Species kinds: Wong particles of finite mass, infinitely massive static
 * quarks (Sec. 5.1), eikonal light-like partons along +x (Sec. 5.2). */
enum { OR_KIND_WONG = 0, OR_KIND_STATIC = 1, OR_KIND_EIKONAL = 2 };
#define OR_MAX_SPECIES 8
/* One Euler + CPIC step of all particles from t_n to t_n + dt.
 * site: site fields at t_n; U1, phi1: links and scalar at t_{n+1}.
 * mass[s], kind[s] per species, active[s] nonzero if species s is active at
 * t_n.  Particle records are updated in place.  Eikonal partons move by dt
 * along +x, keep y and eta, add the kicks dt Q.(E_x, E_y - B_z, E_z + B_y) to
 * p^x, p^y and the P_eta slot, and rotate Q with the crossed x link. */
void or_push_kinds(int N, double t, double dt, const double* site, const double* U1,
                   const double* phi1, int64_t n, double* part, const double* mass,
                   const int* kind, const int* active);
/* or_push_kinds with the kinds from the masses (INFINITY = static, else Wong). */
void or_push(int N, double t, double dt, const double* site, const double* U1,
             const double* phi1, int64_t n, double* part, const double* mass,
             const int* active);
/* Longitudinal momentum p_L = p^z of one particle at time t (lab frame,
 * p^z = p^tau sinh(eta) + tau p^eta cosh(eta)); static and eikonal species
 * return the accumulated value. */
double or_pL_kind(const double* rec16, double t, double mass, int kind);
/* or_pL_kind with the kind from the mass (INFINITY = static). */
double or_pL(const double* rec16, double t, double mass);

/* Temporal constraint: one Euler step of p^tau from its own equation of
 * motion (Sec. 3.1), for the active Wong particles, with the state at t_n
 * (call before or_push_kinds).  ptau[n]: NaN entries are first set to the
 * mass-shell p^tau.  The mass-shell value after the push minus this one is
 * the constraint violation of the temporal-constraint diagnostic. */
void or_ptau_step(int N, double t, double dt, const double* site, int64_t n, const double* part,
                  const double* mass, const int* kind, const int* active, double* ptau);

/* Light-like jet correlator (Sec. 5.2): probe records of OR_JET_LEN doubles,
 * x0, y0, W (3x3 complex, row-major re/im), X_x, X_y, X_z (8 each).  A probe
 * starts at (x0, y0) at tau = 0, moves along +x at the speed of light,
 * multiplies W by each x link it crosses (links at t_{n+1}) and accumulates
 * X_i += dt W f_i W^+ with f = (E_x, E_y - B_z, E_z + B_y) at its cell at
 * t_n.  A parton of charge Q0 on that path receives the kicks Q0 . X_i; the
 * charge-averaged broadening is <dp_i^2> = (q2 / 8) <X_i . X_i>. */
#define OR_JET_LEN 44
/* Probes at uniform positions from Philox counters (j, 0, 4, 0). */
void or_jets_init(int N, uint64_t seed, int64_t n, double* jets);
/* One step of every probe from t_n = t (site fields at t_n, links U1 at t_{n+1}). */
void or_jets_step(int N, double t, double dt, const double* site, const double* U1, int64_t n, double* jets);
/* out3[i] = mean over probes of X_i . X_i. */
void or_jets_obs(int64_t n, const double* jets, double* out3);

/* ---- MV initial conditions (init.c) ------------------------------------ */
/* Wilson lines V^+ of one nucleus (nucleus 0 = A, 1 = B) from Ns sheets of
 * Gaussian colour charge: variance (g2mu_a)^2 / Ns per site and colour,
 * Poisson kernel 1/(k^2 + m^2) with lattice k^2, k = 0 removed, |k| > Lambda
 * removed when Lambda > 0.  out: [N*N][18] (V^+ per site). */
void or_wilson_lines(int N, int Ns, double g2mu_a, double m_a, double Lambda_a,
                     uint64_t seed, int nucleus, double* vdag);
/* Full tau = 0 state: U [2][N*N][18], pi [N*N][8] (phi = e = 0).
 * Returns the number of links whose Newton solve did not converge. */
int or_mv_init(int N, int Ns, double g2mu_a, double m_a, double Lambda_a, uint64_t seed,
               double* U, double* pi);
/* Solve for the Glasma link U from the two pure-gauge links (Newton). */
int or_solve_link(const double* ua18, const double* ub18, double* u18);
/* Plain complex FFT (radix 2 when n is a power of two, else direct DFT),
 * sign = -1 forward, +1 inverse (unnormalised); data interleaved re/im. */
void or_fft(double* data, int n, int sign);

/* ---- observables (obs.c) ---------------------------------------------- */
/* Per-species sums over active particles at time t:
 * out[s*8 + k]: k=0 count, 1 sum px^2, 2 sum py^2, 3 sum pL^2,
 * 4 sum (pT^2 - pT0^2), 5 max |q2 - q2_0|, 6 max |q3 - q3_0|, 7 unused. */
void or_particle_obs(int64_t n, const double* part, double t, const double* mass,
                     const int* kind, const int* active, const int* rep, int n_species, double* out);

/* OpenMP threads used by the site and particle loops. */
int or_threads(void);

#ifdef __cplusplus
}
#endif
#endif
