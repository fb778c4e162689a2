"""Pins of the oracle's Glasma leapfrog (Sec. 2.1) and MV initial conditions:
exact Gauss-law conservation, unitarity, the Abelian single-mode Bessel
solutions with O(dt^2) convergence, a hand-worked 4x4 step, gauge covariance,
and the Poisson / Wilson-line / link-matching construction of the initial state."""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.special

import oracle as O
from tests import helpers as H


def mv_state(N, seed=0, g2mu_a=0.95, m_a=0.095, Ns=8):
    st, bad = O.mv_init(N, Ns, g2mu_a, m_a, 10.0, seed)
    assert bad == 0
    return st


def test_gauss_law_exact_and_unitarity():
    st = mv_state(16)
    dt = 0.125
    scale = np.abs(st.pi).max()
    worst = 0.0
    for n in range(60):
        st = O.field_step(st, n * dt, dt)
        worst = max(worst, np.abs(O.gauss(st)).max())
    assert worst < 1e-13 * max(1.0, scale)
    u, d = O.unitarity(st)
    assert u < 1e-13 and d < 1e-13
    # the evolution does something: electric fields grew from zero
    assert np.abs(st.e).max() > 1e-2


def _scalar_mode(N, nx, dt, steps, eps=1e-4):
    V = N * N
    xs = np.arange(V) % N
    st = O.FieldState(N)
    st.pi[:, 2] = eps * np.cos(2 * math.pi * nx * xs / N)
    for n in range(steps):
        st = O.field_step(st, n * dt, dt)
    k = 2 * math.sin(math.pi * nx / N)
    t_half = (steps - 0.5) * dt
    return st.pi[0, 2] / eps - scipy.special.j0(k * t_half)


def test_bessel_scalar_mode_second_order():
    # linearised boost-invariant scalar: E_eta = pi ~ J0(k t) with lattice k
    e1 = _scalar_mode(16, 2, 0.125, 160)
    e2 = _scalar_mode(16, 2, 0.0625, 320)
    assert abs(e1) < 3e-3
    assert 3.0 < abs(e1 / e2) < 5.0  # O(dt^2)


def _transverse_mode(N, my, dt, steps, eps=1e-4):
    V = N * N
    ys = np.arange(V) // N
    u = H.links(O.unit_links(N)).copy()
    for s in range(V):
        u[0, s] = scipy.linalg.expm(1j * H.alg2mat(np.array([0, 0, eps * math.cos(2 * math.pi * my * ys[s] / N), 0, 0, 0, 0, 0])))
    st = O.FieldState(N, H.links_to_canon(u))
    probe = (N // 4) * N
    k = 2 * math.sin(math.pi * my / N)
    b_ref = None
    for n in range(steps):
        new = O.field_step(st, n * dt, dt)
        site = O.site_fields(st, new, n * dt)
        if n == 0:
            b_ref = site[5, probe, 2]
        st = new
    return site[5, probe, 2] / b_ref - scipy.special.j0(k * (steps - 1) * dt)


def test_bessel_transverse_mode_second_order():
    # linearised transverse field: B_eta ~ J0(k t)
    e1 = _transverse_mode(16, 1, 0.125, 160)
    e2 = _transverse_mode(16, 1, 0.0625, 320)
    assert abs(e1) < 3e-3
    assert 3.0 < abs(e1 / e2) < 5.0


def _diag(c3, c8):
    return np.array([c3 / 2 + c8 / (2 * math.sqrt(3)), -c3 / 2 + c8 / (2 * math.sqrt(3)), -c8 / math.sqrt(3)])


def test_hand_worked_single_link_4x4():
    # One link U_x(0,0) = exp(i theta T^3), all else trivial, t = 1, dt = 1/8.
    # Both plaquettes containing it carry the phases (theta/2, -theta/2, 0), so
    # each contributes i t [.]_ah = -t sin(theta/2) diag(1,-1,0) to the force:
    #   e_x(0,0)^3 = -4 t dt sin(theta/2),  e_x(0,1)^3 = +2 t dt sin(theta/2),
    #   e_y(0,0)^3 = +2 t dt sin(theta/2),  e_y(1,0)^3 = -2 t dt sin(theta/2).
    N, theta, t, dt = 4, 0.3, 1.0, 0.125
    u = H.links(O.unit_links(N)).copy()
    u[0, 0] = np.diag(np.exp(1j * _diag(theta, 0.0)))
    st = O.FieldState(N, H.links_to_canon(u))
    new = O.field_step(st, t, dt)
    s = 2 * t * dt * math.sin(theta / 2)
    assert abs(new.e[0, 0, 2] + 2 * s) < 1e-15
    assert abs(new.e[0, 1 * N + 0, 2] - s) < 1e-15
    assert abs(new.e[1, 0, 2] - s) < 1e-15
    assert abs(new.e[1, 1, 2] + s) < 1e-15
    assert abs(new.e[0, 2 * N + 2]).max() == 0.0


def test_hand_worked_abelian_4x4_random_angles():
    # Cartan-diagonal links and scalar: every plaquette is a diagonal phase and
    # the step reduces to compact U(1)^2 arithmetic on the angles, done here in
    # plain scalars.
    N, t, dt = 4, 1.7, 0.125
    V = N * N
    rng = np.random.default_rng(11)
    c = rng.normal(size=(2, V, 2)) * 0.7       # (c3, c8) per link
    ph = rng.normal(size=(V, 2)) * 0.5
    e = rng.normal(size=(2, V, 2)) * 0.3
    pi = rng.normal(size=(V, 2)) * 0.3
    th = np.array([[_diag(*c[d, s]) for s in range(V)] for d in range(2)])  # phases [2, V, 3]

    def full(a2):
        out = np.zeros(a2.shape[:-1] + (8,))
        out[..., 2] = a2[..., 0]
        out[..., 7] = a2[..., 1]
        return out

    u = np.zeros((2, V, 3, 3), dtype=np.complex128)
    for d in range(2):
        for s in range(V):
            u[d, s] = np.diag(np.exp(1j * th[d, s]))
    st = O.FieldState(N, H.links_to_canon(u), full(ph), full(e), full(pi))
    new = O.field_step(st, t, dt)

    def S(s, dx, dy):
        return H.shift(N, s, dx, dy)

    th_h = t + dt / 2
    for s in range(V):
        for d in range(2):
            o = 1 - d
            dxi, dyi = (1, 0) if d == 0 else (0, 1)
            dxj, dyj = (0, 1) if d == 0 else (1, 0)
            up = th[d, s] + th[o, S(s, dxi, dyi)] - th[d, S(s, dxj, dyj)] - th[o, s]
            dn = th[d, s] - th[o, S(s, dxi - dxj, dyi - dyj)] - th[d, S(s, -dxj, -dyj)] + th[o, S(s, -dxj, -dyj)]
            sn = np.sin(up) + np.sin(dn)
            force = -t * (sn - sn.mean())
            ediag = np.array([(e[d, s, 0] / 2 + e[d, s, 1] / (2 * math.sqrt(3))),
                              (-e[d, s, 0] / 2 + e[d, s, 1] / (2 * math.sqrt(3))),
                              -e[d, s, 1] / math.sqrt(3)]) + dt * force
            e3 = ediag[0] - ediag[1]
            e8 = (ediag[0] + ediag[1] - 2 * ediag[2]) / math.sqrt(3)
            assert abs(new.e[d, s, 2] - e3) < 1e-14
            assert abs(new.e[d, s, 7] - e8) < 1e-14
            assert np.abs(np.delete(new.e[d, s], [2, 7])).max() < 1e-15
            newphase = th[d, s] + dt / th_h * ediag
            assert np.abs(H.links(new.U)[d, s] - np.diag(np.exp(1j * newphase))).max() < 1e-14
        lap = -4 * ph[s] + ph[S(s, 1, 0)] + ph[S(s, -1, 0)] + ph[S(s, 0, 1)] + ph[S(s, 0, -1)]
        pin = pi[s] + dt / t * lap
        assert np.abs(new.pi[s, [2, 7]] - pin).max() < 1e-14
        assert np.abs(new.phi[s, [2, 7]] - (ph[s] + dt * th_h * pin)).max() < 1e-14


def test_gauge_covariance_of_step_and_site_fields():
    N = 8
    rng = np.random.default_rng(2)
    st = mv_state(N)
    dt = 0.125
    for n in range(10):
        st = O.field_step(st, n * dt, dt)
    t = 10 * dt
    Om = H.random_su3(rng, N * N)
    g = O.FieldState(N, *H.gauge_transform(N, st.U, st.phi, st.e, st.pi, Om))
    a = O.field_step(st, t, dt)
    b = O.field_step(g, t, dt)
    ga = O.FieldState(N, *H.gauge_transform(N, a.U, a.phi, a.e, a.pi, Om))
    for x, y in [(ga.U, b.U), (ga.phi, b.phi), (ga.e, b.e), (ga.pi, b.pi)]:
        assert np.abs(x - y).max() < 1e-12
    sa = O.site_fields(st, a, t)
    sb = O.site_fields(g, b, t)
    Od = Om.conj().transpose(0, 2, 1)
    for k in range(6):
        assert np.abs(H.mat2alg(Om @ H.alg2mat(sa[k]) @ Od) - sb[k]).max() < 1e-12


def test_uniform_abelian_E_eta_is_static():
    # uniform Cartan pi with trivial links: D^2 phi = 0 and all commutators
    # vanish, so E_eta stays exactly constant while phi = E t^2 / 2 grows
    N, dt = 4, 0.125
    st = O.FieldState(N)
    st.pi[:, 7] = 0.3
    for n in range(20):
        st = O.field_step(st, n * dt, dt)
    assert np.abs(st.pi[:, 7] - 0.3).max() < 1e-15
    assert np.abs(st.phi[:, 7] - 0.3 * (20 * dt) ** 2 / 2).max() < 1e-14
    assert np.abs(st.e).max() == 0.0


def test_site_E_is_P_over_t_in_a_uniform_abelian_field():
    # Sec. 3.2 defines the site field as E_i = P^i / tau.  In lattice units
    # that is e_i / t; for a field uniform in space and time it must hold
    # exactly, whatever the interpolation.  Cartan-diagonal links (random,
    # non-uniform) commute with a Cartan e, so the transport of the backward
    # link momentum is exact too.  Different e at n -+ 1/2 give their mean.
    N, t = 6, 2.3
    V = N * N
    rng = np.random.default_rng(3)
    u = np.zeros((2, V, 3, 3), dtype=np.complex128)
    for d in range(2):
        for s in range(V):
            u[d, s] = np.diag(np.exp(1j * _diag(*rng.normal(size=2))))
    e_old = np.zeros((2, V, 8))
    e_new = np.zeros((2, V, 8))
    e_old[0, :, 2], e_old[0, :, 7] = 0.37, -0.21
    e_new[0, :, 2], e_new[0, :, 7] = 0.41, -0.19
    e_old[1, :, 2] = e_new[1, :, 2] = -0.53
    old = O.FieldState(N, H.links_to_canon(u), None, e_old, None)
    new = O.FieldState(N, H.links_to_canon(u), None, e_new, None)
    site = O.site_fields(old, new, t)
    assert np.abs(site[0, :, 2] - 0.39 / t).max() < 1e-15
    assert np.abs(site[0, :, 7] - (-0.20) / t).max() < 1e-15
    assert np.abs(site[1, :, 2] - (-0.53) / t).max() < 1e-15
    for a in (0, 1, 3, 4, 5, 6):
        assert np.abs(site[0:2, :, a]).max() < 1e-16


def _rho_python(N, Ns, sigma, seed, nucleus, sheet):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    rho = np.zeros((8, N * N))
    for s in range(N * N):
        z = []
        for j in range(2):
            w = H.philox([s, (nucleus * Ns + sheet) * 2 + j, 1, 0], key)
            z += list(H.box_muller(H.u01(w[0]), H.u01(w[1]))) + list(H.box_muller(H.u01(w[2]), H.u01(w[3])))
        rho[:, s] = sigma * np.array(z)
    return rho


def test_wilson_lines_from_poisson_solution():
    # V^+ = exp(-i alpha_1) exp(-i alpha_2) with (-Lap + m^2) alpha_n = rho_n,
    # zero mode removed and |k| > Lambda cut; solved here with numpy's FFT
    N, Ns, g2mu_a, m_a, Lam, seed = 8, 2, 0.8, 0.1, 2.5, 3
    vd = O.wilson_lines(N, Ns, g2mu_a, m_a, Lam, seed, 1).view(np.complex128).reshape(-1, 3, 3)
    k = 2 * np.sin(np.pi * np.arange(N) / N)
    k2 = k[None, :] ** 2 + k[:, None] ** 2
    G = 1.0 / (k2 + m_a ** 2)
    G[0, 0] = 0.0
    G[k2 > Lam ** 2] = 0.0
    want = np.broadcast_to(np.eye(3, dtype=np.complex128), (N * N, 3, 3)).copy()
    for sheet in range(Ns):
        rho = _rho_python(N, Ns, g2mu_a / math.sqrt(Ns), seed, 1, sheet)
        alpha = np.stack([np.fft.ifft2(np.fft.fft2(rho[a].reshape(N, N)) * G).real.reshape(-1) for a in range(8)], 1)
        for s in range(N * N):
            want[s] = want[s] @ scipy.linalg.expm(-1j * H.alg2mat(alpha[s]))
    assert np.abs(vd - want).max() < 1e-12


def test_link_matching_abelian_and_residual():
    rng = np.random.default_rng(4)
    # commuting (diagonal) nuclear links: the Glasma link is their product
    a = np.diag(np.exp(1j * _diag(0.4, -0.2)))
    b = np.diag(np.exp(1j * _diag(-0.1, 0.5)))
    u, bad = O.solve_link(a.reshape(-1).view(np.float64), b.reshape(-1).view(np.float64))
    assert bad == 0
    assert np.abs(u.view(np.complex128).reshape(3, 3) - a @ b).max() < 1e-13
    # general: residual tr(T^a [(UA + UB)(1 + U^+) - h.c.]) = 0 and U in SU(3)
    for _ in range(5):
        A = H.random_su3(rng, 1, 0.6)[0]
        B = H.random_su3(rng, 1, 0.6)[0]
        u, bad = O.solve_link(A.reshape(-1).view(np.float64), B.reshape(-1).view(np.float64))
        U = u.view(np.complex128).reshape(3, 3)
        M = (A + B) @ (np.eye(3) + U.conj().T)
        assert bad == 0
        assert np.abs(np.einsum("aij,ji->a", H.T, M - M.conj().T)).max() < 1e-12
        assert np.abs(U @ U.conj().T - np.eye(3)).max() < 1e-13
        assert abs(np.linalg.det(U) - 1) < 1e-13


def test_mv_init_gauss_zero_and_links_unitary():
    # at tau = 0 the Gauss residual is exactly 0 (e = phi = 0); the links are
    # SU(3) and the initial E_eta is not trivially zero
    st = mv_state(8)
    assert np.abs(O.gauss(st)).max() == 0.0
    assert np.abs(st.pi).max() > 1e-3
    u, d = O.unitarity(st)
    assert u < 1e-13 and d < 1e-13


def _poisson(rho, N, m_a, Lam):
    k = 2 * np.sin(np.pi * np.arange(N) / N)
    k2 = k[None, :] ** 2 + k[:, None] ** 2
    G = 1.0 / (k2 + m_a ** 2)
    G[0, 0] = 0.0
    G[k2 > Lam ** 2] = 0.0
    return np.stack([np.fft.ifft2(np.fft.fft2(rho[a].reshape(N, N)) * G).real.reshape(-1) for a in range(8)], 1)


def _E_eta_weak_field(N, alpha_A, alpha_B):
    """-i sum_i [d_i alpha_A, d_i alpha_B] on the lattice, the commutators of
    the forward and the backward differences averaged at each site."""
    s = np.arange(N * N)
    A = H.alg2mat(alpha_A)
    B = H.alg2mat(alpha_B)
    out = np.zeros((N * N, 3, 3), dtype=np.complex128)
    for dx, dy in ((1, 0), (0, 1)):
        fw = H.shift(N, s, dx, dy)
        dA = A[fw] - A
        dB = B[fw] - B
        c = dA @ dB - dB @ dA                 # forward difference commutator at x
        out += 0.5 * (c + c[H.shift(N, s, -dx, -dy)])  # and the backward one (at x - i)
    return H.mat2alg(-1j * out)


def test_mv_init_E_eta_weak_field_limit():
    # Initial condition of Sec. 2: A^eta(0) = (ig/2)[alpha_A^i, alpha_B^i] with
    # P^eta = (1/tau) d_tau A_eta and A_eta = -tau^2 A^eta gives
    # E_eta(0) = -ig [alpha_A^i, alpha_B^i].  For one colour sheet per nucleus
    # scaled by eps, the pure-gauge fields are alpha^i = -d_i Lambda + O(eps^2)
    # with Lambda the Poisson solution of each nucleus, so the lattice E_eta(0)
    # must equal -i sum_i [d_i Lambda_A, d_i Lambda_B] up to a relative O(eps).
    # A wrong factor, sign or a dropped average fails at O(1).
    N, m_a, Lam, seed = 8, 0.1, 2.5, 5
    res = []
    for eps in (2e-3, 1e-3):
        st, bad = O.mv_init(N, 1, eps, m_a, Lam, seed)
        assert bad == 0
        la = _poisson(_rho_python(N, 1, eps, seed, 0, 0), N, m_a, Lam)
        lb = _poisson(_rho_python(N, 1, eps, seed, 1, 0), N, m_a, Lam)
        want = _E_eta_weak_field(N, la, lb)
        assert np.abs(want).max() > 1e-3 * eps ** 2   # the commutator is not degenerate
        res.append(np.abs(st.pi - want).max() / np.abs(want).max())
    # relative residual O(eps): small, and halves with eps
    assert res[1] < 2e-2
    assert 1.6 < res[0] / res[1] < 2.4
