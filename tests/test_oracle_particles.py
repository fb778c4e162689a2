"""Pins of the oracle's test-particle part: the Haar colour-charge sampler
(Sec. 4.2, App. C), Casimir conservation (App. A), the two limiting cases of
Sec. 5 (static quarks vs the integrated E correlator, light-like jets vs the
transported Lorentz-force correlator), lab-frame closed forms (hyperbolic
motion in a uniform E_eta, cyclotron motion in a uniform B_eta), a conserved
canonical momentum that fixes the B_i components and the rapidity Wilson line,
and gauge covariance of the push."""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle as O
from tests import helpers as H


def mv_state(N, seed=0):
    st, bad = O.mv_init(N, 8, 0.95, 0.095, 10.0, seed)
    assert bad == 0
    return st


# ------------------------------------------------------------------ sampler
@pytest.mark.parametrize("rep,TR,AR", [(0, 0.5, 1.0), (1, 3.0, 0.0)])
def test_haar_n_point_functions(rep, TR, AR):
    n = 200_000
    rec = O.sample_species(32, 12345, 3, rep, 0, 0.0, 0.0, n)
    Q = rec[:, 6:14]
    q2w, q3w = O.casimirs(O.q0(rep))
    # Casimirs fixed per draw
    q2 = (Q * Q).sum(1)
    d = O.d_abc()
    q3 = np.einsum("abc,na,nb,nc->n", d, Q, Q, Q)
    assert np.abs(q2 - q2w).max() < 1e-12
    assert np.abs(q3 - q3w).max() < 1e-11
    # <Q^a> = 0, <Q^a Q^b> = T_R delta^ab, <Q^a Q^b Q^c> = (A_R/4) d^abc (eq. for the n-point functions)
    m1 = Q.mean(0)
    s1 = Q.std(0) / math.sqrt(n)
    assert np.all(np.abs(m1) < 5 * s1)
    P2 = np.einsum("na,nb->nab", Q, Q)
    m2 = P2.mean(0)
    s2 = P2.std(0) / math.sqrt(n)
    assert np.all(np.abs(m2 - TR * np.eye(8)) < 5 * s2 + 1e-12)
    P3 = np.einsum("na,nb,nc->abc", Q, Q, Q) / n
    s3 = np.sqrt(np.einsum("na,nb,nc->abc", Q ** 2, Q ** 2, Q ** 2) / n - P3 ** 2) / math.sqrt(n)
    assert np.all(np.abs(P3 - AR / 4 * d) < 5 * s3 + 1e-12)
    # kinematics: positions uniform on the lattice, |p_T| as requested
    assert 0 <= rec[:, 0].min() and rec[:, 0].max() < 32
    assert abs(rec[:, 0].mean() - 16) < 5 * 32 / math.sqrt(12 * n)


def test_haar_unitaries_are_haar_on_u3():
    rng = np.random.default_rng(0)
    n = 50_000
    acc = np.zeros((3, 3))
    for _ in range(n):
        u = O.haar_from_normals(rng.normal(size=18))
        assert np.abs(u @ u.conj().T - np.eye(3)).max() < 1e-13
        acc += np.abs(u) ** 2
    # Haar on U(3): E|u_ij|^2 = 1/3 for every entry
    assert np.abs(acc / n - 1 / 3).max() < 5 * math.sqrt(1 / 3 * (1 - 1 / 3) / n) * 1.5


# ------------------------------------------------------------------ Casimirs
def test_casimirs_conserved_by_the_push():
    N, dt = 16, 0.125
    st = mv_state(N)
    parts = [O.sample_species(N, 9, s, rep, 0, p, 0.0, 200) for s, (rep, p) in enumerate([(0, 0.6), (1, 0.3), (0, 5.0)])]
    part = np.concatenate(parts)
    r = O.Run(st, part, [0.6, 2.0, 0.0], [0.0, 0.25, 0.0], [0, 1, 0], dt)
    moved = part[:, 6:14].copy()
    for _ in range(60):
        r.step()
    obs = r.observables()
    assert obs[:, 5].max() < 1e-13 * 24 and obs[:, 6].max() < 1e-12 * 24
    assert np.abs(part[:, 6:14] - moved).max() > 1e-2  # charges did rotate


# ------------------------------------------------------------------ static limit
def _static_run(N, st, part, dt, steps, tf):
    r = O.Run(st.copy(), part, [math.inf], [tf], [0], dt)
    n = part.shape[0]
    X = np.zeros((n, 3, 8))
    for _ in range(steps):
        act = r.t() >= tf
        cells = (np.floor(part[:, 1] + 0.5).astype(int) % N) * N + np.floor(part[:, 0] + 0.5).astype(int) % N
        r.step()
        if act:
            X += dt * r.site[[0, 1, 2]][:, cells].transpose(1, 0, 2)
    return X, r


def test_static_limit_equals_integrated_E_correlator():
    # m -> infinity: no motion and no colour rotation, so each particle's
    # momentum is Q^a X^a with X_i = sum_n dt E_i(t_n) at its site
    N, dt, tf = 16, 0.125, 0.5
    st = mv_state(N)
    part = O.sample_species(N, 1, 0, 0, 0, 0.0, 0.0, 300)
    Q = part[:, 6:14].copy()
    x0 = part[:, :3].copy()
    X, r = _static_run(N, st, part, dt, 40, tf)
    for i, slot in enumerate((3, 4, 5)):
        pred = np.einsum("na,na->n", Q, X[:, i])
        assert np.abs(part[:, slot] - pred).max() < 1e-13 * max(1, np.abs(pred).max())
    assert np.array_equal(part[:, :3], x0) and np.array_equal(part[:, 6:14], Q)
    assert np.abs(part[:, 3]).max() > 0.05


def test_static_quark_in_a_uniform_E_x_gets_Q_E_integral():
    # Trivial links, phi = pi = 0 and a uniform Abelian e_x = c T^3: every
    # force term vanishes, so e_x stays c T^3 and the site field is
    # E_x = c / t_n (Sec. 3.2: E_i = P^i / tau).  A static quark then gets
    # p_x = Q^3 c sum_n dt / t_n over its active steps, which approaches
    # Q^3 c ln(t / t_form) at O(dt); p_y and p_L stay 0.
    N, dt, tf, c, steps = 4, 0.0625, 0.5, 0.8, 120
    st = O.FieldState(N)
    st.e[0, :, 2] = c
    part = O.sample_species(N, 9, 0, 0, 0, 0.0, 0.0, 40)
    Q3 = part[:, 8].copy()
    r = O.Run(st, part, [math.inf], [tf], [0], dt)
    acc = 0.0
    for _ in range(steps):
        if r.t() >= tf:
            acc += dt / r.t()
        r.step()
    assert np.abs(r.st.e[0, :, 2] - c).max() < 1e-14
    assert np.abs(part[:, 3] - Q3 * c * acc).max() < 1e-13
    assert np.abs(part[:, 4:6]).max() < 1e-15
    assert abs(acc - math.log(r.t() / tf)) < dt / tf
    assert np.abs(part[:, 3]).max() > 0.3


def test_static_ensemble_average_and_casimir_scaling():
    # <(Q.X)^2> over the Haar ensemble = T_R X^a X^a (Fierz with <Q^a Q^b> =
    # T_R delta^ab); adjoint over fundamental = q2(A)/q2(F) = 6, i.e. 9/4 after
    # dividing by D_R (Sec. 6 and App. D)
    rng = np.random.default_rng(5)
    X = rng.normal(size=8)
    n = 200_000
    out = {}
    for rep in (0, 1):
        Q = O.sample_species(8, 77, rep, rep, 0, 0.0, 0.0, n)[:, 6:14]
        v = (Q @ X) ** 2
        out[rep] = (v.mean(), v.std() / math.sqrt(n))
    assert abs(out[0][0] - 0.5 * X @ X) < 5 * out[0][1]
    assert abs(out[1][0] - 3.0 * X @ X) < 5 * out[1][1]
    ratio = (out[1][0] / 8) / (out[0][0] / 3)
    assert abs(ratio - 9 / 4) < 0.05


def test_large_mass_converges_to_static_and_pz_is_the_longitudinal_momentum():
    N, dt, tf = 16, 0.125, 0.5
    st = mv_state(N)
    base = O.sample_species(N, 1, 0, 0, 0, 0.0, 0.0, 64)
    ps = base.copy()
    _static_run(N, st, ps, dt, 40, tf)
    gaps = []
    for m in (1e2, 1e3, 1e4):
        pm = base.copy()
        r = O.Run(st.copy(), pm, [m], [tf], [0], dt)
        for _ in range(40):
            r.step()
        gaps.append(np.abs(pm[:, 3:5] - ps[:, 3:5]).max())
        t = r.t()
    assert gaps[1] < gaps[0] / 5 and gaps[2] < gaps[1] / 5 and gaps[2] < 1e-4
    # lab p^z (not tau p^eta) approaches the static E_eta integral
    pz = np.array([O.p_long(pm[i], t, 1e4) for i in range(len(pm))])
    scale = np.abs(ps[:, 5]).max()
    assert np.abs(pz - ps[:, 5]).max() < 0.1 * scale
    assert np.abs(pm[:, 5] / t - ps[:, 5]).max() > 0.5 * scale


# ------------------------------------------------------------------ light-like limit
def _jet_vs_correlator(dt, n=40, T=7.5):
    N = 16
    st = mv_state(N)
    part = O.sample_species(N, 2, 0, 0, 2, 1e8, 0.0, n)
    x0, y0, Q0 = part[:, 0].copy(), part[:, 1].copy(), part[:, 6:14].copy()
    r = O.Run(st, part, [0.0], [0.0], [0], dt)
    W = np.broadcast_to(np.eye(3, dtype=complex), (n, 3, 3)).copy()
    X = np.zeros((n, 3, 3, 3), dtype=complex)
    iy = np.floor(y0 + 0.5).astype(int) % N
    steps = int(round(T / dt))
    for k in range(steps):
        ix = np.floor(x0 + k * dt + 0.5).astype(int)
        r.step()
        cell = iy * N + ix % N
        Ex, Ey, Ee, Bx, By, Be = [H.alg2mat(r.site[j][cell]) for j in range(6)]
        # Lorentz force of a light-like parton moving along +x: (E_x, E_y - B_z, E_z + B_y)
        for i, f in enumerate((Ex, Ey - Be, Ee + By)):
            X[:, i] += dt * W @ f @ W.conj().transpose(0, 2, 1)
        cross = np.floor(x0 + (k + 1) * dt + 0.5).astype(int) != ix
        W[cross] = W[cross] @ H.links(r.st.U)[0][cell][cross]
    pred = np.einsum("na,nia->ni", Q0, np.stack([H.mat2alg(X[:, i]) for i in range(3)], 1))
    pz = np.array([O.p_long(part[i], r.t(), 0.0) for i in range(n)])
    return part, pred, pz, x0


def test_light_like_limit_equals_jet_correlator():
    part, pred, pz, x0 = _jet_vs_correlator(0.125)
    assert np.allclose(part[:, 0], (x0 + 7.5) % 16, atol=1e-9)
    assert np.abs(part[:, 3] - 1e8 - pred[:, 0]).max() < 1e-6
    assert np.abs(part[:, 4] - pred[:, 1]).max() < 1e-6
    # the longitudinal kick converges at O(dt) (Euler from tau = 0)
    g1 = np.abs(pz - pred[:, 2]).max()
    _, pred2, pz2, _ = _jet_vs_correlator(0.0625)
    g2 = np.abs(pz2 - pred2[:, 2]).max()
    assert g2 < 0.75 * g1 and g1 < 0.2 * np.abs(pred[:, 2]).max()


def _probes_at(x0, y0):
    jets = np.zeros((len(x0), O.JET_LEN))
    jets[:, 0], jets[:, 1] = x0, y0
    for i in range(3):
        jets[:, 2 + 2 * (3 * i + i)] = 1.0
    return jets


def test_oracle_jet_correlator_equals_direct_sum():
    """The oracle's jet correlator (Sec. 5.2) against the transported-force
    sum written out here with numpy on the oracle's own site fields and links
    (W <- W U_x on each crossing, X_i += dt W f_i W^+)."""
    N, n, dt, T = 16, 30, 0.125, 7.5
    st = mv_state(N)
    rng = np.random.default_rng(5)
    x0, y0 = rng.uniform(0, N, n), rng.uniform(0, N, n)
    jets = _probes_at(x0, y0)
    r = O.Run(st, None, [0.0], [0.0], [0], dt, jets=jets)
    W = np.broadcast_to(np.eye(3, dtype=complex), (n, 3, 3)).copy()
    X = np.zeros((n, 3, 3, 3), dtype=complex)
    iy = np.floor(y0 + 0.5).astype(int) % N
    for k in range(int(round(T / dt))):
        ix = np.floor(x0 + k * dt + 0.5).astype(int)
        r.step()
        cell = iy * N + ix % N
        Ex, Ey, Ee, Bx, By, Be = [H.alg2mat(r.site[j][cell]) for j in range(6)]
        for i, f in enumerate((Ex, Ey - Be, Ee + By)):
            X[:, i] += dt * W @ f @ W.conj().transpose(0, 2, 1)
        cross = np.floor(x0 + (k + 1) * dt + 0.5).astype(int) != ix
        W[cross] = W[cross] @ H.links(r.st.U)[0][cell][cross]
    want = np.stack([H.mat2alg(X[:, i]) for i in range(3)], 1)
    got = jets[:, 20:44].reshape(n, 3, 8)
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
    Wgot = jets[:, 2:20].view(np.complex128).reshape(n, 3, 3)
    assert np.abs(Wgot - W).max() < 1e-12
    assert np.allclose(O.jets_obs(jets), (want ** 2).sum(axis=2).mean(axis=0), rtol=1e-12)


def test_eikonal_partons_receive_the_correlator_kicks():
    """Eikonal partons (fixed light-like path along +x, no momentum feedback)
    rotate their charge instead of transporting the force: their kicks equal
    Q0 . X_i of probes on the same paths to rounding, whatever the charge."""
    N, n, dt, T = 16, 40, 0.125, 6.0
    st = mv_state(N)
    part = O.sample_species(N, 9, 0, 0, 3, 0.0, 0.0, n)
    assert np.all(part[:, 3:6] == 0.0) and np.all(part[:, 14] == 0.0)
    x0, y0, Q0 = part[:, 0].copy(), part[:, 1].copy(), part[:, 6:14].copy()
    jets = _probes_at(x0, y0)
    r = O.Run(st, part, [0.0], [0.0], [0], dt, kind=[O.KIND_EIKONAL], jets=jets)
    steps = int(round(T / dt))
    for _ in range(steps):
        r.step()
    X = jets[:, 20:44].reshape(n, 3, 8)
    kick = np.einsum("na,nia->ni", Q0, X)
    assert np.abs(part[:, 3:6] - kick).max() < 1e-12 * np.abs(kick).max()
    assert np.allclose(part[:, 0], (x0 + steps * dt) % N, atol=1e-12)
    assert np.array_equal(part[:, 1], y0) and np.all(part[:, 2] == 0.0)
    # the charge moved on the colour sphere: Casimirs unchanged
    q2 = (part[:, 6:14] ** 2).sum(axis=1)
    assert np.abs(q2 - 4.0).max() < 1e-12
    # p_L of an eikonal parton is the accumulated lab p_z
    assert O.p_long(part[0], r.t(), 0.0, O.KIND_EIKONAL) == part[0, 5]


# ------------------------------------------------------------------ closed forms
def _hyperbolic_gap(dt):
    # uniform Abelian E_eta on a trivial background = uniform lab E_z; a
    # particle formed at rest in z at t0 follows p_z = qE (t_lab - t0),
    # z = (sqrt(mT^2 + p_z^2) - mT)/qE  (textbook hyperbolic motion)
    N, E, m, tf = 4, 0.2, 0.5, 0.5
    st = O.FieldState(N)
    st.pi[:, 2] = E
    part = np.zeros((1, 16))
    part[0, :2] = (1.3, 2.2)
    part[0, 3] = 0.3
    part[0, 8] = 1.0   # Q^3 = 1
    r = O.Run(st, part, [m], [tf], [0], dt)
    for _ in range(int(round(3.0 / dt))):
        r.step()
    pz = O.p_long(part[0], r.t(), m)
    mT = math.hypot(m, 0.3)
    tl = tf + pz / E
    z = (math.sqrt(mT * mT + pz * pz) - mT) / E
    return math.sqrt(tl * tl - z * z) - r.t(), part[0]


def test_uniform_E_eta_hyperbolic_motion():
    g1, p1 = _hyperbolic_gap(0.125)
    g2, _ = _hyperbolic_gap(0.0625)
    assert abs(g1) < 0.2 and 1.7 < g1 / g2 < 2.3   # O(dt) Euler
    assert p1[3] == 0.3 and p1[4] == 0.0            # no transverse force


def _cyclotron(dt, T=4.0):
    # flux theta N^2 = 2 pi through the torus in the T^3 direction: every
    # plaquette is exp(i theta 2T^3), so B_eta = -2 sin(theta) T^3 uniformly
    N = 8
    th = 2 * math.pi / N ** 2
    D = 2 * H.T[2]
    u = H.links(O.unit_links(N)).copy()
    for s in range(N * N):
        x, y = s % N, s // N
        u[1, s] = scipy.linalg.expm(1j * th * x * D)
        if x == N - 1:
            u[0, s] = scipy.linalg.expm(-1j * th * N * y * D)
    st = O.FieldState(N, H.links_to_canon(u))
    site = O.site_fields(st, st, 1.0)
    assert np.abs(site[5, :, 2] + 2 * math.sin(th)).max() < 1e-14
    assert np.abs(np.delete(site, 5, axis=0)).max() < 1e-15
    q3, m, p = 2.0, 0.4, 0.5
    part = np.zeros((1, 16))
    part[0, :2] = (3.3, 4.6)
    part[0, 3] = p
    part[0, 8] = q3
    ang, prev = 0.0, 0.0
    for n in range(int(round(T / dt))):
        O.push(N, 1.0 + n * dt, dt, site, st.U, st.phi, part, [m], [1])
        a = math.atan2(part[0, 4], part[0, 3])
        ang += (a - prev + math.pi) % (2 * math.pi) - math.pi
        prev = a
    # Lorentz force q v x B with B = B_z: clockwise at omega = qB / p^tau
    qB = -2 * math.sin(th) * q3
    omega = qB / math.hypot(p, m)
    return ang - (-omega * T), math.hypot(part[0, 3], part[0, 4]) - p, part[0]


def test_cyclotron_in_uniform_B_eta():
    a1, r1, p1 = _cyclotron(0.125)
    a2, r2, _ = _cyclotron(0.0625)
    assert abs(a1) < 0.1 and abs(r1) < 0.15 * 0.5    # |p_T| conserved up to Euler's O(dt) growth
    assert abs(r2) < 0.6 * abs(r1) and abs(a2) < 0.1
    assert np.allclose(p1[6:14], [0, 0, 2, 0, 0, 0, 0, 0])


def _canonical_px(dt, flip_eta=False, swap_B=False, T=6.0):
    # uniform, static, non-Abelian: U_x = exp(i c1 T^1), U_y = 1, phi = c3 T^3.
    # Translation invariance in x conserves p^x - Q^a A_x^a with A_x = c1 T^1
    # (follows from Wong's equations: dp^x = -Q.F_x_eta v^eta with
    # F_x_eta = i[A_x, A_eta], and dQ = -i[A_eta, Q] d eta)
    N, c1, c3, t0, m = 6, 0.05, 0.8, 1.0, 1.0
    u = H.links(O.unit_links(N)).copy()
    Ux = scipy.linalg.expm(1j * c1 * H.T[0])
    u[0, :] = Ux
    st = O.FieldState(N, H.links_to_canon(u))
    st.phi[:, 2] = c3
    part = np.zeros((1, 16))
    part[0, :2] = (2.0, 3.0)
    part[0, 5] = 2.0 * t0 * t0
    q = np.random.default_rng(0).normal(size=8)
    part[0, 6:14] = 2 * q / np.linalg.norm(q)
    Ax = H.mat2alg(-1j * scipy.linalg.logm(Ux))
    inv0 = part[0, 3] - part[0, 6:14] @ Ax
    for n in range(int(round(t0 / dt)), int(round(T / dt))):
        t = n * dt
        site = O.site_fields(st, st, t)
        if swap_B:  # literal reading B_i = -(1/t) D_i A_eta of the interpolation formula
            site = site.copy()
            bx, by = site[3].copy(), site[4].copy()
            site[3], site[4] = -by, bx
        O.push(N, t, dt, site, st.U, -st.phi if flip_eta else st.phi, part, [m], [1])
    return part[0, 3] - part[0, 6:14] @ Ax - inv0, part[0, 3]


def test_canonical_momentum_fixes_B_components_and_rapidity_rotation():
    d1, px = _canonical_px(0.125)
    d2, _ = _canonical_px(0.0625)
    assert abs(px) > 1e-3                      # a real force acted
    assert abs(d1) < 0.1 * abs(px) and abs(d2) < 0.6 * abs(d1)
    # planted mistakes are caught: opposite rapidity rotation, or B_x <-> B_y
    assert abs(_canonical_px(0.0625, flip_eta=True)[0]) > 3 * abs(px)
    assert abs(_canonical_px(0.0625, swap_B=True)[0]) > 0.5 * abs(px)


def test_push_is_gauge_covariant():
    N, dt = 12, 0.125
    rng = np.random.default_rng(8)
    st = mv_state(N)
    for n in range(8):
        st = O.field_step(st, n * dt, dt)
    t = 8 * dt
    part = np.concatenate([O.sample_species(N, 4, 0, 0, 0, 3.0, 0.0, 300),
                           O.sample_species(N, 4, 1, 0, 2, 8.0, 0.0, 100)])
    part[:, 5] = rng.normal(size=len(part)) * 0.5
    part[100:200, 3] *= -1
    Om = H.random_su3(rng, N * N)
    new = O.field_step(st, t, dt)
    g = O.FieldState(N, *H.gauge_transform(N, st.U, st.phi, st.e, st.pi, Om))
    gnew = O.FieldState(N, *H.gauge_transform(N, new.U, new.phi, new.e, new.pi, Om))
    site = O.site_fields(st, new, t)
    gsite = O.site_fields(g, gnew, t)

    def cells(p):
        return (np.floor(p[:, 1] + 0.5).astype(int) % N) * N + np.floor(p[:, 0] + 0.5).astype(int) % N

    gpart = part.copy()
    c0 = cells(part)
    gpart[:, 6:14] = H.mat2alg(Om[c0] @ H.alg2mat(part[:, 6:14]) @ Om[c0].conj().transpose(0, 2, 1))
    O.push(N, t, dt, site, new.U, new.phi, part, [0.7, 0.0], [1, 1])
    O.push(N, t, dt, gsite, gnew.U, gnew.phi, gpart, [0.7, 0.0], [1, 1])
    assert np.abs(gpart[:, :6] - part[:, :6]).max() < 1e-12
    c1 = cells(part)
    assert (c1 != c0).sum() > 10
    want = H.mat2alg(Om[c1] @ H.alg2mat(part[:, 6:14]) @ Om[c1].conj().transpose(0, 2, 1))
    assert np.abs(gpart[:, 6:14] - want).max() < 1e-12


# ------------------------------------------------------------------ temporal constraint
def _ptau_gap(dt, field):
    """Integrated p^tau against the mass shell after free streaming in Milne
    coordinates (P_eta conserved, w = P_eta / t falls) or after acceleration
    by a uniform Abelian E_x (work-energy); both equations are exact, so the
    gap is the Euler error, O(dt)."""
    N, m = 4, 0.6
    st = O.FieldState(N)
    if field:
        st.e[0, :, 2] = 0.3   # e_x along T^3: uniform Abelian E_x = e / t
    part = np.zeros((1, 16))
    part[0, :2] = (1.2, 2.1)
    part[0, 3], part[0, 4] = 0.4, -0.2
    part[0, 5] = 0.0 if field else 1.5   # P_eta = tau^2 p^eta
    part[0, 8] = 1.0                      # Q^3 = 1
    ptau = np.full(1, np.nan)
    r = O.Run(st, part, [m], [1.0], [0], dt, step=int(round(1.0 / dt)), ptau=ptau)
    for _ in range(int(round(4.0 / dt))):
        r.step()
    t = r.t()
    w = part[0, 5] / t
    shell = math.sqrt(part[0, 3] ** 2 + part[0, 4] ** 2 + w * w + m * m)
    return ptau[0] - shell, shell


@pytest.mark.parametrize("field", [False, True])
def test_integrated_ptau_follows_the_mass_shell(field):
    g1, s1 = _ptau_gap(0.125, field)
    g2, _ = _ptau_gap(0.0625, field)
    g3, _ = _ptau_gap(0.03125, field)
    assert abs(g1) < 0.15 * s1
    assert 1.8 < g1 / g2 < 2.2 and 1.8 < g2 / g3 < 2.2   # first order (Euler), converging to the shell


def test_ptau_skips_static_eikonal_and_inactive():
    N = 4
    st = O.FieldState(N)
    part = np.zeros((3, 16))
    part[:, 15] = [0, 1, 2]
    part[:, 6] = 2.0
    ptau = np.full(3, np.nan)
    r = O.Run(st, part, [0.5, math.inf, 0.0], [0.0, 0.0, 100.0], [0, 0, 0], 0.125,
              kind=[O.KIND_WONG, O.KIND_STATIC, O.KIND_EIKONAL], ptau=ptau)
    r.step()
    assert ptau[0] == pytest.approx(0.5) and np.isnan(ptau[1]) and np.isnan(ptau[2])
