"""Python face of the FP64 CPU oracle (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``liboracle_glasma.so`` (plain
C, see ``oracle.h`` for the physics and layouts) with numpy arrays and adds the
two limiting-case correlators of Sec. 5 (static quarks, light-like jets),
which are assembled here from the oracle's lattice fields.

All quantities are in lattice units (a = 1); see ``oracle.h``.
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        d = ctypes.c_double
        i = ctypes.c_int
        i64 = ctypes.c_int64
        u64 = ctypes.c_uint64
        P = ctypes.c_void_p
        sig = {
            "or_generator": (None, [i, P]),
            "or_f": (d, [i, i, i]),
            "or_d": (d, [i, i, i]),
            "or_exp_i_alg": (None, [P, P]),
            "or_expm": (None, [P, P]),
            "or_philox4x32_10": (None, [P, P, P]),
            "or_field_step": (None, [i, d, d, P, P, P, P, P, P, P, P]),
            "or_gauss": (None, [i, P, P, P, P, P]),
            "or_site_fields": (None, [i, d, P, P, P, P, P, P, P]),
            "or_unitarity": (None, [i, P, P, P]),
            "or_q0": (None, [i, P]),
            "or_casimirs": (None, [P, P, P]),
            "or_haar_from_normals": (None, [P, P]),
            "or_sample_species": (None, [i, u64, i, i, i, d, d, i64, P]),
            "or_push": (None, [i, d, d, P, P, P, i64, P, P, P]),
            "or_push_kinds": (None, [i, d, d, P, P, P, i64, P, P, P, P]),
            "or_pL": (d, [P, d, d]),
            "or_pL_kind": (d, [P, d, d, i]),
            "or_jets_init": (None, [i, u64, i64, P]),
            "or_ptau_step": (None, [i, d, d, P, i64, P, P, P, P, P]),
            "or_jets_step": (None, [i, d, d, P, P, i64, P]),
            "or_jets_obs": (None, [i64, P, P]),
            "or_wilson_lines": (None, [i, i, d, d, d, u64, i, P]),
            "or_mv_init": (i, [i, i, d, d, d, u64, P, P]),
            "or_solve_link": (i, [P, P, P]),
            "or_fft": (None, [P, i, i]),
            "or_particle_obs": (None, [i64, P, d, P, P, P, P, i, P]),
            "or_threads": (i, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- algebra
def generators():
    """T^a = lambda^a / 2 as an array [8, 3, 3] complex."""
    out = np.zeros((8, 18))
    for a in range(8):
        lib().or_generator(a, _p(out[a]))
    return out.view(np.complex128).reshape(8, 3, 3)


def f_abc():
    return np.array([[[lib().or_f(a, b, c) for c in range(8)] for b in range(8)] for a in range(8)])


def d_abc():
    return np.array([[[lib().or_d(a, b, c) for c in range(8)] for b in range(8)] for a in range(8)])


def exp_i_alg(x):
    """exp(i x^a T^a) as a 3x3 complex matrix."""
    x = _f64(x)
    out = np.zeros(18)
    lib().or_exp_i_alg(_p(x), _p(out))
    return out.view(np.complex128).reshape(3, 3)


def expm(m):
    m = np.ascontiguousarray(m, dtype=np.complex128)
    out = np.zeros(9, dtype=np.complex128)
    lib().or_expm(_p(m), _p(out))
    return out.reshape(3, 3)


def philox(ctr, key):
    c = np.array(ctr, dtype=np.uint32)
    k = np.array(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


# ---------------------------------------------------------------- fields
class FieldState:
    """Oracle field state at integer step n: U(n), phi(n) and the momenta
    e(n-1/2), pi(n-1/2) in the canonical layouts of ``oracle.h``."""

    def __init__(self, N, U=None, phi=None, e=None, pi=None):
        V = N * N
        self.N = N
        self.U = _f64(U) if U is not None else unit_links(N)
        self.phi = _f64(phi) if phi is not None else np.zeros((V, 8))
        self.e = _f64(e) if e is not None else np.zeros((2, V, 8))
        self.pi = _f64(pi) if pi is not None else np.zeros((V, 8))

    def copy(self):
        return FieldState(self.N, self.U.copy(), self.phi.copy(), self.e.copy(), self.pi.copy())


def unit_links(N):
    U = np.zeros((2, N * N, 9), dtype=np.complex128)
    U[:, :, 0] = U[:, :, 4] = U[:, :, 8] = 1.0
    return U.view(np.float64).reshape(2, N * N, 18).copy()


def field_step(st, t, dt):
    """One leapfrog step at t = t_n; returns the new state (n+1)."""
    N = st.N
    nw = FieldState(N, np.empty_like(st.U), np.empty_like(st.phi), np.empty_like(st.e), np.empty_like(st.pi))
    lib().or_field_step(N, t, dt, _p(st.U), _p(st.phi), _p(st.e), _p(st.pi),
                        _p(nw.U), _p(nw.phi), _p(nw.e), _p(nw.pi))
    return nw


def gauss(st):
    g = np.zeros((st.N * st.N, 8))
    lib().or_gauss(st.N, _p(st.U), _p(st.phi), _p(st.e), _p(st.pi), _p(g))
    return g


def site_fields(old, new, t):
    """Site E, B at t_n from the state before (U(n), phi(n), e(n-1/2), pi(n-1/2))
    and after (e(n+1/2), pi(n+1/2)) the step; returns [6, N*N, 8]."""
    N = old.N
    out = np.zeros((6, N * N, 8))
    lib().or_site_fields(N, t, _p(old.U), _p(old.phi), _p(old.e), _p(new.e),
                         _p(old.pi), _p(new.pi), _p(out))
    return out


def unitarity(st):
    a = ctypes.c_double()
    b = ctypes.c_double()
    lib().or_unitarity(st.N, _p(st.U), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


# ---------------------------------------------------------------- particles
def q0(rep):
    out = np.zeros(8)
    lib().or_q0(rep, _p(out))
    return out


def casimirs(q):
    q = _f64(q)
    a = ctypes.c_double()
    b = ctypes.c_double()
    lib().or_casimirs(_p(q), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def haar_from_normals(g18):
    g = _f64(g18)
    out = np.zeros(18)
    lib().or_haar_from_normals(_p(g), _p(out))
    return out.view(np.complex128).reshape(3, 3)


def sample_species(N, seed, species, rep, mom_mode, p0, p1, n):
    out = np.zeros((n, 16))
    lib().or_sample_species(N, seed, species, rep, mom_mode, p0, p1, n, _p(out))
    return out


KIND_WONG, KIND_STATIC, KIND_EIKONAL = 0, 1, 2
JET_LEN = 44


def kinds_of(mass, mom_mode=None):
    """Species kinds: static for INFINITY mass, eikonal for momentum mode 3."""
    out = []
    for k, m in enumerate(mass):
        if np.isinf(m):
            out.append(KIND_STATIC)
        elif mom_mode is not None and mom_mode[k] == 3:
            out.append(KIND_EIKONAL)
        else:
            out.append(KIND_WONG)
    return np.asarray(out, dtype=np.int32)


def push(N, t, dt, site, U1, phi1, part, mass, active, kind=None):
    """Euler + CPIC step of ``part`` (modified in place)."""
    m = _f64(mass)
    act = np.ascontiguousarray(active, dtype=np.int32)
    kd = kinds_of(mass) if kind is None else np.ascontiguousarray(kind, dtype=np.int32)
    lib().or_push_kinds(N, t, dt, _p(_f64(site)), _p(_f64(U1)), _p(_f64(phi1)), part.shape[0],
                        _p(part), _p(m), _p(kd), _p(act))


def p_long(rec, t, mass, kind=None):
    rec = _f64(rec)
    if kind is None:
        return lib().or_pL(_p(rec), t, mass)
    return lib().or_pL_kind(_p(rec), t, mass, int(kind))


def particle_obs(part, t, mass, active, rep, kind=None):
    ns = len(mass)
    out = np.zeros((ns, 8))
    kd = kinds_of(mass) if kind is None else np.ascontiguousarray(kind, dtype=np.int32)
    lib().or_particle_obs(part.shape[0], _p(part), t, _p(_f64(mass)), _p(kd),
                          _p(np.ascontiguousarray(active, dtype=np.int32)),
                          _p(np.ascontiguousarray(rep, dtype=np.int32)), ns, _p(out))
    return out


def ptau_step(N, t, dt, site, part, mass, kind, active, ptau):
    """Euler step of the integrated p^tau (in place) from the state at t_n."""
    lib().or_ptau_step(N, t, dt, _p(_f64(site)), part.shape[0], _p(part), _p(_f64(mass)),
                       _p(np.ascontiguousarray(kind, dtype=np.int32)),
                       _p(np.ascontiguousarray(active, dtype=np.int32)), _p(ptau))


def jets_init(N, seed, n):
    """Jet-correlator probes [n][44]: x0, y0, W (18), X_x, X_y, X_z (8 each)."""
    out = np.zeros((n, JET_LEN))
    lib().or_jets_init(N, seed, n, _p(out))
    return out


def jets_step(N, t, dt, site, U1, jets):
    lib().or_jets_step(N, t, dt, _p(_f64(site)), _p(_f64(U1)), jets.shape[0], _p(jets))


def jets_obs(jets):
    out = np.zeros(3)
    lib().or_jets_obs(jets.shape[0], _p(jets), _p(out))
    return out


# ---------------------------------------------------------------- init
def fft(x, sign):
    d = np.ascontiguousarray(x, dtype=np.complex128).copy()
    lib().or_fft(_p(d), d.size, sign)
    return d


def wilson_lines(N, Ns, g2mu_a, m_a, Lambda_a, seed, nucleus):
    out = np.zeros((N * N, 18))
    lib().or_wilson_lines(N, Ns, g2mu_a, m_a, Lambda_a, seed, nucleus, _p(out))
    return out


def solve_link(ua, ub):
    out = np.zeros(18)
    bad = lib().or_solve_link(_p(_f64(ua)), _p(_f64(ub)), _p(out))
    return out, bad


def mv_init(N, Ns, g2mu_a, m_a, Lambda_a, seed):
    """tau = 0 state (U(0), phi = 0, e(-1/2) = 0, pi(-1/2) = E_eta(0))."""
    U = np.zeros((2, N * N, 18))
    pi = np.zeros((N * N, 8))
    bad = lib().or_mv_init(N, Ns, g2mu_a, m_a, Lambda_a, seed, _p(U), _p(pi))
    return FieldState(N, U, None, None, pi), bad


def threads():
    return lib().or_threads()


# ---------------------------------------------------------------- coupled run
class Run:
    """Coupled field + particle evolution in the oracle (the method's time
    step: leapfrog n -> n+1, site fields at t_n, Euler/CPIC push of the
    particles active at t_n, and the jet-correlator probes if any)."""

    def __init__(self, state, particles, mass, t_form, rep, dt, step=0, kind=None, jets=None, ptau=None):
        self.st = state
        self.part = particles
        self.mass = np.asarray(mass, dtype=np.float64)
        self.t_form = np.asarray(t_form, dtype=np.float64)
        self.rep = np.asarray(rep, dtype=np.int32)
        self.kind = kinds_of(self.mass) if kind is None else np.asarray(kind, dtype=np.int32)
        self.dt = dt
        self.n = step
        self.site = None
        self.jets = jets
        self.ptau = ptau  # integrated p^tau per particle (NaN: not started), or None

    def t(self):
        return self.n * self.dt

    def active(self):
        return (self.t() >= self.t_form).astype(np.int32)

    def step(self):
        t = self.t()
        new = field_step(self.st, t, self.dt)
        self.site = site_fields(self.st, new, t)
        if self.part is not None and len(self.part):
            if self.ptau is not None:
                ptau_step(self.st.N, t, self.dt, self.site, self.part, self.mass, self.kind, self.active(), self.ptau)
            push(self.st.N, t, self.dt, self.site, new.U, new.phi, self.part, self.mass, self.active(), self.kind)
        if self.jets is not None and len(self.jets):
            jets_step(self.st.N, t, self.dt, self.site, new.U, self.jets)
        self.st = new
        self.n += 1

    def observables(self):
        """Particle sums after the last push (time t_n of the new step) with
        the species activity of the step that was pushed."""
        act = (((self.n - 1) * self.dt) >= self.t_form).astype(np.int32)
        return particle_obs(self.part, self.t(), self.mass, act, self.rep, self.kind)
