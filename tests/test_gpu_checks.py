"""GPU tests of the FP32 re-unitarisation and of the FP64 check values,
through the C ABI.

Re-unitarisation: FP32 links are stored as two rows and, once every
`reunit_every` steps (row y in the steps n with (n + 1 + y) % reunit_every ==
0), Gram-Schmidt orthonormalised in FP64.  Runs of several periods stay
within the FP32 bound of the FP64 oracle, each row is unitary to FP32
rounding right after its re-unitarising step, a link field made non-unitary
on purpose is restored row by row within one period, and a run resumed from
a snapshot taken in the middle of a period is bitwise the uninterrupted one
(single events and batches).

Check values: on a state with a Gauss-law violation, a non-unitary link and
charges off their Casimir shells, gauss_max, gauss_rms, unitarity_max and the
Casimir deviations equal the oracle's (Gauss constraint of Sec. 2; Casimirs
of App. A) at 1e-10; on an FP32 state, the check values and the squared site
fields equal the oracle's of the same stored values."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2303_05599_gb300 import _binding as B
from paper_2303_05599_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP32_FIELD_TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2303_05599_gb300 import build
    build.build()
    B.lib()


def wl(N, prec, reunit_every=64, species=(), seed=3):
    w = W.Workload("checks", N=N, L_fm=0.09375 * N, precision=prec, seed=seed, Ns=6, species=list(species))
    w.reunit_every = reunit_every
    return w


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(1e-300, np.abs(b).max())


def oracle_init(w):
    st, bad = O.mv_init(w.N, w.Ns, w.g2mu_a, w.m_a, w.Lambda_a, w.seed)
    assert bad == 0
    return st


def upload_state(ev, st):
    ev.upload(B.GL_BUF_LINKS, st.U)
    ev.upload(B.GL_BUF_PHI, st.phi)
    ev.upload(B.GL_BUF_E, st.e)
    ev.upload(B.GL_BUF_PI, st.pi)


def download_state(ev):
    return O.FieldState(ev.N, ev.download(B.GL_BUF_LINKS), ev.download(B.GL_BUF_PHI), ev.download(B.GL_BUF_E),
                        ev.download(B.GL_BUF_PI))


# ------------------------------------------------------------------ re-unitarisation
# The links of row y are re-unitarised in FP64 in the steps n with
# (n + 1 + y) % reunit_every == 0: every link once per period, the FP64 work
# spread evenly over the steps.


# bound on ||U U^+ - 1||_F per step of FP32 link updates since the last
# re-unitarisation: a few ulps (2^-23 = 1.2e-7) of each updated row; measured
# 1.3e-6 after 3 steps and 2.1e-6 after 15
DRIFT = 5e-7
# right after its re-unitarisation a link is orthonormal to FP32 storage
# rounding: each entry rounded at 2^-24 = 6e-8 gives |r_i|^2 - 1 and <r0, r1>
# of ~2e-7 and a Frobenius norm of ~4e-7 over the 3 x 3 (measured 4.4e-7)
FRESH = 1e-6


def row_unitarity(ev):
    """max over the links of each row of ||U U^+ - 1||_F, from the downloaded
    links (FP32 two-row links with their rebuilt third row)."""
    u = H.links(ev.download(B.GL_BUF_LINKS))
    d = u @ u.conj().transpose(0, 1, 3, 2) - np.eye(3)
    nrm = np.sqrt((np.abs(d) ** 2).sum(axis=(2, 3)))       # [2, V]
    return nrm.reshape(2, ev.N, ev.N).max(axis=(0, 2))      # [N] rows


@pytest.mark.parametrize("every", [4, 16])
def test_fp32_reunitarised_run_stays_within_the_oracle_bound(every):
    # 3 periods and a bit; 37 is not a multiple of the strip width or the
    # segment length
    w = wl(37, W.FP32_2ROW, every)
    st = oracle_init(w)
    ev = B.Event(w)
    upload_state(ev, st)
    steps = 3 * every + 2 if every > 4 else 14
    fresh, worst = [], 0.0
    for n in range(steps):
        ev.glasma_step(1)
        st = O.field_step(st, n * w.dt, w.dt)
        rows = row_unitarity(ev)
        done = [y for y in range(w.N) if (n + 1 + y) % every == 0]
        fresh.append(float(rows[done].max()))
        worst = max(worst, float(rows.max()))
    g = download_state(ev)
    errs = {k: rel(a, b) for k, a, b in [("U", g.U, st.U), ("phi", g.phi, st.phi), ("e", g.e, st.e),
                                         ("pi", g.pi, st.pi)]}
    print("reunit_every %d, %d FP32 steps: field errors %s; rows just re-unitarised: max %.3e; all rows: max %.3e"
          % (every, steps, errs, max(fresh), worst))
    assert max(errs.values()) < 2e-5
    # right after its re-unitarisation a row is unitary to FP32 rounding; in
    # between, each step's FP32 link update adds at most a few ulps of drift
    assert max(fresh) <= FRESH
    assert worst <= DRIFT * every


def test_reunitarisation_restores_non_unitary_links():
    # links made non-unitary by (1 + eps H) U with H Hermitian: ||U U^+ - 1||
    # is O(eps) and the unitary link update keeps it; each row is brought to
    # FP32 rounding by its re-unitarising step, so after one period all are
    every, eps = 8, 1e-3
    w = wl(16, W.FP32_2ROW, every)
    st = oracle_init(w)
    u = H.links(st.U).copy()
    rng = np.random.default_rng(1)
    Hm = H.alg2mat(rng.normal(size=(2, w.N * w.N, 8)))
    u = (np.eye(3) + eps * Hm) @ u
    st.U = H.links_to_canon(u)
    u0, _ = O.unitarity(st)
    ev = B.Event(w)
    upload_state(ev, st)
    restored = set()
    seen = []
    for n in range(every + 2):
        ev.glasma_step(1)
        rows = row_unitarity(ev)
        now = [y for y in range(w.N) if (n + 1 + y) % every == 0]
        restored |= set(now)
        other = [y for y in range(w.N) if y not in restored]
        assert rows[now].max() < FRESH, (n, rows)                     # just re-unitarised
        assert rows[sorted(restored)].max() < DRIFT * every, (n, rows)  # since then: FP32 drift only
        if other:
            assert rows[other].min() > 1e-4, (n, rows)   # untouched by ordinary steps
        seen.append(ev.observables(B.GL_OBS_FIELDS).unitarity_max)
    print("uploaded non-unitarity %.3e; unitarity_max after each step %s" % (u0, seen))
    assert u0 > 1e-3
    assert min(seen[:every - 1]) > 0.3 * u0       # some row not yet re-unitarised
    assert max(seen[every - 1:]) < DRIFT * every  # every row restored after one period


def _species():
    return [W.Species(W.M_CHARM, 0.0, 400, W.REP_F, W.MOM_UNIFORM_PT, 0.0, 5.0),
            W.Species(math.inf, 0.0, 50, W.REP_A, W.MOM_FIXED_PT, 0.0)]


def _same(a, b):
    for which in (B.GL_BUF_LINKS, B.GL_BUF_PHI, B.GL_BUF_E, B.GL_BUF_PI, B.GL_BUF_PARTICLES):
        assert np.array_equal(a.download(which), b.download(which)), which


def test_resume_inside_a_reunitarisation_period_is_bitwise():
    # checkpoint at step 10 of a 16-step period; the resumed run re-unitarises
    # every row at the same steps as the uninterrupted one (a rule of the step
    # index and the row alone)
    w = wl(40, W.FP32_2ROW, 16, _species(), seed=7)
    w.sort_every = 8
    a = B.Event(w)
    a.glasma_init()
    a.wong_init()
    a.step(10)
    f = a.download_native(B.GL_NATIVE_FIELDS)
    p = a.download_native(B.GL_NATIVE_PARTICLES)
    a.step(30)
    b = B.Event(w)
    b.glasma_init()
    b.wong_init()
    b.upload_native(B.GL_NATIVE_FIELDS, f)
    b.upload_native(B.GL_NATIVE_PARTICLES, p)
    b.set_step(10)
    b.step(30)
    _same(a, b)
    # and the canonical FP64 checkpoint path (gl_download / gl_upload / gl_set_step)
    c = B.Event(w)
    c.glasma_init()
    c.wong_init()
    c.step(10)
    canon = {k: c.download(k) for k in (B.GL_BUF_LINKS, B.GL_BUF_PHI, B.GL_BUF_E, B.GL_BUF_PI, B.GL_BUF_PARTICLES)}
    d = B.Event(w)
    d.glasma_init()
    d.wong_init()
    for k, v in canon.items():
        d.upload(k, v)
    d.set_step(10)
    c.step(30)
    d.step(30)
    _same(c, d)


def test_batched_resume_inside_a_reunitarisation_period_is_bitwise():
    ws = []
    for e, N in enumerate([24, 40, 64]):
        w = wl(N, W.FP32_2ROW, 16, _species(), seed=20 + e)
        w.sort_every = 8
        ws.append(w)
    a = B.Batch(ws)
    b = B.Batch(ws)
    with torch.cuda.stream(a.stream):
        a.init()
        a.step(10)
        fs = [ev.download_native(B.GL_NATIVE_FIELDS) for ev in a.events]
        ps = [ev.download_native(B.GL_NATIVE_PARTICLES) for ev in a.events]
        a.step(30)
    with torch.cuda.stream(b.stream):
        b.init()
        b.upload_native(B.GL_NATIVE_FIELDS, fs)
        b.upload_native(B.GL_NATIVE_PARTICLES, ps)
        for ev in b.events:
            ev.set_step(10)
        b.step(30)
    for ea, eb in zip(a.events, b.events):
        _same(ea, eb)
    # the batched event equals the same event run alone, re-unitarisations included
    solo = B.Event(ws[1])
    solo.glasma_init()
    solo.wong_init()
    solo.step(40)
    _same(a.events[1], solo)


# ------------------------------------------------------------------ FP64 check values
def test_field_check_values_equal_the_oracle():
    w = wl(16, W.FP64)
    st = oracle_init(w)
    for n in range(6):
        st = O.field_step(st, n * w.dt, w.dt)
    rng = np.random.default_rng(2)
    # a Gauss-law violation at one site and a non-unitary link elsewhere
    st.e[0, 37] += rng.normal(size=8) * 0.3
    u = H.links(st.U).copy()
    u[1, 100] = (np.eye(3) + 0.1j * H.T[0]) @ u[1, 100]
    st.U = H.links_to_canon(u)
    ev = B.Event(w)
    upload_state(ev, st)
    ev.set_step(6)
    o = ev.observables(B.GL_OBS_FIELDS)
    G = O.gauss(st)
    g2 = (G * G).sum(1)
    want_max, want_rms = math.sqrt(g2.max()), math.sqrt(g2.mean())
    want_u, _ = O.unitarity(st)
    print("gauss_max %.6e/%.6e gauss_rms %.6e/%.6e unitarity_max %.6e/%.6e"
          % (o.gauss_max, want_max, o.gauss_rms, want_rms, o.unitarity_max, want_u))
    assert want_max > 1e-2 and want_u > 1e-3
    assert abs(o.gauss_max - want_max) <= 1e-10 * want_max
    assert abs(o.gauss_rms - want_rms) <= 1e-10 * want_rms
    assert abs(o.unitarity_max - want_u) <= 1e-10 * want_u


def test_fp32_check_values_equal_the_oracle_on_the_same_state():
    """The FP64 checks of an FP32 state (links with their third row rebuilt
    from the two stored ones, momenta and site fields as stored) against the
    oracle's Gauss residual, unitarity and squared site fields of the same
    values, downloaded exactly.  The residuals are small differences of O(1)
    terms summed in another order on each side (relative 1e-8); the squared
    site fields are summed as exact float pairs on the GPU (relative 1e-12)."""
    sp = [W.Species(W.M_CHARM, 0.0, 200, W.REP_F, W.MOM_FIXED_PT, 0.5)]
    w = wl(24, W.FP32_2ROW, species=sp, seed=7)
    ev = B.Event(w)
    ev.glasma_init()
    ev.wong_init()
    ev.step(12)
    o = ev.observables()
    st = download_state(ev)
    G = O.gauss(st)
    g2 = (G * G).sum(1)
    want_max, want_rms = math.sqrt(g2.max()), math.sqrt(g2.mean())
    want_u, _ = O.unitarity(st)
    site = ev.download(B.GL_BUF_SITE)
    tr = 0.5 * (site ** 2).sum(axis=2)
    V = w.N * w.N
    want = {"mean_trE_T2": (tr[0] + tr[1]).sum() / V, "mean_trE_L2": tr[2].sum() / V,
            "mean_trB_T2": (tr[3] + tr[4]).sum() / V, "mean_trB_L2": tr[5].sum() / V}
    print("gauss_max %.6e/%.6e gauss_rms %.6e/%.6e unitarity_max %.6e/%.6e"
          % (o.gauss_max, want_max, o.gauss_rms, want_rms, o.unitarity_max, want_u))
    assert 0 < want_max < 1e-4 and 0 < want_u < 1e-4
    assert abs(o.gauss_max - want_max) <= 1e-8 * want_max
    assert abs(o.gauss_rms - want_rms) <= 1e-8 * want_rms
    assert abs(o.unitarity_max - want_u) <= 1e-8 * want_u
    for f, v in want.items():
        assert v > 0 and abs(getattr(o, f) - v) <= 1e-12 * v, (f, getattr(o, f), v)


def test_casimir_deviations_equal_the_oracle():
    sp = [W.Species(W.M_CHARM, 0.0, 200, W.REP_F, W.MOM_FIXED_PT, 0.5),
          W.Species(W.M_BEAUTY, 0.0, 100, W.REP_A, W.MOM_UNIFORM_PT, 0.0, 3.0)]
    w = wl(16, W.FP64, species=sp, seed=4)
    st = oracle_init(w)
    part = np.concatenate([O.sample_species(w.N, w.seed, k, s.rep, s.mom_mode, *w.lattice_species()[k][2:4],
                                            s.count) for k, s in enumerate(sp)])
    # charges moved off their Casimir shells by different amounts
    rng = np.random.default_rng(8)
    part[:, 6:14] *= 1.0 + 1e-3 * rng.random(len(part))[:, None]
    part[::7, 6:14] += 1e-3 * rng.normal(size=(len(part[::7]), 8))
    ev = B.Event(w)
    upload_state(ev, st)
    ev.upload(B.GL_BUF_PARTICLES, part)
    ls = w.lattice_species()
    run = O.Run(st, part.copy(), [s[0] for s in ls], [s[1] for s in ls], [s.rep for s in sp], w.dt)
    for _ in range(3):
        run.step()
    ev.step(3)
    o = ev.observables(B.GL_OBS_PARTICLES)
    want = run.observables()
    for k in range(len(sp)):
        print("species %d: casimir2 %.6e/%.6e casimir3 %.6e/%.6e"
              % (k, o.casimir2_dev[k], want[k, 5], o.casimir3_dev[k], want[k, 6]))
        assert want[k, 5] > 1e-4 and want[k, 6] > 1e-4
        assert abs(o.casimir2_dev[k] - want[k, 5]) <= 1e-10 * want[k, 5]
        assert abs(o.casimir3_dev[k] - want[k, 6]) <= 1e-10 * want[k, 6]
