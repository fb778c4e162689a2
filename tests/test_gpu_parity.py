"""GPU parity of the CUDA path against the FP64 oracle, called through the
C ABI.  FP64: 1e-10 relative on fields, site fields, single trajectories and
observables (1e-3 on late-time ensemble averages of the full small run); FP32
two-row path: error bounds checked and printed.  Full-size cases compare one
step from a downloaded GPU state with the oracle's step from the same state."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2303_05599_gb300 import _binding as B
from paper_2303_05599_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP64_TOL = 1e-10
# FP32 particles without a cell flip, per-particle relative error after 40
# coupled steps (Euler amplifies field rounding linearly in the step count)
FP32_PARTICLE_TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2303_05599_gb300 import build
    build.build()
    B.lib()


def wl(N, prec=W.FP64, species=(), seed=3, Ns=6, L=None):
    return W.Workload("test", N=N, L_fm=L if L else 0.09375 * N, precision=prec, seed=seed, Ns=Ns,
                      species=list(species))


def rel(a, b):
    scale = max(1e-300, np.abs(b).max())
    return np.abs(np.asarray(a) - np.asarray(b)).max() / scale


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


def oracle_particles(w):
    parts = []
    for k, s in enumerate(w.species):
        m, tf, p0, p1 = w.lattice_species()[k]
        parts.append(O.sample_species(w.N, w.seed, k, s.rep, s.mom_mode, p0, p1, s.count))
    return np.concatenate(parts) if parts else np.zeros((0, 16))


def oracle_run(w, st, part, jets=None):
    ls = w.lattice_species()
    kind = O.kinds_of([s[0] for s in ls], [s.mom_mode for s in w.species])
    return O.Run(st, part, [s[0] for s in ls], [s[1] for s in ls], [s.rep for s in w.species], w.dt, kind=kind,
                 jets=jets)


MIXED = [W.Species(W.M_CHARM, 0.06, 120, W.REP_F, W.MOM_FIXED_PT, 0.5),
         W.Species(math.inf, 0.0, 60, W.REP_F, W.MOM_FIXED_PT, 0.0),
         W.Species(0.0, 0.0, 60, W.REP_A, W.MOM_ALONG_X, 10.0),
         W.Species(W.M_BEAUTY, 0.02, 60, W.REP_A, W.MOM_UNIFORM_PT, 0.0, 5.0)]


# ------------------------------------------------------------------ init
@pytest.mark.parametrize("N", [8, 37])
def test_mv_init_parity(N):
    w = wl(N)
    ev = B.Event(w)
    ev.glasma_init()
    st = oracle_init(w)
    g = download_state(ev)
    assert rel(g.U, st.U) < FP64_TOL
    assert rel(g.pi, st.pi) < FP64_TOL
    assert np.abs(g.phi).max() == 0 and np.abs(g.e).max() == 0


@pytest.mark.parametrize("N", [16, 37])
def test_sampling_parity(N):
    w = wl(N, species=MIXED)
    ev = B.Event(w)
    ev.wong_init()
    got = ev.download(B.GL_BUF_PARTICLES)
    want = oracle_particles(w)
    assert np.array_equal(got[:, 15], want[:, 15])
    assert np.abs(got[:, :2] - want[:, :2]).max() < 1e-12
    assert rel(got[:, 3:5], want[:, 3:5]) < 1e-13
    assert rel(got[:, 6:14], want[:, 6:14]) < 1e-12
    assert rel(got[:, 14], want[:, 14]) < 1e-13


# ------------------------------------------------------------------ fields
@pytest.mark.parametrize("N", [4, 16, 37])
def test_field_steps_fp64_parity(N):
    w = wl(N)
    st = oracle_init(w)
    ev = B.Event(w)
    upload_state(ev, st)
    k = 12
    ev.glasma_step(k)
    for n in range(k):
        st = O.field_step(st, n * w.dt, w.dt)
    g = download_state(ev)
    for a, b in [(g.U, st.U), (g.phi, st.phi), (g.e, st.e), (g.pi, st.pi)]:
        assert rel(a, b) < FP64_TOL
    o = ev.observables()
    assert o.gauss_max < 1e-12 and o.unitarity_max < 1e-12


def test_field_steps_fp32_error_bounds():
    w = wl(32, prec=W.FP32_2ROW)
    st = oracle_init(w)
    ev = B.Event(w)
    upload_state(ev, st)
    k = 24
    ev.glasma_step(k)
    for n in range(k):
        st = O.field_step(st, n * w.dt, w.dt)
    g = download_state(ev)
    errs = {name: rel(a, b) for name, a, b in [("U", g.U, st.U), ("phi", g.phi, st.phi), ("e", g.e, st.e),
                                               ("pi", g.pi, st.pi)]}
    print("FP32 two-row field error vs FP64 oracle after %d steps:" % k, errs)
    assert max(errs.values()) < 2e-5
    o = ev.observables()
    print("FP32 gauss_max %.3e unitarity_max %.3e" % (o.gauss_max, o.unitarity_max))
    assert o.unitarity_max < 1e-5


# ------------------------------------------------------------------ coupled
def _coupled(N, prec, steps, species=MIXED, seed=3):
    w = wl(N, prec=prec, species=species, seed=seed)
    st = oracle_init(w)
    part = oracle_particles(w)
    ev = B.Event(w)
    upload_state(ev, st)
    ev.upload(B.GL_BUF_PARTICLES, part)
    run = oracle_run(w, st, part)
    for _ in range(steps):
        run.step()
    ev.step(steps)
    return w, ev, run


# 4 and 5: a single tile wraps around the whole lattice several times, and
# every particle crosses the periodic boundary within a few cells
@pytest.mark.parametrize("N", [4, 5, 16, 37])
def test_coupled_fp64_parity(N):
    w, ev, run = _coupled(N, W.FP64, 30)
    got = ev.download(B.GL_BUF_PARTICLES)
    assert rel(got[:, :2], run.part[:, :2]) < FP64_TOL
    for sl in (slice(2, 3), slice(3, 5), slice(5, 6), slice(6, 14)):
        assert rel(got[:, sl], run.part[:, sl]) < FP64_TOL
    site = ev.download(B.GL_BUF_SITE)
    assert rel(site, run.site) < FP64_TOL
    g = download_state(ev)
    assert rel(g.U, run.st.U) < FP64_TOL and rel(g.e, run.st.e) < FP64_TOL
    # observables through the ABI against the oracle's sums (lattice units -> GeV^2)
    o = ev.observables()
    want = run.observables()
    a2 = w.a_GeVinv ** 2
    for k in range(len(w.species)):
        assert o.n_active[k] == int(want[k, 0])
        for got_v, want_v in [(o.sum_px2[k], want[k, 1]), (o.sum_py2[k], want[k, 2]),
                              (o.sum_pL2[k], want[k, 3]), (o.sum_dpT2[k], want[k, 4])]:
            assert abs(got_v * a2 - want_v) <= FP64_TOL * max(1.0, abs(want_v))
        # Casimirs conserved to rounding, relative to q2 = 4 (F) or 24 (A)
        qscale = 24.0 if w.species[k].rep == W.REP_A else 4.0
        assert o.casimir2_dev[k] < 1e-13 * qscale and o.casimir3_dev[k] < 1e-12 * qscale
    assert o.gauss_max < 1e-12


def per_particle_rel(got, want):
    scale = np.abs(want).max(axis=0, keepdims=True) + 1e-300
    return (np.abs(got - want) / scale).max(axis=1)


def ngp_cells(part, N, fp32):
    """NGP cell of every particle, floor(x + 1/2) in the state's precision
    (the rule both sides use), wrapped onto the lattice."""
    if fp32:
        x = part[:, :2].astype(np.float32)
        c = np.floor(x + np.float32(0.5)).astype(np.int64)
    else:
        c = np.floor(part[:, :2] + 0.5).astype(np.int64)
    return c % N


@pytest.mark.parametrize("N", [5, 32])
def test_coupled_fp32_error_bounds(N):
    # An FP32 position can round to the other side of a cell edge; the particle
    # then gathers another cell's fields and takes another colour rotation.
    # Those particles are found exactly, by comparing every step's NGP cells
    # with the oracle's, and left out; the maximum error of all the others is
    # bounded.
    w = wl(N, prec=W.FP32_2ROW, species=MIXED, seed=3)
    st = oracle_init(w)
    part = oracle_particles(w)
    ev = B.Event(w)
    upload_state(ev, st)
    ev.upload(B.GL_BUF_PARTICLES, part)
    run = oracle_run(w, st, part)
    got = ev.download(B.GL_BUF_PARTICLES)
    flipped = (ngp_cells(got, N, True) != ngp_cells(run.part, N, False)).any(axis=1)
    steps = 40
    for _ in range(steps):
        run.step()
        ev.step(1)
        got = ev.download(B.GL_BUF_PARTICLES)
        flipped |= (ngp_cells(got, N, True) != ngp_cells(run.part, N, False)).any(axis=1)
    keep = ~flipped
    e = {k: per_particle_rel(got[:, sl], run.part[:, sl])
         for k, sl in [("x", slice(0, 2)), ("p", slice(3, 5)), ("P_eta", slice(5, 6)), ("Q", slice(6, 14))]}
    summary = {k: (float(np.median(v[keep])), float(v[keep].max())) for k, v in e.items()}
    print("FP32 particle error vs FP64 oracle after %d steps, %d of %d particles without a cell flip "
          "(median, max):" % (steps, keep.sum(), len(keep)), summary)
    assert keep.sum() >= 0.9 * len(keep)
    assert all(s[1] < FP32_PARTICLE_TOL for s in summary.values())
    o = ev.observables()
    print("FP32 Casimir drift q2 %s q3 %s" % (list(o.casimir2_dev)[:4], list(o.casimir3_dev)[:4]))
    # relative to the species' q2 (4 fundamental, 24 adjoint): FP32 rounding of
    # the rotations and of the link unitarity
    for k, sp in enumerate(w.species):
        q2 = 24.0 if sp.rep == W.REP_A else 4.0
        assert o.casimir2_dev[k] / q2 < 2e-5 and o.casimir3_dev[k] / q2 < 2e-5


def test_small_workload_full_run_fp64():
    """32x32, L = 3 fm, 1000 charm quarks, 86 steps to tau = 1 fm/c, entirely
    from the GPU's own initial state and sampler, against the oracle."""
    w = W.config_small()
    ev = B.Event(w)
    ev.glasma_init()
    ev.wong_init()
    st = oracle_init(w)
    part = oracle_particles(w)
    run = oracle_run(w, st, part)
    short = 20
    ev.step(short)
    for _ in range(short):
        run.step()
    got = ev.download(B.GL_BUF_PARTICLES)
    assert rel(got[:, :6], run.part[:, :6]) < FP64_TOL      # single trajectories, short horizon
    ev.step(w.n_steps - short)
    for _ in range(w.n_steps - short):
        run.step()
    g = download_state(ev)
    field_err = max(rel(g.U, run.st.U), rel(g.e, run.st.e), rel(g.phi, run.st.phi), rel(g.pi, run.st.pi))
    print("full small run: field rel error %.3e" % field_err)
    assert field_err < FP64_TOL
    o = ev.observables()
    want = run.observables()
    a2 = w.a_GeVinv ** 2
    pT2 = (o.sum_px2[0] + o.sum_py2[0]) * a2 / o.n_active[0]
    pL2 = o.sum_pL2[0] * a2 / o.n_active[0]
    wpT2 = (want[0, 1] + want[0, 2]) / want[0, 0]
    wpL2 = want[0, 3] / want[0, 0]
    print("<pT^2> %.6e vs %.6e, <pL^2> %.6e vs %.6e (lattice units)" % (pT2, wpT2, pL2, wpL2))
    assert abs(pT2 - wpT2) < 1e-3 * wpT2 and abs(pL2 - wpL2) < 1e-3 * wpL2


# ------------------------------------------------------------------ full size, sampled
@pytest.mark.parametrize("prec,tol", [(W.FP64, FP64_TOL), (W.FP32_2ROW, 2e-5)])
def test_full_size_one_step_parity(prec, tol):
    """256x256 with 1e5 charm + 1e5 static quarks (the benchmark workload):
    GPU init and sampler, a few coupled steps, then one more coupled step on
    the GPU against the oracle's step from the downloaded state."""
    w = W.config_n256(precision=prec)
    ev = B.Event(w)
    ev.glasma_init()
    ev.wong_init()
    ev.step(10)
    st = download_state(ev)
    part = ev.download(B.GL_BUF_PARTICLES)
    run = oracle_run(w, st, part.copy())
    run.n = 10
    run.step()
    ev.step(1)
    g = download_state(ev)
    errs = [rel(g.U, run.st.U), rel(g.e, run.st.e), rel(g.phi, run.st.phi), rel(g.pi, run.st.pi)]
    site = ev.download(B.GL_BUF_SITE)
    errs.append(rel(site, run.site))
    got = ev.download(B.GL_BUF_PARTICLES)
    # exclude particles within 1e-3 of a cell edge before or after the step (FP32
    # rounding may put them in the other cell); none are excluded in FP64
    def near_edge(x):
        f = (x + 0.5) % 1.0
        return (np.minimum(f, 1 - f) < 1e-3).any(axis=1)
    keep = ~(near_edge(part[:, :2]) | near_edge(run.part[:, :2])) if prec == W.FP32_2ROW else np.ones(len(got), bool)
    perr = [rel(got[keep, sl], run.part[keep, sl]) for sl in (slice(0, 2), slice(3, 5), slice(5, 6), slice(6, 14))]
    print("full size one-step errors (fields, site, particles; %d of %d particles compared):" % (keep.sum(), len(keep)),
          errs, perr)
    assert max(errs) < tol
    assert max(perr) < tol
    o = ev.observables()
    assert o.gauss_max < (1e-11 if prec == W.FP64 else 1e-3)


# ------------------------------------------------------------------ edge cases
def test_zero_particles_and_inactive_species():
    late = W.Species(W.M_CHARM, 1e6, 10, W.REP_F, W.MOM_FIXED_PT, 1.0)
    w = wl(8, species=[late])
    ev = B.Event(w)
    ev.glasma_init()
    ev.wong_init()
    before = ev.download(B.GL_BUF_PARTICLES)
    ev.step(5)
    assert np.array_equal(ev.download(B.GL_BUF_PARTICLES), before)
    assert ev.observables().n_active[0] == 0
    w0 = wl(8)
    e0 = B.Event(w0)
    e0.glasma_init()
    e0.step(3)
    assert e0.observables().gauss_max < 1e-12


def test_cell_edge_ties_and_degenerate_momenta():
    # positions exactly on x = k + 1/2 (NGP rounds up), a massless particle at
    # rest (p^tau = 0: no motion), and static quarks
    sp = [W.Species(0.0, 0.0, 4, W.REP_F, W.MOM_FIXED_PT, 0.0), W.Species(2.0, 0.0, 4, W.REP_F, W.MOM_FIXED_PT, 1.0)]
    w = wl(8, species=sp)
    st = oracle_init(w)
    part = oracle_particles(w)
    part[:, 0] = [0.5, 3.5, 7.5, 2.0, 0.5, 6.5, 7.49999999, 1.5]
    part[:, 1] = [1.5, 0.5, 7.5, 4.5, 6.5, 3.0, 7.5, 2.5]
    ev = B.Event(w)
    upload_state(ev, st)
    ev.upload(B.GL_BUF_PARTICLES, part)
    run = oracle_run(w, st, part.copy())
    for _ in range(16):
        run.step()
    ev.step(16)
    got = ev.download(B.GL_BUF_PARTICLES)
    assert rel(got[:, :14], run.part[:, :14]) < FP64_TOL
    assert np.all(np.isfinite(got))


@pytest.mark.parametrize("prec", [W.FP64, W.FP32_2ROW])
def test_fields_independent_of_the_particles(prec):
    """The fields do not feel the particles: coupled steps, fields-only steps
    and an event without particles evolve them bitwise alike (one field
    kernel writes the site fields on every path).  Site fields overwritten by
    later field steps are not handed out."""
    def make(count):
        return wl(40, prec=prec, species=[W.Species(W.M_CHARM, 0.06, count, W.REP_F, W.MOM_UNIFORM_PT, 0.0, 5.0)])
    a = B.Event(make(300)); a.glasma_init(); a.wong_init(); a.step(8)
    b = B.Event(make(300)); b.glasma_init(); b.wong_init(); b.glasma_step(8)
    c = B.Event(make(0)); c.glasma_init(); c.step(8)
    for which in (B.GL_BUF_LINKS, B.GL_BUF_E, B.GL_BUF_PHI, B.GL_BUF_PI):
        ref = a.download(which)
        assert np.array_equal(ref, b.download(which)) and np.array_equal(ref, c.download(which))
    a.download(B.GL_BUF_SITE)                 # the last push's site fields are held
    for ev in (a, c):
        ev.glasma_step(2)                     # overwrites the buffer of that time's parity
        with pytest.raises(B.GlasmaError) as e:
            ev.download(B.GL_BUF_SITE)
        assert e.value.status == B.GL_ERR_STATE
        assert math.isnan(ev.observables().mean_trE_T2)


def test_call_order_errors():
    w = wl(8, species=[W.Species(W.M_CHARM, 0.0, 4)])
    ev = B.Event(w)
    ev.glasma_init()
    ev.wong_init()
    with pytest.raises(B.GlasmaError) as e:
        ev.wong_push()
    assert e.value.status == B.GL_ERR_STATE
    ev.glasma_step(2)
    with pytest.raises(B.GlasmaError) as e:
        ev.wong_push()
    assert e.value.status == B.GL_ERR_STATE
    with pytest.raises(B.GlasmaError) as e:
        ev.upload(B.GL_BUF_LINKS, np.zeros(10))
    assert e.value.status == B.GL_ERR_SIZE


# ------------------------------------------------------------------ light-like jets
JET_SPECIES = [W.Species(0.0, 0.0, 64, W.REP_F, W.MOM_EIKONAL_X, 0.0),
               W.Species(W.M_CHARM, 0.0, 32, W.REP_A, W.MOM_FIXED_PT, 0.5)]


@pytest.mark.parametrize("prec,tol", [(W.FP64, FP64_TOL), (W.FP32_2ROW, 2e-4)])
def test_jets_and_eikonal_parity(prec, tol):
    """Light-like jet-correlator probes and eikonal partons (Sec. 5.2) against
    the oracle: probe Wilson lines and force integrals, the partons' kicks and
    charges, and the charge-averaged broadening through the C ABI."""
    w = wl(24, prec=prec, species=JET_SPECIES, seed=5)
    w.n_jets = 50
    st = oracle_init(w)
    part = oracle_particles(w)
    jets = O.jets_init(w.N, w.seed, w.n_jets)
    ev = B.Event(w)
    upload_state(ev, st)
    ev.upload(B.GL_BUF_PARTICLES, part)
    ev.upload(B.GL_BUF_JETS, jets)
    run = oracle_run(w, st, part, jets=jets.copy())
    steps = 40
    for _ in range(steps):
        run.step()
    ev.step(steps)
    gj = ev.download(B.GL_BUF_JETS)
    assert rel(gj[:, :2], run.jets[:, :2]) < tol
    assert rel(gj[:, 2:20], run.jets[:, 2:20]) < tol       # Wilson lines
    assert rel(gj[:, 20:44], run.jets[:, 20:44]) < tol     # force integrals
    gp = ev.download(B.GL_BUF_PARTICLES)
    eik = gp[:, 15] == 0
    for sl in (slice(0, 3), slice(3, 6), slice(6, 14)):
        assert rel(gp[eik, sl], run.part[eik, sl]) < tol
    a2 = w.a_GeVinv ** 2
    got = np.array(ev.jets_observables()) * a2
    want = O.jets_obs(run.jets)
    assert np.abs(got - want).max() <= tol * np.abs(want).max()
    o = ev.observables()
    want_o = run.observables()
    assert abs(o.sum_pL2[0] * a2 - want_o[0, 3]) <= tol * abs(want_o[0, 3])


def test_eikonal_kicks_equal_probe_integrals_on_gpu():
    """Eikonal partons and probes started on the same paths: the partons'
    kicks are Q0 . X_i of the probes (charge rotated vs force transported), and
    the GPU's own probe initialisation equals the oracle's Philox positions."""
    w = wl(24, prec=W.FP64, species=JET_SPECIES[:1], seed=8)
    w.n_jets = 64
    ev = B.Event(w)
    ev.glasma_init()
    ev.wong_init()
    gj0 = ev.download(B.GL_BUF_JETS)
    assert np.array_equal(gj0[:, :2], O.jets_init(w.N, w.seed, w.n_jets)[:, :2])
    part = ev.download(B.GL_BUF_PARTICLES)
    probes = np.zeros((len(part), B.JET_LEN))
    probes[:, :2] = part[:, :2]
    for i in range(3):
        probes[:, 2 + 2 * (3 * i + i)] = 1.0
    w2 = wl(24, prec=W.FP64, species=JET_SPECIES[:1], seed=8)
    w2.n_jets = len(part)
    ev2 = B.Event(w2)
    for which in (B.GL_BUF_LINKS, B.GL_BUF_PHI, B.GL_BUF_E, B.GL_BUF_PI, B.GL_BUF_PARTICLES):
        ev2.upload(which, ev.download(which))
    ev2.upload(B.GL_BUF_JETS, probes)
    ev2.step(30)
    gp = ev2.download(B.GL_BUF_PARTICLES)
    X = ev2.download(B.GL_BUF_JETS)[:, 20:44].reshape(-1, 3, 8)
    kick = np.einsum("na,nia->ni", part[:, 6:14], X)
    assert np.abs(gp[:, 3:6] - kick).max() < 1e-12 * np.abs(kick).max()


def test_jets_need_a_single_event():
    w = wl(16, prec=W.FP32_2ROW, species=JET_SPECIES[:1])
    w.n_jets = 4
    with pytest.raises(B.GlasmaError):
        B.Batch([w])
    w.n_jets = 0
    ev = B.Event(w)
    with pytest.raises(B.GlasmaError) as e:
        ev.jets_observables()
    assert e.value.status == B.GL_ERR_STATE


def test_energy_density_download():
    """GL_BUF_ENERGY: tr of the squared site fields per site at the last pushed
    time, against the oracle's site fields, and its lattice mean against the
    FP64 field means of the observables."""
    w, ev, run = _coupled(16, W.FP64, 12)
    e = ev.download(B.GL_BUF_ENERGY)
    want = 0.5 * (run.site ** 2).sum(axis=(0, 2))
    assert rel(e, want) < FP64_TOL
    o = ev.observables()
    mean = o.mean_trE_T2 + o.mean_trE_L2 + o.mean_trB_T2 + o.mean_trB_L2
    assert abs(e.mean() - mean) <= 1e-12 * abs(mean)
    with pytest.raises(B.GlasmaError):
        ev.upload(B.GL_BUF_ENERGY, e)


def test_half_time_step_jets_parity():
    """dtau = a/16, the paper's time step for jets (Sec. 7.1): quark jets
    (m = 1 GeV, p^x = 10 GeV), eikonal partons and correlator probes through
    the coupled step, FP64 against the oracle."""
    species = [W.Species(1.0, 0.0, 40, W.REP_F, W.MOM_ALONG_X, 10.0),
               W.Species(0.0, 0.0, 40, W.REP_A, W.MOM_EIKONAL_X, 0.0)]
    w = wl(20, prec=W.FP64, species=species, seed=12)
    w.dtau_over_a = 1.0 / 16
    w.n_jets = 30
    st = oracle_init(w)
    part = oracle_particles(w)
    jets = O.jets_init(w.N, w.seed, w.n_jets)
    ev = B.Event(w)
    upload_state(ev, st)
    ev.upload(B.GL_BUF_PARTICLES, part)
    ev.upload(B.GL_BUF_JETS, jets)
    run = oracle_run(w, st, part, jets=jets.copy())
    for _ in range(48):
        run.step()
    ev.step(48)
    gp = ev.download(B.GL_BUF_PARTICLES)
    for sl in (slice(0, 2), slice(3, 6), slice(6, 14)):
        assert rel(gp[:, sl], run.part[:, sl]) < FP64_TOL
    assert rel(ev.download(B.GL_BUF_JETS), run.jets) < FP64_TOL
    g = download_state(ev)
    assert rel(g.U, run.st.U) < FP64_TOL and rel(g.e, run.st.e) < FP64_TOL


@pytest.mark.parametrize("prec,tol", [(W.FP64, FP64_TOL), (W.FP32_2ROW, 2e-4)])
def test_temporal_constraint_parity(prec, tol):
    """p^tau integrated from its own equation of motion (GL_BUF_PTAU) against
    the oracle's integration, with the same start at the first push and NaN
    for static, eikonal and not yet formed particles."""
    species = MIXED + [W.Species(0.0, 0.0, 20, W.REP_F, W.MOM_EIKONAL_X, 0.0)]
    w = wl(20, prec=prec, species=species, seed=6)
    w.ptau_diagnostic = True
    st = oracle_init(w)
    part = oracle_particles(w)
    ev = B.Event(w)
    upload_state(ev, st)
    ev.upload(B.GL_BUF_PARTICLES, part)
    assert np.all(np.isnan(ev.download(B.GL_BUF_PTAU)))
    run = oracle_run(w, st, part)
    run.ptau = np.full(len(part), np.nan)
    for _ in range(25):
        run.step()
    ev.step(25)
    got = ev.download(B.GL_BUF_PTAU)
    want = run.ptau
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    assert ok.sum() > 100
    assert rel(got[ok], want[ok]) < tol
    # checkpoint: the integration state can be saved and restored
    ev.upload(B.GL_BUF_PARTICLES, ev.download(B.GL_BUF_PARTICLES))
    assert np.all(np.isnan(ev.download(B.GL_BUF_PTAU)))
    ev.upload(B.GL_BUF_PTAU, got)
    assert np.array_equal(ev.download(B.GL_BUF_PTAU), got, equal_nan=True)
