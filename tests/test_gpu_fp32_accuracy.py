"""Accuracy of the FP32 two-row path at late tau against the FP64 oracle.

Two runs are taken to their tau_max from the oracle's own initial state and
particles, on the GPU in FP32 (links stored as two rows, re-unitarised in
FP64 once every 64 steps per row) and in the oracle in FP64:

- the 32x32 workload (L = 3 fm, 1000 charm quarks from tau_form = 0.06 fm/c,
  86 steps to tau = 1 fm/c);
- one 256x256 event (L = 10 fm, 1e5 charm quarks with p_T = 0.5 GeV and 1e5
  static quarks, 205 steps to tau = 1 fm/c, three re-unitarisation periods).

At tau_max the relative errors of the per-species ensemble averages <p_T^2>,
<p_L^2> and <delta p_T^2> (Sec. 3.1, momentum broadening), of the fields and
of the lattice means of the squared site fields (the energy density, Figs. 6
and 9) are printed and bounded.  The FP32 bounds follow from FP32 rounding
(2^-24 per operation) accumulated over a few hundred steps: the fields drift
by ~1e-5 relative, and ensemble averages over 1e3-1e5 particles, whose
individual momenta carry that error, stay within a few 1e-5 (cell-edge
flips of single particles are O(1) for those particles but a small fraction
of the ensemble)."""
import numpy as np
import pytest

import oracle as O
from paper_2303_05599_gb300 import _binding as B
from paper_2303_05599_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2303_05599_gb300 import build
    build.build()
    B.lib()


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(1e-300, np.abs(b).max()))


def ensemble(obs_rows, n_species):
    """<p_T^2>, <p_L^2>, <delta p_T^2> per species (lattice units) from the
    oracle's per-species sums [n, px2, py2, pL2, dpT2, ...]."""
    out = []
    for k in range(n_species):
        n = obs_rows[k, 0]
        out.append(((obs_rows[k, 1] + obs_rows[k, 2]) / n, obs_rows[k, 3] / n, obs_rows[k, 4] / n))
    return np.array(out)


def gpu_ensemble(o, w):
    a2 = w.a_GeVinv ** 2
    out = []
    for k in range(len(w.species)):
        n = o.n_active[k]
        out.append(((o.sum_px2[k] + o.sum_py2[k]) * a2 / n, o.sum_pL2[k] * a2 / n, o.sum_dpT2[k] * a2 / n))
    return np.array(out)


def site_means(site):
    """Lattice means of tr E_T^2, tr E_L^2, tr B_T^2, tr B_L^2 (tr X^2 = X^a X^a / 2)."""
    sq = 0.5 * (site ** 2).sum(axis=2)  # [6, V]
    return np.array([sq[0].mean() + sq[1].mean(), sq[2].mean(), sq[3].mean() + sq[4].mean(), sq[5].mean()])


def run_both(w):
    w.precision = W.FP32_2ROW
    st, bad = O.mv_init(w.N, w.Ns, w.g2mu_a, w.m_a, w.Lambda_a, w.seed)
    assert bad == 0
    ls = w.lattice_species()
    part = np.concatenate([O.sample_species(w.N, w.seed, k, s.rep, s.mom_mode, ls[k][2], ls[k][3], s.count)
                           for k, s in enumerate(w.species)])
    ev = B.Event(w)
    for which, arr in ((B.GL_BUF_LINKS, st.U), (B.GL_BUF_PHI, st.phi), (B.GL_BUF_E, st.e), (B.GL_BUF_PI, st.pi),
                       (B.GL_BUF_PARTICLES, part)):
        ev.upload(which, arr)
    kind = O.kinds_of([s[0] for s in ls], [s.mom_mode for s in w.species])
    run = O.Run(st, part.copy(), [s[0] for s in ls], [s[1] for s in ls], [s.rep for s in w.species], w.dt, kind=kind)
    for _ in range(w.n_steps):
        run.step()
    ev.step(w.n_steps)
    return ev, run


def report(w, ev, run):
    g = O.FieldState(w.N, ev.download(B.GL_BUF_LINKS), ev.download(B.GL_BUF_PHI), ev.download(B.GL_BUF_E),
                     ev.download(B.GL_BUF_PI))
    fields = {"U": rel(g.U, run.st.U), "phi": rel(g.phi, run.st.phi), "e": rel(g.e, run.st.e),
              "pi": rel(g.pi, run.st.pi)}
    site_g = site_means(ev.download(B.GL_BUF_SITE))
    site_o = site_means(run.site)
    means = np.abs(site_g / site_o - 1)
    o = ev.observables()
    ens_g = gpu_ensemble(o, w)
    ens_o = ensemble(run.observables(), len(w.species))
    ens = np.abs(ens_g / ens_o - 1)
    print("\n%s, FP32 vs FP64 oracle at tau = %.3f fm/c after %d steps:" % (w.name, w.n_steps * w.dt * w.a_fm,
                                                                           w.n_steps))
    print("  fields (max relative):", {k: "%.2e" % v for k, v in fields.items()})
    print("  site-field means tr E_T^2, E_L^2, B_T^2, B_L^2 (relative):", ["%.2e" % v for v in means])
    for k, s in enumerate(w.species):
        print("  species %d (m = %s GeV): <p_T^2> %.3e rel err %.2e; <p_L^2> %.3e rel err %.2e; "
              "<delta p_T^2> %.3e rel err %.2e" % (k, s.mass_GeV, ens_o[k, 0], ens[k, 0], ens_o[k, 1], ens[k, 1],
                                                   ens_o[k, 2], ens[k, 2]))
    print("  gauss_max %.2e unitarity_max %.2e" % (o.gauss_max, o.unitarity_max))
    return fields, means, ens, o


def test_fp32_small_workload_to_tau_max():
    w = W.config_small()
    ev, run = run_both(w)
    fields, means, ens, o = report(w, ev, run)
    assert max(fields.values()) < 1e-4
    assert means.max() < 1e-4
    assert ens.max() < 1e-3
    assert o.unitarity_max < 2e-5


def test_fp32_256_event_to_tau_max():
    w = W.config_n256()
    ev, run = run_both(w)
    fields, means, ens, o = report(w, ev, run)
    assert w.n_steps >= 3 * w.reunit_every
    assert max(fields.values()) < 2e-4
    assert means.max() < 1e-4
    assert ens.max() < 1e-3
    assert o.unitarity_max < 3e-5
