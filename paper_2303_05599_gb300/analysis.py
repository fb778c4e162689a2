"""Post-processing of the ensemble observables, on the host.

The library reports per-species sums at each report time (gl_obs).  The
paper turns them into the quantities it plots:

- the momentum broadening <delta p_i^2>(tau) (Sec. 3.1);
- its classical-to-quantum mapping, a division by the dimension of the
  representation D_R = q2(R) / C2(R) (Sec. 6): D_F = 3 and D_A = 8 with the
  classical Casimirs q2(F) = 4, q2(A) = 24 of App. B;
- the instantaneous transport coefficients kappa_{L,T} = d<delta p_{L,T}^2>/dtau
  for heavy quarks and qhat_i = d<delta p_i^2>/dtau for jets (Sec. 7);
- the anisotropies <delta p_L^2>/<delta p_T^2> (heavy quarks) and
  <delta p_z^2>/<delta p_y^2> (jets);
- the Glasma energy density behind Figs. 6 and 9, from the lattice means of
  tr E^2 and tr B^2 or the per-site GL_BUF_ENERGY download.

Everything here is plain numpy on a handful of numbers per report.
"""
import numpy as np

HBARC = 0.1973269804  # GeV fm

REP_F, REP_A = 0, 1
# classical quadratic Casimirs (App. B) and group-theoretical ones of SU(3)
Q2 = {REP_F: 4.0, REP_A: 24.0}
C2 = {REP_F: 4.0 / 3.0, REP_A: 3.0}


def dimension(rep):
    """D_R = q2(R) / C2(R): 3 for the fundamental, 8 for the adjoint."""
    return Q2[rep] / C2[rep]


def quantum_broadening(dp2_classic, rep):
    """Classical <delta p^2> mapped to its quantum counterpart (Sec. 6):
    <dp^2>_classic / q2(R) = <dp^2>_quantum / C2(R)."""
    return np.asarray(dp2_classic, dtype=float) / dimension(rep)


def species_broadening(obs, k):
    """<delta p_T^2>, <delta p_L^2>, <p_x^2>, <p_y^2> of species k from one
    gl_obs record (GeV^2; NaN when no particle is active).  delta p_T^2 is
    p_T^2(tau) - p_T^2(tau_form); p_L starts at 0, so <delta p_L^2> = <p_L^2>."""
    n = obs.n_active[k]
    if n <= 0:
        return (np.nan,) * 4
    return (obs.sum_dpT2[k] / n, obs.sum_pL2[k] / n, obs.sum_px2[k] / n, obs.sum_py2[k] / n)


def instantaneous_rate(tau, dp2):
    """d<delta p^2>/dtau at the report times (kappa or qhat, Sec. 7):
    second-order central differences inside, one-sided at the ends."""
    tau = np.asarray(tau, dtype=float)
    dp2 = np.asarray(dp2, dtype=float)
    if tau.size < 2:
        raise ValueError("need at least two report times")
    return np.gradient(dp2, tau, edge_order=2 if tau.size > 2 else 1)


def anisotropy(numerator, denominator):
    """Ratio of two broadening components, e.g. <dp_L^2>/<dp_T^2>."""
    return np.asarray(numerator, dtype=float) / np.asarray(denominator, dtype=float)


def energy_density_GeV_fm3(tr_sum_lattice, a_fm, g):
    """Physical energy density from the lattice value tr(E^2 + B^2) of the
    site fields (E^ = g a^2 E, B^ = g a^2 B): eps = value / (g^2 a^4), in
    GeV^4, then / (hbar c)^3 for GeV/fm^3."""
    a = a_fm / HBARC  # GeV^-1
    return np.asarray(tr_sum_lattice, dtype=float) / (g * g * a ** 4) / HBARC ** 3


def mean_energy_lattice(obs):
    """Lattice mean of tr(E^2 + B^2) from one gl_obs record (GL_OBS_FIELDS)."""
    return obs.mean_trE_T2 + obs.mean_trE_L2 + obs.mean_trB_T2 + obs.mean_trB_L2


def ptau_constraint(records, ptau_integrated, mass_lattice, t):
    """Temporal-constraint diagnostic: relative difference between p^tau on the
    mass shell, sqrt(p_T^2 + w^2 + m^2) with w = P_eta / t, and p^tau
    integrated from its own equation of motion (GL_BUF_PTAU), per particle.
    records: canonical particle records [n][16] (lattice units); mass_lattice:
    lattice mass per species; t: lattice time of the records.  NaN where the
    integration has not started (inactive, static or eikonal particles)."""
    rec = np.asarray(records, dtype=float)
    pint = np.asarray(ptau_integrated, dtype=float)
    m = np.asarray(mass_lattice, dtype=float)[rec[:, 15].astype(int)]
    w = rec[:, 5] / t if t > 0 else np.zeros(len(rec))
    with np.errstate(invalid="ignore"):
        shell = np.sqrt(rec[:, 3] ** 2 + rec[:, 4] ** 2 + w * w + m * m)
        return (shell - pint) / shell
