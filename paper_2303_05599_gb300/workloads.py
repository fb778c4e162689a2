"""Workload definitions: the synthetic MV events and particle ensembles of the
paper's production setup (Sec. 7.1) at the five sizes the benchmarks and
parity tests use, and their conversion to lattice units.

This module holds configuration only (sizes, seeds, physical parameters and
unit conversion); it contains none of the method's arithmetic and is shared by
the CUDA path's callers and by the tests that drive the oracle.
"""
from dataclasses import dataclass, field
import math
from typing import List

HBARC = 0.1973269804  # GeV fm

M_CHARM = 1.27   # GeV (Sec. 7.1)
M_BEAUTY = 4.18  # GeV (Sec. 7.1)

# momentum modes of a species
MOM_FIXED_PT = 0     # |p_T| = p0, uniform azimuth
MOM_UNIFORM_PT = 1   # |p_T| ~ U[p0, p1], uniform azimuth
MOM_ALONG_X = 2      # p^x = p0, p^y = 0
MOM_EIKONAL_X = 3    # eikonal light-like parton along +x: fixed path, momenta record the kicks

REP_F = 0  # fundamental classical charge, q2 = 4, q3 = 10/3
REP_A = 1  # adjoint classical charge, q2 = 24, q3 = 0

FP64 = 0
FP32_2ROW = 1


@dataclass
class Species:
    mass_GeV: float
    tau_form_fm: float
    count: int
    rep: int = REP_F
    mom_mode: int = MOM_FIXED_PT
    p0_GeV: float = 0.0
    p1_GeV: float = 0.0


@dataclass
class Workload:
    name: str
    N: int
    L_fm: float
    g2mu_GeV: float = 2.0
    mIR_GeV: float = 0.2
    LambdaUV_GeV: float = 10.0
    Ns: int = 50
    dtau_over_a: float = 0.125
    tau_max_fm: float = 1.0
    precision: int = FP64
    reunit_every: int = 64
    sort_every: int = 32
    n_jets: int = 0              # light-like jet-correlator probes (single events)
    ptau_diagnostic: bool = False  # integrate p^tau beside the mass shell (GL_BUF_PTAU)
    seed: int = 0
    species: List[Species] = field(default_factory=list)
    report_every_fm: float = 0.0

    # lattice-unit values (identical expressions to the C library's)
    @property
    def a_fm(self):
        return self.L_fm / self.N

    @property
    def a_GeVinv(self):
        return self.L_fm / self.N / HBARC

    @property
    def g2mu_a(self):
        return self.g2mu_GeV * (self.L_fm / self.N / HBARC)

    @property
    def m_a(self):
        return self.mIR_GeV * (self.L_fm / self.N / HBARC)

    @property
    def Lambda_a(self):
        return self.LambdaUV_GeV * (self.L_fm / self.N / HBARC) if self.LambdaUV_GeV > 0 else 0.0

    @property
    def dt(self):
        return self.dtau_over_a

    @property
    def n_steps(self):
        return int(math.ceil(self.tau_max_fm / (self.dtau_over_a * self.L_fm / self.N) - 1e-9))

    @property
    def n_particles(self):
        return sum(s.count for s in self.species)

    def lattice_species(self):
        """(mass, t_form, p0, p1) per species in lattice units."""
        a = self.L_fm / self.N / HBARC
        out = []
        for s in self.species:
            m = math.inf if math.isinf(s.mass_GeV) else s.mass_GeV * a
            out.append((m, s.tau_form_fm * self.N / self.L_fm, s.p0_GeV * a, s.p1_GeV * a))
        return out


def config_small():
    """32x32, L = 3 fm, FP64, 1000 charm quarks at rest, tau_form = 0.06 fm/c."""
    return Workload("small_N32_fp64", N=32, L_fm=3.0, precision=FP64, seed=0,
                    species=[Species(M_CHARM, 0.06, 1000, REP_F, MOM_FIXED_PT, 0.0)])


def config_n256(precision=FP32_2ROW):
    """256x256, L = 10 fm: 1e5 charm (p_T = 0.5 GeV) + 1e5 static quarks."""
    return Workload("n256_charm_static", N=256, L_fm=10.0, precision=precision, seed=0,
                    species=[Species(M_CHARM, 0.06, 100_000, REP_F, MOM_FIXED_PT, 0.5),
                             Species(math.inf, 0.06, 100_000, REP_F, MOM_FIXED_PT, 0.0)])


def config_n512(precision=FP32_2ROW):
    """512x512, L = 10 fm: 5e5 beauty (p_T = 2 GeV) + 5e5 light-like jets (|p| = 10 GeV)."""
    return Workload("n512_beauty_jets", N=512, L_fm=10.0, precision=precision, seed=0,
                    species=[Species(M_BEAUTY, 0.02, 500_000, REP_F, MOM_FIXED_PT, 2.0),
                             Species(0.0, 0.0, 500_000, REP_F, MOM_FIXED_PT, 10.0)])


def config_batched_events():
    """64 events, N in {64, 128, 256} (event e: [64,128,256][e % 3]), a = 0.04 fm,
    1e4 charm quarks each with p_T ~ U[0, 5] GeV, seed e."""
    evs = []
    for e in range(64):
        N = (64, 128, 256)[e % 3]
        evs.append(Workload("batched_e%d" % e, N=N, L_fm=0.04 * N, precision=FP32_2ROW, seed=e,
                            species=[Species(M_CHARM, 0.06, 10_000, REP_F, MOM_UNIFORM_PT, 0.0, 5.0)]))
    return evs


def config_n1024(precision=FP32_2ROW):
    """1024x1024, L = 10 fm, to tau = 2 fm/c: 4e6 particles in equal thirds of
    charm (p_T = 0.5 GeV), beauty (p_T = 2 GeV) and light-like jets (|p| = 10 GeV)."""
    n = 4_000_000
    c = [n - 2 * (n // 3), n // 3, n // 3]
    return Workload("n1024_mixed", N=1024, L_fm=10.0, precision=precision, seed=0, tau_max_fm=2.0,
                    report_every_fm=0.05,
                    species=[Species(M_CHARM, 0.06, c[0], REP_F, MOM_FIXED_PT, 0.5),
                             Species(M_BEAUTY, 0.02, c[1], REP_F, MOM_FIXED_PT, 2.0),
                             Species(0.0, 0.0, c[2], REP_F, MOM_FIXED_PT, 10.0)])


def config_jets_dt16(precision=FP32_2ROW):
    """The paper's jet setup (Sec. 7.1): 1024x1024, L = 10 fm, dtau = a/16, to
    tau = 1 fm/c; quark jets with m = 1 GeV and p^x = 10 GeV (Sec. 7.3), eikonal
    light-like partons along +x (the limit they approach) and jet-correlator
    probes on the same kind of paths (single event)."""
    return Workload("jets_n1024_dt16", N=1024, L_fm=10.0, precision=precision, seed=0, dtau_over_a=1.0 / 16,
                    n_jets=100_000,
                    species=[Species(1.0, 0.0, 100_000, REP_F, MOM_ALONG_X, 10.0),
                             Species(0.0, 0.0, 100_000, REP_F, MOM_EIKONAL_X, 0.0)])


WORKLOADS = {
    "small_N32_fp64": config_small,
    "n256_charm_static": config_n256,
    "n512_beauty_jets": config_n512,
    "n1024_mixed": config_n1024,
    "jets_n1024_dt16": config_jets_dt16,
}
