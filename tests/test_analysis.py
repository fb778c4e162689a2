"""Host post-processing of the ensemble observables (Sec. 6 and 7): the
classical-to-quantum mapping by D_R, the transport coefficients as time
derivatives, anisotropies and the energy density in physical units."""
import math
from types import SimpleNamespace

import numpy as np
import pytest

from paper_2303_05599_gb300 import analysis as A


def test_dimension_of_the_representation():
    # D_R = q2(R) / C2(R) with the classical Casimirs of App. B: the SU(3)
    # dimensions 3 and 8
    assert A.dimension(A.REP_F) == pytest.approx(3.0, rel=1e-15)
    assert A.dimension(A.REP_A) == pytest.approx(8.0, rel=1e-15)
    # Casimir scaling after the mapping: a classical ratio q2(A)/q2(F) = 6
    # becomes C2(A)/C2(F) = 9/4
    q = A.quantum_broadening(6.0, A.REP_A) / A.quantum_broadening(1.0, A.REP_F)
    assert q == pytest.approx(9.0 / 4.0, rel=1e-15)


def test_instantaneous_rate_is_exact_for_quadratics():
    tau = np.array([0.1, 0.15, 0.3, 0.35, 0.6, 1.0])
    dp2 = 2.0 + 3.0 * tau - 0.7 * tau ** 2
    assert np.allclose(A.instantaneous_rate(tau, dp2), 3.0 - 1.4 * tau, rtol=0, atol=1e-12)
    with pytest.raises(ValueError):
        A.instantaneous_rate([0.1], [1.0])


def test_species_broadening_and_anisotropy():
    o = SimpleNamespace(n_active=[4, 0], sum_dpT2=[8.0, 0], sum_pL2=[2.0, 0], sum_px2=[5.0, 0], sum_py2=[3.0, 0])
    dT, dL, px2, py2 = A.species_broadening(o, 0)
    assert (dT, dL, px2, py2) == (2.0, 0.5, 1.25, 0.75)
    assert all(math.isnan(v) for v in A.species_broadening(o, 1))
    assert A.anisotropy(dL, dT) == 0.25


def test_energy_density_units():
    # a lattice value v at spacing a (fm) and coupling g is v / (g^2 a^4) in
    # GeV^4; 1 GeV^4 = 1 / (hbar c)^3 GeV/fm^3
    a_fm, g, v = 0.04, 2.0, 0.5
    a = a_fm / A.HBARC
    assert A.energy_density_GeV_fm3(v, a_fm, g) == pytest.approx(v / (g * g * a ** 4) / A.HBARC ** 3, rel=1e-15)
    assert A.energy_density_GeV_fm3(1.0, A.HBARC, 1.0) == pytest.approx(1.0 / A.HBARC ** 3, rel=1e-15)
    o = SimpleNamespace(mean_trE_T2=1.0, mean_trE_L2=2.0, mean_trB_T2=3.0, mean_trB_L2=4.0)
    assert A.mean_energy_lattice(o) == 10.0


def test_ptau_constraint_relative_difference():
    rec = np.zeros((3, 16))
    rec[:, 3] = [0.3, 0.0, 1.0]
    rec[:, 5] = [0.0, 2.0, 0.0]
    rec[:, 15] = [0, 0, 1]
    t = 4.0
    shell = np.sqrt(np.array([0.09 + 0.25, 0.25 + 0.25, 1.0 + np.inf]))
    got = A.ptau_constraint(rec, [shell[0], 0.99 * shell[1], np.nan], [0.5, np.inf], t)
    assert got[0] == 0.0 and got[1] == pytest.approx(0.01) and np.isnan(got[2])
