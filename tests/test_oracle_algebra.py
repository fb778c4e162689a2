"""Pins of the oracle's SU(3) algebra, RNG and colour-charge constants against
what the paper prints (Tables I and II, the initial colour vectors of App. B)
and against textbook identities and library routines."""
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def test_generators_textbook():
    T = O.generators()
    for a in range(8):
        assert np.allclose(T[a], T[a].conj().T)
        assert abs(np.trace(T[a])) < 1e-15
        for b in range(8):
            assert abs(np.trace(T[a] @ T[b]) - 0.5 * (a == b)) < 1e-15
    # quadratic Casimir of the fundamental: sum_a T^a T^a = C2(F) 1 = 4/3 (App. B)
    assert np.allclose(sum(T[a] @ T[a] for a in range(8)), 4.0 / 3.0 * np.eye(3), atol=1e-15)


def test_structure_constants_match_tables():
    f = O.f_abc()
    d = O.d_abc()
    want_f = np.zeros((8, 8, 8))
    want_d = np.zeros((8, 8, 8))
    for kind, a, b, c, v in _read("su3_structure_constants.txt"):
        a, b, c, v = int(a) - 1, int(b) - 1, int(c) - 1, float(v)
        if kind == "f":
            for (i, j, k), s in [((a, b, c), 1), ((b, c, a), 1), ((c, a, b), 1),
                                 ((b, a, c), -1), ((a, c, b), -1), ((c, b, a), -1)]:
                want_f[i, j, k] = s * v
        else:
            for i, j, k in [(a, b, c), (b, c, a), (c, a, b), (b, a, c), (a, c, b), (c, b, a)]:
                want_d[i, j, k] = v
    assert np.abs(f - want_f).max() < 1e-14
    assert np.abs(d - want_d).max() < 1e-14


def test_commutator_and_cubic_casimir():
    T = O.generators()
    f = O.f_abc()
    d = O.d_abc()
    for a in range(8):
        for b in range(8):
            comm = T[a] @ T[b] - T[b] @ T[a]
            assert np.allclose(comm, 1j * np.einsum("c,cij->ij", f[a, b], T), atol=1e-15)
    # sum d_abc T^a T^b T^c = C3(F) 1 with C3(F) = (Nc^2-4)(Nc^2-1)/(4 Nc^2) = 10/9 (App. B)
    c3 = np.einsum("abc,aij,bjk,ckl->il", d, T, T, T)
    assert np.allclose(c3, 10.0 / 9.0 * np.eye(3), atol=1e-14)


def test_exp_against_library():
    rng = np.random.default_rng(7)
    T = O.generators()
    for scale in (1e-6, 0.1, 1.0, 4.0):
        x = rng.normal(size=8) * scale
        X = np.einsum("a,aij->ij", x, T)
        U = O.exp_i_alg(x)
        assert np.abs(U - scipy.linalg.expm(1j * X)).max() < 2e-15 * max(1.0, scale)
        assert np.abs(U @ U.conj().T - np.eye(3)).max() < 1e-14
        assert abs(np.linalg.det(U) - 1) < 1e-14
    M = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    assert np.abs(O.expm(M) - scipy.linalg.expm(M)).max() < 1e-13


def test_q3_is_four_trace_q_cubed():
    # App. A: tr(T^a T^b T^c) = (d_abc + i f_abc)/4 gives q3 = 4 tr(Q^3)
    rng = np.random.default_rng(3)
    T = O.generators()
    for _ in range(5):
        q = rng.normal(size=8)
        Q = np.einsum("a,aij->ij", q, T)
        q2, q3 = O.casimirs(q)
        assert abs(q2 - q @ q) < 1e-13
        assert abs(q3 - 4 * np.trace(Q @ Q @ Q).real) < 1e-12


def test_q0_vectors_match_paper():
    for rep_label, q2w, q3w, *vec in _read("q0_vectors.txt"):
        rep = 0 if rep_label == "F" else 1
        q = O.q0(rep)
        assert np.abs(q - np.array([float(v) for v in vec])).max() < 6e-6  # six printed digits
        q2, q3 = O.casimirs(q)
        assert abs(q2 - float(q2w)) < 1e-13
        assert abs(q3 - float(q3w)) < 1e-13
    # closed forms of App. B with Nc = 3
    Nc = 3
    assert abs(O.casimirs(O.q0(0))[0] - (Nc * Nc - 1) / 2) < 1e-13
    assert abs(O.casimirs(O.q0(0))[1] - (Nc * Nc - 4) * (Nc * Nc - 1) / (4 * Nc)) < 1e-13
    assert abs(O.casimirs(O.q0(1))[0] - Nc * (Nc * Nc - 1)) < 1e-13


def test_philox_known_answers():
    for row in _read("philox4x32_10_kat.txt"):
        vals = [int(v, 16) for v in row]
        out = O.philox(vals[0:4], vals[4:6])
        assert [int(v) for v in out] == vals[6:10]


def test_fft_against_numpy():
    rng = np.random.default_rng(5)
    for n in (8, 64, 12):
        x = rng.normal(size=n) + 1j * rng.normal(size=n)
        assert np.abs(O.fft(x, -1) - np.fft.fft(x)).max() < 1e-12
        assert np.abs(O.fft(x, +1) - np.fft.ifft(x) * n).max() < 1e-12
