"""Small numpy helpers for the tests: Gell-Mann generators, algebra/matrix
conversion, gauge transformations and a pure-Python Philox4x32-10.  These are
written independently of both the oracle and the CUDA library."""
import math

import numpy as np


def gellmann_half():
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1] = -1j; l[1][1, 0] = 1j
    l[2][0, 0] = 1; l[2][1, 1] = -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2] = -1j; l[4][2, 0] = 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2] = -1j; l[6][2, 1] = 1j
    l[7] = np.diag([1, 1, -2]) / math.sqrt(3)
    return l / 2


T = gellmann_half()


def alg2mat(x):
    return np.einsum("...a,aij->...ij", x, T)


def mat2alg(m):
    return 2 * np.einsum("...ij,aji->...a", m, T).real


def links(U):
    """canonical [2][V][18] doubles -> [2, V, 3, 3] complex"""
    return np.ascontiguousarray(U).view(np.complex128).reshape(2, -1, 3, 3)


def links_to_canon(u):
    return np.ascontiguousarray(u, dtype=np.complex128).reshape(2, -1, 9).view(np.float64).reshape(2, -1, 18)


def shift(N, s, dx, dy):
    x = s % N
    y = s // N
    return ((y + dy) % N) * N + (x + dx) % N


def random_su3(rng, n, scale=1.0):
    import scipy.linalg
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for k in range(n):
        out[k] = scipy.linalg.expm(1j * alg2mat(rng.normal(size=8) * scale))
    return out


def gauge_transform(N, U, phi, e, pi, Om):
    """U_i(x) -> O(x) U_i(x) O(x+i)^+, site and left-end link fields -> O X O^+"""
    V = N * N
    s = np.arange(V)
    u = links(U).copy()
    for d, (dx, dy) in enumerate([(1, 0), (0, 1)]):
        u[d] = Om @ u[d] @ Om[shift(N, s, dx, dy)].conj().transpose(0, 2, 1)
    Od = Om.conj().transpose(0, 2, 1)
    ph = mat2alg(Om @ alg2mat(phi) @ Od)
    p = mat2alg(Om @ alg2mat(pi) @ Od)
    ee = np.stack([mat2alg(Om @ alg2mat(e[d]) @ Od) for d in range(2)])
    return links_to_canon(u), ph, ee, p


M0, M1, W0, W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85


def philox(c, k):
    c = list(c)
    k = list(k)
    for _ in range(10):
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        c = [(p1 >> 32) ^ c[1] ^ k[0], p1 & 0xFFFFFFFF, (p0 >> 32) ^ c[3] ^ k[1], p0 & 0xFFFFFFFF]
        k = [(k[0] + W0) & 0xFFFFFFFF, (k[1] + W1) & 0xFFFFFFFF]
    return c


def u01(r):
    return (r + 0.5) / 4294967296.0


def box_muller(u1, u2):
    rad = math.sqrt(-2.0 * math.log(u1))
    return rad * math.cos(2 * math.pi * u2), rad * math.sin(2 * math.pi * u2)
