"""The allocation-free entry point gl_ensemble_sums_noalloc, for callers that
cannot allocate device memory (their host owns every device allocation, or
their device footprint is fixed after start-up).  It is called through the C
ABI on particle records the test holds on the device and must agree with the
sums that observables() reports for the same state, and with the oracle's
per-species sums of the same records, on two calls in a row with different
states (its fixed scratch array keeps the previous call's contents, which
must not leak into the next result).  The ensemble includes Wong quarks,
static quarks and eikonal light-like partons, whose p_L is the accumulated
longitudinal momentum; a NaN charge shows up as a NaN Casimir deviation."""
import ctypes
import math

import numpy as np
import pytest

import oracle as O
from paper_2303_05599_gb300 import _binding as B
from paper_2303_05599_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2303_05599_gb300 import build
    build.build()
    B.lib()


def _context_sums(ev, w):
    """observables() sums per species, converted back to lattice units."""
    o = ev.observables()
    a2 = w.a_GeVinv ** 2
    out = []
    for k in range(len(w.species)):
        out.append([o.n_active[k], o.sum_px2[k] * a2, o.sum_py2[k] * a2, o.sum_pL2[k] * a2, o.sum_dpT2[k] * a2,
                    o.casimir2_dev[k], o.casimir3_dev[k]])
    return np.array(out)


def _kinds(w):
    ls = w.lattice_species()
    return O.kinds_of([s[0] for s in ls], [s.mom_mode for s in w.species])


def _mask(w, pushed_step):
    mask = 0
    for k, s in enumerate(w.lattice_species()):
        if pushed_step * w.dt >= s[1]:
            mask |= 1 << k
    return mask


def _noalloc_call(rec_host, w, mask, t):
    rec = torch.from_numpy(np.ascontiguousarray(rec_host)).cuda()
    ns = len(w.species)
    ls = w.lattice_species()
    mass = (ctypes.c_double * ns)(*[s[0] for s in ls])
    rep = (ctypes.c_int32 * ns)(*[s.rep for s in w.species])
    kind = (ctypes.c_int32 * ns)(*[int(k) for k in _kinds(w)])
    out = torch.full((ns * 7,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    st = B.lib().gl_ensemble_sums_noalloc(ctypes.c_void_p(rec.data_ptr()), rec.shape[0], ns, mass, rep, kind, mask,
                                          t, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert st == B.GL_OK
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(ns, 7)


def _oracle_sums(rec, w, mask, t):
    ls = w.lattice_species()
    act = [(mask >> k) & 1 for k in range(len(ls))]
    return O.particle_obs(np.ascontiguousarray(rec), t, [s[0] for s in ls], act, [s.rep for s in w.species],
                          _kinds(w))[:, :7]


def _close(a, b):
    scale = np.maximum(1.0, np.abs(b))
    assert np.all(np.abs(a - b) <= TOL * scale + 1e-13), (a, b)


WORKLOAD = dict(N=16, L_fm=1.5, Ns=4, precision=W.FP64, seed=7,
                species=[W.Species(W.M_CHARM, 0.0, 700, W.REP_F, W.MOM_FIXED_PT, 0.5),
                         W.Species(float("inf"), 0.0, 300, W.REP_A, W.MOM_FIXED_PT, 0.0),
                         W.Species(0.0, 0.05, 500, W.REP_F, W.MOM_ALONG_X, 10.0),
                         W.Species(0.0, 0.0, 400, W.REP_A, W.MOM_EIKONAL_X, 0.0)])


def test_noalloc_sums_match_observables_and_the_oracle_on_two_calls():
    w = W.Workload("noalloc", **WORKLOAD)
    ev = B.Event(w)
    ev.glasma_init()
    ev.wong_init()
    results = []
    for steps, total in ((5, 5), (4, 9)):
        ev.step(steps)
        rec = ev.download(B.GL_BUF_PARTICLES)
        mask, t = _mask(w, total - 1), total * w.dt
        got = _noalloc_call(rec, w, mask, t)
        _close(got, _context_sums(ev, w))
        _close(got, _oracle_sums(rec, w, mask, t))
        results.append(got)
    assert not np.allclose(results[0][:, 1:5], results[1][:, 1:5])
    # the eikonal partons have a non-zero accumulated p_L
    assert results[1][3, 3] > 0


def test_noalloc_propagates_nan():
    w = W.Workload("noalloc", **WORKLOAD)
    ev = B.Event(w)
    ev.glasma_init()
    ev.wong_init()
    ev.step(3)
    rec = ev.download(B.GL_BUF_PARTICLES)
    clean = _noalloc_call(rec, w, _mask(w, 2), 3 * w.dt)
    bad = rec.copy()
    i = int(np.flatnonzero(bad[:, 15] == 1)[17])   # a static quark
    bad[i, 8] = math.nan
    got = _noalloc_call(bad, w, _mask(w, 2), 3 * w.dt)
    assert math.isnan(got[1, 5]) and math.isnan(got[1, 6])
    assert np.array_equal(got[1, :5], clean[1, :5])
    assert np.array_equal(np.delete(got, 1, axis=0), np.delete(clean, 1, axis=0))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    mass = (ctypes.c_double * 1)(1.0)
    rep = (ctypes.c_int32 * 1)(0)
    kind = (ctypes.c_int32 * 1)(0)
    st = B.lib().gl_ensemble_sums_noalloc(ctypes.c_void_p(dummy.data_ptr()), B.GL_NOALLOC_MAX_PARTICLES + 1, 1,
                                          mass, rep, kind, 1, 1.0, ctypes.c_void_p(out.data_ptr()), None)
    assert st == B.GL_ERR_SIZE
    bad_kind = (ctypes.c_int32 * 1)(5)
    st = B.lib().gl_ensemble_sums_noalloc(ctypes.c_void_p(dummy.data_ptr()), 1, 1, mass, rep, bad_kind, 1, 1.0,
                                          ctypes.c_void_p(out.data_ptr()), None)
    assert st == B.GL_ERR_ARG
