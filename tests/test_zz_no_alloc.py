"""The allocation-free entry point gl_ensemble_sums_noalloc, for callers that
cannot allocate device memory (their host owns every device allocation, or
their device footprint is fixed after start-up).  It is called through the C
ABI on particle records the test holds on the device and must agree with the
sums that observables() reports for the same state, on two calls in a row
with different states (its fixed scratch array keeps the previous call's
contents, which must not leak into the next result)."""
import ctypes

import numpy as np
import pytest

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


def _noalloc_sums(ev, w, pushed_step, t):
    rec = torch.from_numpy(ev.download(B.GL_BUF_PARTICLES)).cuda()
    ns = len(w.species)
    ls = w.lattice_species()
    mass = (ctypes.c_double * ns)(*[s[0] for s in ls])
    rep = (ctypes.c_int32 * ns)(*[s.rep for s in w.species])
    mask = 0
    for k, s in enumerate(ls):
        if pushed_step * w.dt >= s[1]:
            mask |= 1 << k
    out = torch.full((ns * 7,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    st = B.lib().gl_ensemble_sums_noalloc(ctypes.c_void_p(rec.data_ptr()), rec.shape[0], ns, mass, rep, mask, t,
                                          ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert st == B.GL_OK
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(ns, 7)


def _close(a, b):
    scale = np.maximum(1.0, np.abs(b))
    assert np.all(np.abs(a - b) <= TOL * scale + 1e-13), (a, b)


def test_noalloc_sums_match_observables_on_two_calls():
    w = W.Workload("noalloc", N=16, L_fm=1.5, Ns=4, precision=W.FP64, seed=7,
                   species=[W.Species(W.M_CHARM, 0.0, 700, W.REP_F, W.MOM_FIXED_PT, 0.5),
                            W.Species(float("inf"), 0.0, 300, W.REP_A, W.MOM_FIXED_PT, 0.0),
                            W.Species(0.0, 0.05, 500, W.REP_F, W.MOM_ALONG_X, 10.0)])
    ev = B.Event(w)
    ev.glasma_init()
    ev.wong_init()
    ev.step(5)
    first = _noalloc_sums(ev, w, 4, 5 * w.dt)
    _close(first, _context_sums(ev, w))
    ev.step(4)
    second = _noalloc_sums(ev, w, 8, 9 * w.dt)
    _close(second, _context_sums(ev, w))
    assert not np.allclose(first[:, 1:5], second[:, 1:5])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    mass = (ctypes.c_double * 1)(1.0)
    rep = (ctypes.c_int32 * 1)(0)
    st = B.lib().gl_ensemble_sums_noalloc(ctypes.c_void_p(dummy.data_ptr()), B.GL_NOALLOC_MAX_PARTICLES + 1, 1,
                                          mass, rep, 1, 1.0, ctypes.c_void_p(out.data_ptr()), None)
    assert st == B.GL_ERR_SIZE
