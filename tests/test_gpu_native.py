"""Native snapshots (gl_download_native, gl_upload_native,
gl_batch_upload_native): the fields of the current time slice and the particle
arrays as the bytes of the device layout.  A run restored from them evolves
bitwise like the uninterrupted one, per event and per batch; sizes are
checked; and out-of-range species or original indices in an uploaded particle
snapshot are reported (GL_ERR_ARG) and repaired on the device, so that later
calls stay inside their arrays."""
import ctypes
import math

import numpy as np
import pytest

from paper_2303_05599_gb300 import _binding as B
from paper_2303_05599_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CANON = (B.GL_BUF_LINKS, B.GL_BUF_PHI, B.GL_BUF_E, B.GL_BUF_PI, B.GL_BUF_PARTICLES)
OBS_ARRAYS = ("n_active", "sum_px2", "sum_py2", "sum_pL2", "sum_dpT2", "casimir2_dev", "casimir3_dev")


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2303_05599_gb300 import build
    build.build()
    B.lib()


def events(prec):
    out = []
    for e, N in enumerate([16, 40, 24]):
        out.append(W.Workload("nat%d" % e, N=N, L_fm=0.04 * N * 2, Ns=4, precision=prec, seed=41 + e,
                              sort_every=4,
                              species=[W.Species(W.M_CHARM, 0.06, 300 + 50 * e, W.REP_F, W.MOM_UNIFORM_PT, 0.0, 5.0),
                                       W.Species(math.inf, 0.0, 40, W.REP_A, W.MOM_FIXED_PT, 0.0)]))
    return out


def same_state(a, b, n_species):
    for which in CANON:
        assert np.array_equal(a.download(which), b.download(which)), which
    oa, ob = a.observables(), b.observables()
    for f in OBS_ARRAYS:
        x, y = list(getattr(oa, f))[:n_species], list(getattr(ob, f))[:n_species]
        assert np.array_equal(x, y), (f, x, y)


@pytest.mark.parametrize("prec", [W.FP64, W.FP32_2ROW])
def test_event_restored_from_a_native_snapshot(prec):
    w = events(prec)[1]
    a = B.Event(w)
    a.glasma_init()
    a.wong_init()
    a.step(7)
    f = a.download_native(B.GL_NATIVE_FIELDS)
    p = a.download_native(B.GL_NATIVE_PARTICLES)
    # the device layout: FP32 two-row links, phi, e, pi = 14 float4 per site
    # (FP64: 34 double2); particles at least 76 (FP32) or 136 (FP64) bytes each
    per_site = 14 * 16 if prec == W.FP32_2ROW else 34 * 16
    assert f.nbytes == w.N * w.N * per_site
    assert p.nbytes >= w.n_particles * (76 if prec == W.FP32_2ROW else 136)
    a.step(6)
    b = B.Event(w)
    b.glasma_init()
    b.wong_init()
    b.upload_native(B.GL_NATIVE_FIELDS, f)
    b.upload_native(B.GL_NATIVE_PARTICLES, p)
    b.set_step(7)
    b.step(6)
    same_state(a, b, len(w.species))
    with pytest.raises(B.GlasmaError) as e:
        b.upload_native(B.GL_NATIVE_FIELDS, f[:-16])
    assert e.value.status == B.GL_ERR_SIZE
    assert B.lib().gl_upload_native(b.ctx, 7, f.ctypes.data_as(ctypes.c_void_p), f.nbytes) == B.GL_ERR_ARG


def test_batch_restored_from_native_snapshots():
    ws = events(W.FP32_2ROW)
    a = B.Batch(ws)
    b = B.Batch(ws)
    with torch.cuda.stream(a.stream):
        a.init()
        a.step(7)
        fs = [ev.download_native(B.GL_NATIVE_FIELDS) for ev in a.events]
        ps = [ev.download_native(B.GL_NATIVE_PARTICLES) for ev in a.events]
        a.step(6)
    with torch.cuda.stream(b.stream):
        b.init()
        b.upload_native(B.GL_NATIVE_FIELDS, fs)
        b.upload_native(B.GL_NATIVE_PARTICLES, ps)
        for ev in b.events:
            ev.set_step(7)
        b.step(6)
        short = [x[:-256] for x in fs]
        ptrs = (ctypes.c_void_p * len(ws))(*[x.ctypes.data for x in short])
        sizes = (ctypes.c_size_t * len(ws))(*[x.nbytes for x in short])
        assert B.lib().gl_batch_upload_native(b.b, B.GL_NATIVE_FIELDS, ptrs, sizes) == B.GL_ERR_SIZE
    for ea, eb, w in zip(a.events, b.events, ws):
        same_state(ea, eb, len(w.species))


def _a256(n):
    return (n + 255) // 256 * 256


def test_out_of_range_indices_are_reported_and_repaired():
    w = events(W.FP32_2ROW)[0]
    ev = B.Event(w)
    ev.glasma_init()
    ev.wong_init()
    ev.step(3)
    p = ev.download_native(B.GL_NATIVE_PARTICLES)
    n = w.n_particles
    # FP32 particle arrays, each 256-byte aligned: float4 (x, y, p^x, p^y),
    # float2 (eta, P_eta), float4 q[2], int32 species, double p_T^2(tau_form),
    # int32 original index, float p^tau
    o_sp = _a256(16 * n) + _a256(8 * n) + _a256(32 * n)
    o_id = o_sp + _a256(4 * n) + _a256(8 * n)
    sp = p[o_sp:o_sp + 4 * n].view(np.int32)
    idx = p[o_id:o_id + 4 * n].view(np.int32)
    assert sorted(idx.tolist()) == list(range(n))
    assert set(sp.tolist()) <= {0, 1}
    bad = p.copy()
    bad[o_sp:o_sp + 4 * n].view(np.int32)[3] = 99
    bad[o_id:o_id + 4 * n].view(np.int32)[5] = n + 1000
    bad[o_id:o_id + 4 * n].view(np.int32)[6] = -2
    with pytest.raises(B.GlasmaError) as e:
        ev.upload_native(B.GL_NATIVE_PARTICLES, bad)
    assert e.value.status == B.GL_ERR_ARG
    fixed = ev.download_native(B.GL_NATIVE_PARTICLES)
    assert fixed[o_sp:o_sp + 4 * n].view(np.int32)[3] == 0
    assert fixed[o_id:o_id + 4 * n].view(np.int32)[5] == 5
    assert fixed[o_id:o_id + 4 * n].view(np.int32)[6] == 6
    ev.download(B.GL_BUF_PARTICLES)  # every record lands inside the host buffer
    ev.upload_native(B.GL_NATIVE_PARTICLES, p)
    assert np.array_equal(ev.download_native(B.GL_NATIVE_PARTICLES), p)


def test_batch_upload_reports_and_repairs_the_event_with_bad_indices():
    """The batched upload checks every event's particle indices in one launch:
    the event with a bad species and a bad original index is named in the
    error, its records are repaired, and the other events are unchanged."""
    ws = events(W.FP32_2ROW)
    b = B.Batch(ws)
    with torch.cuda.stream(b.stream):
        b.init()
        b.step(3)
        ps = [ev.download_native(B.GL_NATIVE_PARTICLES) for ev in b.events]
        n = ws[1].n_particles
        o_sp = _a256(16 * n) + _a256(8 * n) + _a256(32 * n)
        o_id = o_sp + _a256(4 * n) + _a256(8 * n)
        bad = [p.copy() for p in ps]
        bad[1][o_sp:o_sp + 4 * n].view(np.int32)[7] = -1
        bad[1][o_id:o_id + 4 * n].view(np.int32)[2] = n
        with pytest.raises(B.GlasmaError) as e:
            b.upload_native(B.GL_NATIVE_PARTICLES, bad)
        assert e.value.status == B.GL_ERR_ARG
        assert "event 1" in str(e.value)
        fixed = b.events[1].download_native(B.GL_NATIVE_PARTICLES)
        assert fixed[o_sp:o_sp + 4 * n].view(np.int32)[7] == 0
        assert fixed[o_id:o_id + 4 * n].view(np.int32)[2] == 2
        for k in (0, 2):
            assert np.array_equal(b.events[k].download_native(B.GL_NATIVE_PARTICLES), ps[k])
        b.upload_native(B.GL_NATIVE_PARTICLES, ps)
        for k in range(3):
            assert np.array_equal(b.events[k].download_native(B.GL_NATIVE_PARTICLES), ps[k])
    b.close()
