"""Ensemble sums of the momentum broadening (Sec. 3.1: <p_T^2> and <dp_T^2> as
sums over the particles of a species) against their exact values.

The square of an FP32 momentum is exact in FP64 (a 24-bit significand squared
needs 48 bits), so math.fsum over the downloaded state's squares is the
correctly rounded sum.  The device sums FP32 squares as float pairs; the test
holds every sum to 1e-11 relative, well below what a plain FP32 sum (about
1e-7 per addition) or a pair sum that dropped the low parts of the squares
(about 1e-10 here) would give.  The FP64 state sums in FP64 and is held to
1e-13.  Both the single-event path and the batched path are checked, over
several reduction blocks of 4096 particles and a ragged last block."""
import math

import numpy as np
import pytest

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


def workload(prec, seed):
    # 17,000 particles: five blocks of the per-event reduction, the last one ragged
    return W.Workload("obs_sums", N=32, L_fm=2.0, Ns=4, precision=prec, seed=seed,
                      species=[W.Species(W.M_CHARM, 0.0, 9000, W.REP_F, W.MOM_UNIFORM_PT, 0.0, 5.0),
                               W.Species(math.inf, 0.0, 5000, W.REP_A, W.MOM_FIXED_PT, 0.0),
                               W.Species(0.0, 0.0, 3000, W.REP_F, W.MOM_ALONG_X, 10.0)])


def exact_sums(rec, ns):
    """(count, sum p_x^2, sum p_y^2, sum p_T^2(tau_form)) per species, in
    lattice units, from canonical records [np][16]."""
    sp = rec[:, 15].astype(np.int64)
    out = []
    for k in range(ns):
        r = rec[sp == k]
        out.append((len(r), math.fsum(r[:, 3] ** 2), math.fsum(r[:, 4] ** 2), math.fsum(r[:, 14])))
    return out


def check(o, rec, w, tol):
    a2 = w.a_GeVinv ** 2
    for k, (n, px2, py2, pt0) in enumerate(exact_sums(rec, len(w.species))):
        assert o.n_active[k] == n, (k, o.n_active[k], n)
        assert abs(o.sum_px2[k] * a2 - px2) <= tol * px2, (k, o.sum_px2[k] * a2, px2)
        assert abs(o.sum_py2[k] * a2 - py2) <= tol * py2, (k, o.sum_py2[k] * a2, py2)
        # <dp_T^2> = sum p_x^2 + sum p_y^2 - sum p_T^2(tau_form): a difference,
        # so its error is relative to the terms
        dpt2 = px2 + py2 - pt0
        assert abs(o.sum_dpT2[k] * a2 - dpt2) <= tol * (px2 + py2 + pt0), (k, o.sum_dpT2[k] * a2, dpt2)


TOLS = {W.FP32_2ROW: 1e-11, W.FP64: 1e-13}


@pytest.mark.parametrize("prec", [W.FP32_2ROW, W.FP64])
def test_single_event_sums_are_exact_to_the_bound(prec):
    w = workload(prec, 21)
    ev = B.Event(w)
    ev.glasma_init()
    ev.wong_init()
    ev.step(6)
    o = ev.observables()
    rec = ev.download(B.GL_BUF_PARTICLES).reshape(-1, 16)
    assert np.any(rec[:, 3] != 0.0) and np.any(rec[:, 4] != 0.0)
    check(o, rec, w, TOLS[prec])


@pytest.mark.parametrize("prec", [W.FP32_2ROW, W.FP64])
def test_batched_sums_are_exact_to_the_bound(prec):
    ws = [workload(prec, 31), workload(prec, 32)]
    batch = B.Batch(ws)
    with torch.cuda.stream(batch.stream):
        batch.init()
        batch.step(6)
        obs = batch.observables()
        for o, ev, w in zip(obs, batch.events, ws):
            check(o, ev.download(B.GL_BUF_PARTICLES).reshape(-1, 16), w, TOLS[prec])
