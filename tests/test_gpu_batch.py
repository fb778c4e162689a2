"""Batched events on the GPU: many MV events of different N advanced by one
field launch and one push launch per step (CUDA-graph replays) give bitwise
the same fields and particles as each event stepped on its own, for any tile
shape the autotuner picks; ragged lattices (N not a multiple of the tile)
included."""
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


def events(prec):
    out = []
    for e, N in enumerate([16, 40, 24, 64]):
        out.append(W.Workload("b%d" % e, N=N, L_fm=0.04 * N * 2, Ns=4, precision=prec, seed=11 + e, sort_every=0,
                              species=[W.Species(W.M_CHARM, 0.06, 300 + 50 * e, W.REP_F, W.MOM_UNIFORM_PT, 0.0, 5.0),
                                       W.Species(math.inf, 0.0, 40, W.REP_A, W.MOM_FIXED_PT, 0.0)]))
    return out


@pytest.mark.parametrize("prec", [W.FP64, W.FP32_2ROW])
def test_batch_equals_single_events(prec):
    ws = events(prec)
    batch = B.Batch(ws)
    with torch.cuda.stream(batch.stream):
        batch.init()
        tune = batch.autotune()
        print("autotune:", tune)
        steps = 21
        batch.step(7)
        batch.step(steps - 7)
        torch.cuda.synchronize()
        for e, w in enumerate(ws):
            single = B.Event(w, stream=batch.stream)
            single.glasma_init()
            single.wong_init()
            single.step(steps)
            be = batch.events[e]
            for buf in (B.GL_BUF_LINKS, B.GL_BUF_E, B.GL_BUF_PI, B.GL_BUF_PHI, B.GL_BUF_PARTICLES, B.GL_BUF_SITE):
                a, b = be.download(buf), single.download(buf)
                assert np.array_equal(a, b), (e, buf, np.abs(a - b).max())
        obs = batch.observables()
        assert all(o.step == steps for o in obs)
        assert all(o.n_active[0] > 0 for o in obs)


def test_batch_rejects_events_at_different_steps():
    ws = events(W.FP32_2ROW)[:2]
    batch = B.Batch(ws)
    with torch.cuda.stream(batch.stream):
        batch.init()
        batch.events[0].step(1)
        with pytest.raises(B.GlasmaError) as e:
            batch.step(1)
        assert e.value.status == B.GL_ERR_STATE


@pytest.mark.parametrize("prec", [W.FP64, W.FP32_2ROW])
def test_autotuned_tile_shape_changes_nothing(prec):
    """The fused kernel computes every site with the same operations whatever
    the tile shape, so a context tuned to any shape evolves bitwise like one
    with the default shape."""
    w = events(prec)[1]
    w.sort_every = 16
    a = B.Event(w)
    b = B.Event(w)
    for ev in (a, b):
        ev.glasma_init()
        ev.wong_init()
    tune = a.autotune()
    print("single-event autotune:", tune)
    a.step(19)
    b.step(19)
    for buf in (B.GL_BUF_LINKS, B.GL_BUF_E, B.GL_BUF_PI, B.GL_BUF_PHI, B.GL_BUF_PARTICLES):
        assert np.array_equal(a.download(buf), b.download(buf))
