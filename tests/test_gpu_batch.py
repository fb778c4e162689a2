"""Batched events on the GPU: many MV events of different N advanced by one
field launch and one push launch per step (CUDA-graph replays) give bitwise
the same fields and particles as each event stepped on its own, for any tile
shape the autotuner picks; ragged lattices (N not a multiple of the tile)
included."""
import ctypes
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


def events(prec, sort_every=0):
    # the 5x5 event: one tile wraps around its lattice, and every particle
    # stays within a few cells of the periodic boundary
    out = []
    for e, N in enumerate([16, 40, 24, 64, 5]):
        out.append(W.Workload("b%d" % e, N=N, L_fm=0.04 * N * 2, Ns=4, precision=prec, seed=11 + e,
                              sort_every=sort_every,
                              species=[W.Species(W.M_CHARM, 0.06, 300 + 50 * e, W.REP_F, W.MOM_UNIFORM_PT, 0.0, 5.0),
                                       W.Species(math.inf, 0.0, 40, W.REP_A, W.MOM_FIXED_PT, 0.0)]))
    return out


OBS_ARRAYS = ("n_active", "sum_px2", "sum_py2", "sum_pL2", "sum_dpT2", "casimir2_dev", "casimir3_dev")
OBS_SCALARS = ("gauss_max", "gauss_rms", "unitarity_max", "mean_trE_T2", "mean_trE_L2", "mean_trB_T2",
               "mean_trB_L2")


def same_obs(a, b, n_species):
    for f in OBS_ARRAYS:
        x, y = list(getattr(a, f))[:n_species], list(getattr(b, f))[:n_species]
        assert np.array_equal(x, y, equal_nan=True), (f, x, y)
    for f in OBS_SCALARS:
        x, y = getattr(a, f), getattr(b, f)
        assert x == y or (math.isnan(x) and math.isnan(y)), (f, x, y)


@pytest.mark.parametrize("prec,sort_every", [(W.FP64, 0), (W.FP32_2ROW, 0), (W.FP32_2ROW, 4)])
def test_batch_equals_single_events(prec, sort_every):
    """Fields, particles and observables (the particle sums come from the
    batched reduction) bitwise equal to each event run alone, with and
    without the periodic cell sort."""
    ws = events(prec, sort_every)
    batch = B.Batch(ws)
    with torch.cuda.stream(batch.stream):
        batch.init()
        tune = batch.autotune()
        print("autotune:", tune)
        steps = 21
        batch.step(7)
        batch.step(steps - 7)
        torch.cuda.synchronize()
        obs = batch.observables()
        for e, w in enumerate(ws):
            single = B.Event(w, stream=batch.stream)
            single.glasma_init()
            single.wong_init()
            single.step(steps)
            be = batch.events[e]
            for buf in (B.GL_BUF_LINKS, B.GL_BUF_E, B.GL_BUF_PI, B.GL_BUF_PHI, B.GL_BUF_PARTICLES, B.GL_BUF_SITE):
                a, b = be.download(buf), single.download(buf)
                assert np.array_equal(a, b), (e, buf, np.abs(a - b).max())
            same_obs(obs[e], single.observables(), 2)
        assert all(o.step == steps for o in obs)
        assert all(o.n_active[0] > 0 for o in obs)
        assert all(o.what == B.GL_OBS_ALL for o in obs)


def test_observables_parts():
    """GL_OBS_PARTICLES and GL_OBS_FIELDS each give their part of the full
    observables bitwise and NaN (counts 0) for the other."""
    ws = events(W.FP32_2ROW)
    batch = B.Batch(ws)
    with torch.cuda.stream(batch.stream):
        batch.init()
        batch.step(9)
        full = batch.observables()
        part = batch.observables(B.GL_OBS_PARTICLES)
        fld = batch.observables(B.GL_OBS_FIELDS)
        single_part = [ev.observables(B.GL_OBS_PARTICLES) for ev in batch.events]
    for e in range(len(ws)):
        assert part[e].what == B.GL_OBS_PARTICLES and fld[e].what == B.GL_OBS_FIELDS
        for f in OBS_ARRAYS:
            assert np.array_equal(list(getattr(part[e], f))[:2], list(getattr(full[e], f))[:2])
            assert np.array_equal(list(getattr(single_part[e], f))[:2], list(getattr(full[e], f))[:2])
            if f == "n_active":
                assert list(fld[e].n_active)[:2] == [0, 0]
            else:
                assert all(math.isnan(v) for v in list(getattr(fld[e], f))[:2])
        for f in OBS_SCALARS:
            assert getattr(fld[e], f) == getattr(full[e], f)
            assert math.isnan(getattr(part[e], f))


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(1e-300, np.abs(b).max()))


@pytest.mark.parametrize("workload", ["n256_charm_static", "batched64", "n1024_mixed"])
def test_full_size_batch_step_against_the_oracle(workload):
    """The benchmark's configurations at full size: their events (30 x 256^2,
    the 64 events of 64/128/256, or one 1024^2 event with 4e6 charm, beauty
    and light-like particles), autotuned launch shapes, CUDA-graph
    steps until every species is formed; then one more batched step of
    sampled events (one per lattice size) against one oracle step from their
    downloaded states.  FP32 two-row: 2e-5 relative on every field, the site
    fields and the particles away from cell edges."""
    import oracle as O
    if workload == "batched64":
        ws = W.config_batched_events()
        sample = [min(i for i, v in enumerate(ws) if v.N == N) for N in (64, 128, 256)]
    elif workload == "n1024_mixed":
        ws = [W.config_n1024()]
        sample = [0]
    else:
        ws = []
        for e in range(30):
            w = W.config_n256()
            w.seed = e
            ws.append(w)
        sample = [0, 29]
    batch = B.Batch(ws)
    n_form = max(int(math.ceil(sp.tau_form_fm / (w.dtau_over_a * w.a_fm) - 1e-9)) for w in ws for sp in w.species)
    with torch.cuda.stream(batch.stream):
        batch.init()
        batch.autotune()
        batch.step(n_form + 1)
        saved = {}
        for e in sample:
            ev = batch.events[e]
            st = O.FieldState(ev.N, ev.download(B.GL_BUF_LINKS), ev.download(B.GL_BUF_PHI),
                              ev.download(B.GL_BUF_E), ev.download(B.GL_BUF_PI))
            saved[e] = (st, ev.download(B.GL_BUF_PARTICLES))
        batch.step(1)
    for e in sample:
        w, ev = ws[e], batch.events[e]
        st, part = saved[e]
        ls = w.lattice_species()
        kind = O.kinds_of([s[0] for s in ls], [s.mom_mode for s in w.species])
        run = O.Run(st, part.copy(), [s[0] for s in ls], [s[1] for s in ls], [s.rep for s in w.species], w.dt,
                    step=n_form + 1, kind=kind)
        run.step()
        errs = [_rel(ev.download(B.GL_BUF_LINKS), run.st.U), _rel(ev.download(B.GL_BUF_E), run.st.e),
                _rel(ev.download(B.GL_BUF_PHI), run.st.phi), _rel(ev.download(B.GL_BUF_PI), run.st.pi),
                _rel(ev.download(B.GL_BUF_SITE), run.site)]
        got = ev.download(B.GL_BUF_PARTICLES)

        def near_edge(x):
            f = (x + 0.5) % 1.0
            return (np.minimum(f, 1 - f) < 1e-3).any(axis=1)
        keep = ~(near_edge(part[:, :2]) | near_edge(run.part[:, :2]))
        perr = [_rel(got[keep, sl], run.part[keep, sl]) for sl in (slice(0, 2), slice(3, 5), slice(5, 6), slice(6, 14))]
        print(workload, "event", e, "N", w.N, "errors", errs, perr, "compared", int(keep.sum()), "of", len(keep))
        assert max(errs) < 2e-5 and max(perr) < 2e-5


def test_batch_with_an_event_without_particles():
    """An event whose species are all empty sits in a batch beside normal
    events: it gets no push chunks and no sort, zero sums, and every event
    still evolves bitwise as it does alone."""
    ws = events(W.FP32_2ROW, sort_every=3)[:3]
    empty = ws[1]
    empty.species = [W.Species(s.mass_GeV, s.tau_form_fm, 0, s.rep, s.mom_mode, s.p0_GeV, s.p1_GeV)
                     for s in empty.species]
    batch = B.Batch(ws)
    with torch.cuda.stream(batch.stream):
        batch.init()
        batch.autotune()
        batch.step(8)
        obs = batch.observables()
        singles = []
        for w in ws:
            ev = B.Event(w, stream=batch.stream)
            ev.glasma_init()
            ev.wong_init()
            ev.step(8)
            singles.append(ev)
    assert list(obs[1].n_active)[:2] == [0, 0]
    assert list(obs[1].sum_px2)[:2] == [0.0, 0.0]
    for eb, es in zip(batch.events, singles):
        for which in (B.GL_BUF_LINKS, B.GL_BUF_E, B.GL_BUF_PHI, B.GL_BUF_PARTICLES):
            assert np.array_equal(eb.download(which), es.download(which))


RESTORE_BUFS = (B.GL_BUF_LINKS, B.GL_BUF_PHI, B.GL_BUF_E, B.GL_BUF_PI, B.GL_BUF_PARTICLES)


def test_batch_upload_restores_a_run():
    """A batch restored with gl_batch_upload (one wait per buffer for all
    events) from the downloads of another batch at step 7 evolves bitwise
    like the uninterrupted one; a wrong size is rejected with GL_ERR_SIZE."""
    ws = events(W.FP32_2ROW, sort_every=4)
    a = B.Batch(ws)
    b = B.Batch(ws)
    with torch.cuda.stream(a.stream):
        a.init()
        a.step(7)
        saved = {which: [ev.download(which) for ev in a.events] for which in RESTORE_BUFS}
        a.step(6)
    with torch.cuda.stream(b.stream):
        b.init()
        for which in RESTORE_BUFS:
            b.upload(which, saved[which])
        for ev in b.events:
            ev.set_step(7)
        b.step(6)
        bad = [np.zeros(3)] * len(ws)
        ptrs = (ctypes.c_void_p * len(ws))(*[x.ctypes.data for x in bad])
        counts = (ctypes.c_size_t * len(ws))(*[x.size for x in bad])
        assert B.lib().gl_batch_upload(b.b, B.GL_BUF_PHI, ptrs, counts) == B.GL_ERR_SIZE
    for ea, eb in zip(a.events, b.events):
        for which in RESTORE_BUFS:
            assert np.array_equal(ea.download(which), eb.download(which))


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


def test_particle_order_changes_nothing():
    """The sort (by row, motion class and cell) changes only where particles
    sit in memory: with or without it, and whatever the sort period, every
    particle (in the caller's order) and every field evolves bitwise alike;
    the per-species counts of the observables agree exactly and their sums to
    summation order."""
    runs = []
    for se in (0, 3, 16):
        w = events(W.FP32_2ROW)[3]
        w.sort_every = se
        ev = B.Event(w)
        ev.glasma_init()
        ev.wong_init()
        ev.step(23)
        runs.append((ev.download(B.GL_BUF_PARTICLES), ev.download(B.GL_BUF_LINKS), ev.observables()))
    p0, u0, o0 = runs[0]
    for p, u, o in runs[1:]:
        assert np.array_equal(p, p0)
        assert np.array_equal(u, u0)
        assert list(o.n_active)[:2] == list(o0.n_active)[:2]
        for f in ("sum_px2", "sum_py2", "sum_pL2", "sum_dpT2"):
            np.testing.assert_allclose(list(getattr(o, f))[:2], list(getattr(o0, f))[:2], rtol=1e-12)


def test_sort_of_particles_all_in_one_cell():
    """A legal but degenerate ensemble, 120k particles of two motion classes
    uploaded into one cell: the radix sort takes linear work whatever the
    keys, and the ensemble evolves bitwise as it does without any sort."""
    import time
    runs = []
    for se in (0, 2):
        w = W.Workload("one_cell", N=32, L_fm=1.28, Ns=4, precision=W.FP32_2ROW, seed=5, sort_every=se,
                       species=[W.Species(W.M_CHARM, 0.0, 100_000, W.REP_F, W.MOM_UNIFORM_PT, 0.0, 5.0),
                                W.Species(math.inf, 0.0, 20_000, W.REP_A, W.MOM_FIXED_PT, 0.0)])
        ev = B.Event(w)
        ev.glasma_init()
        ev.wong_init()
        rec = ev.download(B.GL_BUF_PARTICLES)
        rec[:, 0] = 7.2
        rec[:, 1] = 19.9
        t0 = time.perf_counter()
        ev.upload(B.GL_BUF_PARTICLES, rec)
        ev.step(9)
        got = ev.download(B.GL_BUF_PARTICLES)
        dt = time.perf_counter() - t0
        runs.append(got)
        assert dt < 30.0, "sorting one crowded cell took %.1f s" % dt
    assert np.array_equal(runs[0], runs[1])


@pytest.mark.parametrize("prec", [W.FP64, W.FP32_2ROW])
def test_schedules_agree(prec):
    """One persistent fused launch per step (any push chunk) and the two-stream
    schedules (push one block per chunk, or resident push blocks) evolve the
    batch bitwise alike, across sort segments."""
    ws = events(prec, sort_every=5)
    tile = "32x4" if prec == W.FP64 else "strip16"
    shapes = [dict(tile=tile, push_block=128, push_chunk=1024, fused=False, push_grid=0),
              dict(tile=tile, push_block=256, push_chunk=512, fused=True, push_grid=0),
              dict(tile=tile, push_block=128, push_chunk=2048, fused=True, push_grid=0),
              dict(tile=tile, push_block=128, push_chunk=1024, fused=False, push_grid=1),
              dict(tile=tile, push_block=128, push_chunk=512, fused=False, push_grid=2),
              dict(tile=tile, push_block=128, push_chunk=128, fused=False, push_grid=0),
              dict(tile=tile, push_block=256, push_chunk=256, fused=False, push_grid=0)]
    if prec != W.FP64:
        # the other strip launch shapes: rows split among 12 or 8 warps per SM
        shapes.append(dict(tile="strip12", push_block=512, push_chunk=1024, fused=False, push_grid=0))
        shapes.append(dict(tile="strip8", push_block=128, push_chunk=512, fused=False, push_grid=1))
    results = []
    for sh in shapes:
        batch = B.Batch(ws)
        with torch.cuda.stream(batch.stream):
            batch.init()
            batch.set_launch(**sh)
            got = batch.launch()
            assert {k: got[k] for k in sh} == sh
            batch.step(3)
            batch.step(10)
            torch.cuda.synchronize()
            results.append([[ev.download(buf) for buf in (B.GL_BUF_LINKS, B.GL_BUF_E, B.GL_BUF_PI, B.GL_BUF_PHI,
                                                          B.GL_BUF_PARTICLES, B.GL_BUF_SITE)]
                            for ev in batch.events])
        batch.close()
    for r in results[1:]:
        for e in range(len(ws)):
            for a, b in zip(results[0][e], r[e]):
                assert np.array_equal(a, b)


def test_set_launch_rejects_bad_shapes():
    ws = events(W.FP64)[:1]
    batch = B.Batch(ws)
    with pytest.raises(B.GlasmaError):
        batch.set_launch("32x8")          # FP64 batches use 32x4
    with pytest.raises(B.GlasmaError):
        batch.set_launch("strip16")       # FP32 launch shapes only
    with pytest.raises(B.GlasmaError):
        batch.set_launch("32x4", push_block=100)
    with pytest.raises(B.GlasmaError):
        batch.set_launch("32x4", push_chunk=1000)
    batch.close()


def test_segment_length_changes_nothing():
    """The FP32 field kernel cuts the strips of all events into segments of a
    per-launch length (the unit of work of one warp; a segment's first row gets
    its carries from a dry row, the column left of a strip from the halo
    pass): any length, shorter or longer than a lattice, evolves the batch
    bitwise alike, re-unitarisations and sorts included."""
    ws = events(W.FP32_2ROW, sort_every=5)
    for w in ws:
        w.reunit_every = 4
    results = []
    for rows in (0, 5, 23, 64):
        batch = B.Batch(ws)
        with torch.cuda.stream(batch.stream):
            batch.init()
            batch.set_launch("strip12", 128, 256, False, 0)
            batch.set_segment_rows(rows)
            before = batch.launch()["segment_rows"]  # the next launch's, reported before it
            assert rows == 0 or before == rows
            batch.step(13)
            torch.cuda.synchronize()
            assert batch.launch()["segment_rows"] == before
            results.append([[ev.download(buf) for buf in (B.GL_BUF_LINKS, B.GL_BUF_E, B.GL_BUF_PI, B.GL_BUF_PHI,
                                                          B.GL_BUF_PARTICLES, B.GL_BUF_SITE)]
                            for ev in batch.events])
        batch.close()
    for r in results[1:]:
        for e in range(len(ws)):
            for a, b in zip(results[0][e], r[e]):
                assert np.array_equal(a, b)
    fp64 = B.Batch(events(W.FP64)[:1])
    with pytest.raises(B.GlasmaError):
        fp64.set_segment_rows(16)
    fp64.close()


def test_observables_begin_end_equal_the_synchronous_call():
    """gl_batch_observables_begin/_end with up to two requests outstanding (a
    step enqueued between a request and its read) give bitwise the values the
    synchronous call gives at the same steps; misuse is GL_ERR_STATE."""
    ws = events(W.FP32_2ROW, sort_every=3)
    a, b = B.Batch(ws), B.Batch(ws)
    got_a, got_b = [], []
    with torch.cuda.stream(a.stream):
        a.init()
        for _ in range(7):
            a.step(1)
            got_a.append(a.observables(B.GL_OBS_PARTICLES))
        got_a.append(a.observables())
    with torch.cuda.stream(b.stream):
        b.init()
        with pytest.raises(B.GlasmaError) as e:
            b.observables_end()
        assert e.value.status == B.GL_ERR_STATE
        for k in range(7):
            b.step(1)
            b.observables_begin(B.GL_OBS_PARTICLES)
            if k > 0:
                got_b.append(b.observables_end())
        b.observables_begin()
        with pytest.raises(B.GlasmaError) as e:
            b.observables_begin()
        assert e.value.status == B.GL_ERR_STATE
        with pytest.raises(B.GlasmaError) as e:
            b.observables()
        assert e.value.status == B.GL_ERR_STATE
        got_b.append(b.observables_end())
        got_b.append(b.observables_end())
    n_species = len(ws[0].species)
    assert len(got_a) == len(got_b) == 8
    for ra, rb in zip(got_a, got_b):
        for oa, ob in zip(ra, rb):
            same_obs(oa, ob, n_species)
    a.close()
    b.close()
