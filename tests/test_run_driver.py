"""The report driver (paper_2303_05599_gb300.run): health checks and report
rows on the host, and a short run on the GPU; checkpoint / resume and
host-side fault injection through the C ABI."""
import io
import json
import math
from contextlib import redirect_stdout
from types import SimpleNamespace

import numpy as np
import pytest

from paper_2303_05599_gb300 import run as R
from paper_2303_05599_gb300 import workloads as W


def fake_obs(n=2, bad=None, gauss=1e-7, unit=1e-6):
    arr = [1.0, 2.0]
    o = SimpleNamespace(n_species=n, sum_px2=list(arr), sum_py2=list(arr), sum_pL2=list(arr), sum_dpT2=list(arr),
                        gauss_max=gauss, unitarity_max=unit)
    if bad:
        getattr(o, bad)[1] = float("nan")
    return o


def test_health_checks():
    assert R.health([fake_obs()], 1e-3, 1e-4, True) == []
    probs = R.health([fake_obs(bad="sum_pL2")], 1e-3, 1e-4, False)
    assert len(probs) == 1 and "sum_pL2" in probs[0]
    assert len(R.health([fake_obs(gauss=1.0)], 1e-3, 1e-4, True)) == 1
    assert len(R.health([fake_obs(unit=float("nan"))], 1e-3, 1e-4, True)) == 1
    assert R.health([fake_obs(gauss=1.0)], 1e-3, 1e-4, False) == []   # fields not checked


def test_report_line_maps_to_quantum_values():
    sp = [W.Species(W.M_CHARM, 0.06, 10, W.REP_F), W.Species(math.inf, 0.0, 10, W.REP_A)]
    red = [{"n_active": 10, "mean_dpT2": 0.3, "mean_pL2": 0.6, "casimir2_dev": 0.0, "casimir3_dev": 0.0},
           {"n_active": 10, "mean_dpT2": 0.8, "mean_pL2": 1.6, "casimir2_dev": 0.0, "casimir3_dev": 0.0}]
    row = R.report_line(0.5, red, sp)
    assert row["species"][0]["dpT2_quantum_GeV2"] == pytest.approx(0.1)   # / D_F = 3
    assert row["species"][1]["dpL2_quantum_GeV2"] == pytest.approx(0.2)   # / D_A = 8
    assert row["species"][0]["anisotropy_L_over_T"] == pytest.approx(2.0)
    assert row["species"][1]["mass_GeV"] == "inf"
    json.dumps(row)


@pytest.mark.gpu
def test_driver_runs_a_small_workload():
    buf = io.StringIO()
    with redirect_stdout(buf):
        R.main(["--workload", "small_N32_fp64", "--events", "2", "--tau-max", "0.5", "--report-every", "0.1",
                "--field-checks"])
    rows = [json.loads(l) for l in buf.getvalue().splitlines()]
    assert len(rows) == 5
    assert rows[-1]["tau_fm"] == pytest.approx(0.5, abs=0.02)
    last = rows[-1]["species"][0]
    assert last["n_active"] == 2000 and last["dpT2_GeV2"] > 0 and last["dpL2_GeV2"] > 0
    assert rows[-1]["gauss_max"] < 1e-10 and math.isfinite(rows[-1]["energy_density_lattice"])
    assert "d_dpT2_dtau_GeV2_per_fm" in last


@pytest.mark.gpu
def test_checkpoint_resume_is_bitwise():
    """Run 2k coupled steps, or run k, download every buffer, create a new
    context, upload, set the step and run k more: the same bits."""
    import torch
    from paper_2303_05599_gb300 import _binding as B
    assert torch.cuda.is_available()
    w = W.Workload("ckpt", N=24, L_fm=2.25, Ns=4, precision=W.FP32_2ROW, seed=4, n_jets=16, ptau_diagnostic=True,
                   sort_every=8,  # sorts before and after the checkpoint
                   species=[W.Species(W.M_CHARM, 0.0, 300, W.REP_F, W.MOM_UNIFORM_PT, 0.0, 3.0),
                            W.Species(0.0, 0.0, 50, W.REP_A, W.MOM_EIKONAL_X, 0.0)])
    bufs = (B.GL_BUF_LINKS, B.GL_BUF_PHI, B.GL_BUF_E, B.GL_BUF_PI, B.GL_BUF_PARTICLES, B.GL_BUF_PTAU, B.GL_BUF_JETS)
    a = B.Event(w)
    a.glasma_init()
    a.wong_init()
    a.step(10)
    saved = {b: a.download(b) for b in bufs}
    a.step(10)
    c = B.Event(w)
    for b in bufs:
        c.upload(b, saved[b])
    c.set_step(10)
    c.step(10)
    for b in bufs + (B.GL_BUF_SITE,):
        assert np.array_equal(a.download(b), c.download(b), equal_nan=True), b


@pytest.mark.gpu
def test_host_side_fault_injection_is_detected():
    """A corrupted checkpoint (one non-finite link component injected on the
    host before the upload) is caught by the report health check instead of
    silently polluting the ensemble."""
    from paper_2303_05599_gb300 import _binding as B
    w = W.Workload("fault", N=16, L_fm=1.5, Ns=4, precision=W.FP32_2ROW, seed=2,
                   species=[W.Species(W.M_CHARM, 0.0, 400, W.REP_F, W.MOM_FIXED_PT, 0.5)])
    ev = B.Event(w)
    ev.glasma_init()
    ev.wong_init()
    ev.step(3)
    good = ev.observables()
    assert R.health([good], 1e-3, 1e-4, True) == []
    U = ev.download(B.GL_BUF_LINKS)
    U[0, 37, 4] = float("nan")
    ev.upload(B.GL_BUF_LINKS, U)
    ev.step(3)
    probs = R.health([ev.observables()], 1e-3, 1e-4, True)
    assert probs, "the injected fault went unnoticed"
