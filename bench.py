"""Benchmark of the coupled CPIC time step (Glasma leapfrog + Wong push).

A step is one pass of the whole hot path over every event of the batch: the
fused field kernel (leapfrog step of Sec. 2 with the E/B interpolation of
Sec. 3.2 to the sites) and the particle push (Wong equations with the CPIC
colour rotation, Sec. 3).  The default workload is the batched one: 64
independent MV events with N drawn from {64, 128, 256} (event e has
N = [64, 128, 256][e % 3]), a = 0.04 fm, g^2 mu = 2 GeV, m = 0.2 GeV, Ns = 50,
dtau = a/8, each with 1e4 charm quarks of p_T ~ U[0, 5] GeV, FP32 two-row
links re-unitarised in FP64 every 64 steps.  All events advance together:
one field launch and one push launch per step, replayed from a CUDA graph,
with the field step of t_s overlapping the push of t_{s-1}.  The timed window
ends on a re-unitarising step, so its cost is inside the number.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--precision fp32|fp64] [--events E]

Under torchrun each rank runs its own events (seeds offset by rank): events
are independent, so they shard with no data-path collective (weak scaling);
only the ensemble sums of the report are reduced.  Rank 0 prints one JSON
line.
"""
import argparse
import ctypes
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "lattice site-updates/s + particle-steps/s, % HBM peak; FP32 vs FP64 at stated error"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched64")
    ap.add_argument("--precision", default=None, choices=[None, "fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=6,
                    help="oracle steps compared with the same GPU steps (error_vs_oracle)")
    ap.add_argument("--cpu-sample-seconds", type=float, default=10.0,
                    help="the oracle keeps stepping until its timed sample reaches this much CPU time")
    ap.add_argument("--reunit-every", type=int, default=None)
    ap.add_argument("--events", type=int, default=0, help="events per GPU (default 30; 1 for n1024_mixed)")
    ap.add_argument("--launch", default=None, help="fixed launch shapes and schedule "
                                                   "TILE:PUSH_BLOCK:PUSH_CHUNK:fused|streams[:PUSH_GRID[:SEGMENT_ROWS]] "
                                                   "(e.g. strip12:128:256:streams:0:16) "
                                                   "instead of the autotuner")
    return ap.parse_args()


BATCHED = "batched64"

# DRAM traffic per launch from ncu (dram__bytes_read.sum + dram__bytes_write.sum
# of one single-kernel capture of a full launch at the autotuner's launch
# shapes), keyed by (workload, events per GPU, kernel, precision).  Absent:
# not captured for the current kernels.
TRAFFIC = {
    ("batched64", 64, "field_step", 1): 514717696 + 694459904,
    ("batched64", 64, "wong_push", 1): 376806400 + 28170496,
    ("n1024_mixed", 1, "field_step", 1): 301978624 + 377472000,
    ("n1024_mixed", 1, "wong_push", 1): 589935360 + 197241088,
}


# FP64 path: bound by the FP64 pipe (ncu: 90 % of its cycles active), so its
# roofline is arithmetic.  Peak: 152 SMs x 2 FP64 FMA per clock x 2 flops x
# 2.07 GHz = 1.26 TFLOP/s (NVIDIA's nominal 1.25).  Flops counted with ncu
# (sm__sass_thread_inst_executed_op_{dfma,dadd,dmul}_pred_on; 2 per DFMA):
# per site of the field step (the 64 uneven events), and per active particle
# of the push, which depends on the species mix (all Wong charm quarks in the
# 64-event batch; half Wong, half static in 30 x 256^2).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP64_FLOP_PER_SITE = 4815
FP64_FLOP_PER_PARTICLE = {"batched64": 958, "n256_charm_static": 498}


def sort_launches(ws):
    """Kernels of one batched particle sort: keys, then per 8-bit digit pass a
    histogram, three scan kernels and a scatter, then the gather.  The passes
    cover the largest key, (number of motion classes) x N^2 - 1, of any event."""
    top = 1
    for w in ws:
        classes = {"static" if math.isinf(s.mass_GeV) else ("eikonal" if s.mom_mode == 3 else "wong")
                   for s in w.species}
        top = max(top, len(classes) * w.N * w.N - 1)
    passes = (max(1, top.bit_length()) + 7) // 8
    return 2 + 5 * passes


def leapfrog_bytes_per_site(prec):
    """The leapfrog's own algorithmic bytes: every field of step n read once and
    the fields of step n+1 written once (U: 2 links, phi, e: 2, pi); FP32 links
    are stored as two rows."""
    r = 8 if prec == 0 else 4
    links = 36 if prec == 0 else 24
    return (links + 8 + 16 + 8) * 2 * r


def site_field_bytes_per_site(prec):
    """The six site fields E, B at t_n (48 reals) written once by the same launch."""
    return 48 * (8 if prec == 0 else 4)


def field_bytes_per_site(prec):
    """Fused leapfrog + site-field kernel: the leapfrog's bytes and the site-field write."""
    return leapfrog_bytes_per_site(prec) + site_field_bytes_per_site(prec)


def timed_window_start(pre, K, every):
    """First timed step: `pre`, or later so that the K timed steps end on a
    re-unitarising step (step n re-unitarises when (n + 1) % every == 0)."""
    if every <= 0:
        return pre
    r = every * ((pre + 1 + every - 1) // every) - 1   # first re-unitarising step >= pre
    return pre if r < pre + K else r - K + 1


def representatives(ws):
    """One event of each lattice size, with the number of events of that size:
    the CPU samples time these and weight them by the counts."""
    reps = {}
    for i, w in enumerate(ws):
        if w.N not in reps:
            reps[w.N] = [i, 0]
        reps[w.N][1] += 1
    return [(i, c) for i, c in sorted(reps.values())]


def push_bytes(prec, n_active, V):
    """Push kernel: each active particle's state read and written once (x, y,
    eta, p^x, p^y, P_eta, Q: 14 reals) plus its species index; the site fields
    (48 reals per site) and the scalar at t_{n+1} (8 reals per site) read once."""
    r = 8 if prec == 0 else 4
    return n_active * (14 * 2 * r + 4) + V * (48 + 8) * r


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        # the samples are read back into the JSON line; BENCH_CLOCKS_DIR keeps the raw file
        self.path = os.path.join(os.environ.get("BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 "clocks_bench_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            return self.summarise(f)

    @staticmethod
    def summarise(lines):
        """Median SM clock, the highest maximum clock and the throttle reasons
        seen active, from lines of the query in Q (CSV, no header, no units)."""
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        samples = []
        for line in lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm, mx = float(p[1]), float(p[2])
            except ValueError:
                continue
            samples.append((sm, mx, {n for k, n in enumerate(names) if p[5 + k].lower().startswith("active")}))
        return summarise_clock_samples(samples)


def summarise_clock_samples(samples):
    """(SM MHz, max SM MHz, set of active reasons) samples -> the JSON record."""
    if not samples:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    sm = sorted(x[0] for x in samples)
    reasons = set()
    for x in samples:
        reasons |= x[2]
    return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(x[1] for x in samples), "reasons": sorted(reasons),
            "samples": len(samples)}


# NVML throttle-reason bits (nvmlClocksThrottleReason*) reported in the JSON line
NVML_REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}


class NvmlClockSampler:
    """The same record from NVML read queries (SM clock, its maximum and the
    active throttle reasons) polled every 0.25 ms by a thread, so that a timed
    region of a few milliseconds still holds many samples.  Needs
    libnvidia-ml from the driver; start() returns False without it."""

    def __init__(self, device):
        self.device = device
        self.samples = []
        self.thread = None

    def start(self):
        import threading
        try:
            import torch
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                return False
            p = torch.cuda.get_device_properties(self.device)
            bus = b"%08x:%02x:%02x.0" % (getattr(p, "pci_domain_id", 0), p.pci_bus_id, p.pci_device_id)
            h = ctypes.c_void_p()
            if nv.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus), ctypes.byref(h)) != 0:
                return False
        except Exception:
            return False
        self.nv, self.h = nv, h
        self.stop_flag = False
        mx = ctypes.c_uint()
        if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) != 0:  # NVML_CLOCK_SM
            return False
        first = threading.Event()

        def poll():
            # two queries a sample (each takes a fraction of a millisecond);
            # the maximum clock does not change
            clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
            while not self.stop_flag:
                if (nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and
                        nv.nvmlDeviceGetCurrentClocksThrottleReasons(h, ctypes.byref(rs)) == 0):
                    self.samples.append((float(clk.value), float(mx.value),
                                         {n for bit, n in NVML_REASONS.items() if rs.value & bit}))
                first.set()
                time.sleep(0.00025)

        self.thread = threading.Thread(target=poll, daemon=True)
        self.thread.start()
        first.wait(timeout=0.5)  # the timed region starts after the first sample
        return True

    def stop(self):
        if self.thread is None:
            return summarise_clock_samples([])
        self.stop_flag = True
        self.thread.join(timeout=5)
        self.nv.nvmlShutdown()
        return dict(summarise_clock_samples(self.samples), source="nvml")


def _rel(a, b):
    import numpy as np
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(1e-300, np.abs(b).max()))


def _ensemble(part, mass, t, static):
    """<p_T^2>, <p_L^2> per species (lattice units) from canonical particle
    records: p_L = p^tau sinh(eta) + w cosh(eta), w = P_eta / t (static: P_eta)."""
    import numpy as np
    out = {}
    for k in range(len(mass)):
        m = part[:, 15] == k
        if not m.any():
            continue
        px, py, eta, Pe = part[m, 3], part[m, 4], part[m, 2], part[m, 5]
        if static[k]:
            pl = Pe
        else:
            w = Pe / t if t > 0 else 0 * Pe
            pl = np.sqrt(px * px + py * py + w * w + mass[k] ** 2) * np.sinh(eta) + w * np.cosh(eta)
        out[k] = (float(np.mean(px * px + py * py)), float(np.mean(pl * pl)))
    return out


def _oracle_sample(w, ev, args, budget_s):
    """The oracle on one event from the GPU state: `cpu_sample_steps` coupled
    steps, the same steps taken by the GPU on that event, the GPU's errors, and
    more oracle steps until the sample reaches `budget_s` of CPU time.
    Returns (seconds per step, steps, errors, step0)."""
    import math
    import numpy as np
    import oracle as O
    from paper_2303_05599_gb300 import _binding as B
    st = O.FieldState(w.N, ev.download(B.GL_BUF_LINKS), ev.download(B.GL_BUF_PHI), ev.download(B.GL_BUF_E),
                      ev.download(B.GL_BUF_PI))
    part = ev.download(B.GL_BUF_PARTICLES)
    ls = w.lattice_species()
    obs = ev.observables()
    step0 = int(obs.step)
    run = O.Run(st, part, [s[0] for s in ls], [s[1] for s in ls], [s.rep for s in w.species], w.dt, step=step0)
    k = args.cpu_sample_steps
    t0 = time.perf_counter()
    for _ in range(k):
        run.step()
    dt = time.perf_counter() - t0
    # the same k steps on the GPU (this event alone), then the errors
    ev.step(k)
    gp = ev.download(B.GL_BUF_PARTICLES)
    mass = [s[0] for s in ls]
    static = [math.isinf(s.mass_GeV) for s in w.species]
    t_end = run.n * w.dt
    ens_g, ens_o = _ensemble(gp, mass, t_end, static), _ensemble(run.part, mass, t_end, static)
    dpos = np.abs(gp[:, :2] - run.part[:, :2])
    dpos = np.minimum(dpos, w.N - dpos)  # periodic
    err = {
        "steps": k, "from_step": step0,
        "links": _rel(ev.download(B.GL_BUF_LINKS), run.st.U),
        "e": _rel(ev.download(B.GL_BUF_E), run.st.e),
        "phi": _rel(ev.download(B.GL_BUF_PHI), run.st.phi),
        "pi": _rel(ev.download(B.GL_BUF_PI), run.st.pi),
        "site_fields": _rel(ev.download(B.GL_BUF_SITE), run.site),
        "positions_max_abs_lattice_units": float(dpos.max()),
        "momenta": _rel(gp[:, 3:6], run.part[:, 3:6]),
        "momenta_per_particle_p50_p99": [float(v) for v in np.percentile(
            np.abs(gp[:, 3:6] - run.part[:, 3:6]).max(axis=1) / max(1e-300, np.abs(run.part[:, 3:6]).max()), [50, 99])],
        "charges": _rel(gp[:, 6:14], run.part[:, 6:14]),
        "ensemble_pT2": {str(s): abs(ens_g[s][0] / ens_o[s][0] - 1) for s in ens_o if ens_o[s][0] > 0},
        "ensemble_pL2": {str(s): abs(ens_g[s][1] / ens_o[s][1] - 1) for s in ens_o if ens_o[s][1] > 0},
    }
    # the timed sample goes on past the compared steps, to a bounded amount of CPU work
    n_steps = k
    t1 = time.perf_counter()
    while dt + (time.perf_counter() - t1) < budget_s:
        run.step()
        n_steps += 1
    dt += time.perf_counter() - t1
    return dt / n_steps, n_steps, err, step0


def cpu_baseline(ws, events, args):
    """The oracle as it stands on the host cores, on a bounded sample of the
    workload: one event of each lattice size, from the GPU state after the
    run, for an equal share of `cpu_sample_seconds` each.  The per-step times
    are weighted by the number of events of each size, so the rate is the
    oracle's on the whole workload.  The same steps are taken by the GPU on
    each sampled event, and its errors against the FP64 oracle are reported
    for every observable."""
    import oracle as O
    reps = representatives(ws)
    budget = args.cpu_sample_seconds / len(reps)
    t_all = sites = parts = 0.0
    errors, desc = {}, []
    for i, count in reps:
        w = ws[i]
        t_step, n, err, step0 = _oracle_sample(w, events[i], args, budget)
        t_all += count * t_step
        sites += count * w.N * w.N
        parts += count * w.n_particles
        errors["N%d" % w.N] = err
        desc.append("%d steps of a %dx%d event with %d particles from step %d (x%d events)"
                    % (n, w.N, w.N, w.n_particles, step0, count))
    return {"value": sites / t_all, "unit": "site-updates/s", "cores": O.threads(), "kind": "oracle",
            "sample": "FP64 coupled steps of the full lattice with all particles, from the GPU state: " +
                      "; ".join(desc) + " (%.1f s of CPU time; the per-step times weighted by the event counts; "
                      "the first %d steps of each also taken by the GPU for error_vs_oracle)"
                      % (args.cpu_sample_seconds, args.cpu_sample_steps),
            "particle_steps_per_s": parts / t_all,
            "error_vs_oracle": errors,
            "cell_flips": "the max values come from the few particles whose FP32 position rounds to the other "
                          "side of a cell edge (different NGP cell); the percentiles show the rest"}


def events_for(args, rank):
    """The events one rank runs: `--events` replicas of a single-event
    workload (the paper averages 30 events, Sec. 7.1), or the 64 uneven events
    of the batched workload."""
    from paper_2303_05599_gb300 import workloads as W

    def options(w):
        if args.reunit_every is not None:
            w.reunit_every = args.reunit_every
        if args.precision == "fp64":
            w.precision = W.FP64
        elif args.precision == "fp32":
            w.precision = W.FP32_2ROW
        return w

    if args.workload == BATCHED:
        evs = W.config_batched_events()
        for w in evs:
            w.seed = w.seed + 64 * rank
            options(w)
        return evs
    n = args.events if args.events else (1 if W.WORKLOADS[args.workload]().N >= 1024 else 30)
    evs = []
    for e in range(n):
        w = options(W.WORKLOADS[args.workload]())
        w.n_jets = 0  # jet-correlator probes run on the single-event API only
        w.seed = rank * n + e
        evs.append(w)
    return evs


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2303_05599_gb300 import _binding as B
    from paper_2303_05599_gb300 import multi

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl")
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    B.lib()

    ws = events_for(args, rank)
    K = args.steps
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        batch = B.Batch(ws, stream=stream)
        batch.init()
        if args.launch:
            parts = args.launch.split(":")
            tile, pb, pc, mode = parts[:4]
            batch.set_launch(tile, int(pb), int(pc), mode == "fused", int(parts[4]) if len(parts) > 4 else 0)
            if len(parts) > 5:
                batch.set_segment_rows(int(parts[5]))
            tune = dict(batch.launch(), fixed=True)
        else:
            tune = batch.autotune()
        # untimed: W warm-up steps, at least up to the first step at which every
        # species is formed (the steady state of the run)
        n_form = max(int(math.ceil(sp.tau_form_fm / (w.dtau_over_a * w.a_fm) - 1e-9)) for w in ws for sp in w.species)
        pre = timed_window_start(max(args.warmup, n_form + 1), K, ws[0].reunit_every if ws[0].precision else 0)
        batch.step(pre)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clocks = NvmlClockSampler(local)
        if not clocks.start():
            clocks = ClockSampler(local)
            clocks.start()
        e0.record(stream)
        batch.step(K)                      # K coupled steps: CUDA-graph replays
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ck = clocks.stop()
        t_step = e0.elapsed_time(e1) / 1e3
        # per-kernel durations: the same K steps with events around every launch
        f_ms, p_ms = batch.step_timed(K)
        obs = batch.observables()
        # end to end through the public API: every event's state (the fields of
        # one time slice and the particles, as native snapshots) uploaded from
        # pinned host memory, then K steps with the observables of every event
        # read back each step
        parts = (B.GL_NATIVE_FIELDS, B.GL_NATIVE_PARTICLES)
        host = []
        for ev in batch.events:
            bufs = {}
            for part in parts:
                t = torch.empty(ev.native_bytes(part), dtype=torch.uint8, pin_memory=True)
                ev.download_native(part, out=t.numpy())
                bufs[part] = t
            host.append(bufs)
        h2d = sum(t.numel() for bufs in host for t in bufs.values())
        # one untimed restore from the same pinned buffers first: the first DMA
        # from freshly pinned pages has shown one-off costs (14 ms against 3 ms)
        for part in parts:
            batch.upload_native(part, [bufs[part].numpy() for bufs in host])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for part in parts:
            batch.upload_native(part, [bufs[part].numpy() for bufs in host])
        t1 = time.perf_counter()
        # each step's particle sums are requested behind it and read back
        # while the next step runs
        for k in range(K):
            batch.step(1)
            batch.observables_begin(B.GL_OBS_PARTICLES)
            if k > 0:
                batch.observables_end()
        batch.observables_end()
        final = batch.observables()        # the report: particle sums and FP64 field checks
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        e2e_t = t2 - t0
        e2e_parts = {"upload_s": t1 - t0, "steps_and_reads_s": t2 - t1}

    n_species = len(ws[0].species)
    ens = multi.ensemble_reduce(obs, n_species)  # report-time reduction over every rank's events
    sites = sum(w.N * w.N for w in ws)
    n_active = sum(sum(o.n_active[k] for k in range(o.n_species)) for o in obs)
    tt = torch.tensor([t_step, e2e_t], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    t_step, e2e_t = float(tt[0]), float(tt[1])
    line = None
    if rank == 0:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        hbm = peaks.get("hbm_gbs", 6800.0)
        peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
        prec = ws[0].precision
        kern = {
            "field_step": (field_bytes_per_site(prec) * sites, f_ms / 1e3 / K),
            "wong_push": (push_bytes(prec, n_active, sites), p_ms / 1e3 / K),
        }
        roof = {}
        for name, (b, t) in kern.items():
            roof[name] = {"bound": "hbm", "achieved": b / t / 1e9, "peak": hbm, "unit": "GB/s",
                          "frac": b / t / 1e9 / hbm, "traffic": TRAFFIC.get((args.workload, len(ws), name, prec)),
                          "bytes_per_launch": b, "us_per_launch": t * 1e6, "peak_source": peak_src}
        # the field launch's bytes itemised: the leapfrog's own (each field of
        # step n read once, step n+1 written once) and the site-field write;
        # the fraction on the leapfrog's bytes alone stands beside the total
        t_f = kern["field_step"][1]
        lf = leapfrog_bytes_per_site(prec) * sites
        roof["field_step"].update({
            "bytes_per_site": {"leapfrog": leapfrog_bytes_per_site(prec),
                               "site_fields": site_field_bytes_per_site(prec)},
            "frac_leapfrog_bytes_only": lf / t_f / 1e9 / hbm,
            "achieved_leapfrog_bytes_only": lf / t_f / 1e9})
        if prec == 0:
            flops = {"field_step": FP64_FLOP_PER_SITE * sites}
            if args.workload in FP64_FLOP_PER_PARTICLE:
                flops["wong_push"] = FP64_FLOP_PER_PARTICLE[args.workload] * n_active
            for name, (b, t) in kern.items():
                if name not in flops:
                    roof[name] = {"bound": "alu", "achieved": None, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                  "frac": None, "traffic": None, "us_per_launch": t * 1e6,
                                  "note": "FP64 flops per particle not counted for this species mix"}
                    continue
                roof[name] = {"bound": "alu", "achieved": flops[name] / t / 1e12, "peak": FP64_PEAK_TFLOPS,
                              "unit": "TFLOP/s", "frac": flops[name] / t / 1e12 / FP64_PEAK_TFLOPS, "traffic": None,
                              "flops_per_launch": flops[name], "us_per_launch": t * 1e6,
                              "peak_source": "derived: 152 SMs x 2 FP64 FMA/clock x 2 x 2.07 GHz"}
        dom = max(kern, key=lambda k: kern[k][1])
        single = args.workload != BATCHED
        line = {
            "metric": METRIC,
            "value": world * sites * K / t_step,
            "unit": "site-updates/s",
            "n_gpus": world,
            "steps": K,
            "warmup": args.warmup,
            "ms_per_step": t_step / K * 1e3,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64" if prec == 0 else "f32",
            "data": "synthetic: MV events generated on the GPU from Philox seeds, Haar-random charges",
            "config": {"workload": args.workload + (" x %d events" % len(ws) if single else ""),
                       "events_per_gpu": len(ws), "N": ws[0].N if single else "64/128/256 by event",
                       "sites_per_gpu": sites, "particles_per_gpu": sum(w.n_particles for w in ws),
                       "precision": "fp32_2row" if prec else "fp64", "dtau_over_a": ws[0].dtau_over_a,
                       "reunit_every": ws[0].reunit_every, "parallelism": "events sharded over ranks",
                       "l2": "per-step working set larger than L2 (no flush)",
                       "timed_from_step": pre,
                       "launch": "one CUDA-graph replay per step: the field step of t_s and the push of t_{s-1}, "
                                 "as one persistent fused launch or on two streams (autotuned)"},
            "particle_steps_per_s": world * n_active * K / t_step,
            "ensemble": {"tau_fm": obs[0].tau_fm, "per_species": ens},
            "kernel_ms_per_step": {"field_step": f_ms / K, "wong_push": p_ms / K},
            "autotune": tune,
            "roofline": dict(roof[dom], kernel=dom),
            "roofline_kernels": roof,
            "e2e": dict({"value": world * sites * K / e2e_t, "unit": "site-updates/s",
                         "h2d_bytes_per_step": h2d / K,
                         # one request of every event's rows a step, and the final report
                         "d2h_bytes_per_step": len(ws) * B.lib().gl_batch_obs_row_bytes() * (K + 1) / K,
                         "includes": "gl_batch_upload_native of every event's fields and particles from pinned "
                                     "host memory (native snapshots: the device layout, from gl_download_native); "
                                     "K x (gl_batch_step(1) + the per-species particle sums of every event read "
                                     "back to the host, each step's while the next step runs: "
                                     "gl_batch_observables_begin/_end); one full report with the FP64 field "
                                     "checks at the end",
                         "gauss_max_final": max(o.gauss_max for o in final)}, **e2e_parts),
            "gpu_launches": 3 * K + sort_launches(ws) * sum(1 for s_ in range(pre + 1, pre + K + 1)
                                                          if ws[0].sort_every > 0 and s_ % ws[0].sort_every == 0),
            "clocks": ck,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(ws, batch.events, args)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line))


def run_reference(args):
    """The oracle (plain FP64 CPU implementation) on the host cores, same
    workload, metric and unit.  Each step is one oracle coupled step (full
    lattice, all particles) of one event of each lattice size of the
    workload; the per-step times are weighted by the number of events of
    each size, so the rate is the oracle's on the whole workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import oracle as O
    from oracle import build as ob
    ob.build()
    evs = events_for(args, 0)
    runs = []
    for i, count in representatives(evs):
        w = evs[i]
        st, bad = O.mv_init(w.N, w.Ns, w.g2mu_a, w.m_a, w.Lambda_a, w.seed)
        ls = w.lattice_species()
        part = np.concatenate([O.sample_species(w.N, w.seed, k, s.rep, s.mom_mode, ls[k][2], ls[k][3], s.count)
                               for k, s in enumerate(w.species)])
        runs.append((w, count, O.Run(st, part, [s[0] for s in ls], [s[1] for s in ls], [s.rep for s in w.species],
                                     w.dt)))
    t_all = sites = parts = 0.0
    for w, count, run in runs:
        for _ in range(args.warmup):
            run.step()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            run.step()
        t = (time.perf_counter() - t0) / args.steps
        t_all += count * t
        sites += count * w.N * w.N
        parts += count * w.n_particles
    value = sites / t_all
    sample = "; ".join("%dx%d with %d particles (x%d events)" % (w.N, w.N, w.n_particles, c) for w, c, _ in runs)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_all * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic: oracle MV events and particles",
        "config": {"workload": args.workload + (" x %d events" % len(evs) if args.workload != BATCHED else ""),
                   "sites": int(sites), "particles": int(parts), "precision": "fp64 oracle (CPU)"},
        "particle_steps_per_s": parts / t_all,
        "cpu_baseline": {"value": value, "unit": "site-updates/s", "cores": O.threads(), "kind": "oracle",
                         "sample": "one event of each lattice size: %s; %d coupled steps of the full lattice with "
                                   "all particles after %d warm-up steps, per-step times weighted by the event "
                                   "counts (ms_per_step: the whole workload's step, extrapolated so)"
                                   % (sample, args.steps, args.warmup)},
        "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
