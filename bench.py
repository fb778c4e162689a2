"""Benchmark of the coupled CPIC time step (Glasma leapfrog + Wong push).

A step is one pass of the whole hot path over one event: the fused kernel
(leapfrog step and site E/B interpolation) and the particle push kernel
(gl_step_coupled).  The default workload is the 256x256 event (L = 10 fm,
g^2 mu = 2 GeV, m = 0.2 GeV, Ns = 50, dtau = a/8) with 1e5 charm quarks
(p_T = 0.5 GeV) and 1e5 static quarks, FP32 two-row links.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--precision fp32|fp64]

Under torchrun each rank runs its own event (seed + rank): events are
independent, so the units shard with no data-path collective (weak scaling).
Rank 0 prints one JSON line.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "lattice site-updates/s + particle-steps/s, % HBM peak; FP32 vs FP64 at stated error"
L2_FLUSH_BYTES = 512 << 20   # written between timed steps (L2 is 129 MB)
L2_CLEAN_BYTES = 256 << 20   # then read, so the written lines are evicted before the step starts


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="n256_charm_static")
    ap.add_argument("--precision", default=None, choices=[None, "fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=6)
    ap.add_argument("--reunit-every", type=int, default=None)
    return ap.parse_args()


BATCHED = "batched64"


def workload(args, rank=0):
    from paper_2303_05599_gb300 import workloads as W
    if args.workload == BATCHED:
        evs = W.config_batched_events()
        for w in evs:
            w.seed = w.seed + 64 * rank
        return evs
    w = W.WORKLOADS[args.workload]()
    if args.reunit_every is not None:
        w.reunit_every = args.reunit_every
    if args.precision == "fp64":
        w.precision = W.FP64
    elif args.precision == "fp32":
        w.precision = W.FP32_2ROW
    w.seed = w.seed + rank
    return w


def field_bytes_per_site(prec):
    """Fused leapfrog + site-field kernel: every field of step n read once, the
    fields of step n+1 written once (U: 2 links, phi, e: 2, pi) and the six site
    fields E, B written once."""
    r = 8 if prec == 0 else 4
    links = 36 if prec == 0 else 24
    return (links + 8 + 16 + 8) * 2 * r + 48 * r


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
        self.path = os.path.join(ROOT, "gpurun_out", "clocks_bench_%d.csv" % os.getpid())

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
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for k, n in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(n)
        if sm:
            sm.sort()
            out = {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}
        return out


def cpu_baseline(w, ev, args):
    """The oracle as it stands on the host cores: a few coupled steps of the
    full lattice and all particles, from the GPU state after warm-up."""
    import numpy as np
    import oracle as O
    from paper_2303_05599_gb300 import _binding as B
    st = O.FieldState(w.N, ev.download(B.GL_BUF_LINKS), ev.download(B.GL_BUF_PHI), ev.download(B.GL_BUF_E),
                      ev.download(B.GL_BUF_PI))
    part = ev.download(B.GL_BUF_PARTICLES)
    ls = w.lattice_species()
    run = O.Run(st, part, [s[0] for s in ls], [s[1] for s in ls], [s.rep for s in w.species], w.dt,
                step=args.warmup)
    k = args.cpu_sample_steps
    t0 = time.perf_counter()
    for _ in range(k):
        run.step()
    dt = time.perf_counter() - t0
    return {"value": w.N * w.N * k / dt, "unit": "site-updates/s", "cores": O.threads(), "kind": "oracle",
            "sample": "%d coupled steps of the full %dx%d lattice with all %d particles, FP64, from the GPU "
                      "state after warm-up (%.1f s)" % (k, w.N, w.N, w.n_particles, dt),
            "particle_steps_per_s": w.n_particles * k / dt}


def run_batch(args, ws, dev, stream, world):
    """64 MV events of N in {64, 128, 256} as one batch: one field launch and
    one push launch per step, replayed from a CUDA graph; the working set
    (about 1.2 GB) is far larger than L2, so no flush is needed."""
    import torch
    from paper_2303_05599_gb300 import _binding as B
    batch = B.Batch(ws, stream=stream)
    batch.init()
    tune = batch.autotune()
    batch.step(args.warmup)
    K = args.steps
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    e0.record(stream)
    batch.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    t_step = e0.elapsed_time(e1) / 1e3
    # per-kernel split from separately timed replays of each launch shape
    sites = sum(w.N * w.N for w in ws)
    obs = batch.observables()
    n_active = sum(sum(o.n_active[k] for k in range(o.n_species)) for o in obs)
    t0 = time.perf_counter()
    for _ in range(K):
        batch.step(1)
        batch.observables()
    e2e_t = time.perf_counter() - t0
    return batch, tune, t_step, e2e_t, sites, n_active, ck


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2303_05599_gb300 import _binding as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    B.lib()

    w = workload(args, rank)
    stream = torch.cuda.Stream(device=dev)
    if args.workload == BATCHED:
        with torch.cuda.stream(stream):
            batch, tune, t_step, e2e_t, sites, n_active, ck = run_batch(args, w, dev, stream, world)
        emit_batch(args, w, tune, t_step, e2e_t, sites, n_active, ck, world, rank)
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    with torch.cuda.stream(stream):
        ev = B.Event(w, stream=stream)
        ev.glasma_init()
        ev.wong_init()
        tune = ev.autotune()
        for _ in range(args.warmup):
            ev.glasma_step(1)
            ev.wong_push()
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        clean = torch.ones(L2_CLEAN_BYTES // 4, dtype=torch.float32, device=dev)
        K = args.steps
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        wall0 = time.perf_counter()
        for k in range(K):
            # L2 flush between timed steps, outside the step's events: write a
            # buffer larger than L2, then read another one so that no dirty line
            # of the flush is left for the timed kernels to write back
            flush.zero_()
            clean.sum()
            e = evs[k]
            e[0].record(stream)
            ev.glasma_step(1)      # fused leapfrog + site E, B kernel
            e[1].record(stream)
            ev.wong_push()         # push kernel
            e[2].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ck = clocks.stop()
        field_each = sorted(e[0].elapsed_time(e[1]) for e in evs)
        t_field = sum(e[0].elapsed_time(e[1]) for e in evs) / 1e3
        t_push = sum(e[1].elapsed_time(e[2]) for e in evs) / 1e3
        t_step = t_field + t_push
        obs = ev.observables()
        n_active = sum(obs.n_active[k] for k in range(len(w.species)))

        # end to end through the public API: coupled step + observables read back every step
        t0 = time.perf_counter()
        for _ in range(K):
            ev.step(1)
            ev.observables()
        e2e_t = time.perf_counter() - t0

    tt = torch.tensor([t_step, e2e_t, float(n_active)], dtype=torch.float64, device=dev)
    if world > 1:
        mx = tt.clone()
        dist.all_reduce(mx[:2], op=dist.ReduceOp.MAX)
        sm = tt.clone()
        dist.all_reduce(sm[2:], op=dist.ReduceOp.SUM)
        t_step, e2e_t, n_active_all = float(mx[0]), float(mx[1]), float(sm[2])
    else:
        n_active_all = float(n_active)
    V = w.N * w.N
    value = world * V * K / t_step
    # report-time ensemble average over every rank's event (outside the timed region)
    from paper_2303_05599_gb300 import multi
    ens = multi.ensemble_reduce([obs], len(w.species))
    line = None
    if rank == 0:
        import json as _json
        peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        hbm = peaks.get("hbm_gbs", 6800.0)
        peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
        kern = {
            "field_step": (field_bytes_per_site(w.precision) * V, t_field / K),
            "wong_push": (push_bytes(w.precision, n_active, V), t_push / K),
        }
        dom = max(kern, key=lambda k: kern[k][1])
        roof = {}
        for name, (b, t) in kern.items():
            roof[name] = {"bound": "hbm", "achieved": b / t / 1e9, "peak": hbm, "unit": "GB/s",
                          "frac": b / t / 1e9 / hbm, "traffic": None, "bytes_per_launch": b, "us_per_launch": t * 1e6,
                          "peak_source": peak_src}
        dtype = "f64" if w.precision == 0 else "f32"
        line = {
            "metric": METRIC,
            "value": value,
            "unit": "site-updates/s",
            "n_gpus": world,
            "steps": K,
            "warmup": args.warmup,
            "ms_per_step": t_step / K * 1e3,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": dtype,
            "data": "synthetic: MV events generated on the GPU from Philox seeds, Haar-random charges",
            "config": {"workload": w.name, "N": w.N, "L_fm": w.L_fm, "particles": w.n_particles,
                       "precision": "fp32_2row" if w.precision else "fp64", "dtau_over_a": w.dtau_over_a,
                       "events_per_gpu": 1, "parallelism": "events sharded over ranks",
                       "l2": "flushed between timed steps (512 MiB write, then 256 MiB read), outside the step's events"},
            "particle_steps_per_s": n_active_all * K / t_step,
            "ensemble": {"tau_fm": obs.tau_fm, "per_species": ens},
            "kernel_ms_per_step": {"field_step": t_field / K * 1e3, "wong_push": t_push / K * 1e3},
            "field_step_ms_min_median_max": [field_each[0], field_each[K // 2], field_each[-1]],
            "autotune": tune,
            "roofline": dict(roof[dom], kernel=dom),
            "roofline_kernels": roof,
            "e2e": {"value": world * V * K / e2e_t, "unit": "site-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 8 * (8 * 7 + 7),
                    "includes": "gl_step_coupled + observables() read back to the host every step, wall clock; "
                                "the step's inputs are the device-resident state"},
            "gpu_launches": 2 * K,
            "clocks": ck,
            "wall_s_timed_loop": wall,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w, ev, args)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line))


def emit_batch(args, ws, tune, t_step, e2e_t, sites, n_active, ck, world, rank):
    import torch
    import torch.distributed as dist
    K = args.steps
    if world > 1:
        t = torch.tensor([t_step, e2e_t], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_step, e2e_t = float(t[0]), float(t[1])
    if rank != 0:
        return
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    prec = ws[0].precision
    step_bytes = field_bytes_per_site(prec) * sites + push_bytes(prec, n_active, sites)
    line = {
        "metric": METRIC, "value": world * sites * K / t_step, "unit": "site-updates/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": t_step / K * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == 0 else "f32",
        "data": "synthetic: MV events generated on the GPU from Philox seeds, Haar-random charges",
        "config": {"workload": BATCHED, "events_per_gpu": len(ws), "N": "64/128/256 by event", "a_fm": 0.04,
                   "sites_per_gpu": sites, "particles_per_gpu": sum(w.n_particles for w in ws),
                   "precision": "fp32_2row" if prec else "fp64", "parallelism": "events sharded over ranks",
                   "l2": "working set (~1.2 GB per step) larger than L2, no flush",
                   "launch": "one CUDA graph replay per step (field, push, clock tick)"},
        "particle_steps_per_s": world * n_active * K / t_step,
        "autotune": tune,
        "roofline": {"bound": "hbm", "achieved": step_bytes / (t_step / K) / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": step_bytes / (t_step / K) / 1e9 / hbm, "traffic": None, "kernel": "whole batched step",
                     "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"},
        "e2e": {"value": world * sites * K / e2e_t, "unit": "site-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": len(ws) * 8 * (8 * 7 + 7),
                "includes": "gl_batch_step + observables of every event read back each step"},
        "gpu_launches": 3 * K,
        "clocks": ck,
    }
    print(json.dumps(line))


def run_reference(args):
    """The oracle (plain FP64 CPU implementation) on the host cores, same
    workload, metric and unit; each step is one oracle coupled step of the
    full lattice with all particles."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import oracle as O
    from oracle import build as ob
    ob.build()
    w = workload(args, 0)
    st, bad = O.mv_init(w.N, w.Ns, w.g2mu_a, w.m_a, w.Lambda_a, w.seed)
    ls = w.lattice_species()
    part = np.concatenate([O.sample_species(w.N, w.seed, k, s.rep, s.mom_mode, ls[k][2], ls[k][3], s.count)
                           for k, s in enumerate(w.species)])
    run = O.Run(st, part, [s[0] for s in ls], [s[1] for s in ls], [s.rep for s in w.species], w.dt)
    for _ in range(args.warmup):
        run.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run.step()
    dt = time.perf_counter() - t0
    V = w.N * w.N
    value = V * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic: oracle MV event and particles",
        "config": {"workload": w.name, "N": w.N, "particles": w.n_particles,
                   "precision": "fp64 oracle (CPU)"},
        "particle_steps_per_s": w.n_particles * args.steps / dt,
        "cpu_baseline": {"value": value, "unit": "site-updates/s", "cores": O.threads(), "kind": "oracle",
                         "sample": "%d coupled steps of the full lattice with all particles" % args.steps},
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
