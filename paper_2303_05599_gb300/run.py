"""Run a workload to tau_max and report the momentum broadening at fixed
proper-time intervals, the way the paper's figures are made (Sec. 7):

    python -m paper_2303_05599_gb300.run --workload n256_charm_static \\
        --events 30 --tau-max 1.0 --report-every 0.05 > broadening.jsonl

All events of a rank advance together as one batch (CUDA-graph replays of the
coupled step).  At every report time the per-species sums of every event are
read back (and, if asked, the FP64 field checks), reduced over events and
ranks, and one JSON line is written with, per species:
<delta p_T^2>, <delta p_L^2>, their values mapped to quantum expectation
values (division by D_R, Sec. 6), the anisotropy <dp_L^2>/<dp_T^2>, and the
Casimir drifts.  After the last report the instantaneous transport
coefficients kappa_{T,L} = d<dp^2>/dtau (Sec. 7) are added to every line.

Under torchrun the events are sharded over ranks (events are independent);
only the report sums are all-reduced.  Health checks stop the run with an
error when a reduction turns non-finite or the Gauss constraint or link
unitarity drift past their bounds.
"""
import argparse
import json
import math
import os
import sys


def parse(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="n256_charm_static")
    ap.add_argument("--events", type=int, default=1, help="events in total (sharded over ranks)")
    ap.add_argument("--tau-max", type=float, default=None, help="fm/c (default: the workload's)")
    ap.add_argument("--report-every", type=float, default=0.05, help="fm/c")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default=None)
    ap.add_argument("--field-checks", action="store_true", help="FP64 Gauss/unitarity checks at every report")
    ap.add_argument("--gauss-tol", type=float, default=1e-3)
    ap.add_argument("--unitarity-tol", type=float, default=1e-4)
    ap.add_argument("--summary", action="store_true",
                    help="end with one JSON line: wall time of the run (steps and reports) and its rates")
    return ap.parse_args(argv)


def health(obs_list, gauss_tol, unitarity_tol, fields):
    """Problems found in a report of gl_obs records (empty list: healthy)."""
    bad = []
    for e, o in enumerate(obs_list):
        for k in range(o.n_species):
            for name in ("sum_px2", "sum_py2", "sum_pL2", "sum_dpT2"):
                v = getattr(o, name)[k]
                if not math.isfinite(v):
                    bad.append("event %d species %d: %s is %r" % (e, k, name, v))
        if fields:
            for name in ("gauss_rms", "mean_trE_T2", "mean_trE_L2", "mean_trB_T2", "mean_trB_L2"):
                v = getattr(o, name, 0.0)
                if not math.isfinite(v):
                    bad.append("event %d: %s is %r" % (e, name, v))
            if not (o.gauss_max <= gauss_tol):
                bad.append("event %d: Gauss residual %r above %g" % (e, o.gauss_max, gauss_tol))
            if not (o.unitarity_max <= unitarity_tol):
                bad.append("event %d: link unitarity %r above %g" % (e, o.unitarity_max, unitarity_tol))
    return bad


def report_line(tau, reduced, species):
    """One JSON-ready report from the ensemble reduction of multi.ensemble_reduce."""
    from . import analysis as A
    row = {"tau_fm": tau, "species": []}
    for k, (s, r) in enumerate(zip(species, reduced)):
        dT, dL = r["mean_dpT2"], r["mean_pL2"]
        row["species"].append({
            "index": k, "mass_GeV": s.mass_GeV if math.isfinite(s.mass_GeV) else "inf", "rep": s.rep,
            "n_active": r["n_active"], "dpT2_GeV2": dT, "dpL2_GeV2": dL,
            "dpT2_quantum_GeV2": float(A.quantum_broadening(dT, s.rep)),
            "dpL2_quantum_GeV2": float(A.quantum_broadening(dL, s.rep)),
            "anisotropy_L_over_T": dL / dT if dT > 0 else None,
            "casimir2_dev": r["casimir2_dev"], "casimir3_dev": r["casimir3_dev"]})
    return row


def main(argv=None):
    args = parse(argv)
    import torch
    import torch.distributed as dist
    from . import _binding as B
    from . import analysis as A
    from . import multi
    from . import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    mine = multi.shard_events(args.events, rank, world)
    ws = []
    for e in mine:
        w = W.WORKLOADS[args.workload]()
        w.seed = e
        w.n_jets = 0
        if args.precision == "fp64":
            w.precision = W.FP64
        elif args.precision == "fp32":
            w.precision = W.FP32_2ROW
        ws.append(w)
    tau_max = args.tau_max if args.tau_max is not None else W.WORKLOADS[args.workload]().tau_max_fm
    w0 = W.WORKLOADS[args.workload]()
    dtau = w0.dtau_over_a * w0.a_fm
    n_total = int(math.ceil(tau_max / dtau - 1e-9))
    every = max(1, int(round(args.report_every / dtau)))
    what = B.GL_OBS_ALL if args.field_checks else B.GL_OBS_PARTICLES
    rows = []
    if ws:
        batch = B.Batch(ws)
        stream = batch.stream
    else:
        batch, stream = None, torch.cuda.current_stream()
    import time
    with torch.cuda.stream(stream):
        if batch:
            batch.init()
            batch.autotune()
        torch.cuda.synchronize()
        t_start = time.perf_counter()
        done = 0
        while done < n_total:
            k = min(every, n_total - done)
            if batch:
                batch.step(k)
                obs = batch.observables(what)
            else:
                obs = []
            done += k
            bad = health(obs, args.gauss_tol, args.unitarity_tol, args.field_checks)
            if bad:
                raise RuntimeError("unhealthy run at step %d: %s" % (done, "; ".join(bad[:4])))
            red = multi.ensemble_reduce(obs, len(w0.species))
            row = report_line(done * dtau, red, w0.species)
            if args.field_checks and obs:
                row["gauss_max"] = max(o.gauss_max for o in obs)
                row["unitarity_max"] = max(o.unitarity_max for o in obs)
                row["energy_density_lattice"] = sum(A.mean_energy_lattice(o) for o in obs) / len(obs)
            rows.append(row)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_start
    # instantaneous transport coefficients over the report series
    if len(rows) >= 2:
        tau = [r["tau_fm"] for r in rows]
        for k in range(len(w0.species)):
            for comp in ("dpT2_GeV2", "dpL2_GeV2"):
                series = [r["species"][k][comp] for r in rows]
                rate = A.instantaneous_rate(tau, series)
                for r, v in zip(rows, rate):
                    r["species"][k]["d_" + comp.replace("_GeV2", "") + "_dtau_GeV2_per_fm"] = float(v)
    if rank == 0:
        for r in rows:
            sys.stdout.write(json.dumps(r) + "\n")
        if args.summary:
            sites = sum(w.N * w.N for w in ws) * world
            parts = sum(w.n_particles for w in ws) * world
            sys.stdout.write(json.dumps({"summary": {
                "workload": args.workload, "events": args.events, "steps": n_total, "reports": len(rows),
                "tau_max_fm": n_total * dtau, "wall_s": wall, "field_checks": bool(args.field_checks),
                "site_updates_per_s": sites * n_total / wall, "particle_steps_per_s": parts * n_total / wall,
                "health": "ok", "launch": batch.launch() if batch else None}}) + "\n")
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
