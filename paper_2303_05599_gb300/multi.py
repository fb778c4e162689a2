"""Events across ranks.

The paper's observables are averages over many independent MV events
(Sec. 7.1).  Events share nothing while they evolve, so they are sharded over
ranks (one process per GPU) with no collective on the data path; only the
per-species ensemble sums of a report are combined: sums are added and the
Casimir-drift maxima are maxed, over a torch.distributed process group (NCCL
on GPUs, gloo on CPUs).
"""
import numpy as np

# columns of one species' sums, in the order of gl_obs
SUM_FIELDS = ("n_active", "sum_px2", "sum_py2", "sum_pL2", "sum_dpT2")
MAX_FIELDS = ("casimir2_dev", "casimir3_dev")


def shard_events(n_events, rank, world):
    """Event indices of this rank: contiguous blocks, the first n_events % world
    ranks one event longer."""
    base, extra = divmod(n_events, world)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


def local_sums(obs_list, n_species):
    """Per-species sums and maxima over this rank's events, as two arrays
    [n_species, 5] and [n_species, 2] (from gl_obs records or dicts).  A NaN
    in any event's maximum makes that maximum NaN (np.maximum propagates it)."""
    s = np.zeros((n_species, len(SUM_FIELDS)))
    m = np.zeros((n_species, len(MAX_FIELDS)))
    for o in obs_list:
        for k in range(n_species):
            for j, f in enumerate(SUM_FIELDS):
                s[k, j] += _get(o, f, k)
            for j, f in enumerate(MAX_FIELDS):
                m[k, j] = np.maximum(m[k, j], _get(o, f, k))
    return s, m


def _get(o, f, k):
    v = o[f] if isinstance(o, dict) else getattr(o, f)
    return float(v[k])


def ensemble_reduce(obs_list, n_species, group=None):
    """Combine this rank's event observables with every other rank's.
    Returns per-species dicts with the mean <p_x^2>, <p_y^2>, <p_L^2>,
    <delta p_T^2> (GeV^2) over all active particles of all events, the
    particle count and the largest Casimir drifts."""
    import torch
    import torch.distributed as dist
    s, m = local_sums(obs_list, n_species)
    if dist.is_available() and dist.is_initialized():
        dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
        # a collective's MAX need not propagate NaN: the maxima travel with
        # NaN replaced by -inf, and a count of NaN entries travels beside them
        nan = np.isnan(m)
        ts = torch.tensor(s, dtype=torch.float64, device=dev)
        tm = torch.tensor(np.where(nan, -np.inf, m), dtype=torch.float64, device=dev)
        tn = torch.tensor(nan.astype(np.float64), dtype=torch.float64, device=dev)
        dist.all_reduce(ts, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(tm, op=dist.ReduceOp.MAX, group=group)
        dist.all_reduce(tn, op=dist.ReduceOp.SUM, group=group)
        s, m = ts.cpu().numpy(), tm.cpu().numpy()
        m = np.where(tn.cpu().numpy() > 0, np.nan, m)
    out = []
    for k in range(n_species):
        n = s[k, 0]
        d = {"n_active": int(round(n)), "casimir2_dev": m[k, 0], "casimir3_dev": m[k, 1]}
        for j, f in enumerate(("px2", "py2", "pL2", "dpT2")):
            d["mean_" + f] = s[k, j + 1] / n if n > 0 else 0.0
        out.append(d)
    return out
