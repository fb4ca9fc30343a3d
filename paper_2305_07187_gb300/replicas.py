"""End-of-run gather of replica results over ranks (host side).

The replicas of one instance are independent and J is read-only, so the path
shards replicas across GPUs with no exchange during the run.  What the ranks
share is one gather after it: the best replica (its cut, energy, spins and
where it ran), the distribution of final cuts, and the time-to-target cut,
which for the whole job is the earliest time any rank reached the target.
Every rank gets the same result (all-gather of small host objects; works on
gloo and NCCL process groups).
"""
from __future__ import annotations

import numpy as np


def local_summary(cuts, energies, spins, rank=0, ttt_s=None):
    """This rank's contribution: best replica (largest cut; ties to the lower
    energy, then the lower replica index), its spins, the cut histogram and
    the rank's time-to-target (None if it never reached the target)."""
    cuts = np.asarray(cuts).astype(np.int64).ravel()
    energies = np.asarray(energies).astype(np.int64).ravel()
    spins = np.asarray(spins)
    if cuts.size == 0:
        return {"rank": rank, "best": None, "hist": {}, "ttt_s": ttt_s}
    order = np.lexsort((np.arange(cuts.size), energies, -cuts))
    r = int(order[0])
    vals, counts = np.unique(cuts, return_counts=True)
    return {"rank": rank,
            "best": {"cut": int(cuts[r]), "energy": int(energies[r]), "replica": r,
                     "spins": spins[r].astype(np.int8).copy()},
            "hist": {int(v): int(c) for v, c in zip(vals, counts)},
            "ttt_s": None if ttt_s is None else float(ttt_s)}


def merge(summaries):
    """Combine the ranks' summaries: the best replica over all ranks (ties to
    the lower energy, then the lower rank), the summed cut histogram and the
    smallest time-to-target of the ranks that reached it."""
    best, hist, ttts = None, {}, []
    for sm in sorted(summaries, key=lambda x: x["rank"]):
        b_ = sm["best"]
        if b_ is not None and (best is None or (b_["cut"], -b_["energy"]) > (best["cut"], -best["energy"])):
            best = dict(b_, rank=sm["rank"])
        for v, c in sm["hist"].items():
            hist[v] = hist.get(v, 0) + c
        if sm["ttt_s"] is not None:
            ttts.append(sm["ttt_s"])
    return {"best": best, "hist": dict(sorted(hist.items())), "replicas": int(sum(hist.values())),
            "ttt_s": min(ttts) if ttts else None}


def gather_best(cuts, energies, spins, dist=None, ttt_s=None):
    """All-gather every rank's local_summary and merge them (one rank: no
    collective).  Returns the merged dict on every rank."""
    rank, world = 0, 1
    if dist is not None and dist.is_initialized():
        rank, world = dist.get_rank(), dist.get_world_size()
    mine = local_summary(cuts, energies, spins, rank, ttt_s)
    if world == 1:
        return merge([mine])
    everyone = [None] * world
    dist.all_gather_object(everyone, mine)
    return merge(everyone)
