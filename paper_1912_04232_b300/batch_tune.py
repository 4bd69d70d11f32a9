"""Autotuner of the batched-replica engine (Sec. 4.2: many independent
systems advanced together).  Per replica size class it chooses

  * the cell-size multiplier of the replicas' cell grids
    (md_replica_desc.cell_mult: cells of side >= mult x (r_cut + skin)), and
  * the threads per particle of the force kernel (md_batch_set_class_tpp),

by coordinate descent on the measured time (CUDA events) of a short
graph-launched NVE run from the caller's state, starting from the default
(multiplier 1, 4 threads).  The choice does not change what is computed:
the rows hold the same partners and each particle's forces are those of the
single-system kernels with its replica's threads per particle, so tuned and
default trajectories agree to rounding.  Results are cached in a JSON file
keyed by the replica set.
"""
from __future__ import annotations

import hashlib
import json
import os

from . import jmd as J

CLASS_EDGES = (512, 2048)        # size classes: N < 512, 512 <= N < 2048, N >= 2048
MULTS = (1.0, 1.5, 2.0)
TPPS = (4, 8, 16)


def size_class(n: int) -> int:
    return 0 if n < CLASS_EDGES[0] else (1 if n < CLASS_EDGES[1] else 2)


def replica_key(descs) -> str:
    """Stable key of a replica set (sizes, kinds, boxes, cutoffs)."""
    h = hashlib.sha256()
    for d in descs:
        h.update(f"{d.N}:{d.kind}:{d.L:.9g}:{d.r_cut:.6g}:{d.skin:.6g};".encode())
    return h.hexdigest()[:16]


def with_mults(descs, mult_of_class):
    """Copies of the descriptors with each replica's class multiplier."""
    out = []
    for d in descs:
        e = J.md_replica_desc.from_buffer_copy(d)
        e.cell_mult = float(mult_of_class[size_class(d.N)])
        out.append(e)
    return out


def tpp_per_replica(descs, tpp_of_class):
    return [int(tpp_of_class[size_class(d.N)]) for d in descs]


def coordinate_descent(trial, present, mults=MULTS, tpps=TPPS):
    """Search the multipliers, then the threads per particle, one class at a
    time, keeping a change only if the trial is faster.  trial(mult, tpp) ->
    time; present[c]: class c has replicas.  Returns (mult, tpp, t0, t)."""
    mult, tpp = [1.0, 1.0, 1.0], [4, 4, 4]
    t0 = best = trial(mult, tpp)
    for c in range(3):
        if not present[c]:
            continue
        for m in mults:
            if m == mult[c]:
                continue
            cand = list(mult)
            cand[c] = m
            t = trial(cand, tpp)
            if t < best:
                best, mult = t, cand
    for c in range(3):
        if not present[c]:
            continue
        for q in tpps:
            if q == tpp[c]:
                continue
            cand = list(tpp)
            cand[c] = q
            t = trial(mult, cand)
            if t < best:
                best, tpp = t, cand
    return mult, tpp, t0, best


def tune(descs, r0, v0, probe=20, cap=128, cache_path=None, stream=None):
    """Tuned {"cell_mult": [3], "tpp": [3], "ms_default", "ms_tuned"} for the
    replicas `descs` from positions r0 / velocities v0 (device [N][4]; not
    modified).  Reads and extends the cache at cache_path."""
    import torch
    key = replica_key(descs)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as fp:
                cache = json.load(fp)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return dict(cache[key], cached=True)
    present = [False, False, False]
    for d in descs:
        present[size_class(d.N)] = True
    st = torch.zeros(1, dtype=torch.int32, device=r0.device)

    def trial(mult, tpp):
        b = J.Batch(with_mults(descs, mult), cap=cap, stream=stream)
        J.md_batch_set_class_tpp(b.plan, tpp_per_replica(descs, tpp), stream)
        r, v = r0.clone(), v0.clone()
        f = torch.zeros_like(r)

        def run():
            r.copy_(r0)
            v.copy_(v0)
            J.md_batch_build(b.plan, r, st, stream)
            J.md_batch_forces(b.plan, r, f, st, stream)
            J.md_batch_run_nve(b.plan, r, v, f, probe, None, None, True, st, stream)

        run()   # captures the graph
        ts = []
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        if J.md_status_poll(st) != 0:
            raise J.MDError(J.md_status_poll(st), "batch_tune trial")
        return min(ts)

    mult, tpp, t0, t = coordinate_descent(trial, present)
    res = {"cell_mult": mult, "tpp": tpp, "ms_default": t0, "ms_tuned": t, "probe_steps": probe,
           "classes": [sum(1 for d in descs if size_class(d.N) == c) for c in range(3)]}
    if cache_path:
        cache[key] = res
        try:
            with open(cache_path, "w") as fp:
                json.dump(cache, fp)
        except OSError:
            pass
    return dict(res, cached=False)
