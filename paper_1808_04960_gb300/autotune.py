"""Measured autotuning of the batched stage kernel's schedule.

For one batch (a list of plans with their state and scratch tensors) every
candidate (block size, CTAs per SM) is forced through the library's tuning
cache, a batch plan is built with it, and a few SSP-RK3 steps are timed with
CUDA events on clones of the states.  The fastest candidate is written to the
cache file as "<signature hex> <block> <ctas per SM>", which
gpweno_plan_batch reads for batches with the same instance list.
"""
from __future__ import annotations

import os
import tempfile

from . import gpweno

CANDIDATES = ((128, 1), (128, 2), (128, 3), (128, 4), (256, 1), (256, 2))


def _time_batch(plans, Us, Ss, dt_dev, cache, steps, warmup):
    import torch
    batch = gpweno.BatchPlan(plans, tune_cache=cache)
    Uc = [u.clone() for u in Us]
    Sc = [s.clone() for s in Ss]
    for _ in range(warmup):
        batch.rk3_step(Uc, Sc, dt_dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        batch.rk3_step(Uc, Sc, dt_dev)
    e1.record()
    torch.cuda.synchronize()
    info = batch.info()
    ms = e0.elapsed_time(e1) / steps
    batch.close()
    return ms, info


def tune_batch(plans, Us, Ss, dt_dev, cache_path=None, candidates=CANDIDATES, steps=3, warmup=1):
    """Time every candidate schedule; return (best (block, ctas), {candidate: ms/step}).
    If cache_path is given, the best line replaces any earlier line for this batch."""
    sig = gpweno.BatchPlan(plans).info()["signature"]
    timings = {}
    fd, tmp = tempfile.mkstemp(suffix=".txt")
    os.close(fd)
    try:
        for block, cps in candidates:
            with open(tmp, "w") as f:
                f.write(f"{sig} {block} {cps}\n")
            try:
                ms, info = _time_batch(plans, Us, Ss, dt_dev, tmp, steps, warmup)
            except gpweno.GpwenoError:
                continue
            if info["block"] == block and info["ctas_per_sm"] == cps:
                timings[(block, cps)] = ms
    finally:
        os.unlink(tmp)
    best = min(timings, key=timings.get)
    if cache_path:
        lines = []
        if os.path.exists(cache_path):
            with open(cache_path) as f:
                lines = [ln for ln in f if not ln.startswith(sig)]
        lines.append(f"{sig} {best[0]} {best[1]}\n")
        with open(cache_path, "w") as f:
            f.writelines(lines)
    return best, timings
