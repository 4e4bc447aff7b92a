"""Measured autotuning of the batched stage kernel's schedule and tile shapes.

For one batch (a list of plans with their state and scratch tensors) every
candidate schedule -- block size, resident CTAs per SM, the cap on a strip's
width, the fewest rows of a segment that does not end its strip, and CTA
shares per resident slot -- is forced through the library's tuning cache, a
batch plan is built with it, and a few SSP-RK3 steps are timed with CUDA
events on clones of the states.  The fastest candidate is written to the cache
file as "<signature hex> <block> <ctas per SM> <width cap> <min rows>
<shares per slot>", which gpweno_plan_batch reads for batches with the same
instance list.  Every candidate computes the same faces, so the results do not
depend on the choice (the tests check this bitwise).
"""
from __future__ import annotations

import itertools
import os
import tempfile

from . import gpweno

# (block, CTAs per SM) pairs the register budget allows, then the tile shapes
BLOCKS = ((128, 2), (128, 3), (128, 4), (256, 1), (256, 2))
WIDTH_CAPS = (0, 64, 96)         # 0: the widest strip the block allows (block - 5 columns)
MIN_ROWS = (4, 8, 16, 24)
SHARES_PER_SLOT = (1, 2, 3, 4, 6, 8, 12, 16)
CANDIDATES = tuple((b, c, w, r, o) for (b, c), w, r, o in itertools.product(BLOCKS, WIDTH_CAPS, MIN_ROWS,
                                                                            SHARES_PER_SLOT))


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
    """Time every candidate schedule; return (best candidate, {candidate: ms/step}), a candidate
    being (block, CTAs per SM, width cap, min rows, shares per slot).
    If cache_path is given, the best line replaces any earlier line for this batch."""
    sig = gpweno.BatchPlan(plans).info()["signature"]
    timings = {}
    fd, tmp = tempfile.mkstemp(suffix=".txt")
    os.close(fd)
    try:
        for cand in candidates:
            block, cps = cand[0], cand[1]
            with open(tmp, "w") as f:
                f.write(f"{sig} " + " ".join(str(x) for x in cand) + "\n")
            try:
                ms, info = _time_batch(plans, Us, Ss, dt_dev, tmp, steps, warmup)
            except gpweno.GpwenoError:
                continue
            if info["block"] == block and info["ctas_per_sm"] == cps:
                timings[cand] = ms
    finally:
        os.unlink(tmp)
    best = min(timings, key=timings.get)
    if cache_path:
        lines = []
        if os.path.exists(cache_path):
            with open(cache_path) as f:
                lines = [ln for ln in f if not ln.startswith(sig)]
        lines.append(f"{sig} " + " ".join(str(x) for x in best) + "\n")
        with open(cache_path, "w") as f:
            f.writelines(lines)
    return best, timings


def _main():
    """Tune the seeded batch workload (``workloads.batch_instances``) and write its line into a
    tuning cache: python -m paper_1808_04960_gb300.autotune [--count N] [--cache PATH]."""
    import argparse

    import torch

    from . import workloads
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=256)
    ap.add_argument("--cache", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.txt"))
    ap.add_argument("--steps", type=int, default=5)
    args = ap.parse_args()
    plans, Us, Ss, dts = [], [], [], []
    for inst in workloads.batch_instances(args.count, seed=5):
        m = inst["meta"]
        p = gpweno.Plan(inst["R"], inst["ell_over_dx"], inst["U"].shape[1:], m["dx"], m["bc"], dtype="f32")
        U = torch.from_numpy(inst["U"]).to("cuda", torch.float32).contiguous()
        d = torch.zeros(1, dtype=torch.float64, device="cuda")
        p.cfl_dt(U, 0.4, d)
        plans.append(p)
        Us.append(U)
        Ss.append(p.new_scratch())
        dts.append(d)
    best, timings = tune_batch(plans, Us, Ss, torch.cat(dts), args.cache, steps=args.steps, warmup=2)
    for cand, ms in sorted(timings.items(), key=lambda kv: kv[1]):
        print("block %4d  ctas/SM %d  width cap %3d  min rows %2d  shares/slot %d  %8.3f ms/step" % (cand + (ms,)))
    print("best", best, "->", args.cache)


if __name__ == "__main__":
    _main()
