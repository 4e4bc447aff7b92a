"""Throughput benchmark of the GP-WENO SSP-RK3 step on GB300.

Workload (default): 2D isentropic vortex, periodic [-5,5]^2, 1024^2 cells,
GP-R2, l = 12 dx, sigma = 3 dx, gamma = 1.4, fixed dt = 0.4 / max rate of the
initial state; FP32 is the headline, FP64 is timed beside it.  A step is one
SSP-RK3 step (three fused stage launches).  Metric: cell-updates/s per RK
stage = cells x 3 x steps / time.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead (on a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GP-WENO cell-updates/s per RK stage, FP32 vs FP64, at L1 err vs FP64 oracle"
UNIT = "cell-updates/s"
# FP32 FMA lanes per SM (Blackwell: 4 sub-partitions x 32); the SM count comes from the device
# and the maximum SM clock from the measured peaks (2070 MHz on GB300 when absent)
FP32_LANES = 128


def alu_peak_flops():
    """FP32 ALU peak of the current device: SMs x 128 FMA lanes x 2 FLOP x maximum SM clock;
    returns (FLOP/s, description)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peaks, _ = read_peaks()
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    return sms * FP32_LANES * 2 * mhz * 1e6, f"derived: {sms} SMs x {FP32_LANES} FP32 lanes x 2 x {mhz:.0f} MHz"


def flops_per_cell_stage(R: int, ndim: int = 2) -> float:
    """Algorithmic FP32 operations per cell and RK stage of the GP-WENO stage (FMA = 2)."""
    from paper_1808_04960_gb300 import costmodel
    return costmodel.flops_per_cell_stage(R, ndim)


def hbm_bytes_per_cell_stage(esz: int, nc: int = 4, arrays_per_step: float = 14.0) -> float:
    """Algorithmic HBM bytes per cell and stage of the increment-form SSP-RK3, averaged over
    the three stages (state-sized arrays moved once each): stage 1 reads U and writes D, V1
    (3 arrays); stage 2 reads V1, D, U and writes D, V2 (5); stage 3 reads V2, D, U, lo and
    writes U, lo (6); 14 arrays per step.  In 3D each stage also writes and reads back the
    x+y part of L and reads its stencil state twice (23 arrays per step)."""
    return esz * nc * arrays_per_step / 3.0


def kernel_traffic(key):
    """DRAM bytes per launch of the stage kernel from the committed ncu summary, or None when
    the kernel sources changed since those counters were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            entry = json.load(f)[key]
        h = hashlib.sha256()
        for src in ("face.cuh", "stage.cuh"):
            with open(os.path.join(ROOT, "paper_1808_04960_gb300", "csrc", src), "rb") as f:
                h.update(f.read())
        return entry["traffic_bytes_per_launch"] if h.hexdigest() == entry["kernel_sources_sha256"] else None
    except (OSError, KeyError, ValueError):
        return None


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        load = [s for s in sm if s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return ws, rank, local


def max_over_ranks(x: float, ws: int) -> float:
    """The largest x over the ranks (the job's time is its slowest rank's)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def time_steps(plan, U, scratch, dt, steps, stream, flush, graph=None):
    """Per-step CUDA-event times (ms) of `steps` RK3 steps; L2 flushed between steps outside the events."""
    import torch
    times = []
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if graph is not None:
            graph.replay()
        else:
            plan.rk3_step(U, scratch, dt=dt, stream=stream)
        e1.record(stream)
        times.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in times]


def run_gpu(args):
    import numpy as np
    import torch

    from paper_1808_04960_gb300 import build as libbuild
    from paper_1808_04960_gb300 import gpweno, workloads

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if local == 0:
        libbuild.build()
    barrier(ws)
    libbuild.build()
    if ws > 1:
        return run_gpu_slabs(args, ws, rank, local)
    n, R = args.grid, args.R
    U0, meta = workloads.isentropic_vortex(n)
    cells = n * n
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > 129 MB L2

    # fixed dt of the run from the initial state (computed on the device)
    p64 = gpweno.Plan(R, 12.0, U0.shape[1:], meta["dx"], meta["bc"], dtype="f64")
    U64 = torch.from_numpy(U0).to("cuda", torch.float64)
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    p64.cfl_dt(U64, 0.4, dt_dev)
    dt = float(dt_dev.item())

    results = {}
    states = {}
    for dtype in args.dtypes.split(","):
        tdt = torch.float32 if dtype == "f32" else torch.float64
        plan = gpweno.Plan(R, 12.0, U0.shape[1:], meta["dx"], meta["bc"], dtype=dtype)
        U = torch.from_numpy(U0).to("cuda", tdt).contiguous()
        scratch = torch.zeros((4,) + tuple(U.shape), dtype=tdt, device="cuda")
        steps = args.steps if dtype == "f32" else max(3, min(args.steps, args.fp64_steps))
        for _ in range(args.warmup):
            plan.rk3_step(U, scratch, dt=dt, stream=stream)
        launches = gpweno.last_launch_count()
        graph = None
        if args.graph:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                plan.rk3_step(U, scratch, dt=dt)
            graph.replay()   # one more warm step through the graph
        torch.cuda.synchronize()
        barrier(ws)
        with ClockSampler(local) as clk:
            t_list = time_steps(plan, U, scratch, dt, steps, stream, flush, graph)
        barrier(ws)
        total_ms = max_over_ranks(sum(t_list), ws)
        results[dtype] = dict(ms_per_step=total_ms / steps, steps=steps, launches_per_step=launches,
                              value=ws * cells * 3 * steps / (total_ms * 1e-3), clocks=clk.summary(),
                              kernel_ms=statistics.mean(t_list) / 3.0, schedule=plan.schedule())
        states[dtype] = (plan, U, scratch)
        assert plan.flags() == 0, "non-physical state in benchmark run"

    # accuracy of FP32 against the FP64 path after the same number of steps from the same data
    acc = None
    if "f64" in states:
        n32 = args.acc_steps
        p32, _, s32 = states["f32"]
        U32 = torch.from_numpy(U0).to("cuda", torch.float32).contiguous()
        U64 = torch.from_numpy(U0).to("cuda", torch.float64).contiguous()
        s64 = states["f64"][2]
        for _ in range(n32):
            p32.rk3_step(U32, s32, dt=dt)
            states["f64"][0].rk3_step(U64, s64, dt=dt)
        d = (U32.double() - U64).abs()
        acc = {"steps": n32, "l1_f32_vs_f64_gpu": float(d.mean()), "linf_f32_vs_f64_gpu": float(d.max())}

    # end to end through the public API: pinned host state in, step, state out, every step
    plan, U, scratch = states["f32"]
    host = torch.from_numpy(U0.astype(np.float32)).pin_memory()
    host_out = torch.empty_like(host).pin_memory()
    nb = host.numel() * host.element_size()
    # Every step copies its input in from pinned host memory and its result out.  The copies run
    # on their own streams (one per direction, so both copy engines work) with two device
    # buffers: step k+1's upload and step k-1's download overlap step k's compute.
    bufs = [U, torch.empty_like(U)]
    outs = [host_out, torch.empty_like(host).pin_memory()]
    h2d_s, d2h_s = torch.cuda.Stream(), torch.cuda.Stream()
    up = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    down = [torch.cuda.Event() for _ in range(2)]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for s_ in (h2d_s, d2h_s):
        s_.wait_event(e0)
    for k in range(args.steps):
        b = k % 2
        with torch.cuda.stream(h2d_s):
            if k >= 2:
                h2d_s.wait_event(down[b])          # buffer b's previous result has been read out
            bufs[b].copy_(host, non_blocking=True)
            up[b].record(h2d_s)
        stream.wait_event(up[b])
        plan.rk3_step(bufs[b], scratch, dt=dt, stream=stream)
        done[b].record(stream)
        with torch.cuda.stream(d2h_s):
            d2h_s.wait_event(done[b])
            outs[b].copy_(bufs[b], non_blocking=True)
            down[b].record(d2h_s)
    for ev in down:
        stream.wait_event(ev)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), ws)
    e2e = {"value": ws * cells * 3 * args.steps / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": nb,
           "d2h_bytes_per_step": nb, "ms_per_step": e2e_ms / args.steps,
           "copies": "pinned host, own stream per direction, double-buffered, overlapped with compute"}

    batch = run_batch(args, stream, rank, ws) if args.batch_count > 0 else None
    extra = run_configs(args, stream) if args.configs else None
    variants = run_variants(args, stream) if args.variant_steps > 0 else None

    if rank != 0:
        return None
    peaks, peak_kind = read_peaks()
    r32 = results["f32"]
    kernel_s = r32["kernel_ms"] * 1e-3
    flops = flops_per_cell_stage(R) * cells
    alu_peak_fs, alu_peak_kind = alu_peak_flops()
    alu_peak = alu_peak_fs / 1e12
    achieved = flops / kernel_s / 1e12
    hbm_ach = hbm_bytes_per_cell_stage(4) * cells / kernel_s / 1e9
    line = {
        "metric": METRIC, "value": r32["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r32["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"2D isentropic vortex {n}x{n} periodic [-5,5]^2, GP-R{R}, l=12dx, sigma=3dx, "
                               "SSP-RK3 fixed dt (CFL 0.4)", "grid": [n, n], "R": R, "ell_over_dx": 12.0,
                   "sigma_over_dx": 3.0, "dt": dt, "cuda_graph": bool(args.graph),
                   "l2": "flushed between timed steps (256 MiB write outside the events)",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "fp64": ({"value": results["f64"]["value"], "ms_per_step": results["f64"]["ms_per_step"],
                  "steps": results["f64"]["steps"], "fp32_over_fp64": r32["value"] / results["f64"]["value"]}
                 if "f64" in results else None),
        "accuracy": acc,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": achieved / alu_peak,
                     "traffic": (kernel_traffic(f"stage2d_kernel<float,{R},128> vortex{n}")
                                 if args.graph and n == 1024 and R == 2 else None),
                     "kernel": f"stage2d_kernel<float,{R},128> ({r32['schedule']['ctas_per_sm']}-CTA/SM build, "
                               f"{r32['schedule']['grid']} CTAs, {r32['schedule']['strips']} strips of "
                               f"{r32['schedule']['strip_width']} columns)",
                     "peak_kind": alu_peak_kind,
                     "flops_per_cell_stage": flops_per_cell_stage(R)},
        "roofline_hbm": {"bound": "hbm", "achieved": hbm_ach, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                         "frac": hbm_ach / peaks.get("hbm_gbs"), "peak_kind": peak_kind,
                         "bytes_per_cell_stage": hbm_bytes_per_cell_stage(4)},
        "e2e": e2e,
        "batch": batch,
        "configs": extra,
        "variants": variants,
        "gpu_launches": r32["launches_per_step"] * args.steps,
        "clocks": r32["clocks"],
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, dt)
    return line


def run_gpu_slabs(args, ws, rank, local):
    """N > 1 GPUs: one grid cut into N slabs along y, one slab per GPU, the G = R+3 boundary
    layers of every stage's input exchanged with the neighbouring slabs over NCCL before the
    stage (decomp.SlabStepper).  The grid is N periodic images of the single-GPU vortex stacked
    along y (1024 x 1024 N cells), so every rank steps the single-GPU workload plus the exchange
    (weak scaling).  FP32, fixed dt; the batch is split over the ranks by instance."""
    import numpy as np
    import torch

    from paper_1808_04960_gb300 import decomp, gpweno, workloads
    n, R = args.grid, args.R
    U0, meta = workloads.isentropic_vortex(n)
    cells = n * n
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    p64 = gpweno.Plan(R, 12.0, U0.shape[1:], meta["dx"], meta["bc"], dtype="f64")
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    p64.cfl_dt(torch.from_numpy(U0).to("cuda").contiguous(), 0.4, dt_dev)
    dt = float(dt_dev.item())
    slab = decomp.Slab((n * ws, n), meta["bc"], rank, ws, R + 3)
    assert slab.local_shape == U0.shape[1:]
    plan = gpweno.Plan(R, 12.0, slab.local_shape, meta["dx"], slab.local_bc, dtype="f32")
    stepper = decomp.SlabStepper(plan, slab)
    U = torch.from_numpy(U0).to("cuda", torch.float32).contiguous()
    for _ in range(args.warmup):
        stepper.step(U, dt=dt, stream=stream)
    torch.cuda.synchronize()
    barrier(ws)
    with ClockSampler(local) as clk:
        times = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stepper.step(U, dt=dt, stream=stream)
            e1.record(stream)
            times.append((e0, e1))
        torch.cuda.synchronize()
        t_list = [a.elapsed_time(b) for a, b in times]
    barrier(ws)
    total_ms = max_over_ranks(sum(t_list), ws)
    nonphys = plan.flags()
    # end to end: the slab in from pinned host memory, the step, the slab out, every step
    host = torch.from_numpy(U0.astype(np.float32)).pin_memory()
    host_out = torch.empty_like(host).pin_memory()
    nb = host.numel() * host.element_size()
    torch.cuda.synchronize()
    barrier(ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        U.copy_(host, non_blocking=True)
        stepper.step(U, dt=dt, stream=stream)
        host_out.copy_(U, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), ws)
    batch = run_batch(args, stream, rank, ws) if args.batch_count > 0 else None
    if rank != 0:
        return None
    kernel_s = total_ms / args.steps / 3.0 * 1e-3
    alu_peak_fs, alu_peak_kind = alu_peak_flops()
    achieved = flops_per_cell_stage(R) * cells / kernel_s / 1e12
    peaks, peak_kind = read_peaks()
    hbm_ach = hbm_bytes_per_cell_stage(4) * cells / kernel_s / 1e9
    return {
        "metric": METRIC, "value": ws * cells * 3 * args.steps / (total_ms * 1e-3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"2D isentropic vortex, {ws} periodic images of the {n}x{n} [-5,5]^2 vortex "
                               f"stacked along y ({n}x{n * ws} cells), GP-R{R}, l=12dx, sigma=3dx, SSP-RK3 fixed "
                               "dt (CFL 0.4)", "grid": [n, n * ws], "R": R, "ell_over_dx": 12.0,
                   "sigma_over_dx": 3.0, "dt": dt, "cuda_graph": False,
                   "l2": "flushed between timed steps (256 MiB write outside the events)",
                   "parallelism": f"slabs{ws}: y-slab per GPU, NCCL halo exchange of G={R + 3} layers "
                                  "before every stage"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak_fs / 1e12, "unit": "TFLOP/s",
                     "frac": achieved / (alu_peak_fs / 1e12), "traffic": None,
                     "kernel": f"stage2d_kernel<float,{R},128> (per GPU, step time incl. the exchange)",
                     "peak_kind": alu_peak_kind, "flops_per_cell_stage": flops_per_cell_stage(R)},
        "roofline_hbm": {"bound": "hbm", "achieved": hbm_ach, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                         "frac": hbm_ach / peaks.get("hbm_gbs"), "peak_kind": peak_kind},
        "e2e": {"value": ws * cells * 3 * args.steps / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": nb,
                "d2h_bytes_per_step": nb, "ms_per_step": e2e_ms / args.steps,
                "copies": "per rank: its slab in from pinned host memory and out again, every step, one stream"},
        "batch": batch,
        "gpu_launches": 6 * args.steps,
        "nonphysical_flag": nonphys,
        "clocks": clk.summary(),
    }


def run_batch(args, stream, rank=0, ws=1):
    """Batched workload: `--batch-count` seeded 2D instances (n_x, n_y log-uniform on [64, 1024],
    R in {1,2,3}, l/dx in {6,12,24}, half four-quadrant, half vortex), per-instance CFL dt.
    With N ranks the instances are split over the ranks by estimated cost (no exchange: they are
    independent), each rank one launch per RK stage for its share.  FP32 under a CUDA
    graph against per-instance launches and against the FP64 batch; the FP32 states' error
    against the FP64 batch after the same steps."""
    import torch

    from paper_1808_04960_gb300 import decomp, gpweno, workloads
    insts = workloads.batch_instances(args.batch_count, seed=5)
    costs = [decomp.instance_cost(i["nx"], i["ny"], i["R"]) for i in insts]
    parts, loads = decomp.shard_instances(costs, ws)
    mine = [insts[k] for k in parts[rank]]
    if not mine:
        raise RuntimeError(f"{ws} ranks for {len(insts)} batch instances: rank {rank} has none")
    cache = os.path.join(ROOT, "paper_1808_04960_gb300", "tune_cache.txt")

    def build(dtype):
        tdt = torch.float32 if dtype == "f32" else torch.float64
        plans, Us, Ss, dts = [], [], [], []
        for inst in mine:
            m = inst["meta"]
            p = gpweno.Plan(inst["R"], inst["ell_over_dx"], inst["U"].shape[1:], m["dx"], m["bc"], dtype=dtype)
            U = torch.from_numpy(inst["U"]).to("cuda", tdt).contiguous()
            plans.append(p)
            Us.append(U)
            Ss.append(p.new_scratch())
        # the same per-instance dt for both precisions: CFL 0.4 of the FP64 initial state
        for inst in mine:
            m = inst["meta"]
            p64 = gpweno.Plan(inst["R"], inst["ell_over_dx"], inst["U"].shape[1:], m["dx"], m["bc"], dtype="f64")
            d = torch.zeros(1, dtype=torch.float64, device="cuda")
            p64.cfl_dt(torch.from_numpy(inst["U"]).to("cuda").contiguous(), 0.4, d)
            dts.append(d)
        return plans, Us, Ss, torch.cat(dts)

    def timed(batch, Us, Ss, dt_dev, steps, graph=True):
        for _ in range(2):
            batch.rk3_step(Us, Ss, dt_dev, stream=stream)
        g = None
        if graph:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                batch.rk3_step(Us, Ss, dt_dev)
            g.replay()
        torch.cuda.synchronize()
        barrier(ws)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record(stream)
        for _ in range(steps):
            if g is not None:
                g.replay()
            else:
                batch.rk3_step(Us, Ss, dt_dev, stream=stream)
        e[1].record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        return max_over_ranks(e[0].elapsed_time(e[1]), ws) / steps

    plans, Us, Ss, dt_dev = build("f32")
    cells = sum(i["nx"] * i["ny"] for i in insts)
    batch = gpweno.BatchPlan(plans, tune_cache=cache)
    ms_b = timed(batch, Us, Ss, dt_dev, args.batch_steps)
    # per-instance launches (3 per instance per step), no graph
    dt_host = dt_dev.cpu().tolist()
    barrier(ws)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record(stream)
    for _ in range(args.batch_steps):
        for p, U, S, dt in zip(plans, Us, Ss, dt_host):
            p.rk3_step(U, S, dt=dt, stream=stream)
    e[1].record(stream)
    torch.cuda.synchronize()
    ms_u = max_over_ranks(e[0].elapsed_time(e[1]), ws) / args.batch_steps
    nonphys = batch.flags()
    info = batch.info()
    # ALU fraction on the method's operation count of each instance's radius, over all ranks' peaks
    alu_peak, _ = alu_peak_flops()
    flops_stage = sum(i["nx"] * i["ny"] * flops_per_cell_stage(i["R"]) for i in insts)
    out = {"workload": f"{len(insts)} seeded 2D instances, n_x,n_y log-uniform on [64,1024], R in {{1,2,3}}, "
                       "l/dx in {6,12,24}, four-quadrant/vortex, FP32, per-instance CFL 0.4 (fixed dt)",
           "instances": len(insts), "cells": cells, "steps": args.batch_steps,
           "value": cells * 3 / (ms_b * 1e-3), "unit": UNIT, "ms_per_step": ms_b,
           "unbatched_value": cells * 3 / (ms_u * 1e-3), "unbatched_ms_per_step": ms_u,
           "speedup_vs_unbatched": ms_u / ms_b, "launches_per_step": 3,
           "alu_frac": flops_stage * 3 / (ms_b * 1e-3) / (alu_peak * ws),
           "flops_per_cell_stage_mean": flops_stage / cells,
           "unbatched_launches_per_step": 3 * len(insts), "schedule": info, "nonphysical_flag": nonphys,
           "sharding": {"ranks": ws, "instances_per_rank": [len(p) for p in parts],
                        "cost_share_max_over_mean": max(loads) / (sum(loads) / ws)}}
    # FP64 batch from the same initial data: throughput, and the FP32 error against it after the
    # same number of steps (FP32 states restarted from the initial data; the FP64 GPU path is pinned
    # to the oracle by the tests)
    if args.batch_fp64_steps > 0:
        del batch
        p64, U64, S64, dt64 = build("f64")
        b64 = gpweno.BatchPlan(p64, tune_cache=cache)
        ms_64 = timed(b64, U64, S64, dt64, args.batch_fp64_steps)
        out["fp64"] = {"value": cells * 3 / (ms_64 * 1e-3), "ms_per_step": ms_64, "steps": args.batch_fp64_steps,
                       "fp32_over_fp64": ms_64 / ms_b}
        for U, inst in zip(Us, mine):
            U.copy_(torch.from_numpy(inst["U"]).to("cuda", torch.float32))
        for U, inst in zip(U64, mine):
            U.copy_(torch.from_numpy(inst["U"]).to("cuda", torch.float64))
        for S in Ss + S64:
            S.zero_()
        b32 = gpweno.BatchPlan(plans, tune_cache=cache)
        k = args.acc_batch_steps
        for _ in range(k):
            b32.rk3_step(Us, Ss, dt_dev, stream=stream)
            b64.rk3_step(U64, S64, dt64, stream=stream)
        torch.cuda.synchronize()
        tot, n_el, mx = 0.0, 0, 0.0
        for a, b in zip(Us, U64):
            d = (a.double() - b).abs()
            tot += float(d.sum())
            n_el += d.numel()
            mx = max(mx, float(d.max()))
        out["accuracy"] = {"steps": k, "l1_f32_vs_f64_gpu": tot / max(n_el, 1), "linf_f32_vs_f64_gpu": mx,
                           "fp64_gpu_vs_oracle": "pinned by tests/test_gpu_batch.py (1e-10)"}
    return out


def timed_cfl_run(plan, U, steps, stream, flops_cell, cells, bytes_cell):
    """`steps` SSP-RK3 steps with the CFL time step kept on the device (fused into the last stage),
    one step captured in a CUDA graph; returns throughput and roofline fractions."""
    import torch

    from paper_1808_04960_gb300 import gpweno
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    plan.cfl_dt(U, plan.cfl, dt_dev)
    s = plan.new_scratch()
    for _ in range(2):
        plan.rk3_step(U, s, dt_dev=dt_dev, stream=stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.rk3_step(U, s, dt_dev=dt_dev)
    launches = gpweno.last_launch_count()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    alu_peak, _ = alu_peak_flops()
    per_stage_s = ms * 1e-3 / 3
    peaks, _ = read_peaks()
    return {"value": cells * 3 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "launches_per_step": launches, "dt_last": float(dt_dev.item()), "nonphysical_flag": plan.flags(),
            "alu_frac": flops_cell * cells / per_stage_s / alu_peak,
            "hbm_frac": bytes_cell * cells / per_stage_s / (peaks.get("hbm_gbs", 6800.0) * 1e9)}


def fp32_vs_fp64(R, U0, meta, steps, stream, **opts):
    """FP32 and FP64 GPU runs from the same initial data with the same fixed dt (CFL 0.4 of the
    FP64 initial state): L1 (mean) and L-inf of FP32 - FP64 after `steps` SSP-RK3 steps.  The FP64
    GPU path itself is pinned to the FP64 oracle by the tests (sampled blocks at full size)."""
    import torch

    from paper_1808_04960_gb300 import gpweno
    p64 = gpweno.Plan(R, 12.0, U0.shape[1:], meta["dx"], meta["bc"], dtype="f64", **opts)
    U64 = torch.from_numpy(U0).to("cuda", torch.float64).contiguous()
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    p64.cfl_dt(U64, 0.4, d)
    dt = float(d.item())
    s64 = p64.new_scratch()
    for _ in range(steps):
        p64.rk3_step(U64, s64, dt=dt, stream=stream)
    del s64
    p32 = gpweno.Plan(R, 12.0, U0.shape[1:], meta["dx"], meta["bc"], dtype="f32", **opts)
    U32 = torch.from_numpy(U0).to("cuda", torch.float32).contiguous()
    s32 = p32.new_scratch()
    for _ in range(steps):
        p32.rk3_step(U32, s32, dt=dt, stream=stream)
    del s32
    torch.cuda.synchronize()
    l1, linf = 0.0, 0.0
    for c in range(U32.shape[0]):                     # per component, to bound the extra memory
        dd = (U32[c].double() - U64[c]).abs()
        l1 += float(dd.sum())
        linf = max(linf, float(dd.max()))
    out = {"steps": steps, "dt": dt, "l1_f32_vs_f64_gpu": l1 / U32.numel(), "linf_f32_vs_f64_gpu": linf,
           "nonphysical_flag": max(p32.flags(), p64.flags()),
           "fp64_gpu_vs_oracle": "pinned by the tests (sampled blocks at full size)"}
    del U32, U64
    torch.cuda.empty_cache()
    return out


def run_configs(args, stream):
    """The other measured configurations: the 4096^2 seeded four-quadrant Riemann problem (GP-R2,
    l=12dx, CFL 0.4 from the device each step) and the 3D Mach-3 shock into a 32-mode density field
    (512^3 by default, GP-R3, CFL 0.4), both FP32."""
    import torch

    from paper_1808_04960_gb300 import costmodel, gpweno, workloads
    out = {}
    n = args.fq_grid
    U0, m = workloads.four_quadrant(n, seed=3)
    plan = gpweno.Plan(2, 12.0, U0.shape[1:], m["dx"], m["bc"], dtype="f32", cfl=0.4)
    U = torch.from_numpy(U0).to("cuda", torch.float32).contiguous()
    r = timed_cfl_run(plan, U, args.fq_steps, stream, costmodel.flops_per_cell_stage(2, 2), n * n,
                      hbm_bytes_per_cell_stage(4, 4))
    r["workload"] = f"four-quadrant Riemann problem {n}x{n} on [0,1]^2, seeded states, outflow, GP-R2, l=12dx, " \
                    f"sigma=3dx, SSP-RK3, CFL 0.4 (device dt), FP32"
    r["flops_per_cell_stage"] = costmodel.flops_per_cell_stage(2, 2)
    del U, plan
    torch.cuda.empty_cache()
    if args.acc_config_steps > 0:
        r["accuracy"] = fp32_vs_fp64(2, U0, m, args.acc_config_steps, stream)
    out["four_quadrant"] = r
    del U0
    n3 = args.shock_grid
    if n3 > 0:
        U0, m = workloads.shock_turbulence_3d(n3, seed=4)
        plan = gpweno.Plan(3, 12.0, U0.shape[1:], m["dx"], m["bc"], dtype="f32", cfl=0.4)
        U = torch.from_numpy(U0).to("cuda", torch.float32).contiguous()
        r = timed_cfl_run(plan, U, args.shock_steps, stream, costmodel.flops_per_cell_stage(3, 3), n3 ** 3,
                          hbm_bytes_per_cell_stage(4, 5, 23.0))
        r["workload"] = f"3D Mach-3 shock into a 32-mode seeded density field, {n3}^3, periodic y/z, " \
                        f"zero-gradient x, GP-R3, l=12dx, sigma=3dx, SSP-RK3, CFL 0.4 (device dt), FP32"
        r["flops_per_cell_stage"] = costmodel.flops_per_cell_stage(3, 3)
        del U, plan
        torch.cuda.empty_cache()
        if args.acc_config_steps > 0:
            r["accuracy"] = fp32_vs_fp64(3, U0, m, max(1, args.acc_config_steps // 5), stream)
        out["shock_turbulence_3d"] = r
        del U0
    torch.cuda.empty_cache()
    return out


def run_variants(args, stream):
    """Throughput of the scheme variants on one workload: the seeded four-quadrant Riemann
    problem (GP-R2, l=12dx, CFL 0.4 from the device each step, FP32), the default scheme
    (FD-Prim, Lax-Friedrichs face flux) beside HLLC, HLL, the non-zero-mean smoothness
    indicators, the polynomial-candidate hybrid, the FD-Flux form and GP-AO(2,3); each with its
    own algorithmic operation count for the ALU fraction."""
    import torch

    from paper_1808_04960_gb300 import costmodel, gpweno, workloads
    n = args.variant_grid
    U0, m = workloads.four_quadrant(n, seed=3)
    cases = [("fdprim_lf", {}, {}), ("fdprim_hllc", {"flux": "hllc"}, {"flux": "hllc"}),
             ("fdprim_hll", {"flux": "hll"}, {"flux": "hll"}),
             ("fdprim_lf_beta_mean", {"beta_mean": True}, {"beta_mean": True}),
             ("fdprim_lf_poly_candidates", {"candidates": "poly"}, {}),
             ("fdflux", {"scheme": "fdflux"}, {"scheme": "fdflux"}),
             ("ao_2_3", {"ao": True}, {"ao": True})]
    out = {"workload": f"four-quadrant Riemann problem {n}x{n} on [0,1]^2, seeded states, outflow, GP-R2, "
                       f"l=12dx, sigma=3dx, SSP-RK3, CFL 0.4 (device dt), FP32, {args.variant_steps} steps each"}
    base = None
    for name, opts, cm in cases:
        plan = gpweno.Plan(2, 12.0, U0.shape[1:], m["dx"], m["bc"], dtype="f32", cfl=0.4, **opts)
        U = torch.from_numpy(U0).to("cuda", torch.float32).contiguous()
        flops = costmodel.flops_per_cell_stage(2, 2, **cm)
        r = timed_cfl_run(plan, U, args.variant_steps, stream, flops, n * n, hbm_bytes_per_cell_stage(4, 4))
        r["flops_per_cell_stage"] = flops
        r["flops_kind"] = "modelled" if cm.get("scheme") == "fdflux" or cm.get("ao") else "oracle tally"
        base = base or r["value"]
        r["vs_default"] = r["value"] / base
        del U, plan
        if args.acc_config_steps > 0:
            r["accuracy"] = fp32_vs_fp64(2, U0, m, args.acc_config_steps, stream, **opts)
        out[name] = r
    torch.cuda.empty_cache()
    return out


def _oracle_sample(job):
    """One oracle run of the bounded sample (a worker of the all-core measurement)."""
    n, R, steps = job
    import oracle
    from paper_1808_04960_gb300 import workloads
    U0, meta = workloads.isentropic_vortex(n)
    o = oracle.Oracle(U0.shape[1:], meta["dx"], meta["bc"], R=R, ell_over_dx=12.0)
    o.run(U0, 0.4 / o.max_rate(U0), steps)
    return n * n * 3 * steps


def oracle_all_cores(n, R, steps):
    """The same sample on every host core at once: independent oracle processes (spawned, so
    no CUDA state is inherited), aggregate cell-updates/s over the wall time."""
    import multiprocessing as mproc
    cores = os.cpu_count() or 1
    ctx = mproc.get_context("spawn")
    try:
        with ctx.Pool(cores) as pool:
            pool.map_async(_oracle_sample, [(16, R, 1)] * cores).get(timeout=300)   # start-up, untimed
            t0 = time.perf_counter()
            work = sum(pool.map_async(_oracle_sample, [(n, R, steps)] * cores).get(timeout=600))
            secs = time.perf_counter() - t0
    except Exception as e:   # the single-thread figure stands on its own
        return {"unavailable": f"{type(e).__name__}: {e}"}
    return {"value": work / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} concurrent copies of the single-thread sample, {secs:.2f} s wall"}


def cpu_baseline(args, dt_full, gpu_compare=True):
    """The FP64 oracle, as it stands, on a bounded sample: the vortex at `--cpu-grid`^2 for
    `--cpu-steps` RK3 steps (single-threaded C).  Also reports the GPU FP32/FP64 error
    against the oracle on that same sample."""
    import numpy as np

    import oracle
    from paper_1808_04960_gb300 import workloads
    n = args.cpu_grid
    U0, meta = workloads.isentropic_vortex(n)
    o = oracle.Oracle(U0.shape[1:], meta["dx"], meta["bc"], R=args.R, ell_over_dx=12.0)
    dt = 0.4 / o.max_rate(U0)
    t0 = time.perf_counter()
    ref = o.run(U0, dt, args.cpu_steps)
    secs = time.perf_counter() - t0
    out = {"value": n * n * 3 * args.cpu_steps / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"vortex {n}x{n}, GP-R{args.R}, {args.cpu_steps} SSP-RK3 steps, FP64 C oracle, "
                     f"1 thread, {secs:.2f} s"}
    out["all_cores"] = oracle_all_cores(n, args.R, args.cpu_steps)
    if gpu_compare:
        import torch

        from paper_1808_04960_gb300 import gpweno
        errs = {}
        for dtype in ("f32", "f64"):
            tdt = torch.float32 if dtype == "f32" else torch.float64
            plan = gpweno.Plan(args.R, 12.0, U0.shape[1:], meta["dx"], meta["bc"], dtype=dtype)
            U = torch.from_numpy(U0).to("cuda", tdt).contiguous()
            s = torch.zeros((4,) + tuple(U.shape), dtype=tdt, device="cuda")
            for _ in range(args.cpu_steps):
                plan.rk3_step(U, s, dt=dt)
            d = np.abs(U.double().cpu().numpy() - ref)
            errs[dtype] = {"l1": float(d.mean()), "linf": float(d.max())}
        out["gpu_error_vs_oracle_on_sample"] = errs
    return out


def run_reference(args):
    """The reference arm: the FP64 CPU oracle, as it stands, one SSP-RK3 step per bench step on a
    bounded sample of the workload (a smaller vortex grid, sized so the whole run takes about two
    minutes at ~3.5 us per cell and RHS evaluation)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import oracle
    from paper_1808_04960_gb300 import workloads
    per_step_budget = 120.0 / (args.steps + args.warmup)
    n = int(math.sqrt(per_step_budget / (3 * 3.5e-6)))
    n = max(32, min(args.cpu_grid, (n // 8) * 8))
    U0, meta = workloads.isentropic_vortex(n)
    o = oracle.Oracle(U0.shape[1:], meta["dx"], meta["bc"], R=args.R, ell_over_dx=12.0)
    dt = 0.4 / o.max_rate(U0)
    U = U0
    for _ in range(args.warmup):
        U = o.rk3_step(U, dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U = o.rk3_step(U, dt)
    secs = time.perf_counter() - t0
    v = n * n * 3 * args.steps / secs
    sample = f"vortex {n}x{n} (bounded sample of the {args.grid}x{args.grid} workload), GP-R{args.R}, " \
             f"1 SSP-RK3 step per bench step, FP64 C oracle, 1 thread"
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"2D isentropic vortex {args.grid}x{args.grid} periodic [-5,5]^2, GP-R{args.R}, "
                                   "l=12dx, sigma=3dx, SSP-RK3 fixed dt (CFL 0.4)", "grid": [args.grid, args.grid],
                       "R": args.R, "sample_grid": [n, n]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpweno", choices=["gpweno", "reference"])
    ap.add_argument("--grid", type=int, default=1024)
    ap.add_argument("--R", type=int, default=2)
    ap.add_argument("--fp64-steps", type=int, default=60)
    ap.add_argument("--acc-steps", type=int, default=100, help="steps of the FP32-vs-FP64 accuracy run")
    ap.add_argument("--cpu-grid", type=int, default=256)
    ap.add_argument("--cpu-steps", type=int, default=4)
    ap.add_argument("--no-graph", dest="graph", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dtypes", default="f32,f64", help="comma list; f32 is always first and required")
    ap.add_argument("--batch-count", type=int, default=256, help="instances of the batched workload (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--batch-fp64-steps", type=int, default=3, help="timed steps of the FP64 batch (0: skip)")
    ap.add_argument("--acc-batch-steps", type=int, default=5, help="steps of the batch FP32-vs-FP64 comparison")
    ap.add_argument("--acc-config-steps", type=int, default=10,
                    help="steps of the FP32-vs-FP64 comparison of the 4096^2 and variant runs (3D: a fifth)")
    ap.add_argument("--no-configs", dest="configs", action="store_false",
                    help="skip the four-quadrant 4096^2 and 3D shock-turbulence measurements")
    ap.add_argument("--fq-grid", type=int, default=4096)
    ap.add_argument("--fq-steps", type=int, default=100)
    ap.add_argument("--shock-grid", type=int, default=512)
    ap.add_argument("--shock-steps", type=int, default=20)
    ap.add_argument("--variant-grid", type=int, default=2048, help="grid of the scheme-variant comparison")
    ap.add_argument("--variant-steps", type=int, default=30, help="steps per variant (0: skip the comparison)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    line = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
