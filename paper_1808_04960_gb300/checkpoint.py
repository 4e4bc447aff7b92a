"""Checkpoint and resume of an SSP-RK3 run.

What a step carries to the next one: the conserved state U, the remainder of
the compensated final-stage sum (the last of the four scratch buffers; the
other three are rewritten inside every step), the device time step of a
CFL-driven run, and the run's time and step count.  A checkpoint holds exactly
these, on the host, with the plan's creation parameters; loading it into
tensors of a plan with the same parameters resumes the run bit for bit (the
stage kernels are deterministic: no atomics touch the state).

A checkpoint is one file written by torch.save:
    {"format": 1, "plan": plan.params, "U": tensor, "lo": tensor,
     "dt": float or None, "t": float, "step": int, "extra": any picklable object}
Tensors are stored on the CPU in the plan's dtype, shape (nc, *grid).
"""
from __future__ import annotations

import os

FORMAT = 1


def save(path, plan, U, scratch, t: float, step: int, dt_dev=None, extra=None) -> None:
    """Write the state of a run on `plan` to `path` (atomically: a temporary file is renamed).

    U: the state after `step` steps; scratch: the run's RK3 scratch (plan.new_scratch());
    dt_dev: the device time step of a CFL-driven run (a one-element double tensor), or None."""
    import torch
    expected = (plan.nc,) + tuple(plan.shape)
    if tuple(U.shape) != expected or tuple(scratch.shape) != (4,) + expected:
        raise ValueError(f"state {tuple(U.shape)} / scratch {tuple(scratch.shape)} do not fit the plan {expected}")
    if U.dtype != plan.dtype or scratch.dtype != plan.dtype:
        raise ValueError(f"state and scratch must be {plan.dtype}")
    blob = {"format": FORMAT, "plan": dict(plan.params), "U": U.detach().to("cpu", copy=True),
            "lo": scratch[3].detach().to("cpu", copy=True),
            "dt": None if dt_dev is None else float(dt_dev.reshape(-1)[0].item()),
            "t": float(t), "step": int(step), "extra": extra}
    tmp = f"{path}.tmp{os.getpid()}"
    torch.save(blob, tmp)
    os.replace(tmp, path)


def load(path, plan, U, scratch, dt_dev=None):
    """Restore a checkpoint into U, scratch and dt_dev (device tensors of `plan`); returns
    (t, step, extra).  Refuses a checkpoint of another format or of a plan with other creation
    parameters, and one that carries a device time step when dt_dev is None (or the reverse)."""
    import torch
    blob = torch.load(path, map_location="cpu", weights_only=False)
    if not isinstance(blob, dict) or blob.get("format") != FORMAT:
        raise ValueError(f"{path}: not a checkpoint of format {FORMAT}")
    if blob["plan"] != plan.params:
        diff = sorted(k for k in set(blob["plan"]) | set(plan.params) if blob["plan"].get(k) != plan.params.get(k))
        raise ValueError(f"{path}: written for another plan (differs in {', '.join(diff)})")
    if (blob["dt"] is None) != (dt_dev is None):
        raise ValueError(f"{path}: device time step {'missing' if dt_dev is not None else 'present'} in the checkpoint")
    expected = (plan.nc,) + tuple(plan.shape)
    if tuple(U.shape) != expected or tuple(scratch.shape) != (4,) + expected:
        raise ValueError(f"state {tuple(U.shape)} / scratch {tuple(scratch.shape)} do not fit the plan {expected}")
    U.copy_(blob["U"])
    scratch.zero_()
    scratch[3].copy_(blob["lo"])
    if dt_dev is not None:
        dt_dev.fill_(blob["dt"])
    return blob["t"], blob["step"], blob["extra"]
