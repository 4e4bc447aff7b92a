"""Checkpoint file round trip and refusal rules (host only; the resume-on-GPU test is
tests/test_gpu_checkpoint.py)."""
import numpy as np
import pytest
import torch

from paper_1808_04960_gb300 import checkpoint


class _Plan:
    """The attributes of gpweno.Plan that checkpoint reads."""

    def __init__(self, shape=(6, 8), dtype=torch.float64, **kw):
        self.shape = tuple(shape)
        self.nc = len(shape) + 2
        self.dtype = dtype
        self.params = {"R": 2, "ell_over_dx": 12.0, "shape": list(shape), "dtype": "f64", "cfl": 0.4}
        self.params.update(kw)


def _state(plan, seed):
    g = torch.Generator().manual_seed(seed)
    U = torch.rand((plan.nc,) + plan.shape, generator=g, dtype=plan.dtype)
    S = torch.rand((4, plan.nc) + plan.shape, generator=g, dtype=plan.dtype)
    return U, S


def test_round_trip_restores_state_remainder_dt_and_counters(tmp_path):
    plan = _Plan()
    U, S = _state(plan, 1)
    dt = torch.tensor([3.25e-4], dtype=torch.float64)
    f = tmp_path / "run.ckpt"
    checkpoint.save(f, plan, U, S, t=0.125, step=17, dt_dev=dt, extra={"note": "x"})
    U2 = torch.zeros_like(U)
    S2 = torch.full_like(S, 7.0)
    dt2 = torch.zeros(1, dtype=torch.float64)
    t, step, extra = checkpoint.load(f, plan, U2, S2, dt_dev=dt2)
    assert (t, step, extra) == (0.125, 17, {"note": "x"})
    assert torch.equal(U2, U) and torch.equal(S2[3], S[3])
    assert torch.count_nonzero(S2[:3]) == 0          # the per-step buffers are not carried
    assert dt2.item() == dt.item()


def test_refuses_other_plan_shape_dtype_and_dt_mismatch(tmp_path):
    plan = _Plan()
    U, S = _state(plan, 2)
    f = tmp_path / "run.ckpt"
    checkpoint.save(f, plan, U, S, t=0.0, step=0)
    with pytest.raises(ValueError, match="ell_over_dx"):
        checkpoint.load(f, _Plan(ell_over_dx=24.0), torch.zeros_like(U), torch.zeros_like(S))
    with pytest.raises(ValueError, match="device time step"):
        checkpoint.load(f, plan, torch.zeros_like(U), torch.zeros_like(S), dt_dev=torch.zeros(1, dtype=torch.float64))
    with pytest.raises(ValueError, match="do not fit"):
        checkpoint.load(f, plan, torch.zeros((plan.nc, 6, 9), dtype=plan.dtype), torch.zeros_like(S))
    with pytest.raises(ValueError):
        checkpoint.save(f, plan, U.float(), S, t=0.0, step=0)
    g = tmp_path / "junk.ckpt"
    torch.save({"format": 99}, g)
    with pytest.raises(ValueError, match="format"):
        checkpoint.load(g, plan, torch.zeros_like(U), torch.zeros_like(S))


def test_save_is_atomic_and_overwrites(tmp_path):
    plan = _Plan(shape=(5,))
    U, S = _state(plan, 3)
    f = tmp_path / "run.ckpt"
    checkpoint.save(f, plan, U, S, t=1.0, step=1)
    checkpoint.save(f, plan, U * 2, S, t=2.0, step=2)
    U2, S2 = torch.zeros_like(U), torch.zeros_like(S)
    t, step, _ = checkpoint.load(f, plan, U2, S2)
    assert (t, step) == (2.0, 2) and torch.equal(U2, U * 2)
    assert [p.name for p in tmp_path.iterdir()] == ["run.ckpt"]
    assert np.array_equal(S2[3].numpy(), S[3].numpy())
