"""Resume from a checkpoint reproduces the uninterrupted SSP-RK3 run bit for bit: the state,
the compensation remainder and the device time step are all that a step carries forward."""
import numpy as np
import pytest

from paper_1808_04960_gb300 import checkpoint, gpweno
from paper_1808_04960_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _case(name):
    if name == "vortex2d":
        U0, meta = W.isentropic_vortex(64)
        return U0, meta, 2
    if name == "quadrant2d":
        U0, meta = W.four_quadrant(48, seed=3)
        return U0, meta, 3
    U0, meta = W.shock_turbulence_3d(20, seed=4)
    return U0, meta, 3


@pytest.mark.parametrize("name", ["vortex2d", "quadrant2d", "shock3d"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_resume_is_bitwise(tmp_path, name, dtype):
    import torch
    U0, meta, R = _case(name)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    n1, n2 = 3, 4

    def fresh():
        p = gpweno.Plan(R, 12.0, U0.shape[1:], meta["dx"], meta["bc"], dtype=dtype, cfl=0.4)
        U = torch.from_numpy(U0).to("cuda", tdt).contiguous()
        return p, U, p.new_scratch(), torch.zeros(1, dtype=torch.float64, device="cuda")

    # uninterrupted run with the device CFL time step
    p, U, S, dt = fresh()
    p.cfl_dt(U, 0.4, dt)
    for _ in range(n1 + n2):
        p.rk3_step(U, S, dt_dev=dt)
    torch.cuda.synchronize()
    ref, ref_lo, ref_dt = U.clone(), S[3].clone(), dt.item()

    # interrupted: n1 steps, checkpoint, everything discarded, a new plan, resume, n2 steps
    p, U, S, dt = fresh()
    p.cfl_dt(U, 0.4, dt)
    t = 0.0
    for _ in range(n1):
        t += dt.item()
        p.rk3_step(U, S, dt_dev=dt)
    f = tmp_path / "run.ckpt"
    checkpoint.save(f, p, U, S, t=t, step=n1, dt_dev=dt)
    del p, U, S, dt
    p2, U2, S2, dt2 = fresh()
    U2.zero_()
    t2, step, _ = checkpoint.load(f, p2, U2, S2, dt_dev=dt2)
    assert step == n1 and t2 == t
    for _ in range(n2):
        p2.rk3_step(U2, S2, dt_dev=dt2)
    torch.cuda.synchronize()
    assert torch.equal(U2, ref), float((U2.double() - ref.double()).abs().max())
    assert torch.equal(S2[3], ref_lo)
    assert dt2.item() == ref_dt
    assert p2.flags() == 0
    assert np.isfinite(U2.double().cpu().numpy()).all()
