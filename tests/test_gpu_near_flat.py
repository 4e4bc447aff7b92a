"""FP32 where the smoothness indicators are tiny and nearly equal: a constant state
carrying a density step of 1e-6 (about eight FP32 ulps of the density) and a smooth
ripple of the same size.  Windows away from the step hold beta ~ (1e-6)^2 (dx k)^2 that
differ in their last digits, the windows across the step a larger beta of the same
tiny scale, so FP32 rounding of beta would decide the nonlinear weights -- the case a
compensated evaluation of beta exists for.  The kernel forms every window from
cell-relative differences d_j = L (V_j - V_s), taken from exact conserved differences,
so beta keeps its relative accuracy at any scale of the variation; the FP32 RHS must
follow the FP64 oracle on the same (FP32-representable) data to a small fraction of
the RHS itself."""
import numpy as np
import pytest

import oracle
from paper_1808_04960_gb300 import gpweno
from paper_1808_04960_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_04960_gb300 import build
    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def near_flat(shape, amp=1e-6, seed=0):
    """rho = 1 + amp (step at the middle of x) + amp/2 sin(2 pi (x + 0.3 y)), u = 0.4, v = -0.2,
    p = 1, then rounded to FP32 (the oracle gets exactly the FP32 data)."""
    ny, nx = shape
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    rho = 1.0 + amp * (X > 0.5) + 0.5 * amp * np.sin(2 * np.pi * (X + 0.3 * Y))
    U = W.conserved(rho, [0.4 * np.ones_like(X), -0.2 * np.ones_like(X)], np.ones_like(X), 1.4)
    U = U.astype(np.float32).astype(np.float64)
    meta = dict(dx=(1.0 / nx, 1.0 / ny), bc=(("periodic", "periodic"), ("periodic", "periodic")), gamma=1.4)
    return np.ascontiguousarray(U), meta


@pytest.mark.parametrize("R", [1, 2, 3])
@pytest.mark.parametrize("amp", [1e-6, 1e-5])
def test_near_flat_f32_rhs_follows_oracle(R, amp):
    import torch
    U, meta = near_flat((40, 130), amp=amp)
    ref = oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=R).rhs(U)
    plan = gpweno.Plan(R, 12.0, U.shape[1:], meta["dx"], meta["bc"], dtype="f32")
    got = plan.rhs(torch.from_numpy(U).to("cuda", torch.float32).contiguous()).double().cpu().numpy()
    assert plan.flags() == 0
    scale = np.abs(ref).max()
    err = np.abs(got - ref)
    print(f"\nNEARFLAT R={R} amp={amp:g} max|L|={scale:.3e} linf/max={err.max() / scale:.3e} "
          f"l1/max={err.mean() / scale:.3e}")
    # relative to the RHS that the 1e-6 variation produces (not to the O(1) state)
    assert err.max() <= 2e-3 * scale and err.mean() <= 2e-4 * scale, (err.max() / scale, err.mean() / scale)


def test_near_flat_f32_steps_follow_oracle():
    """Ten FP32 steps on the near-flat data stay within two FP32 ulps of the density (the
    storage limit of an FP32 state: the 1e-6 variation is only about eight ulps) of the FP64
    oracle's steps."""
    import torch
    U, meta = near_flat((40, 130), amp=1e-6)
    o = oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=2)
    dt = 0.4 / o.max_rate(U)
    ref = o.run(U, dt, 10)
    plan = gpweno.Plan(2, 12.0, U.shape[1:], meta["dx"], meta["bc"], dtype="f32")
    Ud = torch.from_numpy(U).to("cuda", torch.float32).contiguous()
    s = plan.new_scratch()
    for _ in range(10):
        plan.rk3_step(Ud, s, dt=dt)
    got = Ud.double().cpu().numpy()
    var = np.abs(ref[0] - ref[0].mean()).max()          # the size of the density variation
    err = np.abs(got[0] - ref[0])
    print(f"\nNEARFLAT steps variation={var:.3e} linf={err.max():.3e} ({err.max() / var:.3e} of it)")
    assert err.max() <= 2.0 * 2.0 ** -23 * np.abs(ref[0]).max()
