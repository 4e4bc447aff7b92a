"""The allocation-free RK3 step (gpweno_rk3_step_noalloc) against the regular
one (gpweno_rk3_step with a caller-provided scratch buffer).

Callers that may not allocate device memory (their host application owns all
device memory through its own pool, or hands them only the state buffer) use
the variant whose stage buffers sit in the library's static 16 MiB device
array.  Both must give the same state, call after call: the static array keeps
the previous call's contents, so two calls in a row are checked.  Collected
last (file name) so that a run stopping at the first failure has run every
other test first."""
import numpy as np
import pytest

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
    torch.cuda.set_device(0)


@pytest.mark.parametrize("dtype,shape,tol,R", [("f64", (96, 130), 1e-10, 2), ("f32", (256, 300), 1e-6, 2),
                                               ("f64", (300,), 1e-10, 2), ("f32", (32, 32, 32), 1e-6, 3),
                                               ("f64", (30, 34, 36), 1e-10, 3)])
def test_noalloc_matches_scratch_step(dtype, shape, tol, R):
    """Two calls in a row of each step agree; in 3D the x+y part of L passes through the
    static array's first two stage slots in turn (V1, V2, V1), so 3D is checked too."""
    import torch
    if len(shape) == 1:
        U0, meta = W.sod_1d(shape[0])
    elif len(shape) == 3:
        U0, meta = W.shock_turbulence_3d(shape[2], seed=4)
        if U0.shape[1:] != shape:   # a ragged box: a window of the cubic one (same spacing)
            U0 = np.ascontiguousarray(U0[:, :shape[0], :shape[1], :shape[2]])
    else:
        U0, meta = W.four_quadrant(shape[1], seed=3, ny=shape[0])
    plan = gpweno.Plan(R, 12.0, U0.shape[1:], meta["dx"], meta["bc"], dtype=dtype)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    Ua = torch.from_numpy(U0).to("cuda", tdt).contiguous()
    Ub = Ua.clone()
    scratch = torch.zeros((4,) + tuple(Ua.shape), dtype=tdt, device="cuda")
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    plan.cfl_dt(Ua, 0.4, dt_dev)                     # CFL 0.4 of the initial state
    dt = float(dt_dev.item())
    for call in range(2):
        plan.rk3_step(Ua, scratch, dt=dt)
        plan.rk3_step_noalloc(Ub, dt)
        # this call's stage launches only (3D: a plane and a z-marching launch per stage)
        assert gpweno.last_launch_count() == 3 * (2 if len(shape) == 3 else 1)
        torch.cuda.synchronize()
        a, b = Ua.double().cpu().numpy(), Ub.double().cpu().numpy()
        assert np.isfinite(b).all()
        assert np.abs(a - b).max() <= tol * max(1.0, np.abs(a).max()), (call, np.abs(a - b).max())
    assert plan.flags() == 0


def test_noalloc_rejects_grids_beyond_the_static_array():
    import torch
    U0, meta = W.isentropic_vortex(1024)       # 3 x 16 MiB of FP32 stages > 16 MiB
    plan = gpweno.Plan(2, 12.0, U0.shape[1:], meta["dx"], meta["bc"], dtype="f32")
    U = torch.from_numpy(U0).to("cuda", torch.float32).contiguous()
    before = U.clone()
    with pytest.raises(gpweno.GpwenoError) as e:
        plan.rk3_step_noalloc(U, 1e-4)
    assert e.value.status == gpweno.ERR_ARG
    assert "static scratch" in str(e.value)
    torch.cuda.synchronize()
    assert torch.equal(U, before)
