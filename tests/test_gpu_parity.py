"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle,
element by element on the same seeded inputs.

Tolerances (from the stated targets): FP64 GPU vs oracle <= 1e-10 L-inf on
smooth data and <= 1e-9 L1 on shocked data; FP32 GPU vs FP64 oracle <= 1e-5 L1
on the smooth vortex.  Where floating point decides a branch (the max in the
Lax-Friedrichs speed, the min of the smoothness indicators) both sides run
the same formula, so only rounding separates them."""
import math

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


def to_dev(U, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(U)).to("cuda", {"f32": torch.float32, "f64": torch.float64}[dtype])


def to_np(t):
    return t.double().cpu().numpy()


def gpu_rhs(U, meta, R, dtype="f64", ell=12.0, sigma=3.0):
    plan = gpweno.Plan(R, ell, U.shape[1:], meta["dx"], meta["bc"], gamma=meta["gamma"], sigma_over_dx=sigma,
                       dtype=dtype)
    out = to_np(plan.rhs(to_dev(U, dtype)))
    assert plan.flags() == 0
    return out


def gpu_run(U, meta, R, dt, nsteps, dtype="f64", ell=12.0, sigma=3.0):
    import torch
    plan = gpweno.Plan(R, ell, U.shape[1:], meta["dx"], meta["bc"], gamma=meta["gamma"], sigma_over_dx=sigma,
                       dtype=dtype)
    Ud = to_dev(U, dtype)
    scratch = torch.zeros((4,) + tuple(Ud.shape), dtype=Ud.dtype, device="cuda")
    for _ in range(nsteps):
        plan.rk3_step(Ud, scratch, dt=dt)
    out = to_np(Ud)
    assert plan.flags() == 0
    return out


def perturbed_vortex(nx, ny, seed=0):
    U, meta = W.isentropic_vortex(nx, ny=ny)
    rng = np.random.default_rng(seed)
    U = U * (1.0 + 1e-3 * rng.standard_normal(U.shape))
    return U, meta


@pytest.mark.parametrize("R", [1, 2, 3])
@pytest.mark.parametrize("shape", [(48, 64), (37, 300), (260, 29)])
def test_rhs_f64_smooth(R, shape):
    ny, nx = shape
    U, meta = W.isentropic_vortex(nx, ny=ny)
    ref = oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=R).rhs(U)
    out = gpu_rhs(U, meta, R)
    assert np.abs(out - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("R", [1, 2, 3])
def test_rhs_f64_shocked(R):
    U, meta = W.four_quadrant(72, seed=3, ny=50)
    ref = oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=R).rhs(U)
    out = gpu_rhs(U, meta, R)
    assert np.abs(out - ref).mean() <= 1e-9
    assert np.abs(out - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("sigma", [1.5, 12.0])
def test_rhs_f64_sigma_variants(sigma):
    U, meta = perturbed_vortex(40, 33, seed=1)
    ref = oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=2, sigma_over_dx=sigma).rhs(U)
    out = gpu_rhs(U, meta, 2, sigma=sigma)
    assert np.abs(out - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("R", [1, 2, 3])
def test_rk3_f64_vortex_steps(R):
    U, meta = W.isentropic_vortex(64, ny=40)
    o = oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=R)
    dt = 0.4 / o.max_rate(U)
    ref = o.run(U, dt, 8)
    out = gpu_run(U, meta, R, dt, 8)
    assert np.abs(out - ref).max() <= 1e-10


def test_rk3_f64_four_quadrant_steps():
    U, meta = W.four_quadrant(96, seed=3, ny=80)
    o = oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=2)
    dt = 0.4 / o.max_rate(U)
    ref = o.run(U, dt, 10)
    out = gpu_run(U, meta, 2, dt, 10)
    assert np.abs(out - ref).mean() <= 1e-9


def test_sod_1d_f64_to_final_time():
    U, meta = W.sod_1d(256)
    o = oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=2)
    dt = 0.4 / o.max_rate(U)
    steps = int(math.ceil(0.2 / dt))
    dt = 0.2 / steps
    ref = o.run(U, dt, steps)
    out = gpu_run(U, meta, 2, dt, steps)
    assert np.abs(out - ref).mean() <= 1e-9
    # sanity against the exact Riemann solution: contact and shock near their positions
    rho = out[0]
    x = meta["x"]
    assert abs(rho[np.argmin(np.abs(x - 0.6))] - 0.4263) < 0.02   # between contact (0.685) and rarefaction tail
    assert abs(rho[np.argmin(np.abs(x - 0.8))] - 0.2656) < 0.02   # between contact and shock (0.850)


@pytest.mark.parametrize("R", [1, 2, 3])
def test_rhs_1d_f64(R):
    U, meta = W.sod_1d(300)
    ref = oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=R).rhs(U)
    out = gpu_rhs(U, meta, R)
    assert np.abs(out - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("shape", [(4, 4), (1, 7), (7, 1), (3, 500), (300, 2), (251, 251), (5, 252), (17, 503)])
def test_edge_shapes_f64(shape):
    """Narrow and ragged grids: fewer cells than ghost layers (periodic wrap by modulo), exactly one
    strip, one cell more than a strip, single rows and columns."""
    ny, nx = shape
    U, meta = perturbed_vortex(nx, ny, seed=ny * 1000 + nx)
    for bc in ("periodic", "outflow"):
        m = dict(meta)
        m["bc"] = ((bc, bc), (bc, bc))
        ref = oracle.Oracle(U.shape[1:], m["dx"], m["bc"], R=2).rhs(U)
        out = gpu_rhs(U, m, 2)
        assert np.abs(out - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max()), bc


@pytest.mark.parametrize("shape", [(9, 123), (6, 124), (5, 246), (4, 247), (130, 3), (3, 370)])
def test_edge_shapes_f32(shape):
    """FP32 kernels sweep the plane in strips of at most 123 columns (128-thread blocks): exactly
    one strip, one column more, two full strips, one more, and narrow grids, against the oracle
    within FP32 rounding of the RHS."""
    ny, nx = shape
    U, meta = perturbed_vortex(nx, ny, seed=ny * 1000 + nx + 7)
    for bc in ("periodic", "outflow"):
        m = dict(meta)
        m["bc"] = ((bc, bc), (bc, bc))
        ref = oracle.Oracle(U.shape[1:], m["dx"], m["bc"], R=2).rhs(U)
        out = gpu_rhs(U, m, 2, "f32")
        assert np.abs(out - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max()), bc


def test_uniform_state_zero_rhs():
    U = np.zeros((4, 33, 70))
    U[0], U[1], U[2], U[3] = 1.3, 0.4, -0.7, 3.1
    meta = dict(dx=(0.1, 0.2), bc=(("outflow", "outflow"), ("periodic", "periodic")), gamma=1.4)
    for dtype in ("f64", "f32"):
        assert np.abs(gpu_rhs(U, meta, 2, dtype)).max() == 0.0


def test_transpose_bitwise():
    U, meta = W.four_quadrant(64, seed=7, ny=64)
    Ut = np.stack([U[0].T, U[2].T, U[1].T, U[3].T])
    for dtype in ("f64", "f32"):
        L = gpu_rhs(U, meta, 2, dtype)
        Lt = gpu_rhs(Ut, meta, 2, dtype)
        back = np.stack([Lt[0].T, Lt[2].T, Lt[1].T, Lt[3].T])
        assert np.array_equal(back, L), dtype


def test_conservation_periodic_f64():
    U, meta = perturbed_vortex(96, 80, seed=3)
    L = gpu_rhs(U, meta, 2)
    assert np.abs(L.sum(axis=(1, 2))).max() < 1e-10


def test_f32_vortex_error_vs_oracle():
    """FP32 bulk arithmetic: L1 error against the FP64 oracle after 20 steps stays below 1e-5."""
    U, meta = W.isentropic_vortex(128)
    o = oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=2)
    dt = 0.4 / o.max_rate(U)
    ref = o.run(U, dt, 20)
    out = gpu_run(U, meta, 2, dt, 20, dtype="f32")
    l1 = np.abs(out - ref).mean()
    assert l1 <= 1e-5, l1
    L = gpu_rhs(U, meta, 2, "f32")
    Lr = o.rhs(U)
    assert np.abs(L - Lr).max() <= 1e-4 * np.abs(Lr).max()


def test_cfl_dt_and_fused_rate():
    import torch
    U, meta = W.four_quadrant(80, seed=3, ny=60)
    o = oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=2)
    plan = gpweno.Plan(2, 12.0, U.shape[1:], meta["dx"], meta["bc"], dtype="f64", cfl=0.4)
    Ud = to_dev(U, "f64")
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    plan.cfl_dt(Ud, 0.4, dt_dev)
    dt0 = float(dt_dev.item())
    assert abs(dt0 - o.cfl_dt(U, 0.4)) <= 1e-14 * dt0
    scratch = torch.zeros((4,) + tuple(Ud.shape), dtype=Ud.dtype, device="cuda")
    plan.rk3_step(Ud, scratch, dt_dev=dt_dev)   # uses dt0, writes the next dt
    U1 = o.rk3_step(U, dt0)
    assert np.abs(to_np(Ud) - U1).mean() <= 1e-9
    dt1 = float(dt_dev.item())
    assert abs(dt1 - o.cfl_dt(U1, 0.4)) <= 1e-12 * dt1


def test_nonphysical_flag():
    U, meta = W.four_quadrant(40, seed=3)
    U[0, 10:12, 10:12] = -1.0
    plan = gpweno.Plan(2, 12.0, U.shape[1:], meta["dx"], meta["bc"], dtype="f64")
    plan.rhs(to_dev(U, "f64"))
    assert plan.flags() == 1
    assert plan.flags() == 0   # read-and-clear


def test_launch_count():
    import torch
    U, meta = W.isentropic_vortex(32)
    plan = gpweno.Plan(2, 12.0, U.shape[1:], meta["dx"], meta["bc"], dtype="f32", cfl=0.4)
    Ud = to_dev(U, "f32")
    scratch = torch.zeros((4,) + tuple(Ud.shape), dtype=Ud.dtype, device="cuda")
    dt_dev = torch.full((1,), 0.01, dtype=torch.float64, device="cuda")
    plan.rk3_step(Ud, scratch, dt_dev=dt_dev)
    assert gpweno.last_launch_count() == 4
    plan.rk3_step(Ud, scratch, dt=0.01)
    assert gpweno.last_launch_count() == 3
