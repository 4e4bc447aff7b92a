"""HLLC (flux_form = 1, the paper's default solver) and HLL (flux_form = 2) on the GPU
against the oracle's textbook solvers: RHS and RK3 parity in 1D, 2D and 3D,
smooth and shocked, and FP32 against FP64."""
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


def gpu(U, meta, R, dtype="f64", dt=None, steps=0):
    import torch
    plan = gpweno.Plan(R, 12.0, U.shape[1:], meta["dx"], meta["bc"], gamma=meta["gamma"], dtype=dtype, flux="hllc")
    tdt = torch.float32 if dtype == "f32" else torch.float64
    Ud = torch.from_numpy(U).to("cuda", tdt).contiguous()
    if steps == 0:
        out = plan.rhs(Ud)
    else:
        s = plan.new_scratch()
        for _ in range(steps):
            plan.rk3_step(Ud, s, dt=dt)
        out = Ud
    res = out.double().cpu().numpy()
    assert plan.flags() == 0
    return res


def orc(U, meta, R):
    return oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=R, gamma=meta["gamma"], flux="hllc")


@pytest.mark.parametrize("R", [1, 2, 3])
def test_hllc_rhs_2d_smooth(R):
    U, meta = W.isentropic_vortex(48, ny=40)
    ref = orc(U, meta, R).rhs(U)
    assert np.abs(gpu(U, meta, R) - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("R", [1, 2, 3])
def test_hllc_rhs_2d_shocked(R):
    U, meta = W.four_quadrant(64, seed=3, ny=56)
    ref = orc(U, meta, R).rhs(U)
    out = gpu(U, meta, R)
    assert np.abs(out - ref).mean() <= 1e-9
    assert np.abs(out - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())


def test_hllc_sod_1d_run():
    U, meta = W.sod_1d(256)
    o = orc(U, meta, 2)
    dt = 0.4 / o.max_rate(U)
    steps = int(math.ceil(0.2 / dt))
    dt = 0.2 / steps
    ref = o.run(U, dt, steps)
    out = gpu(U, meta, 2, dt=dt, steps=steps)
    assert np.abs(out - ref).mean() <= 1e-9
    x = meta["x"]
    assert abs(out[0][np.argmin(np.abs(x - 0.6))] - 0.4263) < 0.02
    assert abs(out[0][np.argmin(np.abs(x - 0.8))] - 0.2656) < 0.02


def test_hllc_3d_and_steps():
    U, meta = W.shock_turbulence_3d(20, seed=4)
    o = orc(U, meta, 3)
    ref = o.rhs(U)
    out = gpu(U, meta, 3)
    assert np.abs(out - ref).mean() <= 1e-9
    dt = 0.4 / o.max_rate(U)
    ref = o.run(U, dt, 2)
    out = gpu(U, meta, 3, dt=dt, steps=2)
    assert np.abs(out - ref).mean() <= 1e-9


def test_hllc_f32_vs_f64():
    U, meta = W.four_quadrant(128, seed=3)
    dt = 0.2 * meta["dx"][0]
    a = gpu(U, meta, 2, "f32", dt=dt, steps=10)
    b = gpu(U, meta, 2, "f64", dt=dt, steps=10)
    assert np.abs(a - b).mean() <= 1e-5


# ---------------------------------------------------------------------------
# HLL (flux_form = 2, the solver of the paper's Mach-3 wind-tunnel test)

def gpu_flux(U, meta, R, flux, dtype="f64", dt=None, steps=0):
    import torch
    plan = gpweno.Plan(R, 12.0, U.shape[1:], meta["dx"], meta["bc"], gamma=meta["gamma"], dtype=dtype, flux=flux)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    Ud = torch.from_numpy(U).to("cuda", tdt).contiguous()
    if steps == 0:
        out = plan.rhs(Ud)
    else:
        s = plan.new_scratch()
        for _ in range(steps):
            plan.rk3_step(Ud, s, dt=dt)
        out = Ud
    res = out.double().cpu().numpy()
    assert plan.flags() == 0
    return res


def orc_flux(U, meta, R, flux):
    return oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=R, gamma=meta["gamma"], flux=flux)


@pytest.mark.parametrize("R", [1, 2, 3])
def test_hll_rhs_2d(R):
    U, meta = W.isentropic_vortex(48, ny=40)
    ref = orc_flux(U, meta, R, "hll").rhs(U)
    assert np.abs(gpu_flux(U, meta, R, "hll") - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max())
    U, meta = W.four_quadrant(64, seed=3, ny=56)
    ref = orc_flux(U, meta, R, "hll").rhs(U)
    out = gpu_flux(U, meta, R, "hll")
    assert np.abs(out - ref).mean() <= 1e-9
    assert np.abs(out - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())


def test_hll_sod_1d_and_3d_steps():
    U, meta = W.sod_1d(256)
    o = orc_flux(U, meta, 2, "hll")
    dt = 0.4 / o.max_rate(U)
    steps = int(math.ceil(0.2 / dt))
    dt = 0.2 / steps
    ref = o.run(U, dt, steps)
    out = gpu_flux(U, meta, 2, "hll", dt=dt, steps=steps)
    assert np.abs(out - ref).mean() <= 1e-9
    U, meta = W.shock_turbulence_3d(20, seed=4)
    o = orc_flux(U, meta, 3, "hll")
    assert np.abs(gpu_flux(U, meta, 3, "hll") - o.rhs(U)).mean() <= 1e-9
    dt = 0.4 / o.max_rate(U)
    assert np.abs(gpu_flux(U, meta, 3, "hll", dt=dt, steps=2) - o.run(U, dt, 2)).mean() <= 1e-9


def test_hll_f32_vs_f64():
    U, meta = W.four_quadrant(128, seed=3)
    dt = 0.2 * meta["dx"][0]
    a = gpu_flux(U, meta, 2, "hll", "f32", dt=dt, steps=10)
    b = gpu_flux(U, meta, 2, "hll", "f64", dt=dt, steps=10)
    assert np.abs(a - b).mean() <= 1e-5
