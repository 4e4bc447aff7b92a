"""3D path (xy-plane kernel + z-marching kernel per stage) against the FP64
oracle on small grids with a ragged tail in every direction."""
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


def smooth_3d(shape, seed=0):
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*[(np.arange(n) + 0.5) / n for n in shape], indexing="ij")
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * (x + 2 * y)) * np.cos(2 * np.pi * z) + 0.01 * rng.standard_normal(x.shape)
    u = 0.3 + 0.1 * np.cos(2 * np.pi * y)
    v = -0.2 + 0.1 * np.sin(2 * np.pi * z)
    w = 0.1 * np.cos(2 * np.pi * x)
    p = 1.0 + 0.1 * np.sin(2 * np.pi * (x - z))
    U = W.conserved(rho, [u, v, w], p, 1.4)
    meta = dict(dx=(1.0 / nx, 1.0 / ny, 1.0 / nz), bc=(("periodic", "periodic"),) * 3, gamma=1.4)
    return U, meta


def run_gpu(U, meta, R, dtype="f64", dt=None, steps=0):
    import torch
    plan = gpweno.Plan(R, 12.0, U.shape[1:], meta["dx"], meta["bc"], gamma=meta["gamma"], dtype=dtype)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    Ud = torch.from_numpy(U).to("cuda", tdt).contiguous()
    if steps == 0:
        out = plan.rhs(Ud).double().cpu().numpy()
    else:
        s = plan.new_scratch()
        for _ in range(steps):
            plan.rk3_step(Ud, s, dt=dt)
        out = Ud.double().cpu().numpy()
    assert plan.flags() == 0
    return out


@pytest.mark.parametrize("R", [1, 2, 3])
def test_rhs_3d_smooth(R):
    U, meta = smooth_3d((13, 17, 22), seed=R)
    ref = oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=R).rhs(U)
    out = run_gpu(U, meta, R)
    assert np.abs(out - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max())


def test_rhs_3d_shock_turbulence():
    U, meta = W.shock_turbulence_3d(24, seed=4)
    ref = oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=3).rhs(U)
    out = run_gpu(U, meta, 3)
    assert np.abs(out - ref).mean() <= 1e-9
    assert np.abs(out - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("shape", [(4, 5, 6), (1, 9, 300), (30, 3, 7), (9, 1, 1)])
def test_rhs_3d_edge_shapes(shape):
    U, meta = smooth_3d(shape, seed=7)
    for bc in ("periodic", "outflow"):
        m = dict(meta)
        m["bc"] = ((bc, bc),) * 3
        ref = oracle.Oracle(U.shape[1:], m["dx"], m["bc"], R=2).rhs(U)
        out = run_gpu(U, m, 2)
        assert np.abs(out - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max()), bc


def test_rk3_3d_steps():
    U, meta = W.shock_turbulence_3d(20, seed=4)
    o = oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=3)
    dt = 0.4 / o.max_rate(U)
    ref = o.run(U, dt, 3)
    out = run_gpu(U, meta, 3, dt=dt, steps=3)
    assert np.abs(out - ref).mean() <= 1e-9


def test_axis_permutation_3d():
    """Relabelling x <-> z (with u <-> w) permutes the result exactly (same face code per axis)."""
    U, meta = smooth_3d((12, 12, 12), seed=3)
    meta["dx"] = (1 / 12, 1 / 12, 1 / 12)
    Ut = np.stack([U[0].transpose(2, 1, 0), U[3].transpose(2, 1, 0), U[2].transpose(2, 1, 0),
                   U[1].transpose(2, 1, 0), U[4].transpose(2, 1, 0)]).copy()
    for dtype in ("f64", "f32"):
        L = run_gpu(U, meta, 2, dtype)
        Lt = run_gpu(Ut, meta, 2, dtype)
        back = np.stack([Lt[0].transpose(2, 1, 0), Lt[3].transpose(2, 1, 0), Lt[2].transpose(2, 1, 0),
                         Lt[1].transpose(2, 1, 0), Lt[4].transpose(2, 1, 0)])
        tol = 1e-13 if dtype == "f64" else 1e-5
        assert np.abs(back - L).max() <= tol * max(1.0, np.abs(L).max()), dtype
