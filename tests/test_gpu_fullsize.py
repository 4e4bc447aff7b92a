"""Parity at the configured full sizes, in the launch configuration bench.py
times (one SSP-RK3 step through the same plans, CUDA graph, device CFL dt):
the FP64 oracle recomputes sampled blocks one by one.

One RK3 step reads at most 3 (R+3) cells away in each direction, so the
oracle runs each block on a window with that margin: periodic dimensions are
cut out by wrapping, other dimensions are clipped at the domain edge (where the
oracle applies the true boundary condition) and, when clipped, the cut edge is
farther from the block than one step can see."""
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


def window(U, meta, lo, hi, margin):
    """Cut the window [lo-margin, hi+margin) per array axis; return it, the block's offset inside
    it, and the window's boundary conditions in (x, y, z) order."""
    nd = U.ndim - 1
    idx, off, bcs = [], [], []
    for ax in range(nd):
        n = U.shape[1 + ax]
        d = nd - 1 - ax                       # array axis -> (x, y, z) index
        per = meta["bc"][d][0] == "periodic"
        if per:
            r = np.arange(lo[ax] - margin, hi[ax] + margin) % n
            off.append(margin)
            bcs.append(("outflow", "outflow"))
        else:
            a, b = max(0, lo[ax] - margin), min(n, hi[ax] + margin)
            r = np.arange(a, b)
            off.append(lo[ax] - a)
            bcs.append(meta["bc"][d])
        idx.append(r)
    Wd = U[(slice(None),) + np.ix_(*idx)]
    return np.ascontiguousarray(Wd), off, tuple(reversed(bcs))


def sampled_parity(U0, meta, R, out, dt, blocks, size, ell=12.0):
    """Max abs and mean abs difference of `out` against the oracle on the sampled blocks."""
    margin = 3 * (R + 3)
    errs, means = [], []
    for lo in blocks:
        hi = [l + size for l in lo]
        Wd, off, bcs = window(U0, meta, lo, hi, margin)
        o = oracle.Oracle(Wd.shape[1:], meta["dx"], bcs, R=R, ell_over_dx=ell, gamma=meta["gamma"])
        ref = o.rk3_step(Wd, dt)
        sl = (slice(None),) + tuple(slice(o_, o_ + size) for o_ in off)
        got = out[(slice(None),) + tuple(slice(l, l + size) for l in lo)]
        d = np.abs(got - ref[sl])
        errs.append(d.max())
        means.append(d.mean())
    return max(errs), float(np.mean(means))


def gpu_step(U0, meta, R, dtype, cfl=0.4):
    import torch
    plan = gpweno.Plan(R, 12.0, U0.shape[1:], meta["dx"], meta["bc"], gamma=meta["gamma"], dtype=dtype, cfl=cfl)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    U = torch.from_numpy(U0).to("cuda", tdt).contiguous()
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    plan.cfl_dt(U, cfl, dt_dev)
    dt = float(dt_dev.item())
    s = plan.new_scratch()
    g = torch.cuda.CUDAGraph()
    Uw = U.clone()
    plan.rk3_step(Uw, s.clone(), dt_dev=dt_dev.clone())   # warm-up outside the capture
    with torch.cuda.graph(g):
        plan.rk3_step(U, s, dt_dev=dt_dev)
    g.replay()
    torch.cuda.synchronize()
    assert plan.flags() == 0
    return U.double().cpu().numpy(), dt, float(dt_dev.item())


def report(name, dtype, emax, emean):
    """Measured errors on one line (shown with pytest -s), for the record beside the bounds."""
    print(f"\nFULLSIZE {name} {dtype} linf={emax:.3e} l1={emean:.3e}")


def test_vortex_1024_full_size():
    """Smooth run: FP64 within 1e-10 L-inf of the oracle; FP32 within 1e-5 L1 and 8e-6 L-inf."""
    U0, meta = W.isentropic_vortex(1024)
    blocks = [(0, 0), (500, 500), (512, 100), (1000, 1008), (250, 760)]
    for dtype, tol_max, tol_mean in (("f64", 1e-10, 1e-10), ("f32", 8e-6, 1e-5)):
        out, dt, _ = gpu_step(U0, meta, 2, dtype)
        emax, emean = sampled_parity(U0, meta, 2, out, dt, blocks, 16)
        report("vortex1024", dtype, emax, emean)
        assert emax <= tol_max and emean <= tol_mean, (dtype, emax, emean)


def test_four_quadrant_4096_full_size():
    U0, meta = W.four_quadrant(4096, seed=3)
    # interfaces at x, y = 0.5 (cell 2048), their crossing, the outflow edges and corners
    blocks = [(2040, 2040), (0, 0), (4080, 4080), (2040, 0), (0, 2040), (4080, 2040), (1000, 2040), (2040, 3000),
              (1500, 700)]
    for dtype, tol_max, tol_mean in (("f64", 1e-9, 1e-9), ("f32", 2e-4, 1e-6)):
        out, dt, dt_next = gpu_step(U0, meta, 2, dtype)
        emax, emean = sampled_parity(U0, meta, 2, out, dt, blocks, 16)
        report("four_quadrant4096", dtype, emax, emean)
        assert emean <= tol_mean and emax <= tol_max, (dtype, emax, emean)
        assert dt_next > 0


def test_shock_turbulence_512_full_size():
    U0, meta = W.shock_turbulence_3d(512, seed=4)
    blocks = [(0, 0, 120), (200, 300, 125), (511 - 8, 511 - 8, 511 - 8), (100, 7, 300), (256, 256, 0)]
    for dtype, tol_mean in (("f32", 1e-5),):
        out, dt, _ = gpu_step(U0, meta, 3, dtype)
        emax, emean = sampled_parity(U0, meta, 3, out, dt, blocks, 8)
        report("shock_turbulence512", dtype, emax, emean)
        assert emean <= tol_mean, (dtype, emax, emean)
