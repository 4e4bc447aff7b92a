"""Slab decomposition through the C ABI on one GPU: the grid is cut into slabs along its
slowest axis, each slab has its own plan with GPWENO_BC_EXTERNAL cut sides, and before
every stage each slab packs its G = R+3 boundary layers (gpweno_halo_pack) and the
neighbours' layers are copied into its halo buffers (here by device copies; across GPUs
by NCCL, see decomp.halo_exchange).  The slabs put back together must equal the
single-domain step bitwise -- every face sees the same stencil values -- including the
CFL time step from the max-reduced rate maxima."""
import numpy as np
import pytest

from paper_1808_04960_gb300 import decomp, gpweno
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


def _case(name):
    if name == "vortex2d":
        return W.isentropic_vortex(200, ny=157), 2
    if name == "quadrant2d":
        return W.four_quadrant(150, seed=3, ny=131), 2
    if name == "vortex2d_r3":
        return W.isentropic_vortex(96, ny=70), 3
    if name == "sod1d":
        return W.sod_1d(301), 2
    if name == "shock3d":
        return W.shock_turbulence_3d(24, seed=4), 3
    raise KeyError(name)


def _run(name, dtype, world, steps=3, cfl=0.4):
    import torch
    (U0, meta), R = _case(name)
    G = R + 3
    tdt = torch.float32 if dtype == "f32" else torch.float64
    shape = U0.shape[1:]
    # single domain, device CFL dt
    ref_plan = gpweno.Plan(R, 12.0, shape, meta["dx"], meta["bc"], dtype=dtype, cfl=cfl)
    Uref = torch.from_numpy(U0).to("cuda", tdt).contiguous()
    sref = ref_plan.new_scratch()
    dref = torch.zeros(1, dtype=torch.float64, device="cuda")
    ref_plan.cfl_dt(Uref, cfl, dref)
    dts_ref = []
    for _ in range(steps):
        dts_ref.append(float(dref.item()))
        ref_plan.rk3_step(Uref, sref, dt_dev=dref)
    # slabs
    slabs = [decomp.Slab(shape, meta["bc"], r, world, G) for r in range(world)]
    plans = [gpweno.Plan(R, 12.0, s.local_shape, meta["dx"], s.local_bc, dtype=dtype, cfl=cfl) for s in slabs]
    steppers = [decomp.SlabStepper(p, s, exchange=lambda *a: None) for p, s in zip(plans, slabs)]
    Us = [torch.from_numpy(np.ascontiguousarray(U0[(slice(None), s.rows)])).to("cuda", tdt).contiguous()
          for s in slabs]
    dts = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in slabs]
    rates = [torch.zeros(3, dtype=torch.int64, device="cuda") for _ in slabs]

    def common_dt():
        for p, r in zip(plans, rates):
            p.rate_export(r)
        m = torch.stack(rates).max(dim=0).values   # the max-reduction across ranks
        for p, d in zip(plans, dts):
            p.dt_from_rates(m, cfl, d)

    for p, U in zip(plans, Us):
        p.rates(U)
    common_dt()
    for _ in range(steps):
        for k in range(3):
            for st, U in zip(steppers, Us):
                st.pack(k, U)
            for r, (st, s) in enumerate(zip(steppers, slabs)):
                if s.lo_rank is not None:
                    st.recv[0].copy_(steppers[s.lo_rank].send[1])
                if s.hi_rank is not None:
                    st.recv[1].copy_(steppers[s.hi_rank].send[0])
            for st, U, d in zip(steppers, Us, dts):
                st.stage(k, U, dt_dev=d)
        common_dt()
    torch.cuda.synchronize()
    got = torch.cat(Us, dim=1)
    assert all(p.flags() == 0 for p in plans)
    return got, Uref, [float(d.item()) for d in dts], float(dref.item())


@pytest.mark.parametrize("name,world", [("vortex2d", 2), ("vortex2d", 3), ("quadrant2d", 2), ("vortex2d_r3", 3),
                                        ("sod1d", 2), ("shock3d", 2)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_slabs_bitwise_equal_single_domain(name, world, dtype):
    import torch
    got, ref, dts, dref = _run(name, dtype, world)
    assert torch.equal(got, ref), float((got.double() - ref.double()).abs().max())
    assert all(d == dref for d in dts)


def test_external_side_needs_halo_and_stage_stepping():
    import torch
    U0, meta = W.isentropic_vortex(64, ny=40)
    s = decomp.Slab(U0.shape[1:], meta["bc"], 0, 2, 5)
    p = gpweno.Plan(2, 12.0, s.local_shape, meta["dx"], s.local_bc, dtype="f32")
    U = torch.from_numpy(np.ascontiguousarray(U0[:, s.rows])).to("cuda", torch.float32).contiguous()
    scratch = p.new_scratch()
    with pytest.raises(gpweno.GpwenoError):
        p.rk3_stage(0, U, scratch, dt=1e-3)            # no halo registered yet
    with pytest.raises(gpweno.GpwenoError):
        p.rk3_step(U, scratch, dt=1e-3)                # whole steps need the exchange between stages
    with pytest.raises(gpweno.GpwenoError):
        gpweno.Plan(2, 12.0, (4, 64), meta["dx"], (("periodic", "periodic"), ("external", "external")))
    with pytest.raises(gpweno.GpwenoError):          # external sides on a dimension other than the slowest
        gpweno.Plan(2, 12.0, (40, 64), meta["dx"], (("external", "outflow"), ("outflow", "outflow")))
