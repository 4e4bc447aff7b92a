"""Bounds-checked build of the stage kernels (-DGPWENO_CHECKED): every shared-memory and
global access is checked against its array's extent before it is made, and a violation sets
bit `site` (1-11, see CheckSite in csrc/stage.cuh) of the plan's flag word and skips the access.
A child process loads libgpweno_checked.so and steps small ragged cases through every kernel
(1D, 2D R = 1..3, the 3D plane and z kernels, the scheme variants, the batch kernel and the slab
loaders with external halo buffers, FP32 and FP64).  No case may record a violation, and every
result must equal, bit for bit, the default library's result in this process: the checks take
nothing away and add no arithmetic."""
import hashlib
import json
import os
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SITE_MASK = ~1   # bit 0 is the non-physical-state flag


def _digest(t):
    return hashlib.sha1(t.detach().cpu().contiguous().numpy().tobytes()).hexdigest()[:16]


def run_cases():
    """Every case: {name: [digest of the result, flag word]}.  Uses whichever library
    gpweno.load() has loaded in this process."""
    import torch

    from paper_1808_04960_gb300 import decomp, gpweno
    from paper_1808_04960_gb300 import workloads as W
    torch.cuda.set_device(0)
    out = {}

    def single(name, U0, meta, R, dtype, steps=2, **opts):
        tdt = torch.float32 if dtype == "f32" else torch.float64
        p = gpweno.Plan(R, 12.0, U0.shape[1:], meta["dx"], meta["bc"], dtype=dtype, **opts)
        U = torch.from_numpy(U0).to("cuda", tdt).contiguous()
        L = p.rhs(U)
        S = p.new_scratch()
        dt = 0.025 * min(meta["dx"])
        for _ in range(steps):
            p.rk3_step(U, S, dt=dt)
        torch.cuda.synchronize()
        out[name] = [_digest(L) + _digest(U), p.flags()]

    for dtype in ("f32", "f64"):
        for R in (1, 2, 3):
            U0, meta = W.isentropic_vortex(53, ny=37)
            single(f"vortex2d_R{R}_{dtype}", U0, meta, R, dtype)
        U0, meta = W.four_quadrant(131, seed=3, ny=45)                 # two strips in FP32
        single(f"quadrant2d_{dtype}", U0, meta, 2, dtype)
        U0, meta = W.four_quadrant(260, seed=3, ny=19)                 # three strips, short segments
        single(f"quadrant2d_wide_{dtype}", U0, meta, 3, dtype)
        U0, meta = W.sod_1d(150)
        single(f"sod1d_{dtype}", U0, meta, 2, dtype)
        U0, meta = W.shock_turbulence_3d(20, seed=4)
        single(f"shock3d_{dtype}", U0, meta, 3, dtype, steps=1)
    U0, meta = W.four_quadrant(70, seed=3, ny=41)
    for vname, opts in (("fdflux", {"scheme": "fdflux"}), ("ao", {"ao": True}), ("mean", {"beta_mean": True}),
                        ("hllc", {"flux": "hllc"}), ("hll", {"flux": "hll"}), ("poly", {"candidates": "poly"})):
        single(f"variant_{vname}_f32", U0, meta, 2, "f32", **opts)

    # batch kernel
    rng = np.random.default_rng(7)
    plans, Us, Ss, dts = [], [], [], []
    for k in range(7):
        nx, ny, R = int(rng.integers(9, 200)), int(rng.integers(9, 90)), int(rng.integers(1, 4))
        U0, meta = (W.four_quadrant(nx, seed=k, ny=ny) if k % 2 else W.isentropic_vortex(nx, ny=ny))
        p = gpweno.Plan(R, 12.0, U0.shape[1:], meta["dx"], meta["bc"], dtype="f32")
        plans.append(p)
        Us.append(torch.from_numpy(U0).to("cuda", torch.float32).contiguous())
        Ss.append(p.new_scratch())
        dts.append(0.025 * min(meta["dx"]))
    batch = gpweno.BatchPlan(plans)
    dt_dev = torch.tensor(dts, dtype=torch.float64, device="cuda")
    for _ in range(2):
        batch.rk3_step(Us, Ss, dt_dev)
    torch.cuda.synchronize()
    out["batch_f32"] = ["".join(_digest(u) for u in Us), batch.flags()]

    # slabs with external halo buffers (the kVarSlab loaders), exchanged by device copies
    for name, (U0, meta), R in (("slabs2d", W.isentropic_vortex(60, ny=40), 2),
                                ("slabs3d", W.shock_turbulence_3d(18, seed=4), 1),
                                ("slabs1d", W.sod_1d(90), 2)):
        world = 2
        slabs = [decomp.Slab(U0.shape[1:], meta["bc"], r, world, R + 3) for r in range(world)]
        sp = [gpweno.Plan(R, 12.0, s.local_shape, meta["dx"], s.local_bc, dtype="f32") for s in slabs]
        steppers = [decomp.SlabStepper(p, s, exchange=lambda *a: None) for p, s in zip(sp, slabs)]
        Ul = [torch.from_numpy(np.ascontiguousarray(U0[:, s.rows])).to("cuda", torch.float32).contiguous()
              for s in slabs]
        dt = 0.025 * min(meta["dx"])
        for _ in range(2):
            for k in range(3):
                for st, U in zip(steppers, Ul):
                    st.pack(k, U)
                for st, s in zip(steppers, slabs):
                    if s.lo_rank is not None:
                        st.recv[0].copy_(steppers[s.lo_rank].send[1])
                    if s.hi_rank is not None:
                        st.recv[1].copy_(steppers[s.hi_rank].send[0])
                for st, U in zip(steppers, Ul):
                    st.stage(k, U, dt=dt)
        torch.cuda.synchronize()
        out[f"{name}_f32"] = ["".join(_digest(u) for u in Ul), max(p.flags() for p in sp)]
    return out


pytestmark = pytest.mark.gpu


def test_checked_build_records_no_violation_and_changes_no_bit():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_04960_gb300 import build, gpweno
    build.build()
    checked = build.build(checked=True)
    child = subprocess.run([sys.executable, os.path.abspath(__file__), checked], capture_output=True, text=True,
                           timeout=900, cwd=ROOT)
    assert child.returncode == 0, child.stdout[-2000:] + child.stderr[-4000:]
    got = json.loads(child.stdout.strip().splitlines()[-1])
    gpweno.load()
    ref = run_cases()
    assert sorted(got) == sorted(ref)
    bad = {k: v[1] for k, v in got.items() if v[1] & SITE_MASK}
    assert not bad, f"bounds violations (flag bits by site): {bad}"
    assert all(v[1] == 0 for v in got.values()), {k: v[1] for k, v in got.items() if v[1]}
    differ = [k for k in ref if ref[k][0] != got[k][0]]
    assert not differ, f"checked build changed results: {differ}"


if __name__ == "__main__":
    from paper_1808_04960_gb300 import gpweno as _g
    _g.load(sys.argv[1])
    print(json.dumps(run_cases()))
