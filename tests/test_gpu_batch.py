"""Batched persistent stepping (gpweno_plan_batch / gpweno_batch_rk3_step):
many 2D instances of uneven size, radius, length scales and boundary
conditions in one launch per RK stage.  Every face depends only on its own
stencil, so the batch must reproduce the single-instance path bit for bit,
and (FP64) the oracle to the parity tolerance."""
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


def make_instances(count, seed, nmin=16, nmax=300):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        nx = int(rng.integers(nmin, nmax))
        ny = int(rng.integers(nmin, nmax))
        R = int(rng.integers(1, 4))
        ell = float(rng.choice([6.0, 12.0, 24.0]))
        if k % 2 == 0:
            U, meta = W.four_quadrant(nx, seed=int(rng.integers(0, 1000)), ny=ny)
        else:
            U, meta = W.isentropic_vortex(nx, ny=ny, beta=float(rng.uniform(2, 6)))
        out.append((U, meta, R, ell))
    return out


def run_both(insts, dtype, steps=3, tune_cache=None):
    import torch
    tdt = torch.float32 if dtype == "f32" else torch.float64
    plans, Us, Ss, Ub, Sb, dts = [], [], [], [], [], []
    for U, meta, R, ell in insts:
        p = gpweno.Plan(R, ell, U.shape[1:], meta["dx"], meta["bc"], dtype=dtype)
        plans.append(p)
        Us.append(torch.from_numpy(U).to("cuda", tdt).contiguous())
        Ub.append(Us[-1].clone())
        Ss.append(p.new_scratch())
        Sb.append(p.new_scratch())
        dts.append(0.1 * min(meta["dx"]))
    batch = gpweno.BatchPlan(plans, tune_cache=tune_cache)
    dt_dev = torch.tensor(dts, dtype=torch.float64, device="cuda")
    for _ in range(steps):
        for p, U, S, dt in zip(plans, Us, Ss, dts):
            p.rk3_step(U, S, dt=dt)
        batch.rk3_step(Ub, Sb, dt_dev)
    assert gpweno.last_launch_count() == 3
    torch.cuda.synchronize()
    assert batch.flags() == 0
    return Us, Ub, plans, batch, dts


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_bitwise_equals_single(dtype):
    insts = make_instances(14, seed=11)
    Us, Ub, plans, batch, _ = run_both(insts, dtype)
    for k, (a, b) in enumerate(zip(Us, Ub)):
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy()), k
    info = batch.info()
    assert info["grid"] >= 1 and info["segments"] >= len(insts)
    # built-in schedule (no tuning cache): 8 CTA shares per resident slot, 8-row minimum segments
    assert info["ctas_per_slot"] == 8 and info["min_rows"] == 8


def test_batch_f64_matches_oracle():
    insts = make_instances(6, seed=5, nmin=12, nmax=80)
    Us, Ub, plans, batch, dts = run_both(insts, "f64", steps=2)
    for (U, meta, R, ell), b, dt in zip(insts, Ub, dts):
        ref = oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=R, ell_over_dx=ell).run(U, dt, 2)
        assert np.abs(b.cpu().numpy() - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max())


def test_batch_both_block_sizes(tmp_path):
    """The tuning cache forces each block size; results do not depend on it."""
    insts = make_instances(8, seed=21)
    _, ref, _, batch, _ = run_both(insts, "f32", steps=2)
    sig = batch.info()["signature"]
    for block in (128, 256):
        cache = tmp_path / f"tune{block}.txt"
        cache.write_text(f"{sig} {block} 1\n")
        _, Ub, _, b2, _ = run_both(insts, "f32", steps=2, tune_cache=str(cache))
        assert b2.info()["block"] == block and b2.info()["ctas_per_sm"] == 1
        for a, b in zip(ref, Ub):
            assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())


def test_batch_rejects_mixed_dtype():
    U, meta = W.isentropic_vortex(32)
    p1 = gpweno.Plan(2, 12.0, U.shape[1:], meta["dx"], meta["bc"], dtype="f32")
    p2 = gpweno.Plan(2, 12.0, U.shape[1:], meta["dx"], meta["bc"], dtype="f64")
    with pytest.raises(gpweno.GpwenoError):
        gpweno.BatchPlan([p1, p2])


@pytest.mark.parametrize("cand", [(128, 4, 0, 8, 1), (128, 2, 64, 24, 2), (256, 2, 96, 8, 2), (256, 1, 0, 24, 1),
                                  (128, 3, 96, 24, 1), (128, 4, 0, 16, 4), (128, 4, 64, 4, 16)])
def test_batch_tile_shapes_bitwise(tmp_path, cand):
    """Every tile shape the autotuner searches (block, CTAs per SM, strip-width cap, fewest
    segment rows, CTA shares per slot) gives the same bits: the schedule changes which CTA
    evaluates a face, never the face's arithmetic."""
    from paper_1808_04960_gb300 import autotune
    assert cand in autotune.CANDIDATES
    insts = make_instances(10, seed=31)
    _, ref, _, batch, _ = run_both(insts, "f32", steps=2)
    sig = batch.info()["signature"]
    cache = tmp_path / "tune.txt"
    cache.write_text(f"{sig} " + " ".join(str(x) for x in cand) + "\n")
    _, Ub, _, b2, _ = run_both(insts, "f32", steps=2, tune_cache=str(cache))
    info = b2.info()
    assert (info["block"], info["ctas_per_sm"], info["min_rows"], info["ctas_per_slot"]) == \
        (cand[0], cand[1], cand[3], cand[4])
    assert info["strip_width_cap"] == (cand[2] if cand[2] else cand[0] - 5)
    for a, b in zip(ref, Ub):
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
