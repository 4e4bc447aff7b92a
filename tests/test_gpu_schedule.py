"""The 2D launch's kernel-build choice (gpweno_plan_schedule): FP32 takes the build for three
CTAs per SM where the four-CTA schedule is row-limited, and for R = 2 also where it leaves a CTA
fewer than 24 rows; everything else takes four CTAs per SM (FP64: one 256-thread CTA)."""
import pytest

from paper_1808_04960_gb300 import gpweno
from paper_1808_04960_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _schedule(n, R, dtype="f32"):
    import torch
    U0, meta = W.isentropic_vortex(n)
    p = gpweno.Plan(R, 12.0, U0.shape[1:], meta["dx"], meta["bc"], dtype=dtype)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    U = torch.from_numpy(U0).to("cuda", tdt).contiguous()
    assert p.schedule() == dict(strip_width=0, strips=0, grid=0, ctas_per_sm=0)
    p.rk3_step(U, p.new_scratch(), dt=1e-4)
    torch.cuda.synchronize()
    assert p.flags() == 0
    return p.schedule()


def _sms():
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


@pytest.mark.parametrize("n,R,ctas", [(1024, 2, 3),     # 9 strips x 1024 rows over 4 x SMs: ~15 rows per CTA
                                      (512, 2, 3),      # row-limited (fewer than 4 x SMs CTAs of >= 8 rows)
                                      (512, 1, 3),
                                      (1536, 2, 4),     # ~33 rows per CTA
                                      (1024, 1, 4),     # R = 1's four-CTA build is not register-capped
                                      (1024, 3, 4),
                                      (512, 3, 3)])     # row-limited: every radius
def test_build_choice(n, R, ctas):
    s = _schedule(n, R)
    assert s["ctas_per_sm"] == ctas
    strips = -(-n // 123)
    assert s["strips"] == strips and s["strip_width"] == -(-n // strips)
    assert s["grid"] == min(ctas * _sms(), strips * n // 8)


def test_fp64_uses_one_256_thread_cta_per_sm():
    s = _schedule(256, 2, "f64")
    assert s["ctas_per_sm"] == 1 and s["strips"] == 2 and s["strip_width"] == 128


def test_schedule_refuses_other_plans():
    U0, meta = W.sod_1d(64)
    p = gpweno.Plan(2, 12.0, U0.shape[1:], meta["dx"], meta["bc"], dtype="f32")
    with pytest.raises(gpweno.GpwenoError):
        p.schedule()
