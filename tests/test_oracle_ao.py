"""Pins for the oracle's GP-AO (Appendix A): AO(2,3) at R = 2 and the recursive
AO(3,2,3) at R = 3, hybridising the high-order GP prediction (Eq. q-intrp) with
the GP-CWENO combination of the three 3-point stencils (Eqs. cweno_stencil,
CWENO, nonlin-AO, CWENO-lin, GP-AO, recursive-weights, AO-recursive).

The pins use properties the construction must have, not its formulas: with all
nonlinear weights equal (a huge epsilon) AO returns the high-order GP prediction;
its coefficients sum to one (quadratics are reproduced in the flat-kernel limit);
at a jump it takes the smooth small stencils; and the whole scheme keeps the
invariants of the others.  The paper states that AO keeps the high order in smooth
flow because the indicators of all stencils are then nearly equal.  With the bare
data-fit term 1/2 f^T K_N^-1 f they are not (its value on constant data, 1^T K_N^-1 1,
grows with the stencil size N), and the hybrid keeps an O(1) share of the third-order
CWENO part (order ~3.4); dividing each by 1^T K_N^-1 1 makes them agree up to O(dx)
and the order rises above 4.3 (the order tests)."""
import math

import numpy as np
import pytest

import oracle
from oracle import gp_tables as G
from paper_1808_04960_gb300 import workloads as W


def _o(R, **kw):
    return oracle.Oracle((16,), (0.1,), (("periodic", "periodic"),), R=R, ao=True, **kw)


@pytest.mark.parametrize("R", [2, 3])
def test_ao_equal_weights_give_the_high_order_prediction(R):
    """epsilon >> beta makes every (eps + beta)^-p equal: omega^R = gamma_HI, omega_m = gamma_m,
    nu^R' = gamma_HI, so AO(R,3) and AO(R',R,3) return q^R = w . f of the full stencil."""
    rng = np.random.default_rng(R)
    o = _o(R, eps=1e30)
    for right, xs in ((False, 0.5), (True, -0.5)):
        wb = G.tables(R, 12.0, 3.0, xs)["w_big"]
        for _ in range(5):
            f = rng.uniform(-1, 1, 2 * R + 1)
            assert abs(o.gp_weno(f, right=right) - wb @ f) < 1e-13


@pytest.mark.parametrize("R", [2, 3])
@pytest.mark.parametrize("ao_beta", ["normalized", "datafit", "loglik"])
def test_ao_coefficients_sum_to_one(R, ao_beta):
    """Quadratic data in the flat-kernel limit: every candidate is (nearly) exact, so any
    combination whose coefficients sum to one returns the exact face value."""
    o = oracle.Oracle((16,), (0.1,), (("periodic", "periodic"),), R=R, ell_over_dx=1000.0, ao=True, ao_beta=ao_beta)
    x = np.arange(-R, R + 1, dtype=float)
    for a, b, cc in ((1.0, 0.3, -0.2), (2.0, -1.0, 0.5), (-0.5, 0.0, 1.0)):
        f = a + b * x + cc * x * x
        assert abs(o.gp_weno(f) - (a + 0.5 * b + 0.25 * cc)) < 1e-5
        assert abs(o.gp_weno(f, right=True) - (a - 0.5 * b + 0.25 * cc)) < 1e-5


def test_ao_takes_the_smooth_small_stencils_at_a_jump():
    """A jump inside S_R (and S_3) but not inside S_1, S_2 (or S_R-1 for the recursion): the
    prediction comes from the flat data (zero-mean beta is exactly 0 there)."""
    o2 = _o(2)
    assert abs(o2.gp_weno(np.array([0, 0, 0, 0, 1.0]))) < 1e-12
    o3 = _o(3)
    assert abs(o3.gp_weno(np.array([0, 0, 0, 0, 0, 0, 1.0]))) < 1e-12
    assert abs(o3.gp_weno(np.array([1.0, 0, 0, 0, 0, 0, 0]), right=True)) < 1e-12


def _gauss_err(n, R, **kw):
    Ug, m = W.gaussian_1d(n)
    oo = oracle.Oracle((n,), m["dx"], m["bc"], R=R, ell_over_dx=0.1 * n, gamma=m["gamma"], ao=True, **kw)
    dx = m["dx"][0]
    dt = 0.4 * dx / 2.3 * (dx / (1.0 / 25)) ** ((2 * R + 1) / 3.0 - 1.0)
    steps = int(math.ceil(1.0 / dt))
    Un = oo.run(Ug, 1.0 / steps, steps)
    Ue, _ = W.gaussian_1d(n, t=1.0)
    return np.abs(Un[0] - Ue[0]).mean()


@pytest.mark.parametrize("R", [2, 3])
def test_ao_smooth_order(R):
    """Smooth advection (Section 6.1 set-up), 100 -> 200 cells: with the size-normalised
    indicators AO(2,3) and AO(3,2,3) converge at order > 4.3 (measured 4.60 and 4.77, and 4.44
    and 4.75 from 200 to 400 cells); with the bare data-fit term only at the third order of the
    CWENO part (measured 3.38 and 3.39), and the normalised errors are several times smaller."""
    e = [_gauss_err(n, R) for n in (100, 200)]
    assert math.log2(e[0] / e[1]) > 4.3, e
    d = [_gauss_err(n, R, ao_beta="datafit") for n in (100, 200)]
    assert 3.0 < math.log2(d[0] / d[1]) < 3.8, d
    assert e[1] < 0.25 * d[1]


def test_ao_normalised_indicators_agree_on_constant_data():
    """The normalisation makes beta of every stencil size equal on constant data: c^2 / 2."""
    import numpy as np
    for R in (2, 3):
        o = _o(R, eps=1e-36)
        t = G.ao_tables(R, 12.0, 3.0, 0.5)
        for k in ("hi", "3") + (("lo",) if R == 3 else ()):
            K = t["Kinv_" + k]
            one = np.ones(K.shape[0])
            assert abs(0.5 * (2.0 * one) @ K @ (2.0 * one) / (one @ K @ one) - 2.0) < 1e-12
        # equal indicators everywhere: AO returns the high-order prediction on constant data
        f = np.full(2 * R + 1, 1.7)
        assert abs(o.gp_weno(f) - 1.7 * G.ao_tables(R, 12.0, 3.0, 0.5)["w_hi"].sum()) < 1e-12


def test_ao_scheme_invariants_and_sod():
    U = np.empty((4, 9, 14))
    for a, v in enumerate((1.3, 0.4, -0.2, 3.1)):
        U[a] = v
    o = oracle.Oracle((9, 14), (0.1, 0.1), (("outflow", "outflow"),) * 2, R=3, ao=True)
    assert np.abs(o.rhs(U)).max() == 0.0
    U1, m = W.smooth_field((20, 24), seed=3)
    o = oracle.Oracle(U1.shape[1:], m["dx"], m["bc"], R=3, ao=True)
    r = o.rhs(U1)
    assert np.abs(r.sum(axis=(1, 2))).max() < 1e-12 * np.abs(r).max() * r[0].size
    U2, m = W.four_quadrant(24, seed=3, ny=20)
    o = oracle.Oracle(U2.shape[1:], m["dx"], m["bc"], R=2, ao=True)
    Um = U2[:, :, ::-1].copy()
    Um[1] = -Um[1]
    r, rm = o.rhs(U2), o.rhs(Um)
    rm = rm[:, :, ::-1]
    rm[1] = -rm[1]
    np.testing.assert_allclose(rm, r, rtol=0, atol=1e-12 * np.abs(r).max())
    U, meta = W.sod_1d(256)
    o = oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=3, ao=True)
    dt = 0.4 / o.max_rate(U)
    steps = int(math.ceil(0.2 / dt))
    out = o.run(U, 0.2 / steps, steps)
    x = meta["x"]
    assert abs(out[0][np.argmin(np.abs(x - 0.6))] - 0.4263) < 0.02
    assert abs(out[0][np.argmin(np.abs(x - 0.8))] - 0.2656) < 0.02
