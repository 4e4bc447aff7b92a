"""Pins of the oracle's GP weight tables (Section 4, step 1) against facts
that do not depend on the oracle's own code: the flat-kernel limit that
reduces GP interpolation to Lagrange interpolation, LAPACK on well-conditioned
cases, the mirror symmetry of the prediction points, and the exactness of the
linear weights in the flat limit."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import gp_tables


def lagrange_weights(points, xs):
    """Textbook Lagrange basis l_j(x*) = prod_{k != j} (x* - x_k)/(x_j - x_k), exact rationals."""
    xs = Fraction(xs)
    out = []
    for j, xj in enumerate(points):
        v = Fraction(1)
        for k, xk in enumerate(points):
            if k != j:
                v *= (xs - xk) / Fraction(xj - xk)
        out.append(float(v))
    return np.array(out)


# classical polynomial (flat-limit) linear weights at x* = x_i + Delta/2
FLAT_GAMMA = {1: [1 / 4, 3 / 4], 2: [1 / 16, 10 / 16, 5 / 16], 3: [1 / 64, 21 / 64, 35 / 64, 7 / 64]}


@pytest.mark.parametrize("R", [1, 2, 3])
def test_flat_limit_is_lagrange(R):
    """l/Delta -> infinity: GP weights -> Lagrange weights, error O((Delta/l)^2)."""
    ell = 1.0e4
    t = gp_tables.tables(R, ell, 3.0, 0.5)
    big = lagrange_weights(list(range(-R, R + 1)), Fraction(1, 2))
    np.testing.assert_allclose(t["w_big"], big, rtol=0, atol=1e-6)
    for m in range(R + 1):
        sub = lagrange_weights(list(range(-R + m, m + 1)), Fraction(1, 2))
        np.testing.assert_allclose(t["w_sub"][m], sub, rtol=0, atol=1e-6)
    np.testing.assert_allclose(t["gamma"], FLAT_GAMMA[R], rtol=0, atol=1e-6)


@pytest.mark.parametrize("R", [1, 2, 3])
def test_flat_gamma_consistent(R):
    """In the flat limit the overdetermined system M gamma = w (Eq. gamm-system) is consistent."""
    t = gp_tables.tables(R, 1.0e4, 3.0, 0.5)
    res = t["M"] @ t["gamma"] - t["w_big"]
    assert np.abs(res).max() < 1e-6


@pytest.mark.parametrize("R,ell", [(1, 3.0), (2, 3.0), (1, 12.0)])
def test_weights_match_lapack_when_well_conditioned(R, ell):
    K = np.array([[np.exp(-(a - b) ** 2 / (2 * ell * ell)) for b in range(-R, R + 1)] for a in range(-R, R + 1)])
    ks = np.array([np.exp(-(0.5 - b) ** 2 / (2 * ell * ell)) for b in range(-R, R + 1)])
    assert np.linalg.cond(K) < 1e8
    w = np.linalg.solve(K, ks)
    t = gp_tables.tables(R, ell, 3.0, 0.5)
    np.testing.assert_allclose(t["w_big"], w, rtol=0, atol=1e-16 * np.linalg.cond(K) * 10)


@pytest.mark.parametrize("R", [1, 2, 3, 4])
@pytest.mark.parametrize("sigma", [1.5, 3.0])
def test_kinv_and_eigen_forms_agree(R, sigma):
    """beta = f^T K^-1 f (Eq. gp-smooth) equals sum (v_h . f)^2 / lambda_h (Eq. beta-eigen):
    the Gauss-elimination inverse and the Jacobi eigen-system are two independent algorithms;
    LAPACK eigh on the FP64 matrix pins the eigenvalues."""
    t = gp_tables.tables(R, 12.0, sigma, 0.5)
    lam, V = t["lam_sigma"], t["V_sigma"]
    Kinv_eig = V @ np.diag(1.0 / lam) @ V.T
    np.testing.assert_allclose(t["Kinv_sigma"], Kinv_eig, rtol=1e-12, atol=1e-12 * np.abs(Kinv_eig).max())
    K = t["K_sigma"]
    lam_lapack = np.linalg.eigvalsh(K)
    np.testing.assert_allclose(lam, lam_lapack, rtol=1e-10, atol=1e-15)
    assert np.all(lam > 0)
    # beta >= 0 for any data, and beta(c f) = c^2 beta(f)
    rng = np.random.default_rng(R)
    f = rng.normal(size=R + 1)
    b = f @ t["Kinv_sigma"] @ f
    assert b > 0
    assert abs((3 * f) @ t["Kinv_sigma"] @ (3 * f) - 9 * b) < 1e-12 * 9 * b
    # K_m is persymmetric: beta is invariant under reversal of the window
    assert abs(f[::-1] @ t["Kinv_sigma"] @ f[::-1] - b) < 1e-10 * b


@pytest.mark.parametrize("R", [1, 2, 3])
def test_mirror_prediction_point(R):
    """Weights for x* = -1/2 are the x* = +1/2 weights reversed (symmetry of K)."""
    tl = gp_tables.tables(R, 12.0, 3.0, 0.5)
    tr = gp_tables.tables(R, 12.0, 3.0, -0.5)
    np.testing.assert_allclose(tr["w_big"], tl["w_big"][::-1], rtol=1e-13, atol=1e-15)
    for m in range(R + 1):
        np.testing.assert_allclose(tr["w_sub"][m], tl["w_sub"][R - m][::-1], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(tr["gamma"], tl["gamma"][::-1], rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("R", [1, 2, 3])
def test_deviation_from_lagrange_shrinks_like_ell_minus_2(R):
    """The SE kernel's expansion in (Delta/l)^2 makes w - w_Lagrange = O((Delta/l)^2); the
    moment defects (sum w - 1, sum w x - x*) shrink at least that fast."""
    lag = lagrange_weights(list(range(-R, R + 1)), Fraction(1, 2))
    x = np.arange(-R, R + 1)
    dev, mom = [], []
    for ell in (24.0, 48.0):
        w = gp_tables.tables(R, ell, 3.0, 0.5)["w_big"]
        dev.append(np.abs(w - lag).max())
        mom.append((abs(w.sum() - 1.0), abs((w * x).sum() - 0.5)))
    assert 3.5 < dev[0] / dev[1] < 4.5, dev
    for k in range(2):
        assert mom[0][k] / mom[1][k] > 3.5, mom


def test_linear_weights_at_default_hyperparameters():
    """At l/Delta = 12 the linear weights stay positive and close to the flat-limit values,
    and the least-squares residual of Eq. gamm-system is small but non-zero."""
    for R in (1, 2, 3):
        t = gp_tables.tables(R, 12.0, 3.0, 0.5)
        assert np.all(t["gamma"] > 0)
        np.testing.assert_allclose(t["gamma"], FLAT_GAMMA[R], atol=0.05)
        res = np.linalg.norm(t["M"] @ t["gamma"] - t["w_big"])
        assert 0 < res < 1e-2


def test_large_ell_conditioning_handled():
    """R=3 at l/Delta = 96 (cond K ~ 1e24) still reproduces the flat limit trend."""
    t96 = gp_tables.tables(3, 96.0, 3.0, 0.5)
    lag = lagrange_weights(list(range(-3, 4)), Fraction(1, 2))
    err96 = np.abs(t96["w_big"] - lag).max()
    t48 = gp_tables.tables(3, 48.0, 3.0, 0.5)
    err48 = np.abs(t48["w_big"] - lag).max()
    assert 3.5 < err48 / err96 < 4.5


def _mp_gp_linear_weights(R, ell, xs="0.5", dps=60):
    """Linear weights gamma of Eq. gamm-system at l/Delta = ell, computed here from the
    definitions with mpmath (LU solves for w and w_m, Householder-QR least squares for gamma)
    -- a different algorithm and arithmetic from the oracle's decimal normal equations."""
    import mpmath as mp
    with mp.workdps(dps):
        ell = mp.mpf(ell)
        xs = mp.mpf(xs)
        k = lambda a, b: mp.e ** (-(a - b) ** 2 / (2 * ell * ell))
        pts = list(range(-R, R + 1))
        K = mp.matrix([[k(a, b) for b in pts] for a in pts])
        w = mp.lu_solve(K, mp.matrix([k(xs, b) for b in pts]))
        M = mp.zeros(2 * R + 1, R + 1)
        for m in range(R + 1):
            sub = pts[m:m + R + 1]
            Km = mp.matrix([[k(a, b) for b in sub] for a in sub])
            wm = mp.lu_solve(Km, mp.matrix([k(xs, b) for b in sub]))
            for j in range(R + 1):
                M[m + j, m] = wm[j]
        gam, res = mp.qr_solve(M, w)
        return [float(gam[m]) for m in range(R + 1)], float(mp.fsum(gam)), float(res)


@pytest.mark.parametrize("R", [1, 2, 3])
def test_linear_weights_at_ell_12_independent(R):
    """gamma at l/Delta = 12 (the operating point) to 1e-10 against the mpmath computation
    above, and not renormalised: sum(gamma) keeps its least-squares defect (a renormalised
    gamma would pass the flat-limit pins but fail here)."""
    g_mp, sum_mp, res_mp = _mp_gp_linear_weights(R, 12)
    t = gp_tables.tables(R, 12.0, 3.0, 0.5)
    np.testing.assert_allclose(t["gamma"], g_mp, rtol=0, atol=1e-10)
    assert abs(t["gamma"].sum() - sum_mp) < 1e-12
    assert abs(sum_mp - 1.0) > 1e-9          # the least-squares gamma does not sum to one
    assert abs(np.linalg.norm(t["M"] @ t["gamma"] - t["w_big"]) - res_mp) < 1e-9 * max(res_mp, 1e-6)


def test_linear_weights_r2_worked_values():
    """R = 2, l/Delta = 12: the worked values (0.063594, 0.620632, 0.315774) of an
    independent high-precision probe, to 1e-6."""
    t = gp_tables.tables(2, 12.0, 3.0, 0.5)
    np.testing.assert_allclose(t["gamma"], [0.063594, 0.620632, 0.315774], rtol=0, atol=1e-6)


# eigenvalues of the (R+1)-point smoothness covariance K_m(sigma/Delta = 3), ascending, as
# printed by an independent probe to three or four significant digits
SIGMA3_EIGS = {1: [0.0540, 1.946], 2: [0.00395, 0.199, 2.797], 3: [3.89e-4, 0.0213, 0.447, 3.531]}


@pytest.mark.parametrize("R", [1, 2, 3])
def test_smoothness_covariance_eigenvalues(R):
    """lambda_h of K_m(sigma) (Eq. beta-eigen) at sigma/Delta = 3 against the worked values,
    and their sum = trace K_m = R+1 (unit diagonal)."""
    t = gp_tables.tables(R, 12.0, 3.0, 0.5)
    lam = np.sort(t["lam_sigma"])
    np.testing.assert_allclose(lam, SIGMA3_EIGS[R], rtol=3e-3)
    assert abs(lam.sum() - (R + 1)) < 1e-13
