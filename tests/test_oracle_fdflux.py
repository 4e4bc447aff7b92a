"""Pins for the oracle's FD-Flux form (Section 2): the reconstruction tables and the scheme.

The FD-Flux form reads the point fluxes F_j as cell averages of the function F^
whose face values are the numerical fluxes (Eqs. prim_F, exct_num_flux, design),
so its GP weights predict a point value from cell averages.  The pins here do not
reuse the oracle's formulas: covariances against direct numerical quadrature, the
flat-kernel limit against the classical WENO-JS reconstruction coefficients
(exact rationals), polynomial exactness, and for the whole scheme the textbook
invariants plus the paper's statement that point-value weights give at most
second order (Eq. flux_2nd)."""
import math
from decimal import Decimal
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from oracle import gp_tables as G
from paper_1808_04960_gb300 import workloads as W


def test_recon_covariances_match_quadrature():
    """[C]_jk = int int k(x, y) over two unit cells and [T]_j = int k(x*, y) over one,
    by composite Gauss-Legendre quadrature in float64 (independent of the erf closed form)."""
    ell = 2.5
    xg, wg = np.polynomial.legendre.leggauss(40)
    k = lambda u: np.exp(-u * u / (2 * ell * ell))
    pts = [Decimal(j) for j in range(-2, 3)]
    C = G.cell_average_cov(pts, Decimal(ell))
    for a in range(5):
        for b in range(5):
            x = (a - 2) + 0.5 * xg
            y = (b - 2) + 0.5 * xg
            q = 0.25 * np.sum(wg[:, None] * wg[None, :] * k(x[:, None] - y[None, :]))
            assert abs(float(C[a][b]) - q) < 1e-13, (a, b)
    T = G.point_cell_cov(pts, Decimal("0.5"), Decimal(ell))
    for b in range(5):
        y = (b - 2) + 0.5 * xg
        q = 0.5 * np.sum(wg * k(0.5 - y))
        assert abs(float(T[b]) - q) < 1e-14, b


# WENO-JS reconstruction coefficients at x_{i+1/2} (Jiang & Shu 1996; Shu 1998, Table 2.1)
# for sub-stencils left to right, and the optimal linear weights.
JS = {
    1: ([[Fr(-1, 2), Fr(3, 2)], [Fr(1, 2), Fr(1, 2)]], [Fr(1, 3), Fr(2, 3)]),
    2: ([[Fr(1, 3), Fr(-7, 6), Fr(11, 6)], [Fr(-1, 6), Fr(5, 6), Fr(1, 3)], [Fr(1, 3), Fr(5, 6), Fr(-1, 6)]],
        [Fr(1, 10), Fr(6, 10), Fr(3, 10)]),
    3: ([[Fr(-1, 4), Fr(13, 12), Fr(-23, 12), Fr(25, 12)], [Fr(1, 12), Fr(-5, 12), Fr(13, 12), Fr(1, 4)],
         [Fr(-1, 12), Fr(7, 12), Fr(7, 12), Fr(-1, 12)], [Fr(1, 4), Fr(13, 12), Fr(-5, 12), Fr(1, 12)]],
        [Fr(1, 35), Fr(12, 35), Fr(18, 35), Fr(4, 35)]),
}


@pytest.mark.parametrize("R", [1, 2, 3])
def test_recon_flat_limit_is_weno_js(R):
    """Polynomial reconstruction weights equal the WENO-JS coefficients (to 1e-25, the test's
    own 28-digit Decimal division); the GP reconstruction weights tend to them like (dx/l)^2; the right-state
    tables are their mirror images."""
    ws, gam = JS[R]
    tp = G.tables_decimal(R, 12.0, 3.0, Decimal("0.5"), poly=True, recon=True)
    for m in range(R + 1):
        for j in range(R + 1):
            assert abs(tp["w_sub"][m][j] - Decimal(ws[m][j].numerator) / ws[m][j].denominator) < Decimal("1e-25")
        assert abs(tp["gamma"][m] - Decimal(gam[m].numerator) / gam[m].denominator) < Decimal("1e-25")
    devs = []
    for ell in (200.0, 400.0):
        t = G.tables(R, ell, 3.0, 0.5, recon=True)
        devs.append(max(abs(t["w_sub"][m][j] - float(ws[m][j])) for m in range(R + 1) for j in range(R + 1)))
    assert devs[1] < 1e-3 and 3.5 < devs[0] / devs[1] < 4.5, devs
    tr = G.tables(R, 12.0, 3.0, -0.5, recon=True)
    tl = G.tables(R, 12.0, 3.0, 0.5, recon=True)
    np.testing.assert_allclose(tr["w_sub"], tl["w_sub"][::-1, ::-1], rtol=0, atol=1e-14)
    np.testing.assert_allclose(tr["gamma"], tl["gamma"][::-1], rtol=0, atol=1e-14)


@pytest.mark.parametrize("R", [1, 2, 3])
def test_poly_recon_reproduces_polynomials(R):
    """sum_j w_j avg_j(p) = p(x*) exactly for every polynomial of degree <= R on each sub-stencil
    (the definition of reconstruction from cell averages)."""
    t = G.tables_decimal(R, 12.0, 3.0, Decimal("0.5"), poly=True, recon=True)
    half = Decimal(1) / 2
    for deg in range(R + 1):
        for m in range(R + 1):
            cells = [Decimal(-R + m + j) for j in range(R + 1)]
            avg = [((c + half) ** (deg + 1) - (c - half) ** (deg + 1)) / (deg + 1) for c in cells]
            val = sum(w * a for w, a in zip(t["w_sub"][m], avg))
            assert abs(val - half ** deg) < Decimal("1e-25"), (deg, m)


def test_gp_recon_moments_shrink():
    """GP reconstruction weights reproduce low moments of cell averages up to a defect that
    shrinks at least like (dx/l)^2 (the GP prior is not polynomial-exact at finite l)."""
    defects = []
    for ell in (12.0, 24.0):
        t = G.tables(2, ell, 3.0, 0.5, recon=True)
        cells = np.arange(-2, 3, dtype=float)
        avg1 = cells                              # cell averages of p(x) = x
        defects.append(abs(t["w_big"] @ avg1 - 0.5))
    assert defects[0] / defects[1] > 3.5 and defects[1] < 1e-5, defects


def _gauss_err(n, R, **kw):
    Ug, m = W.gaussian_1d(n)
    oo = oracle.Oracle((n,), m["dx"], m["bc"], R=R, ell_over_dx=0.1 * n, gamma=m["gamma"], **kw)
    dx = m["dx"][0]
    dt = 0.4 * dx / 2.3 * (dx / (1.0 / 25)) ** ((2 * R + 1) / 3.0 - 1.0)
    steps = int(math.ceil(1.0 / dt))
    Un = oo.run(Ug, 1.0 / steps, steps)
    Ue, _ = W.gaussian_1d(n, t=1.0)
    return np.abs(Un[0] - Ue[0]).mean()


@pytest.mark.parametrize("R,lo", [(2, 4.5), (3, 6.3)])
def test_fdflux_order_with_recon_weights_and_eq_flux_2nd(R, lo):
    """Smooth advection (Section 6.1 set-up, l = 0.1): FD-Flux with reconstruction weights keeps
    order 2R+1; with the point-value weights it drops to 2, as Eq. flux_2nd states."""
    e = [_gauss_err(n, R, scheme="fdflux") for n in (100, 200)]
    assert math.log2(e[0] / e[1]) > lo, e
    e = [_gauss_err(n, R, scheme="fdflux", recon_weights=False) for n in (100, 200)]
    assert abs(math.log2(e[0] / e[1]) - 2.0) < 0.15, e


def test_fdflux_free_stream_conservation_mirror():
    rng = np.random.default_rng(12)
    U = np.empty((4, 9, 14))
    u0 = np.array([1.3, 0.4, -0.2, 3.1])
    for a in range(4):
        U[a] = u0[a]
    o = oracle.Oracle((9, 14), (0.1, 0.1), (("outflow", "outflow"),) * 2, R=2, scheme="fdflux")
    assert np.abs(o.rhs(U)).max() == 0.0
    # conservation on a periodic grid
    U1, m = W.smooth_field((20, 24), seed=3)
    o = oracle.Oracle(U1.shape[1:], m["dx"], m["bc"], R=3, scheme="fdflux")
    r = o.rhs(U1)
    assert np.abs(r.sum(axis=(1, 2))).max() < 1e-12 * np.abs(r).max() * r[0].size
    # mirror x -> -x with u -> -u
    U2, m = W.four_quadrant(24, seed=3, ny=20)
    o = oracle.Oracle(U2.shape[1:], m["dx"], m["bc"], R=2, scheme="fdflux")
    Um = U2[:, :, ::-1].copy()
    Um[1] = -Um[1]
    r, rm = o.rhs(U2), o.rhs(Um)
    rm = rm[:, :, ::-1]
    rm[1] = -rm[1]
    np.testing.assert_allclose(rm, r, rtol=0, atol=1e-12 * np.abs(r).max())


def test_fdflux_sod():
    U, meta = W.sod_1d(256)
    o = oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=2, scheme="fdflux")
    dt = 0.4 / o.max_rate(U)
    steps = int(math.ceil(0.2 / dt))
    out = o.run(U, 0.2 / steps, steps)
    x = meta["x"]
    assert abs(out[0][np.argmin(np.abs(x - 0.6))] - 0.4263) < 0.02
    assert abs(out[0][np.argmin(np.abs(x - 0.8))] - 0.2656) < 0.02
