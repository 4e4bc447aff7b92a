"""Pins of the oracle's per-face scheme and RHS against facts fixed by the
paper and the mathematics (not by re-typing the oracle's formulas):

* GP-WENO prediction: exact for polynomials of degree <= R in the flat-kernel
  limit whatever the nonlinear weights; selects the smooth sub-stencil at a
  jump; scale covariance; mirror symmetry between the two prediction points.
* Roe eigen-system: L R = I and the Roe property A(U_roe)(U_R - U_L) =
  F(U_R) - F(U_L), with A = R diag(lambda) L and F from this file's own flux.
* High-order correction (Eqs. numFlux_cor, FD-ders): exact for face fluxes that
  are cell averages of a degree-5 polynomial.
* RHS: free-stream preservation, conservation on periodic grids, mirror and
  transpose symmetry, reduction of 2D/3D to 1D, and the (2R+1)th order of
  the whole solver on smooth advection with l fixed in physical units
  (Table 1 reports orders ~2R+1 for the same problem)."""
import math

import numpy as np
import pytest

import oracle
from paper_1808_04960_gb300 import workloads as W


def euler_flux(u, g):
    """Normal-direction flux of a normal-first conserved state (test-side, Eq. euler)."""
    rho = u[0]
    un = u[1] / rho
    ke = sum(u[a] ** 2 for a in range(1, len(u) - 1)) / rho
    p = (g - 1.0) * (u[-1] - 0.5 * ke)
    f = np.array(u, dtype=np.float64) * un
    f[1] += p
    f[-1] += p * un
    return f


def rand_state(rng, nc, g=1.4):
    rho = rng.uniform(0.5, 2.0)
    vel = rng.uniform(-1.0, 1.0, nc - 2)
    p = rng.uniform(0.5, 2.0)
    return np.concatenate([[rho], rho * vel, [p / (g - 1) + 0.5 * rho * (vel ** 2).sum()]])


def conservative_jacobian(vel, H, g):
    """Normal flux Jacobian dF/dU (normal-first) written in terms of velocity and total enthalpy
    (textbook form; test-side)."""
    nv = len(vel)
    nc = nv + 2
    u = vel[0]
    q2 = sum(v * v for v in vel)
    gm = g - 1.0
    A = np.zeros((nc, nc))
    A[0, 1] = 1.0
    A[1, 0] = 0.5 * gm * q2 - u * u
    A[1, 1] = (3.0 - g) * u
    for t in range(1, nv):
        A[1, 1 + t] = -gm * vel[t]
        A[1 + t, 0] = -u * vel[t]
        A[1 + t, 1] = vel[t]
        A[1 + t, 1 + t] = u
    A[1, nc - 1] = gm
    A[nc - 1, 0] = u * (0.5 * gm * q2 - H)
    A[nc - 1, 1] = H - gm * u * u
    for t in range(1, nv):
        A[nc - 1, 1 + t] = -gm * u * vel[t]
    A[nc - 1, nc - 1] = g * u
    return A


def primitive_jacobian(rho, un, c, nc):
    """A_V of V_t + A_V V_x = 0 for V = (rho, u_n, u_t..., p) (test-side, from the primitive
    Euler equations: continuity, momentum with p_x/rho, advection, p_t + u p_x + rho c^2 u_x = 0)."""
    A = np.eye(nc) * un
    A[0, 1] = rho
    A[1, nc - 1] = 1.0 / rho
    A[nc - 1, 1] = rho * c * c
    return A


@pytest.mark.parametrize("nc", [3, 4, 5])
def test_roe_average_and_primitive_eigensystem(nc):
    rng = np.random.default_rng(nc)
    g = 1.4
    for _ in range(5):
        uL, uR = rand_state(rng, nc), rand_state(rng, nc)
        roe, Rm, Lm = oracle.roe_eigensystem(uL, uR, g)
        rho, vel, H, c = roe[0], roe[1:nc - 1], roe[nc - 1], roe[nc]
        # Roe property of the averaged state: A(U_roe)(U_R - U_L) = F(U_R) - F(U_L)
        A = conservative_jacobian(vel, H, g)
        np.testing.assert_allclose(A @ (uR - uL), euler_flux(uR, g) - euler_flux(uL, g), rtol=1e-12, atol=1e-12)
        assert abs(rho - math.sqrt(uL[0] * uR[0])) < 1e-14
        assert abs(c * c - (g - 1) * (H - 0.5 * (vel ** 2).sum())) < 1e-13
        # primitive eigen-system at (rho, c)
        np.testing.assert_allclose(Lm @ Rm, np.eye(nc), atol=1e-13)
        lam = np.array([vel[0] - c] + [vel[0]] * (nc - 2) + [vel[0] + c])
        np.testing.assert_allclose(Rm @ np.diag(lam) @ Lm, primitive_jacobian(rho, vel[0], c, nc), atol=1e-12)


def test_correction_exact_for_degree5():
    """f^ = F + alpha D2 F + beta D4 F with alpha=-1/24, beta=3/640 recovers F^(x_face) when the
    face fluxes are the cell averages of a degree-5 F^ (Eq. prim_F read at faces; Eq. numF_cond, q=5)."""
    rng = np.random.default_rng(0)
    for _ in range(10):
        c = rng.normal(size=6)
        P = np.polynomial.Polynomial(c)
        A = P.integ()
        # faces at x = -2..2 (units of Delta), face flux = average of F^ over [x-1/2, x+1/2]
        F5 = np.array([A(x + 0.5) - A(x - 0.5) for x in (-2, -1, 0, 1, 2)])
        assert abs(oracle.corrected_flux(F5) - P(0.0)) < 1e-12 * max(1.0, abs(P(0.0)))
    # degree 6 is not reproduced (the correction is truncated after the fourth derivative)
    P = np.polynomial.Polynomial([0, 0, 0, 0, 0, 0, 1.0])
    A = P.integ()
    F5 = np.array([A(x + 0.5) - A(x - 0.5) for x in (-2, -1, 0, 1, 2)])
    assert abs(oracle.corrected_flux(F5) - P(0.0)) > 1e-3


def _oracle_1d(R, ell, n=16, **kw):
    return oracle.Oracle((n,), (1.0 / n,), (("periodic", "periodic"),), R=R, ell_over_dx=ell, **kw)


@pytest.mark.parametrize("R", [1, 2, 3])
def test_gp_weno_flat_limit_exact_for_polynomials(R):
    """With l/Delta -> infinity every sub-stencil prediction is Lagrange interpolation, exact for
    degree <= R, so q = sum omega_m q^m is exact whatever omega (Eqs. candidate_interp, weight_sum)."""
    o = _oracle_1d(R, 1.0e4)
    rng = np.random.default_rng(R)
    x = np.arange(-R, R + 1, dtype=np.float64)
    for _ in range(5):
        c = rng.normal(size=R + 1)
        P = np.polynomial.Polynomial(c)
        f = P(x)
        assert abs(o.gp_weno(f) - P(0.5)) < 1e-5 * (1 + np.abs(f).max())
        assert abs(o.gp_weno(f, right=True) - P(-0.5)) < 1e-5 * (1 + np.abs(f).max())


@pytest.mark.parametrize("R", [1, 2, 3])
def test_gp_weno_step_selects_smooth_substencil(R):
    """Jump inside every sub-stencil but the leftmost: that one is constant zero, so beta = 0,
    omega_1 -> 1 and the prediction is 0 to O(eps^2)-relative (Eq. weights with eps = 1e-36)."""
    o = _oracle_1d(R, 12.0)
    f = np.zeros(2 * R + 1)
    f[R + 1:] = 1.0
    assert abs(o.gp_weno(f)) < 1e-20
    # and mirrored for the right-state prediction point
    assert abs(o.gp_weno(f[::-1], right=True)) < 1e-20


@pytest.mark.parametrize("R", [1, 2, 3])
def test_gp_weno_constant_data_uses_linear_weights(R):
    """Constant data has identical beta on every sub-stencil, so omega = gamma / sum(gamma)
    (Eq. weights): q = c sum_m gamma_m sum_j w_mj / sum_m gamma_m, i.e. the big-stencil GP
    prediction up to the least-squares residual of Eq. gamm-system."""
    o = _oracle_1d(R, 12.0)
    t = o.tables
    expect = 2.5 * sum(t["gl"][m] * t["wl"][m].sum() for m in range(R + 1)) / t["gl"].sum()
    assert abs(o.gp_weno(np.full(2 * R + 1, 2.5)) - expect) < 1e-14
    assert abs(expect - 2.5 * t["w_big_l"].sum()) < 1e-3


@pytest.mark.parametrize("R", [1, 2, 3])
def test_gp_weno_scale_and_mirror(R):
    o = _oracle_1d(R, 12.0)
    rng = np.random.default_rng(7 + R)
    for _ in range(5):
        f = rng.normal(size=2 * R + 1)
        q = o.gp_weno(f)
        assert abs(o.gp_weno(3.0 * f) - 3.0 * q) < 1e-13 * (1 + abs(q))
        assert abs(o.gp_weno(f[::-1], right=True) - q) < 1e-12 * (1 + abs(q))


@pytest.mark.parametrize("R", [1, 2])
def test_face_uniform_state_flux(R):
    o = oracle.Oracle((16, 16), (0.1, 0.1), (("periodic", "periodic"),) * 2, R=R, ell_over_dx=1.0e4)
    rng = np.random.default_rng(3)
    u0 = rand_state(rng, 4)
    st = np.tile(u0, (2 * R + 2, 1))
    for d in (0, 1):
        uL, uR, F = o.face(st, d)
        np.testing.assert_allclose(uL, u0, rtol=1e-7)
        np.testing.assert_allclose(uR, u0, rtol=1e-7)
        perm = [0, 1 + d, 2 - d, 3]
        np.testing.assert_allclose(F[perm], euler_flux(u0[perm], 1.4), rtol=1e-6, atol=1e-7)


def test_free_stream_preserved_exactly():
    for shape, dx in (((32,), (0.1,)), ((24, 20), (0.1, 0.2)), ((8, 9, 10), (0.1, 0.1, 0.1))):
        nd = len(shape)
        rng = np.random.default_rng(nd)
        u0 = rand_state(rng, nd + 2)
        U = np.empty((nd + 2,) + shape)
        for a in range(nd + 2):
            U[a] = u0[a]
        for bc in ("periodic", "outflow"):
            o = oracle.Oracle(shape, dx, ((bc, bc),) * nd, R=2)
            assert np.abs(o.rhs(U)).max() == 0.0


@pytest.mark.parametrize("R", [1, 2, 3])
def test_conservation_periodic(R):
    U, m = W.isentropic_vortex(24)
    o = oracle.Oracle(U.shape[1:], m["dx"], m["bc"], R=R)
    L = o.rhs(U)
    s = L.sum(axis=(1, 2))
    assert np.abs(s).max() < 1e-11, s


def test_mirror_symmetry_1d():
    """x -> -x with u -> -u maps the solution onto itself (zero-mean GP, symmetric stencils)."""
    rng = np.random.default_rng(11)
    n = 40
    x = (np.arange(n) + 0.5) / n
    rho = 1 + 0.3 * np.sin(2 * np.pi * x) + 0.1 * rng.normal(size=n)
    u = 0.2 * np.cos(2 * np.pi * x)
    p = 1 + 0.2 * np.cos(4 * np.pi * x)
    U = W.conserved(rho, [u], p, 1.4)
    Um = U[:, ::-1].copy()
    Um[1] *= -1
    for bc in ("periodic", "outflow"):
        o = oracle.Oracle((n,), (1.0 / n,), ((bc, bc),), R=2)
        L = o.rhs(U)
        Lm = o.rhs(Um)
        Lmm = Lm[:, ::-1].copy()
        Lmm[1] *= -1
        np.testing.assert_allclose(Lmm, L, rtol=0, atol=1e-11 * np.abs(L).max())


def test_transpose_symmetry_2d():
    """Swapping x and y (with u <-> v) transposes the result: pins the y-direction indexing."""
    U, m = W.four_quadrant(20, seed=3, ny=20)
    rng = np.random.default_rng(1)
    U = U * (1 + 0.01 * rng.random(U.shape))
    o = oracle.Oracle(U.shape[1:], (0.05, 0.05), (("outflow", "outflow"),) * 2, R=2)
    L = o.rhs(U)
    Ut = np.stack([U[0].T, U[2].T, U[1].T, U[3].T])
    Lt = o.rhs(Ut)
    np.testing.assert_allclose(np.stack([Lt[0].T, Lt[2].T, Lt[1].T, Lt[3].T]), L, rtol=0,
                               atol=1e-12 * np.abs(L).max())


def test_2d_and_3d_reduce_to_1d():
    U1, m1 = W.sod_1d(48)
    o1 = oracle.Oracle((48,), m1["dx"], m1["bc"], R=2)
    L1 = o1.rhs(U1)
    U2 = np.zeros((4, 5, 48))
    U2[0], U2[1], U2[3] = U1[0], U1[1], U1[2]
    o2 = oracle.Oracle((5, 48), (m1["dx"][0], 0.3), (("outflow", "outflow"), ("periodic", "periodic")), R=2)
    L2 = o2.rhs(U2)
    for j in range(5):
        np.testing.assert_allclose(L2[[0, 1, 3], j], L1, rtol=0, atol=1e-12 * np.abs(L1).max())
    assert np.abs(L2[2]).max() == 0.0
    U3 = np.zeros((5, 3, 4, 48))
    U3[0], U3[1], U3[4] = U1[0], U1[1], U1[2]
    o3 = oracle.Oracle((3, 4, 48), (m1["dx"][0], 0.3, 0.2),
                       (("outflow", "outflow"), ("periodic", "periodic"), ("outflow", "outflow")), R=2)
    L3 = o3.rhs(U3)
    np.testing.assert_allclose(L3[[0, 1, 4], 1, 2], L1, rtol=0, atol=1e-12 * np.abs(L1).max())


def _gauss_error(R, n, ell_phys=0.1, t_end=0.2):
    U, m = W.gaussian_1d(n)
    g = m["gamma"]
    o = oracle.Oracle((n,), m["dx"], m["bc"], R=R, ell_over_dx=ell_phys * n, gamma=g)
    dx = m["dx"][0]
    # dt ~ dx^((2R+1)/3) so RK3's temporal error drops at the spatial order
    dt0 = 0.4 * dx / 2.3
    dt = dt0 * (dx / (1.0 / 25)) ** ((2 * R + 1) / 3.0 - 1.0)
    steps = int(math.ceil(t_end / dt))
    Un = o.run(U, t_end / steps, steps)
    Ue, _ = W.gaussian_1d(n, t=t_end)
    return np.abs(Un[0] - Ue[0]).mean()


def _table1():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_gaussian_advection_l1.txt")
    rows = np.loadtxt(path, comments="#")
    return {int(r[0]): r for r in rows}


@pytest.mark.parametrize("R,ns", [(1, (25, 50, 100, 200)), (2, (25, 50, 100, 200)), (3, (25, 50, 100))])
def test_convergence_against_table1(R, ns):
    """Smooth Gaussian advection (Section 6.1) to t = 1 with l = 0.1 fixed in physical units:
    the L1 orders match Table 1 to +-0.5 and the errors are within a factor 2.5 of its values
    (the paper's HLLC + RK4 versus this scheme's Lax-Friedrichs + SSP-RK3)."""
    tab = _table1()
    errs = [_gauss_error(R, n, t_end=1.0) for n in ns]
    for n, e in zip(ns, errs):
        ref = tab[n][1 + 2 * (R - 1)]
        assert ref / 2.5 < e < ref * 2.5, (n, e, ref)
    for k in range(1, len(ns)):
        order = math.log(errs[k - 1] / errs[k], 2)
        ref_order = tab[ns[k]][2 + 2 * (R - 1)]
        assert abs(order - ref_order) < 0.5, (ns[k], order, ref_order)


# ---------------------------------------------------------------------------
# HLLC face flux (the paper's default solver, Section 7)

def _roe_uc(uL, uR, g=1.4):
    roe, _, _ = oracle.roe_eigensystem(uL, uR, g)
    nc = len(uL)
    return roe[1], roe[nc]


@pytest.mark.parametrize("nc", [3, 4, 5])
def test_hllc_consistency_and_supersonic(nc):
    """F(U, U) = F(U); fully supersonic states take the upwind physical flux."""
    g = 1.4
    rng = np.random.default_rng(40 + nc)
    for _ in range(5):
        u = rand_state(rng, nc)
        ur, cr = _roe_uc(u, u)
        np.testing.assert_allclose(oracle.hllc(u, u, ur, cr), euler_flux(u, g), rtol=1e-13, atol=1e-13)
    # supersonic to the right: u - c > 0 on both sides and at the Roe state
    uL = W.conserved(np.array(1.0), [np.array(3.0)] + [np.array(0.1)] * (nc - 3), np.array(1.0), g)
    uR = W.conserved(np.array(0.8), [np.array(2.9)] + [np.array(-0.2)] * (nc - 3), np.array(0.9), g)
    ur, cr = _roe_uc(uL, uR)
    np.testing.assert_allclose(oracle.hllc(uL, uR, ur, cr), euler_flux(uL, g), rtol=1e-13)


def test_hllc_resolves_stationary_and_moving_contacts():
    """An isolated contact (equal u and p, different rho and v) is a single HLLC wave: the flux is
    the exact upwind flux of the contact (mass flux rho*u of the upwind side, zero if u = 0)."""
    g = 1.4
    for u in (0.0, 0.4, -0.3):
        uL = W.conserved(np.array(1.0), [np.array(u), np.array(0.3)], np.array(1.0), g)
        uR = W.conserved(np.array(0.2), [np.array(u), np.array(-0.5)], np.array(1.0), g)
        ur, cr = _roe_uc(uL, uR)
        F = oracle.hllc(uL, uR, ur, cr)
        up = uL if u >= 0 else uR
        np.testing.assert_allclose(F, euler_flux(up, g), rtol=1e-12, atol=1e-13)


def test_hllc_mirror_symmetry():
    """Reflecting x -> -x maps F(UL, UR) to the mirrored flux of (mirror UR, mirror UL)."""
    g = 1.4
    rng = np.random.default_rng(9)
    M = np.diag([1.0, -1.0, 1.0, 1.0])
    for _ in range(10):
        uL, uR = rand_state(rng, 4), rand_state(rng, 4)
        ur, cr = _roe_uc(uL, uR)
        F = oracle.hllc(uL, uR, ur, cr)
        mL, mR = M @ uR, M @ uL
        ur2, cr2 = _roe_uc(mL, mR)
        F2 = oracle.hllc(mL, mR, ur2, cr2)
        np.testing.assert_allclose(-(M @ F2), F, rtol=1e-12, atol=1e-12)


def test_hllc_scheme_free_stream_and_order():
    """The whole scheme with HLLC preserves free streams exactly and keeps the Table 1 orders."""
    rng = np.random.default_rng(2)
    u0 = rand_state(rng, 4)
    U = np.empty((4, 11, 13))
    for a in range(4):
        U[a] = u0[a]
    o = oracle.Oracle((11, 13), (0.1, 0.1), (("outflow", "outflow"),) * 2, R=2, flux="hllc")
    assert np.abs(o.rhs(U)).max() == 0.0
    errs = []
    for n in (50, 100):
        Ug, m = W.gaussian_1d(n)
        oo = oracle.Oracle((n,), m["dx"], m["bc"], R=2, ell_over_dx=0.1 * n, gamma=m["gamma"], flux="hllc")
        dx = m["dx"][0]
        dt = 0.4 * dx / 2.3 * (dx / (1.0 / 25)) ** (5 / 3.0 - 1.0)
        steps = int(math.ceil(1.0 / dt))
        Un = oo.run(Ug, 1.0 / steps, steps)
        Ue, _ = W.gaussian_1d(n, t=1.0)
        errs.append(np.abs(Un[0] - Ue[0]).mean())
    tab = _table1()
    order = math.log(errs[0] / errs[1], 2)
    assert abs(order - tab[100][4]) < 0.5, (errs, order)
    assert tab[100][3] / 2.5 < errs[1] < tab[100][3] * 2.5


# ---------------------------------------------------------------------------
# HLL face flux (the solver of the paper's Mach-3 wind-tunnel test, Section 7)

def _einfeldt(uL, uR, g=1.4):
    ur, cr = _roe_uc(uL, uR, g)
    rL, rR = uL[0], uR[0]
    vL, vR = uL[1] / rL, uR[1] / rR
    pL = (g - 1) * (uL[-1] - 0.5 * np.sum(uL[1:-1] ** 2) / rL)
    pR = (g - 1) * (uR[-1] - 0.5 * np.sum(uR[1:-1] ** 2) / rR)
    SL = min(vL - math.sqrt(g * pL / rL), ur - cr)
    SR = max(vR + math.sqrt(g * pR / rR), ur + cr)
    return ur, cr, SL, SR


@pytest.mark.parametrize("nc", [3, 4, 5])
def test_hll_is_the_integral_average_flux(nc):
    """Toro's derivation of HLL: with the intermediate state U* = (S_R U_R - S_L U_L - (F_R - F_L)) /
    (S_R - S_L) (conservation over the wave fan), F_HLL = F_L + S_L (U* - U_L) = F_R + S_R (U* - U_R);
    F(U, U) = F(U); supersonic states take the upwind flux."""
    g = 1.4
    rng = np.random.default_rng(70 + nc)
    for _ in range(10):
        uL, uR = rand_state(rng, nc), rand_state(rng, nc)
        ur, cr, SL, SR = _einfeldt(uL, uR)
        F = oracle.hll(uL, uR, ur, cr)
        fL, fR = euler_flux(uL, g), euler_flux(uR, g)
        if SL < 0 < SR:
            Us = (SR * uR - SL * uL - (fR - fL)) / (SR - SL)
            np.testing.assert_allclose(F, fL + SL * (Us - uL), rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(F, fR + SR * (Us - uR), rtol=1e-12, atol=1e-12)
        u = rand_state(rng, nc)
        ur, cr = _roe_uc(u, u)
        np.testing.assert_allclose(oracle.hll(u, u, ur, cr), euler_flux(u, g), rtol=1e-13, atol=1e-13)
    uL = W.conserved(np.array(1.0), [np.array(-3.0)] + [np.array(0.1)] * (nc - 3), np.array(1.0), g)
    uR = W.conserved(np.array(0.8), [np.array(-2.9)] + [np.array(-0.2)] * (nc - 3), np.array(0.9), g)
    ur, cr = _roe_uc(uL, uR)
    np.testing.assert_allclose(oracle.hll(uL, uR, ur, cr), euler_flux(uR, g), rtol=1e-13)


def test_hll_smears_a_stationary_contact():
    """A stationary contact (u = 0, equal p): HLLC's mass flux is zero, HLL's is the textbook
    diffusive S_L S_R (rho_R - rho_L) / (S_R - S_L) != 0."""
    g = 1.4
    uL = W.conserved(np.array(1.0), [np.array(0.0), np.array(0.0)], np.array(1.0), g)
    uR = W.conserved(np.array(0.2), [np.array(0.0), np.array(0.0)], np.array(1.0), g)
    ur, cr, SL, SR = _einfeldt(uL, uR)
    F = oracle.hll(uL, uR, ur, cr)
    assert abs(oracle.hllc(uL, uR, ur, cr)[0]) < 1e-15
    np.testing.assert_allclose(F[0], SL * SR * (uR[0] - uL[0]) / (SR - SL), rtol=1e-13)
    assert abs(F[0]) > 0.1


def test_hll_scheme_free_stream_mirror_and_order():
    """The whole scheme with HLL: free streams exactly, mirror symmetry, and the Table 1 order."""
    rng = np.random.default_rng(3)
    u0 = rand_state(rng, 4)
    U = np.empty((4, 11, 13))
    for a in range(4):
        U[a] = u0[a]
    o = oracle.Oracle((11, 13), (0.1, 0.1), (("outflow", "outflow"),) * 2, R=2, flux="hll")
    assert np.abs(o.rhs(U)).max() == 0.0
    U1, m = W.four_quadrant(24, seed=3, ny=20)
    o = oracle.Oracle(U1.shape[1:], m["dx"], m["bc"], R=2, flux="hll")
    Um = U1[:, :, ::-1].copy()
    Um[1] = -Um[1]
    r, rm = o.rhs(U1), o.rhs(Um)
    rm = rm[:, :, ::-1]
    rm[1] = -rm[1]
    np.testing.assert_allclose(rm, r, rtol=0, atol=1e-12 * np.abs(r).max())
    errs = []
    for n in (50, 100):
        Ug, m = W.gaussian_1d(n)
        oo = oracle.Oracle((n,), m["dx"], m["bc"], R=2, ell_over_dx=0.1 * n, gamma=m["gamma"], flux="hll")
        dx = m["dx"][0]
        dt = 0.4 * dx / 2.3 * (dx / (1.0 / 25)) ** (5 / 3.0 - 1.0)
        steps = int(math.ceil(1.0 / dt))
        Un = oo.run(Ug, 1.0 / steps, steps)
        Ue, _ = W.gaussian_1d(n, t=1.0)
        errs.append(np.abs(Un[0] - Ue[0]).mean())
    tab = _table1()
    order = math.log(errs[0] / errs[1], 2)
    assert abs(order - tab[100][4]) < 0.5, (errs, order)


# ---------------------------------------------------------------------------
# Variants: non-zero-mean smoothness indicators and the polynomial-candidate hybrid

@pytest.mark.parametrize("R", [1, 2, 3])
def test_nonzero_mean_beta_is_shift_invariant(R):
    """With beta on (f_m - f_i) the nonlinear weights ignore a constant shift of the data, so
    q(f + c) - q(f) = c sum_m omega_m sum_j w_mj is exactly linear in c; with the zero-mean beta
    of the paper it is not.  Constant data give beta = 0, omega = gamma / sum(gamma); next to a
    jump the flat sub-stencil has beta = 0 exactly and takes all the weight."""
    o = _oracle_1d(R, 12.0, beta_mean=True)
    oz = _oracle_1d(R, 12.0)
    t = o.tables
    rng = np.random.default_rng(3 + R)
    f = rng.normal(size=2 * R + 1)
    d1 = o.gp_weno(f + 0.7) - o.gp_weno(f)
    d2 = o.gp_weno(f + 1.4) - o.gp_weno(f)
    assert abs(d2 - 2.0 * d1) < 1e-12
    z1 = oz.gp_weno(f + 0.7) - oz.gp_weno(f)
    z2 = oz.gp_weno(f + 1.4) - oz.gp_weno(f)
    assert abs(z2 - 2.0 * z1) > 1e-6
    s_m = np.array([t["wl"][m].sum() for m in range(R + 1)])
    qc = o.gp_weno(np.full(2 * R + 1, 2.0))
    assert abs(qc - 2.0 * (t["gl"] * s_m).sum() / t["gl"].sum()) < 1e-14
    g = np.ones(2 * R + 1)
    g[R + 1:] = 2.0
    assert abs(o.gp_weno(g) - s_m[0]) < 1e-12


def test_poly_candidates_are_lagrange():
    """The hybrid's candidate weights are Lagrange interpolation weights and its linear weights
    the classical ones (1/16, 10/16, 5/16 for R=2): exact, not a limit."""
    from fractions import Fraction
    from oracle import gp_tables
    t = gp_tables.tables(2, 12.0, 3.0, 0.5, poly=True)
    np.testing.assert_allclose(t["gamma"], [1 / 16, 10 / 16, 5 / 16], rtol=1e-15)
    np.testing.assert_allclose(t["w_sub"][0], [3 / 8, -5 / 4, 15 / 8], rtol=1e-15)
    np.testing.assert_allclose(t["w_big"], [3 / 128, -5 / 32, 45 / 64, 15 / 32, -5 / 128], rtol=1e-15)
    res = t["M"] @ t["gamma"] - t["w_big"]
    assert np.abs(res).max() < 1e-15


def test_poly_hybrid_convergence():
    """Polynomial candidates with GP smoothness indicators keep the (2R+1)th order on smooth
    advection (R=2: 4.5 between 100 and 200 cells; the GP candidates give 4.8 there)."""
    errs = []
    for n in (100, 200):
        Ug, m = W.gaussian_1d(n)
        oo = oracle.Oracle((n,), m["dx"], m["bc"], R=2, ell_over_dx=0.1 * n, gamma=m["gamma"], candidates="poly")
        dx = m["dx"][0]
        dt = 0.4 * dx / 2.3 * (dx / (1.0 / 25)) ** (5 / 3.0 - 1.0)
        steps = int(math.ceil(1.0 / dt))
        Un = oo.run(Ug, 1.0 / steps, steps)
        Ue, _ = W.gaussian_1d(n, t=1.0)
        errs.append(np.abs(Un[0] - Ue[0]).mean())
    order = math.log(errs[0] / errs[1], 2)
    assert order > 4.2, (errs, order)


def test_nonzero_mean_removes_square_wave_overshoot():
    """Section 7.1's scalar-advection discussion: with the zero mean the GP smoothness
    indicators favour data near zero, so a flat square wave overshoots at its edges;
    beta on f - f_centre removes the overshoot and is more diffusive (larger L1).
    Density square wave (1 and 2) advected once around a periodic 200-cell domain at
    u = p = 1, R = 2, l/dx = 12, CFL 0.4."""
    n = 200
    x = (np.arange(n) + 0.5) / n
    rho = np.where((x > 0.25) & (x < 0.75), 2.0, 1.0)
    U0 = W.conserved(rho, [np.ones(n)], np.ones(n), 1.4)
    res = {}
    for mean in (False, True):
        o = oracle.Oracle((n,), (1.0 / n,), (("periodic", "periodic"),), R=2, ell_over_dx=12.0, beta_mean=mean)
        dt = 0.4 / o.max_rate(U0)
        steps = int(math.ceil(1.0 / dt))
        r = o.run(U0, 1.0 / steps, steps)[0]
        res[mean] = (r.max() - 2.0, 1.0 - r.min(), np.abs(r - rho).mean())
    assert res[False][0] > 0.02                        # several percent of the jump
    assert res[True][0] < 1e-3 and res[True][1] < 1e-3
    assert res[True][2] > res[False][2]                # the price: more diffusion
