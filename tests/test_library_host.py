"""Host-side checks of the CUDA library that need no GPU: it builds, loads,
exports every function include/gpweno.h declares, its double-double GP
precompute agrees with the oracle's independent 100-digit tables, and its
argument checks reject bad plans before touching a device."""
import numpy as np
import pytest

import oracle
from oracle import gp_tables as OT
from paper_1808_04960_gb300 import build as libbuild
from paper_1808_04960_gb300 import gpweno


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return gpweno.load()


def test_exports_every_declared_symbol(lib):
    names = gpweno.header_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("R,ell,sigma", [(1, 12.0, 3.0), (2, 12.0, 3.0), (3, 12.0, 3.0), (2, 6.0, 1.5),
                                         (3, 24.0, 3.0), (1, 24.0, 24.0), (2, 12.0, 12.0), (3, 6.0, 3.0)])
def test_dd_tables_match_oracle(lib, R, ell, sigma):
    """Two independent precomputes (double-double Cholesky/Jacobi in C++ and 100-digit
    decimal Gauss/Jacobi in Python) agree to near FP64 rounding."""
    t = gpweno.gp_tables(R, ell, sigma)
    ol = OT.tables(R, ell, sigma, 0.5)
    orr = OT.tables(R, ell, sigma, -0.5)
    tol = 1e-13
    np.testing.assert_allclose(t["w_sub"], ol["w_sub"], rtol=0, atol=tol * np.abs(ol["w_sub"]).max())
    np.testing.assert_allclose(t["w_big"], ol["w_big"], rtol=0, atol=tol * np.abs(ol["w_big"]).max())
    np.testing.assert_allclose(t["gamma"], ol["gamma"], rtol=tol, atol=0)
    np.testing.assert_allclose(t["w_sub_r"], orr["w_sub"], rtol=0, atol=tol * np.abs(orr["w_sub"]).max())
    np.testing.assert_allclose(t["gamma_r"], orr["gamma"], rtol=tol, atol=0)
    # P^T P = K_m(sigma)^{-1}, whatever the eigenvector signs
    PtP = t["P"].T @ t["P"]
    np.testing.assert_allclose(PtP, ol["Kinv_sigma"], rtol=0, atol=1e-12 * np.abs(ol["Kinv_sigma"]).max())
    # rows of P are orthogonal directions scaled by 1/sqrt(lambda), ascending lambda
    lam = 1.0 / np.sum(t["P"] ** 2, axis=1)
    np.testing.assert_allclose(lam, ol["lam_sigma"], rtol=1e-12)


def test_dd_tables_flat_limit(lib):
    t = gpweno.gp_tables(2, 1000.0, 3.0)
    np.testing.assert_allclose(t["gamma"], [1 / 16, 10 / 16, 5 / 16], atol=1e-5)


@pytest.mark.parametrize("args,status", [((0, 12.0, 3.0), gpweno.ERR_ARG), ((4, 12.0, 3.0), gpweno.ERR_ARG),
                                         ((2, 0.5, 3.0), gpweno.ERR_ARG), ((2, 12.0, 1.0), gpweno.ERR_ARG),
                                         ((3, 1000.0, 3.0), gpweno.ERR_PRECOMPUTE)])
def test_precompute_rejects(lib, args, status):
    with pytest.raises(gpweno.GpwenoError) as e:
        gpweno.gp_tables(*args)
    assert e.value.status == status


def test_plan_argument_checks_before_device(lib):
    """Invalid plans are refused with GPWENO_ERR_ARG before any CUDA call."""
    bad = [
        dict(R=2, ell_over_dx=12.0, shape=(16, 16), dx=(0.1, 0.1), bc=(("periodic", "outflow"),) * 2),
        dict(R=2, ell_over_dx=12.0, shape=(16, 16), dx=(0.1, -0.1), bc=(("periodic", "periodic"),) * 2),
        dict(R=5, ell_over_dx=12.0, shape=(16, 16), dx=(0.1, 0.1), bc=(("periodic", "periodic"),) * 2),
        dict(R=2, ell_over_dx=12.0, shape=(16, 16), dx=(0.1, 0.1), bc=(("periodic", "periodic"),) * 2, p=3),
        dict(R=2, ell_over_dx=12.0, shape=(16, 16), dx=(0.1, 0.1), bc=(("periodic", "periodic"),) * 2, gamma=1.0),
        dict(R=2, ell_over_dx=12.0, shape=(16, 16), dx=(0.1, 0.1), bc=(("periodic", "periodic"),) * 2,
             eps=1e-40),
        # an empty dimension, and a grid beyond the 2^31-cell limit
        dict(R=2, ell_over_dx=12.0, shape=(0, 16), dx=(0.1, 0.1), bc=(("periodic", "periodic"),) * 2),
        dict(R=2, ell_over_dx=12.0, shape=(65536, 32769), dx=(0.1, 0.1), bc=(("periodic", "periodic"),) * 2),
    ]
    for kw in bad:
        with pytest.raises(gpweno.GpwenoError) as e:
            gpweno.Plan(**kw)
        assert e.value.status == gpweno.ERR_ARG, kw


def test_batch_needs_plans(lib):
    with pytest.raises(gpweno.GpwenoError):
        gpweno.BatchPlan([])


@pytest.mark.parametrize("R", [1, 2, 3])
def test_dd_poly_tables_match_oracle(lib, R):
    """Polynomial (Lagrange) candidates: the library's tables agree with the oracle's
    100-digit ones, and at R = 2 the linear weights are the classical 1/16, 10/16, 5/16."""
    t = gpweno.gp_tables(R, 12.0, 3.0, candidates="poly")
    ol = OT.tables(R, 12.0, 3.0, 0.5, poly=True)
    orr = OT.tables(R, 12.0, 3.0, -0.5, poly=True)
    np.testing.assert_allclose(t["w_sub"], ol["w_sub"], rtol=0, atol=1e-14 * np.abs(ol["w_sub"]).max())
    np.testing.assert_allclose(t["w_big"], ol["w_big"], rtol=0, atol=1e-14 * np.abs(ol["w_big"]).max())
    np.testing.assert_allclose(t["gamma"], ol["gamma"], rtol=1e-14, atol=0)
    np.testing.assert_allclose(t["w_sub_r"], orr["w_sub"], rtol=0, atol=1e-14 * np.abs(orr["w_sub"]).max())
    np.testing.assert_allclose(t["gamma_r"], orr["gamma"], rtol=1e-14, atol=0)
    if R == 2:
        np.testing.assert_allclose(t["gamma"], [1 / 16, 10 / 16, 5 / 16], rtol=1e-15)
    # the smoothness-indicator tables do not depend on the candidates
    g = gpweno.gp_tables(R, 12.0, 3.0)
    np.testing.assert_array_equal(t["P"], g["P"])


def test_variant_options_checked(lib):
    """beta_mean, candidates, scheme and ao outside {0, 1}, FD-Flux with a face solver, GP-AO with
    FD-Flux, and gamma_HI outside (0, 1) are refused by the C ABI before any device work."""
    import ctypes
    with pytest.raises(gpweno.GpwenoError) as e:
        gpweno._check(lib.gpweno_gp_tables(2, 12.0, 3.0, 2, 0, None, None, None, None, None, None), "gp_tables")
    assert e.value.status == gpweno.ERR_ARG
    with pytest.raises(gpweno.GpwenoError) as e:
        gpweno._check(lib.gpweno_gp_tables(2, 12.0, 3.0, 0, 2, None, None, None, None, None, None), "gp_tables")
    assert e.value.status == gpweno.ERR_ARG
    dims = gpweno.Dims()
    dims.ndim = 2
    for a in range(3):
        dims.n[a] = 16 if a < 2 else 1
        dims.dx[a] = 0.1
        dims.bc_lo[a] = dims.bc_hi[a] = 0
    for field, val in (("beta_mean", 3), ("candidates", 3), ("scheme", 2), ("flux_form", 3), ("scheme+flux", 1),
                       ("ao", 2), ("ao+scheme", 1), ("ao_gamma", 1.0)):
        o = gpweno.Opts()
        lib.gpweno_default_opts(ctypes.byref(o))
        if field == "scheme+flux":
            o.scheme, o.flux_form = 1, 1
        elif field == "ao+scheme":
            o.ao, o.scheme = 1, 1
        elif field == "ao_gamma":
            o.ao, o.ao_gamma_hi = 1, 1.0
        else:
            setattr(o, field, val)
        h = ctypes.c_void_p()
        st = lib.gpweno_plan_create(ctypes.byref(h), 2, 12.0, ctypes.byref(dims), 1.4, ctypes.byref(o))
        assert st == gpweno.ERR_ARG and not h.value, field


@pytest.mark.parametrize("R,ell", [(1, 12.0), (2, 12.0), (3, 12.0), (2, 4.0), (3, 24.0), (2, 1.5)])
def test_dd_recon_tables_match_oracle(lib, R, ell):
    """Reconstruction weights (FD-Flux): the library's power series of the cell-averaged kernel
    in double-double against the oracle's 100-digit erf closed form."""
    t = gpweno.gp_tables(R, ell, 3.0, scheme="fdflux")
    ol = OT.tables(R, ell, 3.0, 0.5, recon=True)
    orr = OT.tables(R, ell, 3.0, -0.5, recon=True)
    tol = 1e-13
    np.testing.assert_allclose(t["w_sub"], ol["w_sub"], rtol=0, atol=tol * np.abs(ol["w_sub"]).max())
    np.testing.assert_allclose(t["w_big"], ol["w_big"], rtol=0, atol=tol * np.abs(ol["w_big"]).max())
    np.testing.assert_allclose(t["gamma"], ol["gamma"], rtol=tol, atol=0)
    np.testing.assert_allclose(t["w_sub_r"], orr["w_sub"], rtol=0, atol=tol * np.abs(orr["w_sub"]).max())
    np.testing.assert_allclose(t["gamma_r"], orr["gamma"], rtol=tol, atol=0)
    tp = gpweno.gp_tables(R, ell, 3.0, candidates="poly", scheme="fdflux")
    op = OT.tables(R, ell, 3.0, 0.5, poly=True, recon=True)
    np.testing.assert_allclose(tp["w_sub"], op["w_sub"], rtol=0, atol=1e-15 * np.abs(op["w_sub"]).max())
    np.testing.assert_allclose(tp["gamma"], op["gamma"], rtol=1e-14, atol=0)


@pytest.mark.parametrize("R,ell", [(2, 12.0), (3, 12.0), (3, 6.0)])
def test_dd_ao_tables_match_oracle(lib, R, ell):
    """GP-AO tables: the library's double-double weights of the three stencil sizes and the
    K_N(sigma) factors (P^T P = K_N^-1 / 1^T K_N^-1 1) against the oracle's 100-digit ones."""
    t = gpweno.ao_tables(R, ell, 3.0)
    for side, xs in ((0, 0.5), (1, -0.5)):
        o = OT.ao_tables(R, ell, 3.0, xs)
        np.testing.assert_allclose(t["w_hi"][side], o["w_hi"], rtol=0, atol=1e-13 * np.abs(o["w_hi"]).max())
        np.testing.assert_allclose(t["w_3"][side], o["w_3"], rtol=0, atol=1e-13 * np.abs(o["w_3"]).max())
        if R == 3:
            np.testing.assert_allclose(t["w_lo"][side], o["w_lo"], rtol=0, atol=1e-13 * np.abs(o["w_lo"]).max())
    o = OT.ao_tables(R, ell, 3.0, 0.5)
    keys = ("hi", "lo", "3") if R == 3 else ("hi", "3")
    dec = OT._ao_decimal(R, str(OT._D(ell)), str(OT._D(3.0)), str(OT._D(0.5)))
    for k in keys:
        P = t["P_" + k]
        # the factors of the size-normalised indicator: P^T P = K_N^-1 / (1^T K_N^-1 1), the sum
        # taken in the oracle's decimal arithmetic (its entries cancel)
        one = float(sum(sum(row) for row in dec["Kinv_" + k]))
        Kn = o["Kinv_" + k] / one
        np.testing.assert_allclose(P.T @ P, Kn, rtol=0, atol=1e-11 * np.abs(Kn).max())
    with pytest.raises(gpweno.GpwenoError):
        gpweno.ao_tables(1, 12.0, 3.0)
