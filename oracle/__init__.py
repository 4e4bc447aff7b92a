"""FP64 CPU oracle of the GP-WENO finite-difference scheme.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import, call, link or
run anything in this package.  The product path (the CUDA library and its
Python binding) never touches it, and the two share no code: the oracle has
its own arbitrary-precision table precompute (``gp_tables.py``, Python
``decimal``) and its own per-face scheme (``euler_oracle.c``, plain FP64 C).

Parity status per function (pins are in ``tests/test_oracle_*.py``):
  gp_tables.tables          pinned (flat-limit Lagrange weights, direct-solve vs
                            eigen form, moment defects, linear-weight consistency)
  euler_oracle gp_weno      pinned (equal beta => omega = gamma, step data,
                            scaling, mirror symmetry)
  euler_oracle roe/flux     pinned (Roe property of the averaged state with a
                            test-side conservative Jacobian; L R = I and
                            R diag(lambda) L = primitive Jacobian)
  corrected_flux            pinned (exact for degree-5 flux primitives)
  oracle_rhs / rk3          pinned (free-stream preservation, conservation,
                            mirror and rotation symmetry, smooth-vortex order)
  FD-Flux (face_flux_fd)    pinned (reconstruction tables: closed-form covariances
                            against quadrature, flat limit = WENO-JS reconstruction
                            coefficients, exact polynomial reconstruction; scheme:
                            free stream, conservation, mirror symmetry, order 2R+1
                            with reconstruction weights and 2 with point weights,
                            Eq. flux_2nd)
  GP-AO (gp_ao)             pinned (equal weights give the high-order GP
                            prediction; coefficients sum to one; smooth small
                            stencils win at a jump; scheme invariants; smooth order
                            above 4.3 with the size-normalised indicators, 3.4
                            with the bare data-fit term)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

from . import gp_tables

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "euler_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libeuler_oracle.so")
_LIB_OPS = os.path.join(_BUILD, "libeuler_oracle_ops.so")
_lock = threading.Lock()
_lib = None


def _compile(target, extra):
    os.makedirs(_BUILD, exist_ok=True)
    if not os.path.exists(target) or os.path.getmtime(target) < os.path.getmtime(_SRC):
        tmp = target + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math",
                               "-ffp-contract=off", *extra, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, target)
    return target


def build(force: bool = False) -> str:
    """Compile the C oracle with the host gcc (plain -O2, no fast-math), and its
    operation-counting build (-DORACLE_COUNT_OPS) beside it."""
    if force:
        for t in (_LIB, _LIB_OPS):
            if os.path.exists(t):
                os.utime(t, (0, 0))
    _compile(_LIB_OPS, ["-DORACLE_COUNT_OPS"])
    return _compile(_LIB, [])


class _Cfg(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("dx", ctypes.c_double * 3),
                ("bc_lo", ctypes.c_int * 3), ("bc_hi", ctypes.c_int * 3), ("R", ctypes.c_int),
                ("gamma", ctypes.c_double), ("eps", ctypes.c_double), ("p", ctypes.c_int),
                ("wl", ctypes.c_void_p), ("gl", ctypes.c_void_p), ("wr", ctypes.c_void_p),
                ("gr", ctypes.c_void_p), ("Kinv", ctypes.c_void_p), ("flux", ctypes.c_int),
                ("beta_mean", ctypes.c_int), ("scheme", ctypes.c_int), ("ao", ctypes.c_int),
                ("ao_gamma_hi", ctypes.c_double), ("ao_gamma_lo", ctypes.c_double), ("ao_l", ctypes.c_void_p),
                ("ao_r", ctypes.c_void_p), ("ao_kinv", ctypes.c_void_p), ("ao_const", ctypes.c_double * 3),
                ("ao_scale", ctypes.c_double * 3)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Cfg)
            dp = ctypes.c_void_p
            lib.oracle_rhs.argtypes = [P, dp, dp]
            lib.oracle_rhs.restype = ctypes.c_int
            lib.oracle_rk3_step.argtypes = [P, dp, ctypes.c_double]
            lib.oracle_rk3_step.restype = ctypes.c_int
            lib.oracle_max_rate.argtypes = [P, dp]
            lib.oracle_max_rate.restype = ctypes.c_double
            lib.oracle_face.argtypes = [P, ctypes.c_int, dp, dp, dp, dp]
            lib.oracle_face.restype = ctypes.c_int
            lib.oracle_roe.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp, dp, dp, dp]
            lib.oracle_roe.restype = ctypes.c_int
            lib.oracle_gp_weno.argtypes = [P, dp, ctypes.c_int]
            lib.oracle_gp_weno.restype = ctypes.c_double
            lib.oracle_hllc.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp, ctypes.c_double, ctypes.c_double, dp]
            lib.oracle_hllc.restype = None
            lib.oracle_hll.argtypes = lib.oracle_hllc.argtypes
            lib.oracle_hll.restype = None
            lib.oracle_corrected_flux.argtypes = [dp]
            lib.oracle_corrected_flux.restype = ctypes.c_double
            _lib = lib
    return _lib


_lib_ops = None


def _load_ops():
    """The operation-counting build: same source and arithmetic, with the tally enabled."""
    global _lib_ops
    with _lock:
        if _lib_ops is None:
            build()
            lib = ctypes.CDLL(_LIB_OPS)
            lib.oracle_rk3_step.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_void_p, ctypes.c_double]
            lib.oracle_rk3_step.restype = ctypes.c_int
            lib.oracle_ops.argtypes = [ctypes.c_int]
            lib.oracle_ops.restype = ctypes.c_ulonglong
            _lib_ops = lib
    return _lib_ops


def op_count(R=2, ndim=2, n=16, **opts):
    """Floating-point operations the oracle executes for one SSP-RK3 step (three RHS
    evaluations and the stage combinations) of a periodic smooth field on an n^ndim grid,
    counted by the -DORACLE_COUNT_OPS build (see euler_oracle.c for the counting rules)."""
    from paper_1808_04960_gb300 import workloads
    shape = (n,) * ndim
    U, meta = workloads.smooth_field(shape, seed=1)
    o = Oracle(shape, meta["dx"], meta["bc"], R=R, **opts)
    lib = _load_ops()
    lib.oracle_ops(1)
    U = np.ascontiguousarray(U, dtype=np.float64).copy()
    if lib.oracle_rk3_step(ctypes.byref(o.cfg), U.ctypes.data_as(ctypes.c_void_p), 1e-4):
        raise FloatingPointError("non-physical state in the counted step")
    return int(lib.oracle_ops(1))


def ops_per_cell_stage(R=2, ndim=2, **opts):
    """Operations per cell and RK stage, the leading term of the count: a step on n^ndim
    cells costs a n^ndim + b n^(ndim-1) (each grid line evaluates 5 faces beyond its n), so two
    grid sizes give a exactly; a third size checks that form."""
    ns = (12, 18, 24) if ndim < 3 else (8, 10, 12)
    cnt = [op_count(R, ndim, n, **opts) for n in ns]
    # solve for a, b from the first two sizes, check the third
    (n1, n2, n3), (c1, c2, c3) = ns, cnt
    d = ndim
    a = (c2 * n1 ** (d - 1) - c1 * n2 ** (d - 1)) / (n2 ** d * n1 ** (d - 1) - n1 ** d * n2 ** (d - 1))
    b = (c1 - a * n1 ** d) / n1 ** (d - 1)
    assert abs(a * n3 ** d + b * n3 ** (d - 1) - c3) < 1e-6 * c3, (ns, cnt)
    return a / 3.0


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """One configured problem: grid, boundary conditions, R, l/Delta, sigma/Delta, gas gamma.

    ``shape`` is the interior grid (nx,), (ny, nx) or (nz, ny, nx) in array
    order; ``dx`` is the spacing per axis in (x, y, z) order; ``bc`` is a
    sequence of (lo, hi) pairs in (x, y, z) order with 'periodic' or 'outflow'.
    """

    def __init__(self, shape, dx, bc, R=2, ell_over_dx=12.0, sigma_over_dx=3.0,
                 gamma=1.4, eps=1e-36, p=2, flux="lf", beta_mean=False, candidates="gp", scheme="fdprim",
                 recon_weights=None, ao=False, ao_gamma_hi=0.85, ao_gamma_lo=0.85, ao_beta="normalized"):
        """scheme "fdprim": GP-WENO Riemann states, face flux, high-order correction (Section 2,
        Del Zanna's form); "fdflux": reconstruction of the split point fluxes (Section 2,
        Shu-Osher's form) with reconstruction weights unless recon_weights=False (the naive
        point-value weights of Eq. flux_2nd, kept for the order test).
        ao: GP-AO of Appendix A instead of GP-WENO (R = 2: AO(2,3); R = 3: AO(3,2,3)), with
        beta of each stencil the data-fit term of Eq. log-like divided by that of constant data,
        (1/2) f^T K_N^-1 f / (1^T K_N^-1 1) ("normalized", the default: stencils of different
        size then agree on smooth data), the data-fit term alone ("datafit"), or the whole
        negative log-likelihood with Sigma = 1 ("loglik")."""
        self.lib = _load()
        shape = tuple(int(s) for s in shape)
        self.ndim = len(shape)
        self.shape = shape
        self.nc = self.ndim + 2
        if recon_weights is None:
            recon_weights = scheme == "fdflux"
        t = gp_tables.scheme_tables(R, ell_over_dx, sigma_over_dx, poly=(candidates == "poly"),
                                    recon=bool(recon_weights))
        self.tables = t
        self._keep = [np.ascontiguousarray(t[k], dtype=np.float64) for k in ("wl", "gl", "wr", "gr", "Kinv")]
        c = _Cfg()
        c.ndim = self.ndim
        n_xyz = list(reversed(shape)) + [1] * (3 - self.ndim)
        for a in range(3):
            c.n[a] = n_xyz[a]
            c.dx[a] = float(dx[a]) if a < self.ndim else 1.0
            lo, hi = bc[a] if a < self.ndim else ("outflow", "outflow")
            c.bc_lo[a] = 0 if lo == "periodic" else 1
            c.bc_hi[a] = 0 if hi == "periodic" else 1
        c.R = int(R)
        c.gamma = float(gamma)
        c.eps = float(eps)
        c.p = int(p)
        c.wl, c.gl, c.wr, c.gr, c.Kinv = [a.ctypes.data for a in self._keep]
        c.flux = {"lf": 0, "hllc": 1, "hll": 2}[flux]
        c.beta_mean = 1 if beta_mean else 0
        c.scheme = {"fdprim": 0, "fdflux": 1}[scheme]
        c.ao = 1 if ao else 0
        if ao:
            if scheme != "fdprim" or candidates != "gp":
                raise ValueError("GP-AO is built on the FD-Prim scheme with GP candidates")
            tl = gp_tables.ao_tables(R, ell_over_dx, sigma_over_dx, 0.5)
            tr = gp_tables.ao_tables(R, ell_over_dx, sigma_over_dx, -0.5)
            keys = ["hi", "lo", "3"] if R == 3 else ["hi", "3"]
            side = lambda t: np.concatenate([t["w_" + k].ravel() for k in keys])
            kinv = np.concatenate([tl["Kinv_" + k].ravel() for k in keys])
            self._keep += [np.ascontiguousarray(side(tl)), np.ascontiguousarray(side(tr)),
                           np.ascontiguousarray(kinv)]
            c.ao_l, c.ao_r, c.ao_kinv = [a.ctypes.data for a in self._keep[-3:]]
            c.ao_gamma_hi, c.ao_gamma_lo = float(ao_gamma_hi), float(ao_gamma_lo)
            for i, (k, n) in enumerate((("hi", 2 * R + 1), ("lo", 2 * R - 1), ("3", 3))):
                c.ao_scale[i] = 1.0
                if ao_beta == "loglik" and ("logdet_" + k) in tl:
                    c.ao_const[i] = 0.5 * n * math.log(2 * math.pi) + 0.5 * tl["logdet_" + k]
                if ao_beta == "normalized" and ("one_" + k) in tl:
                    # the data-fit term per unit of that of constant data, 1^T K_N^-1 1
                    c.ao_scale[i] = 1.0 / tl["one_" + k]
        self.cfg = c
        self.R = int(R)
        self.gamma = float(gamma)

    def _state(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        assert U.shape == (self.nc,) + self.shape, (U.shape, self.shape)
        return U

    def rhs(self, U):
        """L(U) of Eq. disc_fd; raises if a non-physical state was met."""
        U = self._state(U)
        out = np.empty_like(U)
        if self.lib.oracle_rhs(ctypes.byref(self.cfg), _ptr(U), _ptr(out)):
            raise FloatingPointError("non-physical state in oracle rhs")
        return out

    def rk3_step(self, U, dt):
        U = self._state(U).copy()
        if self.lib.oracle_rk3_step(ctypes.byref(self.cfg), _ptr(U), float(dt)):
            raise FloatingPointError("non-physical state in oracle rk3 step")
        return U

    def max_rate(self, U):
        U = self._state(U)
        return float(self.lib.oracle_max_rate(ctypes.byref(self.cfg), _ptr(U)))

    def cfl_dt(self, U, cfl):
        return cfl / self.max_rate(U)

    def run(self, U, dt, nsteps):
        U = self._state(U).copy()
        for _ in range(int(nsteps)):
            if self.lib.oracle_rk3_step(ctypes.byref(self.cfg), _ptr(U), float(dt)):
                raise FloatingPointError("non-physical state in oracle run")
        return U

    def face(self, stencil, d=0):
        """Riemann states and flux at the middle face of a (2R+2, nc) stencil along axis d (x=0)."""
        st = np.ascontiguousarray(stencil, dtype=np.float64)
        assert st.shape == (2 * self.R + 2, self.nc)
        uL = np.zeros(self.nc)
        uR = np.zeros(self.nc)
        F = np.zeros(self.nc)
        ok = self.lib.oracle_face(ctypes.byref(self.cfg), int(d), _ptr(st), _ptr(uL), _ptr(uR), _ptr(F))
        if not ok:
            raise FloatingPointError("non-physical face state")
        return uL, uR, F

    def gp_weno(self, f, right=False):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (2 * self.R + 1,)
        return float(self.lib.oracle_gp_weno(ctypes.byref(self.cfg), _ptr(f), int(bool(right))))


def roe_eigensystem(uL, uR, gamma=1.4):
    """Roe average (rho, u..., H, c) of two conserved normal-first states and the
    primitive-variable eigenvectors (Rm columns, Lm rows) at it."""
    lib = _load()
    uL = np.ascontiguousarray(uL, dtype=np.float64)
    uR = np.ascontiguousarray(uR, dtype=np.float64)
    nc = uL.shape[0]
    roe = np.zeros(nc + 1)
    Rm = np.zeros((nc, nc))
    Lm = np.zeros((nc, nc))
    if not lib.oracle_roe(nc, float(gamma), _ptr(uL), _ptr(uR), _ptr(roe), _ptr(Rm), _ptr(Lm)):
        raise FloatingPointError("non-physical Roe state")
    return roe, Rm, Lm


def hllc(uL, uR, uroe, croe, gamma=1.4):
    """HLLC flux of two conserved normal-first states (Einfeldt speeds from the given Roe values)."""
    lib = _load()
    uL = np.ascontiguousarray(uL, dtype=np.float64)
    uR = np.ascontiguousarray(uR, dtype=np.float64)
    F = np.zeros(uL.shape[0])
    lib.oracle_hllc(uL.shape[0], float(gamma), _ptr(uL), _ptr(uR), float(uroe), float(croe), _ptr(F))
    return F


def hll(uL, uR, uroe, croe, gamma=1.4):
    """HLL flux of two conserved normal-first states (Einfeldt speeds from the given Roe values)."""
    lib = _load()
    uL = np.ascontiguousarray(uL, dtype=np.float64)
    uR = np.ascontiguousarray(uR, dtype=np.float64)
    F = np.zeros(uL.shape[0])
    lib.oracle_hll(uL.shape[0], float(gamma), _ptr(uL), _ptr(uR), float(uroe), float(croe), _ptr(F))
    return F


def corrected_flux(F5):
    lib = _load()
    F5 = np.ascontiguousarray(F5, dtype=np.float64)
    assert F5.shape == (5,)
    return float(lib.oracle_corrected_flux(_ptr(F5)))
