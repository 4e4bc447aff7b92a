"""Python binding of the C ABI in include/gpweno.h (ctypes; argument marshalling only).

Every step of the numerical path runs in the CUDA library ``libgpweno.so``;
this module only checks tensor shapes/dtypes/devices, passes raw pointers and
the current CUDA stream, and turns status codes into exceptions.  PyTorch is
used for device memory and streams.  There is no CPU fallback: if the
library is missing, importing the functions raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgpweno.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "gpweno.h")

OK, ERR_ARG, ERR_PRECOMPUTE, ERR_CUDA, ERR_NONPHYSICAL, ERR_TIMEOUT = range(6)
F32, F64 = 0, 1
PERIODIC, OUTFLOW, EXTERNAL = 0, 1, 2


class GpwenoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"gpweno status {status}: {msg}")
        self.status = status


class Dims(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("dx", ctypes.c_double * 3),
                ("bc_lo", ctypes.c_int * 3), ("bc_hi", ctypes.c_int * 3)]


class Opts(ctypes.Structure):
    _fields_ = [("sigma_over_dx", ctypes.c_double), ("eps", ctypes.c_double), ("p", ctypes.c_int),
                ("dtype", ctypes.c_int), ("cfl", ctypes.c_double), ("flux_form", ctypes.c_int),
                ("beta_mean", ctypes.c_int), ("candidates", ctypes.c_int), ("scheme", ctypes.c_int),
                ("ao", ctypes.c_int), ("ao_gamma_hi", ctypes.c_double), ("ao_gamma_lo", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libgpweno.so (built by ``paper_1808_04960_gb300.build``).  Raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} not found: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(p)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        dp = ctypes.POINTER(ctypes.c_double)
        sigs = {
            "gpweno_default_opts": (None, [ctypes.POINTER(Opts)]),
            "gpweno_plan_create": (i, [ctypes.POINTER(vp), i, d, ctypes.POINTER(Dims), d, ctypes.POINTER(Opts)]),
            "gpweno_plan_destroy": (i, [vp]),
            "gpweno_plan_tables": (i, [vp, dp, dp, dp, dp]),
            "gpweno_gp_tables": (i, [i, d, d, i, i, dp, dp, dp, dp, dp, dp]),
            "gpweno_ao_tables": (i, [i, d, d, dp, dp, dp, dp, dp, dp]),
            "gpweno_rhs": (i, [vp, vp, vp, vp]),
            "gpweno_rk3_step": (i, [vp, vp, vp, d, vp, vp]),
            "gpweno_rk3_stage": (i, [vp, i, vp, vp, d, vp, vp]),
            "gpweno_set_halo": (i, [vp, vp, vp]),
            "gpweno_halo_pack": (i, [vp, vp, vp, vp, vp]),
            "gpweno_rates": (i, [vp, vp, vp]),
            "gpweno_rate_export": (i, [vp, vp, vp]),
            "gpweno_dt_from_rates": (i, [vp, vp, d, vp, vp]),
            "gpweno_cfl_dt": (i, [vp, vp, d, vp, vp]),
            "gpweno_flags": (i, [vp, ctypes.POINTER(ctypes.c_int)]),
            "gpweno_plan_batch": (i, [ctypes.POINTER(vp), ctypes.POINTER(vp), i, ctypes.c_char_p]),
            "gpweno_batch_rk3_step": (i, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp]),
            "gpweno_last_launch_count": (i, []),
            "gpweno_batch_info": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                                      ctypes.POINTER(i), ctypes.POINTER(ctypes.c_ulonglong)]),
            "gpweno_batch_tiles": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]),
            "gpweno_plan_schedule": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                                         ctypes.POINTER(i)]),
            "gpweno_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def header_functions(path: str = HEADER):
    """Names of the functions declared in include/gpweno.h."""
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gpweno_[a-z0-9_]+)\s*\(", src)))


def _check(status, what=""):
    if status != OK:
        msg = load().gpweno_last_error().decode(errors="replace")
        raise GpwenoError(status, f"{what}: {msg}" if what else msg)


def last_launch_count() -> int:
    return int(load().gpweno_last_launch_count())


def _dbl(n):
    return (ctypes.c_double * n)()


def gp_tables(R: int, ell_over_dx: float, sigma_over_dx: float = 3.0, candidates: str = "gp",
              scheme: str = "fdprim") -> dict:
    """The library's double-double tables, computed on the host (no device needed)."""
    import numpy as np
    S = R + 1
    wm, g, P, wb, wmr, gr = _dbl(S * S), _dbl(S), _dbl(S * S), _dbl(2 * R + 1), _dbl(S * S), _dbl(S)
    _check(load().gpweno_gp_tables(int(R), float(ell_over_dx), float(sigma_over_dx),
                                   {"gp": 0, "poly": 1}[candidates], {"fdprim": 0, "fdflux": 1}[scheme],
                                   wm, g, P, wb, wmr, gr), "gpweno_gp_tables")
    a = lambda x, shape: np.array(list(x), dtype=np.float64).reshape(shape)
    return dict(w_sub=a(wm, (S, S)), gamma=a(g, (S,)), P=a(P, (S, S)), w_big=a(wb, (2 * R + 1,)),
                w_sub_r=a(wmr, (S, S)), gamma_r=a(gr, (S,)))


def ao_tables(R: int, ell_over_dx: float, sigma_over_dx: float = 3.0) -> dict:
    """The library's double-double GP-AO tables, computed on the host (no device needed)."""
    import numpy as np
    nh, nl = 2 * R + 1, 2 * R - 1
    wh, wl, w3 = _dbl(2 * nh), _dbl(2 * nl), _dbl(18)
    Ph, Pl, P3 = _dbl(nh * nh), _dbl(nl * nl), _dbl(9)
    _check(load().gpweno_ao_tables(int(R), float(ell_over_dx), float(sigma_over_dx), wh, wl, w3, Ph, Pl, P3),
           "gpweno_ao_tables")
    a = lambda x, shape: np.array(list(x), dtype=np.float64).reshape(shape)
    out = dict(w_hi=a(wh, (2, nh)), w_3=a(w3, (2, 3, 3)), P_hi=a(Ph, (nh, nh)), P_3=a(P3, (3, 3)))
    if R == 3:
        out.update(w_lo=a(wl, (2, nl)), P_lo=a(Pl, (nl, nl)))
    return out


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _bc_code(b):
    if isinstance(b, int):
        return b
    return {"periodic": PERIODIC, "outflow": OUTFLOW, "external": EXTERNAL}[b]


class Plan:
    """A GP-WENO plan for one grid (see gpweno_plan_create).

    shape: interior grid in array order ((nx,), (ny, nx)); dx: spacing in
    (x, y) order; bc: (lo, hi) pairs in (x, y) order, 'periodic', 'outflow' or
    'external' (a slab side whose ghost layers come from a halo buffer; slowest
    dimension only, see set_halo and rk3_stage).
    """

    def __init__(self, R, ell_over_dx, shape, dx, bc, gamma=1.4, sigma_over_dx=3.0, eps=1e-36, p=2,
                 dtype="f32", cfl=0.0, flux="lf", beta_mean=False, candidates="gp", scheme="fdprim", ao=False,
                 ao_gamma_hi=0.85, ao_gamma_lo=0.85):
        import torch
        self.lib = load()
        self.shape = tuple(int(s) for s in shape)
        self.ndim = len(self.shape)
        self.nc = self.ndim + 2
        self.R = int(R)
        self.dtype = {"f32": torch.float32, "f64": torch.float64}[dtype]
        self.cfl = float(cfl)
        # creation parameters (what a checkpoint must agree with to resume on this plan)
        self.params = {"R": self.R, "ell_over_dx": float(ell_over_dx), "shape": list(self.shape),
                       "dx": [float(dx[a]) for a in range(self.ndim)],
                       "bc": [[str(bc[a][0]), str(bc[a][1])] for a in range(self.ndim)], "gamma": float(gamma),
                       "sigma_over_dx": float(sigma_over_dx), "eps": float(eps), "p": int(p), "dtype": dtype,
                       "cfl": self.cfl, "flux": flux, "beta_mean": bool(beta_mean), "candidates": candidates,
                       "scheme": scheme, "ao": bool(ao), "ao_gamma_hi": float(ao_gamma_hi),
                       "ao_gamma_lo": float(ao_gamma_lo)}
        dims = Dims()
        dims.ndim = self.ndim
        n_xyz = list(reversed(self.shape))
        for a in range(3):
            dims.n[a] = n_xyz[a] if a < self.ndim else 1
            dims.dx[a] = float(dx[a]) if a < self.ndim else 1.0
            lo, hi = bc[a] if a < self.ndim else ("outflow", "outflow")
            dims.bc_lo[a] = _bc_code(lo)
            dims.bc_hi[a] = _bc_code(hi)
        opts = Opts()
        self.lib.gpweno_default_opts(ctypes.byref(opts))
        opts.sigma_over_dx = float(sigma_over_dx)
        opts.eps = float(eps)
        opts.p = int(p)
        opts.dtype = F32 if dtype == "f32" else F64
        opts.cfl = float(cfl)
        opts.flux_form = {"lf": 0, "hllc": 1, "hll": 2}[flux]
        opts.beta_mean = 1 if beta_mean else 0
        opts.candidates = {"gp": 0, "poly": 1}[candidates]
        opts.scheme = {"fdprim": 0, "fdflux": 1}[scheme]
        opts.ao = 1 if ao else 0
        opts.ao_gamma_hi = float(ao_gamma_hi)
        opts.ao_gamma_lo = float(ao_gamma_lo)
        h = ctypes.c_void_p()
        _check(self.lib.gpweno_plan_create(ctypes.byref(h), self.R, float(ell_over_dx), ctypes.byref(dims),
                                           float(gamma), ctypes.byref(opts)), "gpweno_plan_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            self.lib.gpweno_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_state(self, U, name="U"):
        import torch
        if not isinstance(U, torch.Tensor) or not U.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if U.dtype != self.dtype or tuple(U.shape) != (self.nc,) + self.shape or not U.is_contiguous():
            raise ValueError(f"{name} must be contiguous {self.dtype} of shape {(self.nc,) + self.shape}, "
                             f"got {U.dtype} {tuple(U.shape)}")

    def empty_state(self, n=1):
        import torch
        return torch.empty((n, self.nc) + self.shape, dtype=self.dtype, device="cuda")

    def new_scratch(self):
        """Zeroed RK3 scratch of 4 state sizes (the last one is the compensation remainder)."""
        import torch
        return torch.zeros((4, self.nc) + self.shape, dtype=self.dtype, device="cuda")

    def tables(self) -> dict:
        import numpy as np
        S = self.R + 1
        wm, g, P, wb = _dbl(S * S), _dbl(S), _dbl(S * S), _dbl(2 * self.R + 1)
        _check(self.lib.gpweno_plan_tables(self.handle, wm, g, P, wb), "gpweno_plan_tables")
        a = lambda x, shape: np.array(list(x), dtype=np.float64).reshape(shape)
        return dict(w_sub=a(wm, (S, S)), gamma=a(g, (S,)), P=a(P, (S, S)), w_big=a(wb, (2 * self.R + 1,)))

    def rhs(self, U, out=None, stream=None):
        """out = L(U) (Eq. disc_fd)."""
        import torch
        self._check_state(U)
        if out is None:
            out = torch.empty_like(U)
        self._check_state(out, "out")
        _check(self.lib.gpweno_rhs(self.handle, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                   _stream_handle(stream)), "gpweno_rhs")
        return out

    def rk3_step(self, U, scratch, dt=0.0, dt_dev=None, stream=None):
        """One SSP-RK3 step in place on U.  scratch: tensor of shape (4, nc, ...) of the plan's dtype
        (see new_scratch); its last slice carries the compensation remainder between steps and must
        be zero when U is (re)initialised.
        dt_dev: optional CUDA float64 scalar tensor holding dt (updated with the CFL dt if cfl > 0)."""
        import torch
        self._check_state(U)
        if (scratch.dtype != self.dtype or tuple(scratch.shape) != (4, self.nc) + self.shape
                or not scratch.is_contiguous() or not scratch.is_cuda):
            raise ValueError("scratch must be a contiguous CUDA tensor of shape (4, nc, ...) and the plan's dtype")
        dptr = None
        if dt_dev is not None:
            if dt_dev.dtype != torch.float64 or not dt_dev.is_cuda or dt_dev.numel() != 1:
                raise ValueError("dt_dev must be a CUDA float64 tensor with one element")
            dptr = ctypes.c_void_p(dt_dev.data_ptr())
        _check(self.lib.gpweno_rk3_step(self.handle, ctypes.c_void_p(U.data_ptr()),
                                        ctypes.c_void_p(scratch.data_ptr()), float(dt), dptr,
                                        _stream_handle(stream)), "gpweno_rk3_step")
        return U

    def rk3_step_noalloc(self, U, dt, stream=None):
        """gpweno_rk3_step_noalloc: one SSP-RK3 step in place on U whose stage buffers live in the
        library's static 16 MiB device array (for callers that may not allocate device memory)."""
        self._check_state(U)
        fn = self.lib.gpweno_rk3_step_noalloc
        fn.restype = ctypes.c_int
        fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
        _check(fn(self.handle, ctypes.c_void_p(U.data_ptr()), float(dt), _stream_handle(stream)),
               "gpweno_rk3_step_noalloc")
        return U

    # ---- slab decomposition (gpweno_set_halo, gpweno_halo_pack, gpweno_rk3_stage, ...) ----

    @property
    def ghost(self) -> int:
        """G = R+3 ghost layers per side."""
        return self.R + 3

    def halo_shape(self):
        """Shape of one side's halo buffer: (nc, G) + the shape of one layer of the slowest axis."""
        return (self.nc, self.ghost) + self.shape[1:]

    def new_halo(self):
        import torch
        return torch.zeros(self.halo_shape(), dtype=self.dtype, device="cuda")

    def _check_halo(self, h, name):
        import torch
        if h is None:
            return None
        if (not isinstance(h, torch.Tensor) or not h.is_cuda or h.dtype != self.dtype
                or tuple(h.shape) != self.halo_shape() or not h.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous CUDA tensor of shape {self.halo_shape()} and the plan's dtype")
        return ctypes.c_void_p(h.data_ptr())

    def set_halo(self, recv_lo, recv_hi):
        """Register the halo buffers the kernels read for the external sides (kept referenced here)."""
        lo, hi = self._check_halo(recv_lo, "recv_lo"), self._check_halo(recv_hi, "recv_hi")
        _check(self.lib.gpweno_set_halo(self.handle, lo, hi), "gpweno_set_halo")
        self._halo = (recv_lo, recv_hi)

    def halo_pack(self, state, send_lo, send_hi, stream=None):
        """The first and last G layers of `state` along the slowest axis into send_lo / send_hi."""
        self._check_state(state, "state")
        _check(self.lib.gpweno_halo_pack(self.handle, ctypes.c_void_p(state.data_ptr()),
                                         self._check_halo(send_lo, "send_lo"), self._check_halo(send_hi, "send_hi"),
                                         _stream_handle(stream)), "gpweno_halo_pack")

    @staticmethod
    def stage_input(k, U, scratch):
        """The stencil state stage k reads (the state whose halo layers are exchanged before it)."""
        return U if k == 0 else scratch[k]

    def rk3_stage(self, k, U, scratch, dt=0.0, dt_dev=None, stream=None):
        """Stage k (0, 1, 2) of rk3_step on the same buffers."""
        import torch
        self._check_state(U)
        if (scratch.dtype != self.dtype or tuple(scratch.shape) != (4, self.nc) + self.shape
                or not scratch.is_contiguous() or not scratch.is_cuda):
            raise ValueError("scratch must be a contiguous CUDA tensor of shape (4, nc, ...) and the plan's dtype")
        dptr = None
        if dt_dev is not None:
            if dt_dev.dtype != torch.float64 or not dt_dev.is_cuda or dt_dev.numel() != 1:
                raise ValueError("dt_dev must be a CUDA float64 tensor with one element")
            dptr = ctypes.c_void_p(dt_dev.data_ptr())
        _check(self.lib.gpweno_rk3_stage(self.handle, int(k), ctypes.c_void_p(U.data_ptr()),
                                         ctypes.c_void_p(scratch.data_ptr()), float(dt), dptr,
                                         _stream_handle(stream)), "gpweno_rk3_stage")

    def rates(self, U, stream=None):
        """Accumulate the maxima of (|u_d|+c)/dx_d of U in the plan's rate buffer."""
        self._check_state(U)
        _check(self.lib.gpweno_rates(self.handle, ctypes.c_void_p(U.data_ptr()), _stream_handle(stream)),
               "gpweno_rates")

    def rate_export(self, rates, stream=None):
        """Move the plan's three rate maxima (double bit patterns) into `rates` (CUDA int64, 3)."""
        import torch
        if rates.dtype != torch.int64 or not rates.is_cuda or rates.numel() != 3 or not rates.is_contiguous():
            raise ValueError("rates must be a contiguous CUDA int64 tensor with 3 elements")
        _check(self.lib.gpweno_rate_export(self.handle, ctypes.c_void_p(rates.data_ptr()), _stream_handle(stream)),
               "gpweno_rate_export")

    def dt_from_rates(self, rates, cfl, dt_dev, stream=None):
        """dt_dev = cfl / sum_d rates[d] (rates as exported, e.g. after a max-reduction over ranks)."""
        import torch
        if rates.dtype != torch.int64 or not rates.is_cuda or rates.numel() != 3:
            raise ValueError("rates must be a CUDA int64 tensor with 3 elements")
        if dt_dev.dtype != torch.float64 or not dt_dev.is_cuda or dt_dev.numel() != 1:
            raise ValueError("dt_dev must be a CUDA float64 tensor with one element")
        _check(self.lib.gpweno_dt_from_rates(self.handle, ctypes.c_void_p(rates.data_ptr()), float(cfl),
                                             ctypes.c_void_p(dt_dev.data_ptr()), _stream_handle(stream)),
               "gpweno_dt_from_rates")

    def cfl_dt(self, U, cfl, dt_dev, stream=None):
        import torch
        self._check_state(U)
        if dt_dev.dtype != torch.float64 or not dt_dev.is_cuda or dt_dev.numel() != 1:
            raise ValueError("dt_dev must be a CUDA float64 tensor with one element")
        _check(self.lib.gpweno_cfl_dt(self.handle, ctypes.c_void_p(U.data_ptr()), float(cfl),
                                      ctypes.c_void_p(dt_dev.data_ptr()), _stream_handle(stream)), "gpweno_cfl_dt")
        return dt_dev

    def schedule(self) -> dict:
        """Schedule of the last 2D stage launch: strip width, strips, CTAs launched, resident CTAs
        per SM of the kernel build used (zeros before the first launch)."""
        v = [ctypes.c_int() for _ in range(4)]
        _check(self.lib.gpweno_plan_schedule(self.handle, *[ctypes.byref(x) for x in v]), "gpweno_plan_schedule")
        return dict(strip_width=v[0].value, strips=v[1].value, grid=v[2].value, ctas_per_sm=v[3].value)

    def flags(self) -> int:
        v = ctypes.c_int(0)
        _check(self.lib.gpweno_flags(self.handle, ctypes.byref(v)), "gpweno_flags")
        return int(v.value)


class BatchPlan:
    """Batched 2D stepping over several plans (gpweno_plan_batch)."""

    def __init__(self, plans, tune_cache=None):
        self.lib = load()
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(self.lib.gpweno_plan_batch(ctypes.byref(h), arr, len(self.plans),
                                          tune_cache.encode() if tune_cache else None), "gpweno_plan_batch")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            self.lib.gpweno_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        """Schedule of the batch: block size, CTAs per SM, CTAs per launch, segments, signature."""
        v = [ctypes.c_int() for _ in range(4)]
        sig = ctypes.c_ulonglong()
        _check(self.lib.gpweno_batch_info(self.handle, *[ctypes.byref(x) for x in v], ctypes.byref(sig)),
               "gpweno_batch_info")
        t = [ctypes.c_int() for _ in range(3)]
        _check(self.lib.gpweno_batch_tiles(self.handle, *[ctypes.byref(x) for x in t]), "gpweno_batch_tiles")
        return dict(block=v[0].value, ctas_per_sm=v[1].value, grid=v[2].value, segments=v[3].value,
                    signature=f"{sig.value:016x}", strip_width_cap=t[0].value, min_rows=t[1].value,
                    ctas_per_slot=t[2].value)

    def flags(self) -> int:
        v = ctypes.c_int(0)
        _check(self.lib.gpweno_flags(self.handle, ctypes.byref(v)), "gpweno_flags")
        return int(v.value)

    def rk3_step(self, Us, scratches, dt_dev, stream=None):
        import torch
        n = len(self.plans)
        if len(Us) != n or len(scratches) != n:
            raise ValueError("one state and one scratch tensor per instance")
        for p, U, s in zip(self.plans, Us, scratches):
            p._check_state(U)
            if tuple(s.shape) != (4, p.nc) + p.shape or s.dtype != p.dtype or not s.is_contiguous():
                raise ValueError("bad scratch tensor")
        if dt_dev.dtype != torch.float64 or dt_dev.numel() != n or not dt_dev.is_cuda:
            raise ValueError("dt_dev must be a CUDA float64 tensor with one entry per instance")
        ua = (ctypes.c_void_p * n)(*[u.data_ptr() for u in Us])
        sa = (ctypes.c_void_p * n)(*[s.data_ptr() for s in scratches])
        _check(self.lib.gpweno_batch_rk3_step(self.handle, ua, sa, ctypes.c_void_p(dt_dev.data_ptr()),
                                              _stream_handle(stream)), "gpweno_batch_rk3_step")
