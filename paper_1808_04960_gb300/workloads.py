"""Seeded synthetic initial data for the Euler workloads.

This module only builds initial conditions (primitive -> conserved
variables of an ideal gas).  It holds none of the GP-WENO method's
arithmetic, and both the CUDA path's tests/bench and the CPU oracle take
their inputs from here.

Every function returns ``(U, meta)`` where ``U`` is a float64 numpy array in
structure-of-arrays layout ``[nc, (nz,) (ny,) nx]`` with components
(rho, rho*u_1, ..., rho*u_ndim, E), and ``meta`` holds the grid spacing in
(x, y, z) order, the boundary conditions as (lo, hi) pairs in (x, y, z)
order, and the problem's constants.

Problems (shapes and distributions of the paper's test problems):
  sod_1d               Sod shock tube (Section 7.2 family of 1D shock tubes)
  gaussian_1d          smooth density advection, Section 6.1
  isentropic_vortex    Shu's isentropic vortex, Section 6.2 (periodic square)
  four_quadrant        2D four-state Riemann problem with seeded states (Section 7.5 family)
  shock_turbulence_3d  Mach-3 shock into a seeded multi-mode density field
  smooth_field         seeded smooth periodic field, every primitive varying at O(amp)
  batch_instances      list of seeded 2D instances of uneven size, R and l/Delta
"""
from __future__ import annotations

import math

import numpy as np


def conserved(rho, vel, p, gamma):
    """(rho, velocity components, p) -> conserved state array."""
    rho = np.asarray(rho, dtype=np.float64)
    comps = [rho]
    ke = np.zeros_like(rho)
    for v in vel:
        v = np.broadcast_to(np.asarray(v, dtype=np.float64), rho.shape)
        comps.append(rho * v)
        ke = ke + v * v
    E = np.asarray(p, dtype=np.float64) / (gamma - 1.0) + 0.5 * rho * ke
    comps.append(np.broadcast_to(E, rho.shape))
    return np.ascontiguousarray(np.stack(comps))


def primitive(U, gamma):
    """Inverse of ``conserved``: returns (rho, [velocities], p)."""
    rho = U[0]
    vel = [U[a] / rho for a in range(1, U.shape[0] - 1)]
    ke = sum(v * v for v in vel)
    p = (gamma - 1.0) * (U[-1] - 0.5 * rho * ke)
    return rho, vel, p


def _centres(n, lo, hi):
    dx = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * dx, dx


def sod_1d(n=256, gamma=1.4):
    x, dx = _centres(n, 0.0, 1.0)
    left = x < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    U = conserved(rho, [np.zeros(n)], p, gamma)
    return U, dict(dx=(dx,), bc=(("outflow", "outflow"),), gamma=gamma, x=x, t_final=0.2, cfl=0.4)


def gaussian_1d(n=100, gamma=5.0 / 3.0, t=0.0):
    """rho = 1 + exp(-100 (x - x0)^2), u = 1, p = 1/gamma on periodic [0,1]; exact at time t is a shift."""
    x, dx = _centres(n, 0.0, 1.0)
    xs = np.mod(x - t, 1.0)
    # distance on the periodic unit interval to x0 = 0.5 (profile is negligible at the seam)
    rho = 1.0 + np.exp(-100.0 * (xs - 0.5) ** 2)
    U = conserved(rho, [np.ones(n)], np.full(n, 1.0 / gamma), gamma)
    return U, dict(dx=(dx,), bc=(("periodic", "periodic"),), gamma=gamma, x=x)


def isentropic_vortex(n=128, half_width=5.0, beta=5.0, gamma=1.4, t=0.0, ny=None, u0=1.0, v0=1.0):
    """Isentropic vortex on the periodic square [-L, L]^2 with free stream
    rho = 1, (u, v) = (u0, v0), p = 1; exact solution at time t is the initial
    field shifted by (u0 t, v0 t) (periodic images are ignored, the
    perturbation is ~exp(-L^2) at the seam)."""
    nx = int(n)
    ny = nx if ny is None else int(ny)
    L = float(half_width)
    x, dx = _centres(nx, -L, L)
    y, dy = _centres(ny, -L, L)
    X, Y = np.meshgrid(x, y)  # [ny, nx]
    Xs = np.mod(X - u0 * t + L, 2 * L) - L
    Ys = np.mod(Y - v0 * t + L, 2 * L) - L
    r2 = Xs * Xs + Ys * Ys
    dT = -(gamma - 1.0) * beta * beta / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)
    amp = beta / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    u = u0 - amp * Ys
    v = v0 + amp * Xs
    T = 1.0 + dT
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    U = conserved(rho, [u, v], p, gamma)
    return U, dict(dx=(dx, dy), bc=(("periodic", "periodic"), ("periodic", "periodic")),
                   gamma=gamma, period=2 * L / u0 if u0 else None)


def four_quadrant_states(seed=3):
    """Four seeded quadrant states (rho, u, v, p): rho~U[0.1,1.5], u,v~U[-1,1], p~U[0.03,1.5]."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.1, 1.5, 4)
    u = rng.uniform(-1.0, 1.0, 4)
    v = rng.uniform(-1.0, 1.0, 4)
    p = rng.uniform(0.03, 1.5, 4)
    return np.stack([rho, u, v, p], axis=1)


def four_quadrant(n=256, seed=3, gamma=1.4, ny=None):
    """Four constant states meeting at (0.5, 0.5) on [0,1]^2 with outflow boundaries.
    Quadrant q = 0: x>=0.5,y>=0.5; 1: x<0.5,y>=0.5; 2: x<0.5,y<0.5; 3: x>=0.5,y<0.5."""
    nx = int(n)
    ny = nx if ny is None else int(ny)
    x, dx = _centres(nx, 0.0, 1.0)
    y, dy = _centres(ny, 0.0, 1.0)
    X, Y = np.meshgrid(x, y)
    st = four_quadrant_states(seed)
    q = np.where(Y >= 0.5, np.where(X >= 0.5, 0, 1), np.where(X < 0.5, 2, 3))
    rho, u, v, p = (st[q, k] for k in range(4))
    U = conserved(rho, [u, v], p, gamma)
    return U, dict(dx=(dx, dy), bc=(("outflow", "outflow"), ("outflow", "outflow")), gamma=gamma,
                   states=st, cfl=0.4)


def shock_turbulence_3d(n=64, seed=4, gamma=1.4, mach=3.0, nmodes=32, kmax=8, rms=0.1):
    """Mach-`mach` planar shock at x = 0.25 moving in +x into rho = 1 + d rho, u = 0, p = 1,
    with d rho a sum of `nmodes` seeded Fourier modes (integer wave vectors |k| <= kmax,
    phases U[0, 2 pi), amplitudes ~ |k|^(-5/3)) scaled to RMS `rms`.  Periodic in y, z;
    zero-gradient in x (the post-shock inflow is supersonic, so it is held)."""
    rng = np.random.default_rng(seed)
    ks = []
    while len(ks) < nmodes:
        k = rng.integers(-kmax, kmax + 1, 3)
        if 0 < np.dot(k, k) <= kmax * kmax:
            ks.append(k)
    ks = np.array(ks, dtype=np.float64)
    phase = rng.uniform(0.0, 2.0 * math.pi, nmodes)
    amp = np.linalg.norm(ks, axis=1) ** (-5.0 / 3.0)
    x, dx = _centres(n, 0.0, 1.0)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    drho = np.zeros_like(X)
    for k, ph, a in zip(ks, phase, amp):
        drho += a * np.cos(2.0 * math.pi * (k[0] * X + k[1] * Y + k[2] * Z) + ph)
    drho *= rms / np.sqrt(np.mean(drho ** 2))
    # Rankine-Hugoniot for a shock of Mach M into gas at rest with rho1 = 1, p1 = 1
    g, M = gamma, mach
    c1 = math.sqrt(g)
    rho2 = (g + 1) * M * M / ((g - 1) * M * M + 2)
    p2 = 1.0 + 2 * g / (g + 1) * (M * M - 1)
    u2 = M * c1 * (1.0 - 1.0 / rho2)
    post = X < 0.25
    rho = np.where(post, rho2, 1.0 + drho)
    u = np.where(post, u2, 0.0)
    p = np.where(post, p2, 1.0)
    zero = np.zeros_like(X)
    U = conserved(rho, [u, zero, zero], p, gamma)
    return U, dict(dx=(dx, dx, dx),
                   bc=(("outflow", "outflow"), ("periodic", "periodic"), ("periodic", "periodic")),
                   gamma=gamma, cfl=0.4, post=(rho2, u2, p2))


def smooth_field(shape, seed=0, amp=0.2, nmodes=3, gamma=1.4):
    """Seeded smooth periodic field on the unit box: each primitive (rho, u..., p)
    is a base value plus `nmodes` random Fourier modes (wave numbers 1..3 per
    axis, amplitude amp/nmodes each), so that no characteristic field is constant.
    ``shape`` is the grid in array order ((nx,), (ny, nx) or (nz, ny, nx))."""
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    rng = np.random.default_rng(seed)
    axes = [_centres(n, 0.0, 1.0) for n in reversed(shape)]      # x, y, z
    grids = np.meshgrid(*[a[0] for a in reversed(axes)], indexing="ij")[::-1]   # X, Y, Z in array shape
    base = [1.0] + [0.3] * nd + [1.0]
    prims = []
    for b in base:
        f = np.full(shape, b)
        for _ in range(nmodes):
            k = rng.integers(1, 4, nd)
            ph = rng.uniform(0.0, 2.0 * math.pi)
            arg = sum(2.0 * math.pi * k[d] * grids[d] for d in range(nd)) + ph
            f = f + (amp / nmodes) * np.sin(arg)
        prims.append(f)
    U = conserved(prims[0], prims[1:1 + nd], prims[-1], gamma)
    dx = tuple(a[1] for a in axes)
    return U, dict(dx=dx, bc=(("periodic", "periodic"),) * nd, gamma=gamma)


def batch_instances(count=256, seed=5, nmin=64, nmax=1024, gamma=1.4):
    """Seeded list of 2D instances: n_x, n_y log-uniform on [nmin, nmax], R in {1,2,3},
    l/Delta in {6,12,24}, half four-quadrant and half vortex (beta ~ U[2,6])."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        nx = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        ny = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        R = int(rng.integers(1, 4))
        ell = float(rng.choice([6.0, 12.0, 24.0]))
        if k % 2 == 0:
            U, meta = four_quadrant(nx, seed=int(rng.integers(0, 2 ** 31)), gamma=gamma, ny=ny)
        else:
            beta = float(rng.uniform(2.0, 6.0))
            U, meta = isentropic_vortex(nx, beta=beta, gamma=gamma, ny=ny)
        out.append(dict(U=U, meta=meta, R=R, ell_over_dx=ell, nx=nx, ny=ny))
    return out
