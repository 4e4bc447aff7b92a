"""GP-WENO weight tables in arbitrary precision -- part of the test oracle.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this module;
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA library (which has
its own double-double precompute in C++).

Everything here follows the pre-simulation step of the paper's stepwise
algorithm (Section 4, step 1(a)-(d)), written as the plain definitions, with
Python's ``decimal`` module at 100 significant digits so that even the
ill-conditioned covariance systems at large l/Delta (cond K ~ 1e25 at R=3,
l/Delta=96) are solved to far below FP64 rounding.

Units: every length is in units of the grid spacing Delta, so the big stencil
S_R has points x_j = j, j = -R..R, centred on cell i (Eq. 2R1-stencil), and the
face-centre prediction point is x* = +1/2 (face i+1/2) or x* = -1/2 (face
i-1/2).

Tables returned (all numpy float64 after rounding the decimal results):
  w_big[j]      GP weights on S_R, w = K^{-1} k*            (Eqs. kmat, kstar, q-intrp)
  w_sub[m][j]   GP weights on sub-stencil S_{m+1}            (Eqs. sub-stencil, candidate_interp)
  gamma[m]      least-squares linear weights of M gamma = w  (Eqs. gamm-system, M-mat)
  Kinv_sigma    inverse of the sub-stencil covariance K_m built with sigma
                instead of l (Section 3.4); beta_m = f^T Kinv f (Eq. gp-smooth)
  eig_sigma     (lambda, V) of that covariance, for the eigen form of beta
                (Eq. beta-eigen), used only to pin the definition form.
Sub-stencil m (0-based) holds the points -R+m .. m (Eq. sub-stencil with
m_paper = m+1).

Reconstruction tables (recon=True) serve the FD-Flux form of Section 2, where
the point values F_j are read as cell averages of the function F^ whose face
values are wanted (Eqs. prim_F, design).  The GP then conditions on cell
averages: [C]_jk = covariance of the averages over cells j and k, [T]_j =
covariance of the point x* with the average over cell j, and w = C^{-1} T.
For the SE kernel (units of Delta, u = x - y):
  G1(u) = int_0^u k = sqrt(pi/2) l erf(u / (sqrt(2) l))
  G2(u) = int_0^u G1 = sqrt(pi/2) l u erf(u / (sqrt(2) l)) + l^2 (exp(-u^2/(2 l^2)) - 1)
  C(delta) = G2(delta+1) - 2 G2(delta) + G2(delta-1)     (delta = x_j - x_k)
  T_j = G1(x* - x_j + 1/2) - G1(x* - x_j - 1/2).
Polynomial reconstruction weights (recon with poly) differentiate the
Lagrange interpolant of the primitive function at the cell edges.
"""
from __future__ import annotations

import decimal
from decimal import Decimal
from functools import lru_cache

import numpy as np

PREC = 100


def _ctx():
    return decimal.Context(prec=PREC)


def _D(x) -> Decimal:
    if isinstance(x, Decimal):
        return x
    if isinstance(x, float):
        # exact binary value of the double, no rounding
        return Decimal(x)
    return Decimal(x)


def se_kernel(a: Decimal, b: Decimal, ell: Decimal) -> Decimal:
    """Squared-exponential kernel with Sigma = 1 (Eq. se; Sigma cancels, Section 3.1)."""
    with decimal.localcontext(_ctx()):
        d = a - b
        return (-(d * d) / (2 * ell * ell)).exp()


def solve(A, b):
    """Gaussian elimination with partial pivoting on decimal matrices (plain textbook algorithm)."""
    n = len(A)
    with decimal.localcontext(_ctx()):
        M = [list(map(_D, row)) + [_D(b[i])] for i, row in enumerate(A)]
        for c in range(n):
            p = max(range(c, n), key=lambda r: abs(M[r][c]))
            if M[p][c] == 0:
                raise ZeroDivisionError("singular matrix")
            M[c], M[p] = M[p], M[c]
            for r in range(c + 1, n):
                f = M[r][c] / M[c][c]
                if f != 0:
                    for k in range(c, n + 1):
                        M[r][k] -= f * M[c][k]
        x = [Decimal(0)] * n
        for r in range(n - 1, -1, -1):
            s = M[r][n]
            for k in range(r + 1, n):
                s -= M[r][k] * x[k]
            x[r] = s / M[r][r]
        return x


def inverse(A):
    n = len(A)
    cols = [solve(A, [Decimal(1) if i == j else Decimal(0) for i in range(n)]) for j in range(n)]
    return [[cols[j][i] for j in range(n)] for i in range(n)]


def least_squares(M, rhs):
    """argmin ||M g - rhs||_2 through the normal equations (M^T M) g = M^T rhs.

    At 100 digits the squared condition number of the (2R+1)x(R+1) matrix M
    (whose columns are weight vectors) costs nothing measurable."""
    rows, cols = len(M), len(M[0])
    with decimal.localcontext(_ctx()):
        MtM = [[sum((M[r][a] * M[r][b] for r in range(rows)), Decimal(0)) for b in range(cols)]
               for a in range(cols)]
        Mtr = [sum((M[r][a] * rhs[r] for r in range(rows)), Decimal(0)) for a in range(cols)]
    return solve(MtM, Mtr)


def jacobi_eigen(A, sweeps=100):
    """Cyclic Jacobi eigen-decomposition of a symmetric decimal matrix.

    Returns (lam, V) with A V[:,h] = lam[h] V[:,h], eigenvalues ascending.
    Textbook rotation formulas (Golub & Van Loan, Alg. 8.4.2)."""
    n = len(A)
    with decimal.localcontext(_ctx()):
        a = [[_D(x) for x in row] for row in A]
        v = [[Decimal(1) if i == j else Decimal(0) for j in range(n)] for i in range(n)]
        tiny = Decimal(10) ** (-(PREC - 10))
        for _ in range(sweeps):
            off = sum(a[i][j] * a[i][j] for i in range(n) for j in range(n) if i != j)
            if off.sqrt() < tiny:
                break
            for p in range(n - 1):
                for q in range(p + 1, n):
                    if a[p][q] == 0:
                        continue
                    theta = (a[q][q] - a[p][p]) / (2 * a[p][q])
                    sign = 1 if theta >= 0 else -1
                    t = sign / (abs(theta) + (theta * theta + 1).sqrt())
                    c = 1 / (t * t + 1).sqrt()
                    s = t * c
                    for k in range(n):
                        akp, akq = a[k][p], a[k][q]
                        a[k][p] = c * akp - s * akq
                        a[k][q] = s * akp + c * akq
                    for k in range(n):
                        apk, aqk = a[p][k], a[q][k]
                        a[p][k] = c * apk - s * aqk
                        a[q][k] = s * apk + c * aqk
                    for k in range(n):
                        vkp, vkq = v[k][p], v[k][q]
                        v[k][p] = c * vkp - s * vkq
                        v[k][q] = s * vkp + c * vkq
        lam = [a[i][i] for i in range(n)]
        order = sorted(range(n), key=lambda i: lam[i])
        return [lam[i] for i in order], [[v[k][i] for i in order] for k in range(n)]


def covariance(points, ell):
    """[K]_jk = K(x_j, x_k) (Eq. kmat)."""
    return [[se_kernel(a, b, ell) for b in points] for a in points]


def kstar(points, xs, ell):
    """[k*]_k = K(x*, x_k) (Eq. kstar)."""
    return [se_kernel(xs, b, ell) for b in points]


def gp_weights(points, xs, ell):
    """w = K^{-1} k*, so that the GP posterior mean at x* is w^T f (Eqs. zero-mean, q-intrp)."""
    return solve(covariance(points, ell), kstar(points, xs, ell))


def m_matrix(w_sub, R):
    """The (2R+1)x(R+1) matrix of Eq. M-mat: column n carries w_n in rows n..n+R."""
    M = [[Decimal(0)] * (R + 1) for _ in range(2 * R + 1)]
    for n in range(R + 1):
        for j in range(R + 1):
            M[n + j][n] = w_sub[n][j]
    return M


def pi_decimal():
    """pi by Machin's formula, 16 atan(1/5) - 4 atan(1/239), with the atan Taylor series."""
    with decimal.localcontext(_ctx()) as ctx:
        ctx.prec = PREC + 10

        def atan_inv(n):
            x = Decimal(1) / n
            x2 = x * x
            term, total, k = x, x, 1
            while True:
                term *= -x2
                add = term / (2 * k + 1)
                if abs(add) < Decimal(10) ** (-(PREC + 5)):
                    break
                total += add
                k += 1
            return total

        return +(16 * atan_inv(5) - 4 * atan_inv(239))


def erf_decimal(z):
    """erf(z) by its Maclaurin series 2/sqrt(pi) sum_n (-1)^n z^(2n+1) / (n! (2n+1))."""
    with decimal.localcontext(_ctx()) as ctx:
        ctx.prec = PREC + 30          # the alternating series cancels about e^(z^2)
        z = _D(z)
        z2 = z * z
        term, total, n = z, z, 0
        while True:
            n += 1
            term = -term * z2 / n
            add = term / (2 * n + 1)
            total += add
            if abs(add) < Decimal(10) ** (-(PREC + 20)) and n > 2 * z2:
                break
        return +(2 / pi_decimal().sqrt() * total)


def cell_average_cov(points, ell):
    """[C]_jk: covariance of the cell averages over cells centred at points j, k (width 1)."""
    with decimal.localcontext(_ctx()):
        rt = (pi_decimal() / 2).sqrt() * ell
        s2l = Decimal(2).sqrt() * ell

        def G2(u):
            return rt * u * erf_decimal(u / s2l) + ell * ell * ((-(u * u) / (2 * ell * ell)).exp() - 1)

        return [[G2(a - b + 1) - 2 * G2(a - b) + G2(a - b - 1) for b in points] for a in points]


def point_cell_cov(points, xs, ell):
    """[T]_j: covariance of the point value at xs with the average over the cell centred at points j."""
    with decimal.localcontext(_ctx()):
        rt = (pi_decimal() / 2).sqrt() * ell
        s2l = Decimal(2).sqrt() * ell

        def G1(u):
            return rt * erf_decimal(u / s2l)

        half = Decimal(1) / 2
        return [G1(xs - b + half) - G1(xs - b - half) for b in points]


def gp_recon_weights(points, xs, ell):
    """w = C^{-1} T: GP prediction of the point value at xs from cell averages."""
    return solve(cell_average_cov(points, ell), point_cell_cov(points, xs, ell))


def poly_recon_weights(points, xs):
    """Polynomial reconstruction at xs from cell averages on unit cells centred at points:
    the primitive P(e_m) = sum_{j<m} avg_j at the S+1 edges e_m is interpolated and
    differentiated, so w_j = sum_{m>j} L'_m(xs)."""
    with decimal.localcontext(_ctx()):
        half = Decimal(1) / 2
        edges = [points[0] - half] + [p + half for p in points]
        ne = len(edges)
        dL = []
        for m in range(ne):
            den = Decimal(1)
            for l in range(ne):
                if l != m:
                    den *= edges[m] - edges[l]
            num = Decimal(0)
            for l in range(ne):
                if l == m:
                    continue
                prod = Decimal(1)
                for q in range(ne):
                    if q != m and q != l:
                        prod *= xs - edges[q]
                num += prod
            dL.append(num / den)
        return [sum(dL[j + 1:], Decimal(0)) for j in range(len(points))]


def lagrange_weights(points, xs):
    """Lagrange basis values l_j(x*) = prod_{k != j} (x* - x_k) / (x_j - x_k) (polynomial interpolation)."""
    with decimal.localcontext(_ctx()):
        out = []
        for j, xj in enumerate(points):
            v = Decimal(1)
            for k, xk in enumerate(points):
                if k != j:
                    v *= (xs - xk) / (xj - xk)
            out.append(v)
        return out


@lru_cache(maxsize=None)
def _tables_decimal(R: int, ell_s: str, sigma_s: str, xs_s: str, poly: bool = False, recon: bool = False):
    ell, sigma, xs = Decimal(ell_s), Decimal(sigma_s), Decimal(xs_s)
    big = [Decimal(j) for j in range(-R, R + 1)]
    if recon:
        weights = poly_recon_weights if poly else (lambda pts, x: gp_recon_weights(pts, x, ell))
    else:
        weights = lagrange_weights if poly else (lambda pts, x: gp_weights(pts, x, ell))
    w_big = weights(big, xs)
    w_sub = []
    for m in range(R + 1):
        pts = [Decimal(j) for j in range(-R + m, m + 1)]
        w_sub.append(weights(pts, xs))
    M = m_matrix(w_sub, R)
    gam = least_squares(M, w_big)
    # smoothness-indicator covariance: any sub-stencil (they are all identical, Eq. beta-eigen text)
    pts0 = [Decimal(j) for j in range(R + 1)]
    Ks = covariance(pts0, sigma)
    Kinv = inverse(Ks)
    lam, V = jacobi_eigen(Ks)
    return dict(w_big=w_big, w_sub=w_sub, gamma=gam, M=M, K_sigma=Ks, Kinv_sigma=Kinv,
                lam_sigma=lam, V_sigma=V, K_ell=covariance(big, ell))


def tables_decimal(R: int, ell_over_dx, sigma_over_dx, xstar, poly=False, recon=False):
    """Decimal tables (see module docstring) for one prediction point x* in units of Delta.
    poly=True: polynomial (Lagrange) candidate and big-stencil weights instead of the GP
    weights -- the WENO-GP hybrid of the paper's WENO-JS comparison (GP smoothness
    indicators on polynomial candidates); the linear weights then solve Eq. gamm-system
    for those weights.  recon=True: weights that predict the point value from cell
    averages (FD-Flux, Section 2); the smoothness-indicator tables are unchanged."""
    return _tables_decimal(int(R), str(_D(ell_over_dx)), str(_D(sigma_over_dx)), str(_D(xstar)), bool(poly),
                           bool(recon))


def _f64(x):
    if isinstance(x, list):
        return np.array([_f64(v) for v in x], dtype=np.float64)
    return float(x)


def tables(R: int, ell_over_dx: float, sigma_over_dx: float = 3.0, xstar: float = 0.5, poly: bool = False,
           recon: bool = False) -> dict:
    """The same tables rounded to float64 numpy arrays."""
    t = tables_decimal(R, ell_over_dx, sigma_over_dx, xstar, poly, recon)
    out = {k: _f64(v) for k, v in t.items()}
    out["R"] = int(R)
    return out


def scheme_tables(R: int, ell_over_dx: float, sigma_over_dx: float = 3.0, poly: bool = False,
                  recon: bool = False) -> dict:
    """Everything the per-face oracle needs: left-state tables (x* = +1/2 from
    the stencil of cell i), right-state tables (x* = -1/2 from the stencil of
    cell i+1, computed directly, not by reversal) and K_m(sigma)^{-1}."""
    tl = tables(R, ell_over_dx, sigma_over_dx, 0.5, poly, recon)
    tr = tables(R, ell_over_dx, sigma_over_dx, -0.5, poly, recon)
    return dict(R=int(R), wl=tl["w_sub"], gl=tl["gamma"], wr=tr["w_sub"], gr=tr["gamma"],
                Kinv=tl["Kinv_sigma"], w_big_l=tl["w_big"], w_big_r=tr["w_big"])


@lru_cache(maxsize=None)
def _ao_decimal(R: int, ell_s: str, sigma_s: str, xs_s: str):
    ell, sigma, xs = Decimal(ell_s), Decimal(sigma_s), Decimal(xs_s)
    out = {}
    sizes = {"hi": R, "lo": R - 1, "3": 1}
    for key, r in sizes.items():
        pts = [Decimal(j) for j in range(-r, r + 1)]
        out["w_" + key] = gp_weights(pts, xs, ell) if key != "3" else None
        Ks = covariance(pts, sigma)
        out["Kinv_" + key] = inverse(Ks)
        with decimal.localcontext(_ctx()):
            out["one_" + key] = sum((sum(row, Decimal(0)) for row in out["Kinv_" + key]), Decimal(0))   # 1^T K^-1 1
        lam, _ = jacobi_eigen(Ks)
        with decimal.localcontext(_ctx()):
            out["logdet_" + key] = sum((l.ln() for l in lam), Decimal(0))
    # the three 3-point stencils of Eq. cweno_stencil: cells -2..0, -1..1, 0..2
    out["w_3"] = [gp_weights([Decimal(j) for j in range(m - 2, m + 1)], xs, ell) for m in range(3)]
    return out


def ao_tables(R: int, ell_over_dx: float, sigma_over_dx: float = 3.0, xstar: float = 0.5) -> dict:
    """Tables of GP-AO (Appendix A) for one prediction point: GP weights of the high-order
    stencil S_R (2R+1 points, Eq. q-intrp), of S_{R-1} (used by the recursive AO(R, R-1, 3)),
    of the three 3-point stencils of Eq. cweno_stencil, and for each stencil size N the inverse
    and log-determinant of K_N built with sigma (the terms of the log-likelihood, Eq. log-like)."""
    assert R in (2, 3)
    t = _ao_decimal(int(R), str(_D(ell_over_dx)), str(_D(sigma_over_dx)), str(_D(xstar)))
    out = {}
    for k, v in t.items():
        if v is None:
            continue
        out[k] = float(v) if isinstance(v, Decimal) else _f64(v)
    return out
