"""Algorithmic operation count of one GP-WENO stage (used for the ALU roofline).

The count is the closed form of the floating-point operations of the plain
FD-Prim algorithm, step by step in the paper's order, with every quantity
computed once where it belongs:

  per cell       primitive variables (rho, u, p) of the cell;
  per face       Roe average of the two cells sharing the face and the
                 primitive-system eigenvectors at it; characteristic
                 projection of the 2R+2 stencil cells; per characteristic
                 field the smoothness indicators of Eq. gp-smooth as
                 d . (K^-1 d) on the R+2 windows shared by the two states
                 (2(R+1) windows with the non-zero mean), the candidates of
                 Eq. candidate_interp, the weights of Eq. weights and the
                 combination of Eq. weight_sum for both states;
                 back-projection and conserved form of both states; the face
                 flux (local Lax-Friedrichs, or HLLC / HLL on their
                 subsonic branch);
  per cell/dir   the corrected flux of Eqs. numFlux_cor / FD-ders (once per
                 face) and the difference of Eq. disc_fd;
  per cell       the Shu-Osher SSP-RK3 stage combination (mean of the three
                 stages).

Counting rules: an add, subtract, multiply, divide or square root counts one,
as does a max or min that selects a value; sign changes, absolute values and
copies count nothing; a sum of k terms counts k-1 additions; x^p counts p-1
multiplications; terms of the eigenvector products with a structural zero
coefficient are skipped and a coefficient of +-1 costs no multiply.  These
are the rules of the operation-counting build of the FP64 oracle, and the CPU
tests check that this closed form equals the oracle's tally for R = 1, 2, 3 in
1D, 2D and 3D, for each face flux and both smoothness-indicator means.  The
count is the method's work, not the kernel's instruction stream: the kernel's
cell-relative rewriting adds arithmetic that this count does not credit.

The FD-Flux form and GP-AO are modelled with the same rules from their steps
(they are not counted by the oracle, whose FD-Flux path inverts the
conservative eigenvector matrix numerically).
"""


def pressure_ops(nv: int) -> int:
    return 2 * nv + 4                      # |m|^2, /2, /rho, E -, (gamma-1), *


def prim_ops(nv: int) -> int:
    return nv + pressure_ops(nv)           # velocities and pressure of a cell


def conserved_ops(nv: int) -> int:
    return 3 * nv - 1 + 5                  # momenta, |u|^2, E


def roe_ops(nv: int) -> int:
    return 9 * nv + 16                     # sqrt rho x2, H x2, rho, velocities, |u|^2, H, c^2, c


EIGEN_OPS = 7                              # rho/(2c), c^2, 1/(2c^2), 1/c^2, c/rho
PROJECTION_OPS_PER_CELL = 8                # rows (0,-an,0,ap), (1,0,0,-ie), e_t, (0,an,0,ap)
BACK_PROJECTION_OPS = 8                    # rows (1,1,0,1), (-cr,0,0,cr), e_t, (c^2,0,0,c^2)
CORRECTION_OPS = 14                        # D2, D4 and the corrected flux, per component
DIVERGENCE_OPS = 3                         # difference, / dx, accumulate, per component


def window_ops(S: int, mean: bool) -> int:
    """beta = d . (K^-1 d) on S points, d = f - mean."""
    return 2 * S * S + S - 1 + (S if mean else 0)


def state_ops(S: int, p: int = 2) -> int:
    """Candidates, nonlinear weights and their combination for one state of one field."""
    return S * (2 * S - 1) + S * (2 + (p - 1)) + (S - 1) + 3 * S - 1


def normal_flux_ops(nc: int, nv: int) -> int:
    return 1 + 2 + (nc - 3) + 2 + pressure_ops(nv)


def flux_ops(flux: str, nc: int, nv: int) -> int:
    if flux == "hllc":
        star = 1 + 4 + 1 + 2 * (nc - 3) + 9 + 3 * nc
        return 2 + 6 + 6 + 15 + 2 * pressure_ops(nv) + 2 * normal_flux_ops(nc, nv) + star
    if flux == "hll":
        return 2 + 6 + 6 + 2 * pressure_ops(nv) + 2 * normal_flux_ops(nc, nv) + 9 * nc
    # local Lax-Friedrichs: two sound speeds and |u_n| + c, max, alpha/2, two fluxes, combination
    return 2 * 4 + 1 + 1 + 2 * (nc + 1) + 5 * nc


def face_ops(R: int, ndim: int, flux: str = "lf", scheme: str = "fdprim", beta_mean: bool = False,
             ao: bool = False, p: int = 2) -> int:
    nc, nv = ndim + 2, ndim
    S, ns = R + 1, 2 * R + 2
    if scheme == "fdflux":
        return _fdflux_face_ops(R, nc, nv, beta_mean, p)
    ops = roe_ops(nv) + EIGEN_OPS + ns * PROJECTION_OPS_PER_CELL
    if ao:
        ops += nc * 2 * _ao_side_ops(R, beta_mean, p)
    else:
        nwin = 2 * S if beta_mean else R + 2
        ops += nc * nwin * window_ops(S, beta_mean)
        ops += nc * 2 * state_ops(S, p)
    ops += 2 * BACK_PROJECTION_OPS + 2 * conserved_ops(nv)
    ops += flux_ops(flux, nc, nv)
    return ops


def _fdflux_face_ops(R, nc, nv, beta_mean, p):
    """FD-Flux (modelled): splitting speed and physical flux of every stencil cell, projection of
    U and F(U) on the conservative characteristic fields (dense nc x nc rows), the split parts'
    own windows, both reconstructions and one back-projection."""
    S, ns = R + 1, 2 * R + 2
    speed = 1 + 3 + 1 + 1                                   # u_n, c, |u_n| + c, max
    ops = roe_ops(nv) + EIGEN_OPS + ns * (speed + normal_flux_ops(nc, nv))
    ops += ns * 2 * nc * (2 * nc - 1) + ns * nc * 4         # project U and F, split (F +- alpha U)/2
    ops += nc * 2 * S * window_ops(S, beta_mean)
    ops += nc * 2 * state_ops(S, p) + nc                    # both parts, summed
    ops += nc * (2 * nc - 1)                                # back-projection
    return ops


def _ao_side_ops(R, beta_mean, p):
    """GP-AO (modelled), one state of one field: beta (x 1/2) and prediction of the full stencil,
    of S_{R-1} (R = 3) and of the three 3-point stencils, the AO(R,3) hybrid and the recursion."""
    sizes = [2 * R + 1] + ([2 * R - 1] if R == 3 else []) + [3, 3, 3]
    ops = sum(window_ops(n, beta_mean) + 1 + (2 * n - 1) + 2 + (p - 1) for n in sizes)
    hybrid = 4 + 3 + 1 + 2 + 3 * 4                          # weights, sum, 1/sum, omega/gamma, combination
    ops += hybrid * (2 if R == 3 else 1) + (12 if R == 3 else 0)
    return ops


def flops_per_cell_stage(R: int, ndim: int = 2, flux: str = "lf", scheme: str = "fdprim",
                         beta_mean: bool = False, ao: bool = False, p: int = 2) -> int:
    nc, nv = ndim + 2, ndim
    per_dir = face_ops(R, ndim, flux, scheme, beta_mean, ao, p) + DIVERGENCE_OPS * nc
    if scheme != "fdflux":
        per_dir += CORRECTION_OPS * nc
    per_cell = ndim * per_dir + 4 * nc                      # stage combination (2, 5, 5 per component)
    if scheme != "fdflux":
        per_cell += prim_ops(nv)
    return per_cell


if __name__ == "__main__":
    for R in (1, 2, 3):
        print(R, [flops_per_cell_stage(R, d) for d in (1, 2, 3)])
