"""Algorithmic operation count of one GP-WENO stage (used for the ALU roofline).

Counts the floating-point operations the method needs per face and per cell,
written from the steps of the scheme (not from the kernel's instruction
stream): dense characteristic projection L U and back-projection R q, R+2
smoothness windows per field (Eq. beta-eigen, shared by the two sides of a
face), 2(R+1) candidate dot products per field (Eq. candidate_interp), the
nonlinear weights (Eq. weights), the Lax-Friedrichs flux, the
correction of Eqs. numFlux_cor / FD-ders, the divergence of Eq. disc_fd and
the SSP-RK3 stage combination.  An add, multiply, divide, square root or
comparison counts 1; a fused multiply-add counts 2.

Variants change the count where they change the steps: the non-zero-mean
smoothness indicators evaluate 2(R+1) windows per field instead of R+2 (the two
sides no longer share them); HLLC and HLL replace the Lax-Friedrichs
combination; the FD-Flux form projects both U and F(U) of every stencil cell,
evaluates the physical flux and the splitting speed in every stencil cell,
has separate windows for the two split parts, one back-projection, and no
correction.  GP-AO replaces the GP-WENO windows, candidates and weights of each
side by the windows and predictions of the full stencil, of S_{R-1} (R = 3)
and of three 3-point stencils, and the AO hybridisations.
"""


def roe_eigensystem_ops(nv: int) -> int:
    # sqrt x2, 1/(sL+sR), velocities, |v|^2, two pressures, H, c^2, c, 1/c, b1, b2, L entries
    return 2 + 2 + 4 * nv + (2 * nv - 1) + 2 * (2 * nv + 3) + 6 + 5 + 3 + (3 * nv + 12)


def _window(n: int) -> int:
    return n * (2 * n - 1) + 2 * n - 1 + 1                       # P_h . f, squares, + eps


def face_ops(R: int, ndim: int, flux: str = "lf", scheme: str = "fdprim", beta_mean: bool = False,
             ao: bool = False) -> int:
    nc, nv = ndim + 2, ndim
    S, ns = R + 1, 2 * R + 2
    window = _window(S)
    ops = roe_eigensystem_ops(nv)
    if scheme == "fdflux":
        ops += ns * (2 * nv + 8)                                # |u_n| + c per stencil cell, max
        ops += ns * (3 * nv + 13)                               # physical flux per stencil cell
        ops += 2 * ns * nc * (2 * nc - 1) + 2 * ns * nc * 2     # project U and F, split
        ops += nc * 2 * S * window                              # separate windows for F+ and F-
        ops += nc * 2 * S * (2 * S - 1)                         # candidates, both parts
        ops += nc * 2 * (7 * S - 2)                             # nonlinear weights + combination
        ops += nc * (2 * nc - 1)                                # one back-projection of the sum
        return ops
    ops += ns * nc * (2 * nc - 1)                               # projection of 2R+2 cells
    if ao:
        sizes = [2 * R + 1] + ([2 * R - 1] if R == 3 else []) + [3, 3, 3]
        side = sum(_window(n) + 1 + 2 * n for n in sizes)       # beta (x 1/2), prediction
        side += 24 * (2 if R == 3 else 1) + (10 if R == 3 else 0)   # AO(R,3) hybrids, recursion
        ops += nc * 2 * side
    else:
        ops += nc * (2 * S if beta_mean else R + 2) * window    # beta windows
        ops += nc * 2 * S * (2 * S - 1)                         # candidates, both sides
        ops += nc * 2 * (7 * S - 2)                             # nonlinear weights + combination, both sides
    ops += 2 * nc * (2 * nc - 1)                                # back-projection, both sides
    ops += 2 * (3 * nv + 13)                                    # two physical fluxes
    if flux == "hllc":
        ops += 14 + 2 * (3 * nc + 8)                            # speeds, contact speed, two star states
    elif flux == "hll":
        ops += 5 + 5 * nc                                       # speeds and the HLL average
    else:
        ops += 1 + 5 * nc                                       # alpha, LF combination
    return ops


def flops_per_cell_stage(R: int, ndim: int = 2, flux: str = "lf", scheme: str = "fdprim",
                         beta_mean: bool = False, ao: bool = False) -> int:
    nc = ndim + 2
    per_cell = ndim * face_ops(R, ndim, flux, scheme, beta_mean, ao)   # one face per cell per direction
    if scheme != "fdflux":
        per_cell += ndim * nc * 14          # corrected flux
    per_cell += ndim * nc * 2 + nc          # divergence
    per_cell += nc * 5                      # stage combination
    return per_cell


if __name__ == "__main__":
    for R in (1, 2, 3):
        print(R, [flops_per_cell_stage(R, d) for d in (1, 2, 3)])
