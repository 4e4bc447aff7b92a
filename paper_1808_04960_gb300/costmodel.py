"""Algorithmic operation count of one GP-WENO stage (used for the ALU roofline).

Counts the floating-point operations the method needs per face and per cell,
written from the steps of the scheme (not from the kernel's instruction
stream): dense characteristic projection L U and back-projection R q, R+2
smoothness windows per field (Eq. beta-eigen, shared by the two sides of a
face), 2(R+1) candidate dot products per field (Eq. candidate_interp), the
nonlinear weights in ratio form (Eq. weights), the Lax-Friedrichs flux, the
correction of Eqs. numFlux_cor / FD-ders, the divergence of Eq. disc_fd and
the SSP-RK3 stage combination.  An add, multiply, divide, square root or
comparison counts 1; a fused multiply-add counts 2.
"""


def roe_eigensystem_ops(nv: int) -> int:
    # sqrt x2, 1/(sL+sR), velocities, |v|^2, two pressures, H, c^2, c, 1/c, b1, b2, L entries
    return 2 + 2 + 4 * nv + (2 * nv - 1) + 2 * (2 * nv + 3) + 6 + 5 + 3 + (3 * nv + 12)


def face_ops(R: int, ndim: int) -> int:
    nc, nv = ndim + 2, ndim
    S, ns = R + 1, 2 * R + 2
    ops = roe_eigensystem_ops(nv)
    ops += ns * nc * (2 * nc - 1)                               # projection of 2R+2 cells
    ops += nc * ((R + 2) * (S * (2 * S - 1) + 2 * S - 1) + (R + 2))  # beta windows (+ eps)
    ops += nc * 2 * S * (2 * S - 1)                             # candidates, both sides
    ops += nc * 2 * (7 * S - 2)                                 # nonlinear weights + combination, both sides
    ops += 2 * nc * (2 * nc - 1)                                # back-projection, both sides
    ops += 2 * (3 * nv + 13) + 1 + 5 * nc                       # two physical fluxes, alpha, LF combination
    return ops


def flops_per_cell_stage(R: int, ndim: int = 2) -> int:
    nc = ndim + 2
    per_cell = ndim * face_ops(R, ndim)     # one face per cell per direction
    per_cell += ndim * nc * 14              # corrected flux
    per_cell += ndim * nc * 2 + nc          # divergence
    per_cell += nc * 5                      # stage combination
    return per_cell


if __name__ == "__main__":
    for R in (1, 2, 3):
        print(R, [flops_per_cell_stage(R, d) for d in (1, 2, 3)])
