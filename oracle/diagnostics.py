"""Oracle: FP64 volume integrals over the shell (Section 6 Eq. 32; Section 7.2 Eq. 35).

Test infrastructure only (see the package docstring).

Quadrature: integral of u over an element = sum_ijk w_i w_j w_k |J_ijk| u_ijk
with w the interpolatory weights at the solution points.
Returns mass, total energy, kinetic energy sum(|m|^2 / (2 rho)) and the
angular momentum vector L = integral of x cross (rho u) (Eq. 32 written in
Cartesian form).
"""
from __future__ import annotations

import numpy as np


def integrals(disc, Q: np.ndarray) -> dict:
    g = disc.geometry(np.arange(disc.n_elem))
    w = disc.ops.w
    W = w[None, :, None, None] * w[None, None, :, None] * w[None, None, None, :] * g["detJ"]
    rho = Q[:, 0]
    m = Q[:, 1:4]
    x = g["x"]
    ke = 0.5 * np.sum(m * m, axis=1) / rho
    L = np.cross(np.moveaxis(x, 1, -1), np.moveaxis(m, 1, -1))
    return dict(
        mass=float(np.sum(W * rho)),
        energy=float(np.sum(W * Q[:, 4])),
        kinetic=float(np.sum(W * ke)),
        L=np.sum(W[..., None] * L, axis=(0, 1, 2, 3)),
        volume=float(np.sum(W)),
    )
