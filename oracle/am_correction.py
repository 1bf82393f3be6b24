"""Oracle: angular-momentum correction (Section 6, Eqs. 32-34).

Test infrastructure only (see the package docstring).

Step 1 (Eq. 32): the three Cartesian components of the angular momentum, written in spherical
coordinates (r, theta colatitude, phi longitude) as printed:
    L_x = int rho r (w sin(theta) sin(phi) - v cos(theta)) dV
    L_y = int rho r (u cos(theta) - w sin(theta) cos(phi)) dV
    L_z = int rho r (v sin(theta) cos(phi) - u sin(theta) sin(phi)) dV
and the moments of inertia I_x = int rho (y^2 + z^2) dV, etc.
Step 2 (Eq. 33): delta Omega_i = L_i / I_i.
Velocity update (Eq. 34), with atan2 as defined below the equation,
    atan2(m1, m2) = 2 arctan(m1 / (sqrt(m1^2 + m2^2) + m2)):
    u += dOz sqrt(x^2+y^2) sin(atan2(y,x)) - dOy sqrt(x^2+z^2) cos(atan2(x,z))
    v += -dOz sqrt(x^2+y^2) cos(atan2(y,x)) + dOx sqrt(y^2+z^2) sin(atan2(z,y))
    w += dOy sqrt(x^2+z^2) sin(atan2(x,z)) - dOx sqrt(y^2+z^2) cos(atan2(z,y))
Readings: only the velocity changes; density and pressure are kept, so the total energy takes the
new kinetic energy.  The update evaluates atan2 with the library function, which equals the
printed identity wherever that identity is defined (it divides by zero on the negative m2 axis);
`atan2_paper` keeps the identity for the test that checks this.  Volume integrals use the
solution-point quadrature w_i w_j w_k |J|.
"""
from __future__ import annotations

import numpy as np


def atan2_paper(m1, m2):
    """atan2 through the half-angle identity printed below Eq. 34 (undefined on the negative m2 axis)."""
    return 2.0 * np.arctan(m1 / (np.sqrt(m1 * m1 + m2 * m2) + m2))


def _weights(disc):
    g = disc.geometry(np.arange(disc.n_elem))
    w = disc.ops.w
    W = w[None, :, None, None] * w[None, None, :, None] * w[None, None, None, :] * g["detJ"]
    return W, g["x"]


def momentum_and_inertia(disc, Q):
    """(L [3], I [3]) of the state Q [E,5,N,N,N] (Eq. 32 and the inertia integrals of Section 6)."""
    W, x = _weights(disc)
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    r = np.sqrt(X * X + Y * Y + Z * Z)
    theta = np.arccos(Z / r)
    phi = np.arctan2(Y, X)
    rho = Q[:, 0]
    u, v, w = Q[:, 1] / rho, Q[:, 2] / rho, Q[:, 3] / rho
    st, ct, sp, cp = np.sin(theta), np.cos(theta), np.sin(phi), np.cos(phi)
    L = np.array([
        np.sum(W * rho * r * (w * st * sp - v * ct)),
        np.sum(W * rho * r * (u * ct - w * st * cp)),
        np.sum(W * rho * r * (v * st * cp - u * st * sp)),
    ])
    I = np.array([np.sum(W * rho * (Y * Y + Z * Z)), np.sum(W * rho * (X * X + Z * Z)),
                  np.sum(W * rho * (X * X + Y * Y))])
    return L, I


def correct(disc, ph, Q):
    """Returns (Q_new, dOmega): Eq. 33 rates and the Eq. 34 velocity update."""
    L, I = momentum_and_inertia(disc, Q)
    dO = L / I
    _, x = _weights(disc)
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    rho = Q[:, 0]
    u, v, w = Q[:, 1] / rho, Q[:, 2] / rho, Q[:, 3] / rho
    p = (ph.gamma - 1.0) * (Q[:, 4] - 0.5 * rho * (u * u + v * v + w * w))
    rxy, rxz, ryz = np.sqrt(X * X + Y * Y), np.sqrt(X * X + Z * Z), np.sqrt(Y * Y + Z * Z)
    a_yx, a_xz, a_zy = np.arctan2(Y, X), np.arctan2(X, Z), np.arctan2(Z, Y)
    un = u + dO[2] * rxy * np.sin(a_yx) - dO[1] * rxz * np.cos(a_xz)
    vn = v - dO[2] * rxy * np.cos(a_yx) + dO[0] * ryz * np.sin(a_zy)
    wn = w + dO[1] * rxz * np.sin(a_xz) - dO[0] * ryz * np.cos(a_zy)
    Qn = Q.copy()
    Qn[:, 1], Qn[:, 2], Qn[:, 3] = rho * un, rho * vn, rho * wn
    Qn[:, 4] = p / (ph.gamma - 1.0) + 0.5 * rho * (un * un + vn * vn + wn * wn)
    return Qn, dO
