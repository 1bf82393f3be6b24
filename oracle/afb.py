"""Oracle: the almost-flux-balance initial stratification (Section 4.3).

Test infrastructure only (see the package docstring).

Steps, in the paper's order:
  1. the polytropic adiabatic reference rho_a, p_a, T_a (Section 4.2, Physics.polytrope);
  2. the target entropy gradient of Section 4.3,
         Gamma(r) = -(L / (4 pi r^2) + rho_a C_p kappa_r(r) dT_a/dr) / (rho_a T_a kappa),
     with the luminosity L = 4 pi r_i^2 f_b from the imposed bottom flux f_b (Section 5).
     Reading: the printed Gamma has no leading minus, but it is the thermal-balance equation of
     Section 4.1 integrated once with an outward luminosity L (total flux
     -kappa rho T dS/dr - kappa_r rho C_p dT/dr = L / (4 pi r^2)), which gives the minus sign; the
     text calls the result superadiabatic (dS/dr < 0, the Schwarzschild criterion of Section 4) and
     sets kappa_r so that the radiative flux carries L at the bottom, i.e. Gamma(r_i) = 0, both of
     which hold only with the sign;
  3. the hydrostatic stratification with that entropy gradient, solved for rho_0 and p_0:
         drho_0/dr = -rho_0 (Gamma / C_p + g rho_0 / (gamma p_0)),   dp_0/dr = -rho_0 g,
     g = GM / r^2, starting from rho_a and p_a.
Reading (the paper says only that rho_a and p_a serve as the initial guess of its finite-difference
solve): the two first-order equations are integrated from the middle radius r_m = (r_i + r_o)/2
outward and inward with rho_0(r_m) = rho_a(r_m), p_0(r_m) = p_a(r_m).  With L = 0 and kappa_r = 0,
Gamma = 0 and the solution is the polytrope itself (a pin of this module).
The integration uses scipy's adaptive eighth-order Dormand-Prince method at a relative tolerance of
3e-14 (near its floor of 100 machine epsilons) with dense output.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import solve_ivp

from .physics import Physics


def luminosity(ph: Physics) -> float:
    return 4.0 * math.pi * ph.r_inner ** 2 * ph.bottom_flux


def dT_a_dr(ph: Physics, r):
    pt = ph.polytrope
    return -pt["T_c"] * pt["alpha"] * pt["d"] / r ** 2


def target_entropy_gradient(ph: Physics, r):
    """Gamma(r) of Section 4.3 (with the sign of the reading above)."""
    return -(luminosity(ph) / (4.0 * math.pi * r ** 2) + ph.rho_a(r) * ph.Cp * ph.kappa_r_at(r) * dT_a_dr(ph, r)) / (
        ph.rho_a(r) * ph.T_a(r) * ph.kappa)


def _rhs(ph: Physics):
    def f(r, y):
        rho, p = y
        g = ph.GM / r ** 2
        return [-rho * (target_entropy_gradient(ph, r) / ph.Cp + g * rho / (ph.gamma * p)), -rho * g]

    return f


def profile(ph: Physics, margin: float = 0.1):
    """Callable r -> (rho_0(r), p_0(r)) on [r_i, r_o] widened by `margin` of the thickness on each
    side: curved 20-node elements put some solution points slightly outside the spherical walls, and
    the equations continue there."""
    rm = 0.5 * (ph.r_inner + ph.r_outer)
    d = ph.r_outer - ph.r_inner
    y0 = [ph.rho_a(rm), ph.p_a(rm)]
    kw = dict(method="DOP853", rtol=3e-14, atol=1e-300, dense_output=True)
    out = solve_ivp(_rhs(ph), (rm, ph.r_outer + margin * d), y0, **kw)
    inn = solve_ivp(_rhs(ph), (rm, ph.r_inner - margin * d), y0, **kw)

    def at(r):
        r = np.asarray(r, dtype=np.float64)
        res = np.empty((2,) + r.shape)
        hi = r >= rm
        if np.any(hi):
            res[:, hi] = out.sol(r[hi])
        if np.any(~hi):
            res[:, ~hi] = inn.sol(r[~hi])
        return res[0], res[1]

    return at


def background(ph: Physics, x: np.ndarray, prof=None) -> np.ndarray:
    """Q0 [E,5,N,N,N] at rest on the almost-flux-balance stratification, at x [E,3,N,N,N]."""
    prof = profile(ph) if prof is None else prof
    r = np.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2 + x[:, 2] ** 2)
    rho, p = prof(r)
    Q0 = np.zeros((x.shape[0], 5) + x.shape[2:])
    Q0[:, 0] = rho
    Q0[:, 4] = p / (ph.gamma - 1.0)
    return Q0
