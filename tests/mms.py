"""Manufactured solution for pinning the residual: symbolic right-hand side of Eqs. 1-3.

The exact operator L(Q) = -div(F_inv - F_v) - M is built here with sympy
directly from the paper's definitions in Section 2: the inviscid fluxes of
Eq. 6, the stress of Eq. 9 with mu = rho nu, the diffusive flux
f = -kappa rho T grad S - kappa_r(r) rho C_p grad T with S = C_p ln(p^(1/gamma)/rho)
(Eq. 23), T = p/(R rho) (Eq. 22) and the radiative diffusivity
kappa_r(r) = kappa_r + kappa_r1 r + kappa_r2 r^2 (Section 7.2's quadratic profile), the energy
equation of Eq. 3 (so the viscous energy flux is u.tau - f), and the gravity and Coriolis forces of
Eq. 2 (g = -GM r_hat / r^2, rotation Omega about +z).  It shares nothing with the oracle's discrete
arithmetic.

Two families of states:
  * "general": the polytrope of Eqs. 25-27 modulated by smooth lateral and radial functions, with a
    smooth velocity field (it does not satisfy the wall conditions: compare away from the walls);
  * "radial": fluid at rest with a non-adiabatic radial stratification rho(r), p(r).  It satisfies
    the impenetrable stress-free walls of Section 5 exactly, and the thermal ones when the imposed
    bottom flux and top temperature are taken from it (wall_data), so the residual converges to L
    on every element, wall layers included.
"""
import functools

import numpy as np
import sympy as sp


@functools.lru_cache(maxsize=None)
def exact_operator(gamma, R_gas, GM, Omega, nu, kappa, kappa_r, kappa_r1, kappa_r2, rho_c, chi_c, chi_a, p_c, n_poly,
                   amp, family="general"):
    x, y, z = sp.symbols("x y z", real=True)
    X = (x, y, z)
    r = sp.sqrt(x * x + y * y + z * z)
    chi = chi_c + chi_a / r
    if family == "general":
        rho = rho_c * chi ** n_poly * (1 + amp * sp.sin(3 * x) * sp.cos(2 * y) * sp.sin(z + sp.Rational(3, 10)))
        u = [amp * sp.sin(2 * y + z), amp * sp.cos(x - z), amp * sp.sin(x + 2 * y)]
        p = p_c * chi ** (n_poly + 1) * (1 + amp * sp.cos(2 * x + y) * sp.sin(3 * z))
    else:
        rho = rho_c * chi ** n_poly * (1 + amp * sp.sin(7 * r))
        u = [sp.Integer(0)] * 3
        p = p_c * chi ** (n_poly + 1) * (1 + amp * sp.cos(5 * r))
    E = p / (gamma - 1) + rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2) / 2
    Q = [rho, rho * u[0], rho * u[1], rho * u[2], E]

    mu = rho * nu
    du = [[sp.diff(u[a], X[b]) for b in range(3)] for a in range(3)]
    div = du[0][0] + du[1][1] + du[2][2]
    tau = [[mu * (du[a][b] + du[b][a]) - (sp.Rational(2, 3) * mu * div if a == b else 0) for b in range(3)]
           for a in range(3)]
    Cp = gamma * R_gas / (gamma - 1)
    T = p / (R_gas * rho)
    S = Cp * sp.log(p ** (1 / sp.Float(gamma)) / rho)
    kr = kappa_r + kappa_r1 * r + kappa_r2 * r * r
    f = [-kappa * rho * T * sp.diff(S, X[b]) - kr * rho * Cp * sp.diff(T, X[b]) for b in range(3)]

    flux = []  # flux[b][v] = (F_inv - F_v) in direction b
    for b in range(3):
        Finv = [rho * u[b]] + [rho * u[b] * u[a] + (p if a == b else 0) for a in range(3)] + [u[b] * (E + p)]
        Fv = [0] + [tau[a][b] for a in range(3)] + [sum(u[a] * tau[a][b] for a in range(3)) - f[b]]
        flux.append([Finv[v] - Fv[v] for v in range(5)])
    gvec = [-GM * X[a] / r ** 3 for a in range(3)]
    # momentum RHS of Eq. 2: + rho g - 2 rho Omega x u ; energy RHS of Eq. 3: + rho u.g
    cor = [-Omega * u[1], Omega * u[0], 0]
    rhs_src = [0] + [rho * gvec[a] - 2 * rho * cor[a] for a in range(3)] + [rho * sum(u[a] * gvec[a] for a in range(3))]
    L = [-sum(sp.diff(flux[b][v], X[b]) for b in range(3)) + rhs_src[v] for v in range(5)]
    fQ = sp.lambdify((x, y, z), Q, "numpy")
    fL = sp.lambdify((x, y, z), L, "numpy")
    fT = sp.lambdify((x, y, z), T, "numpy")
    fx = sp.lambdify((x, y, z), f[0], "numpy")
    return fQ, fL, fT, fx


def _ops(ph, amp, family):
    pt = ph.polytrope
    return exact_operator(ph.gamma, ph.R_gas, ph.GM, ph.Omega, ph.nu, ph.kappa, ph.kappa_r, ph.kappa_r1, ph.kappa_r2,
                          ph.rho_c, pt["c"], pt["alpha"] * pt["d"], pt["p_c"], ph.poly_n, amp, family)


def evaluate(ph, x, amp, family="general"):
    """Q_m and L(Q_m) at points x [..., 3] for oracle Physics `ph` -> ([...,5], [...,5])."""
    fQ, fL, _, _ = _ops(ph, amp, family)
    X = [x[..., 0], x[..., 1], x[..., 2]]
    Q = np.stack([np.broadcast_to(np.asarray(v, dtype=np.float64), x.shape[:-1]) for v in fQ(*X)], -1)
    L = np.stack([np.broadcast_to(np.asarray(v, dtype=np.float64), x.shape[:-1]) for v in fL(*X)], -1)
    return Q, L


def wall_data(ph, amp):
    """(bottom_flux, T_top) of the radial family: f . r_hat at r_inner and T at r_outer (Section 5's
    thermal wall conditions taken from the exact state)."""
    _, _, fT, fx = _ops(ph, amp, "radial")
    return float(fx(ph.r_inner, 0.0, 0.0)), float(fT(ph.r_outer, 0.0, 0.0))
