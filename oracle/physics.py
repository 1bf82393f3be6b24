"""Oracle: governing equations, fluxes, sources and background (Sections 2 and 4).

Test infrastructure only (see the package docstring).

Conservative form, Eq. 4:  dQ/dt + dF/dx + dG/dy + dH/dz + M = 0,
Q = (rho, rho u, rho v, rho w, E), E = p/(gamma-1) + rho |u|^2 / 2  (Section 2).
Total flux F = F_inv - F_v (Eqs. 6-9).

Readings of garbled or conflicting passages (each stated once here):
  * gravity sign (Eq. 5 against Eqs. 2-3 and g = -GM/r^2 r_hat): the source
    vector follows Eqs. 1-3, M = (0, -rho g + 2 rho Omega x u, -rho u.g) with
    g = -GM x/|x|^3; Eq. 5 agrees with this when its g_x is read as a component
    of +g r_hat.  The Coriolis entries of Eq. 5 already agree.
  * heat-flux sign (Eq. 7 against Eq. 3): the energy viscous flux is
    u.tau - f (Eq. 3), with f = -kappa rho T grad S - kappa_r rho C_p grad T.
  * S = C_p ln(p^{1/gamma}/rho) (Eq. 23) and p = R rho T (Eq. 22) give
    rho T grad S = (C_p/R)(grad p / gamma - (p/rho) grad rho).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Physics:
    gamma: float
    R_gas: float
    GM: float
    Omega: float
    nu: float
    kappa: float
    kappa_r: float
    poly_n: float
    N_rho: float
    rho_c: float
    bottom_flux: float
    T_top: float
    kappa_r1: float
    kappa_r2: float
    r_inner: float
    r_outer: float

    @classmethod
    def from_params(cls, phys, r_inner: float, r_outer: float) -> "Physics":
        return cls(*phys.as_tuple(), r_inner, r_outer)

    @property
    def kappa_r_varies(self) -> bool:
        return self.kappa_r1 != 0.0 or self.kappa_r2 != 0.0

    def kappa_r_at(self, r):
        """Radiative diffusivity kappa_r(r) = kappa_r + kappa_r1 r + kappa_r2 r^2 (the solar
        benchmark's quadratic profile, Section 7.2; constant when the last two vanish)."""
        return self.kappa_r + self.kappa_r1 * r + self.kappa_r2 * r * r

    @property
    def Cp(self) -> float:
        return self.gamma * self.R_gas / (self.gamma - 1.0)

    # ---- polytropic background, Eqs. 25-27 ----
    @property
    def polytrope(self):
        beta = self.r_inner / self.r_outer
        d = self.r_outer - self.r_inner
        n = self.poly_n
        chi_o = (beta + 1.0) / (beta * math.exp(self.N_rho / n) + 1.0)
        chi_i = (1.0 + beta - chi_o) / beta
        c = (2.0 * chi_o - beta - 1.0) / (1.0 - beta)
        alpha = (1.0 + beta) * (1.0 - chi_o) / (1.0 - beta) ** 2
        # hydrostatic balance dp/dr = -rho GM / r^2 (Eq. 20) fixes p_c
        p_c = self.GM * self.rho_c / ((n + 1.0) * alpha * d)
        T_c = p_c / (self.R_gas * self.rho_c)
        return dict(beta=beta, d=d, chi_o=chi_o, chi_i=chi_i, c=c, alpha=alpha, p_c=p_c, T_c=T_c)

    def chi(self, r):
        pt = self.polytrope
        return pt["c"] + pt["alpha"] * pt["d"] / r

    def rho_a(self, r):
        return self.rho_c * self.chi(r) ** self.poly_n

    def p_a(self, r):
        return self.polytrope["p_c"] * self.chi(r) ** (self.poly_n + 1.0)

    def T_a(self, r):
        return self.polytrope["T_c"] * self.chi(r)

    @property
    def T_wall_top(self) -> float:
        return self.T_a(self.r_outer) if math.isnan(self.T_top) else self.T_top


def primitives(Q: np.ndarray, ph: Physics):
    """Q [...,5] -> rho, u [...,3], p."""
    rho = Q[..., 0]
    u = Q[..., 1:4] / rho[..., None]
    p = (ph.gamma - 1.0) * (Q[..., 4] - 0.5 * rho * np.sum(u * u, axis=-1))
    return rho, u, p


def conserved(rho, u, p, ph: Physics) -> np.ndarray:
    Q = np.empty(np.shape(rho) + (5,), dtype=np.result_type(rho, u, p, np.float64))
    Q[..., 0] = rho
    Q[..., 1:4] = rho[..., None] * u
    Q[..., 4] = p / (ph.gamma - 1.0) + 0.5 * rho * np.sum(u * u, axis=-1)
    return Q


def inviscid_flux(Q: np.ndarray, ph: Physics) -> np.ndarray:
    """Eq. 6: F_inv, G_inv, H_inv -> [..., 3(direction n), 5]."""
    rho, u, p = primitives(Q, ph)
    F = np.empty(Q.shape[:-1] + (3, 5), dtype=Q.dtype)
    for n in range(3):
        F[..., n, 0] = rho * u[..., n]
        for a in range(3):
            F[..., n, 1 + a] = rho * u[..., n] * u[..., a] + (p if a == n else 0.0)
        F[..., n, 4] = u[..., n] * (Q[..., 4] + p)
    return F


def grad_primitives(Q: np.ndarray, gradQ: np.ndarray, ph: Physics) -> np.ndarray:
    """Chain rule from conserved-variable gradients to primitive gradients.

    gradQ [...,5,3] (d Q_v / d x_n) -> gradW [...,5,3] for W = (rho, u, v, w, p):
      grad u_a = (grad m_a - u_a grad rho) / rho
      grad p   = (gamma-1) (grad E - u . grad m + |u|^2/2 grad rho)
    """
    rho, u, p = primitives(Q, ph)
    gW = np.empty_like(gradQ)
    gW[..., 0, :] = gradQ[..., 0, :]
    for a in range(3):
        gW[..., 1 + a, :] = (gradQ[..., 1 + a, :] - u[..., a, None] * gradQ[..., 0, :]) / rho[..., None]
    ke = 0.5 * np.sum(u * u, axis=-1)
    gW[..., 4, :] = (ph.gamma - 1.0) * (
        gradQ[..., 4, :] - np.einsum("...a,...an->...n", u, gradQ[..., 1:4, :]) + ke[..., None] * gradQ[..., 0, :]
    )
    return gW


def stress(Q: np.ndarray, gradW: np.ndarray, ph: Physics) -> np.ndarray:
    """Eq. 9: tau[..., a, b] with mu = rho nu, trace-free Newtonian stress."""
    rho = Q[..., 0]
    mu = rho * ph.nu
    gu = gradW[..., 1:4, :]  # gu[..., a, b] = d u_a / d x_b
    div = gu[..., 0, 0] + gu[..., 1, 1] + gu[..., 2, 2]
    tau = mu[..., None, None] * (gu + np.swapaxes(gu, -1, -2))
    for a in range(3):
        tau[..., a, a] -= (2.0 / 3.0) * mu * div
    return tau


def heat_flux(rho, p, grad_rho, grad_p, ph: Physics, kr=None) -> np.ndarray:
    """f = -kappa rho T grad S - kappa_r rho C_p grad T (Section 2), written in rho, p.
    kr: the radiative diffusivity at the points (default: the constant ph.kappa_r)."""
    pr = (p / rho)[..., None]
    rhoT_gradS = (ph.Cp / ph.R_gas) * (grad_p / ph.gamma - pr * grad_rho)
    rhoCp_gradT = (ph.Cp / ph.R_gas) * (grad_p - pr * grad_rho)
    kr = ph.kappa_r if kr is None else np.asarray(kr)[..., None]
    return -ph.kappa * rhoT_gradS - kr * rhoCp_gradT


def viscous_flux(Q: np.ndarray, gradW: np.ndarray, ph: Physics, kr=None) -> np.ndarray:
    """Eqs. 7-8 (energy entry signed per Eq. 3): F_v -> [..., 3(n), 5].  kr: radiative diffusivity at
    the points (default the constant)."""
    rho, u, p = primitives(Q, ph)
    tau = stress(Q, gradW, ph)
    f = heat_flux(rho, p, gradW[..., 0, :], gradW[..., 4, :], ph, kr)
    Fv = np.zeros(Q.shape[:-1] + (3, 5), dtype=np.result_type(Q, gradW))
    for n in range(3):
        for a in range(3):
            Fv[..., n, 1 + a] = tau[..., a, n]
        Fv[..., n, 4] = np.einsum("...a,...a->...", u, tau[..., :, n]) - f[..., n]
    return Fv


def source(Q: np.ndarray, x: np.ndarray, ph: Physics) -> np.ndarray:
    """M of Eq. 4: (0, -rho g + 2 rho Omega x u, -rho u.g), g = -GM x/|x|^3, Omega along +z."""
    r = np.sqrt(np.sum(x * x, axis=-1))
    gvec = -ph.GM * x / (r ** 3)[..., None]
    rho = Q[..., 0]
    m = Q[..., 1:4]
    M = np.zeros_like(Q)
    M[..., 1:4] = -rho[..., None] * gvec
    M[..., 1] += 2.0 * ph.Omega * (-m[..., 1])  # (Omega z_hat x m)_x = -Omega m_y
    M[..., 2] += 2.0 * ph.Omega * (m[..., 0])   # (Omega z_hat x m)_y = +Omega m_x
    M[..., 4] = -np.sum(m * gvec, axis=-1)
    return M


def rusanov(QL: np.ndarray, QR: np.ndarray, nhat: np.ndarray, ph: Physics) -> np.ndarray:
    """Rusanov common inviscid flux along the unit normal nhat (pointing from L to R).

    F = (F_n(Q_L) + F_n(Q_R))/2 - lambda (Q_R - Q_L)/2,
    lambda = max over both sides of |V_n| + c_s (Section 3).
    """
    FL = np.einsum("...n,...nv->...v", nhat, inviscid_flux(QL, ph))
    FR = np.einsum("...n,...nv->...v", nhat, inviscid_flux(QR, ph))
    rl, ul, pl = primitives(QL, ph)
    rr, ur, pr = primitives(QR, ph)
    lam = np.maximum(
        np.abs(np.sum(ul * nhat, axis=-1)) + np.sqrt(ph.gamma * pl / rl),
        np.abs(np.sum(ur * nhat, axis=-1)) + np.sqrt(ph.gamma * pr / rr),
    )
    return 0.5 * (FL + FR) - 0.5 * lam[..., None] * (QR - QL)
