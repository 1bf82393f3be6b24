"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds only problem *inputs*: the node coordinates and 20-node
connectivity of a cubed-sphere spherical-shell mesh, and the raw physical
parameter sets of the shell workloads.  It contains none of the
spectral-difference arithmetic (no points, bases, metrics, fluxes or
time stepping); both the oracle and the GPU library compute all of that
themselves from these inputs.

Mesh (paper Section 3, Fig. 1; Section 5): all-hexahedral shell made of
20-node iso-parametric elements (8 corners + 12 mid-edge nodes) with nodes
uniformly distributed in radius.  The paper fuses eight GAMBIT segments; here
the shell is a gnomonic equiangular cubed sphere, 6 panels x n x n lateral
cells x n_r radial layers.  Mid-edge nodes sit at the mid-angle on the exact
sphere (lateral edges) or at the mid-radius (radial edges).

Local node order of a hexahedron (reference cube [0,1]^3, axes xi, eta, zeta):
  corners  0:(0,0,0) 1:(1,0,0) 2:(1,1,0) 3:(0,1,0)
           4:(0,0,1) 5:(1,0,1) 6:(1,1,1) 7:(0,1,1)
  mid-edge 8:(h,0,0) 9:(1,h,0) 10:(h,1,0) 11:(0,h,0)
           12:(h,0,1) 13:(1,h,1) 14:(h,1,1) 15:(0,h,1)
           16:(0,0,h) 17:(1,0,h) 18:(1,1,h) 19:(0,1,h)      (h = 1/2)
On the cubed sphere xi follows the first panel angle, eta the second and
zeta the radius, which gives positive Jacobians on all six panels.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# reference-cube coordinates of the 20 nodes, in units of 1/2
HEX20_REF2 = np.array(
    [
        [0, 0, 0], [2, 0, 0], [2, 2, 0], [0, 2, 0],
        [0, 0, 2], [2, 0, 2], [2, 2, 2], [0, 2, 2],
        [1, 0, 0], [2, 1, 0], [1, 2, 0], [0, 1, 0],
        [1, 0, 2], [2, 1, 2], [1, 2, 2], [0, 1, 2],
        [0, 0, 1], [2, 0, 1], [2, 2, 1], [0, 2, 1],
    ],
    dtype=np.int64,
)


def _panel_direction(panel: int, ta: np.ndarray, tb: np.ndarray) -> np.ndarray:
    """Unnormalised direction of the gnomonic point (tan a, tan b) on a panel."""
    one = np.ones_like(ta)
    if panel == 0:
        d = (one, ta, tb)
    elif panel == 1:
        d = (-ta, one, tb)
    elif panel == 2:
        d = (-one, -ta, tb)
    elif panel == 3:
        d = (ta, -one, tb)
    elif panel == 4:
        d = (-tb, ta, one)
    elif panel == 5:
        d = (tb, ta, -one)
    else:
        raise ValueError(panel)
    return np.stack(d, axis=-1)


def cubed_sphere_hex20(n: int, n_r: int, r_inner: float, r_outer: float):
    """Return (node_xyz [n_nodes,3] float64, hex20 [E,20] int64).

    Element order: e = ((panel*n + j)*n + i)*n_r + k with i, j the lateral
    cell indices along the two panel angles and k the radial layer (fastest).
    """
    if n < 1 or n_r < 1 or not (0.0 < r_inner < r_outer):
        raise ValueError("bad cubed-sphere parameters")
    m = 2 * n  # fine lateral grid (corners + mid-edge points)
    mr = 2 * n_r
    ang = -math.pi / 4 + (math.pi / 2) * np.arange(m + 1) / m
    tan = np.tan(ang)
    tan[0], tan[-1] = -1.0, 1.0  # exact panel edges: shared edges match bitwise
    radii = r_inner + (r_outer - r_inner) * np.arange(mr + 1) / mr
    radii[-1] = r_outer

    I, J, L = np.meshgrid(np.arange(m + 1), np.arange(m + 1), np.arange(mr + 1), indexing="ij")
    keys = []
    xyz = []
    for panel in range(6):
        d = _panel_direction(panel, tan[I], tan[J])
        d = d / np.sqrt(d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1] + d[..., 2] * d[..., 2])[..., None]
        xyz.append(d * radii[L][..., None])
    xyz = np.stack(xyz)  # [6, m+1, m+1, mr+1, 3]

    # element -> fine-grid indices of its 20 nodes
    E = 6 * n * n * n_r
    pan, jj, ii, kk = np.meshgrid(np.arange(6), np.arange(n), np.arange(n), np.arange(n_r), indexing="ij")
    pan, jj, ii, kk = (a.reshape(-1) for a in (pan, jj, ii, kk))
    gi = 2 * ii[:, None] + HEX20_REF2[None, :, 0]
    gj = 2 * jj[:, None] + HEX20_REF2[None, :, 1]
    gk = 2 * kk[:, None] + HEX20_REF2[None, :, 2]
    pts = xyz[pan[:, None], gi, gj, gk]  # [E,20,3]
    assert pts.shape == (E, 20, 3)

    # merge coincident nodes (shared between elements and across panel seams)
    flat = pts.reshape(-1, 3)
    scale = 2.0 ** 36 / r_outer
    key = np.round(flat * scale).astype(np.int64)
    uniq, inv = np.unique(key, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    node_xyz = np.zeros((uniq.shape[0], 3))
    node_xyz[inv] = flat
    hex20 = inv.reshape(E, 20).astype(np.int64)
    return node_xyz, hex20


@dataclasses.dataclass(frozen=True)
class PhysParams:
    """Raw physical parameters of a shell workload (nondimensional units).

    R_o = 1, GM = 1, rho_c = 1, gas constant 1, gamma = 1 + 1/n (adiabatic
    polytrope, Section 4.2), Omega = nu / (Ek d^2) (Eq. 24).  kappa_r = 0 and
    a zero bottom flux, T_top = NaN meaning "polytrope temperature at r_o".
    """

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
    kappa_r1: float = 0.0  # radiative diffusivity kappa_r(r) = kappa_r + kappa_r1 r + kappa_r2 r^2
    kappa_r2: float = 0.0

    def as_tuple(self):
        return dataclasses.astuple(self)


@dataclasses.dataclass(frozen=True)
class ShellConfig:
    name: str
    n: int  # lateral cells per panel edge
    n_r: int  # radial layers
    p: int  # polynomial degree (N = p + 1 solution points per direction)
    r_inner: float
    r_outer: float
    seed: int
    entropy_amp: float
    steps: int
    phys: PhysParams

    @property
    def n_elem(self) -> int:
        return 6 * self.n * self.n * self.n_r

    @property
    def n_dof(self) -> int:
        return self.n_elem * (self.p + 1) ** 3


def make_phys(beta: float, poly_n: float, N_rho: float, Ek: float, nu: float = 5e-4,
              kappa: float = 5e-4) -> PhysParams:
    d = 1.0 - beta
    return PhysParams(
        gamma=1.0 + 1.0 / poly_n,
        R_gas=1.0,
        GM=1.0,
        Omega=nu / (Ek * d * d),
        nu=nu,
        kappa=kappa,
        kappa_r=0.0,
        poly_n=poly_n,
        N_rho=N_rho,
        rho_c=1.0,
        bottom_flux=0.0,
        T_top=float("nan"),
    )


# Shell workloads: cubed-sphere meshes 6 x n x n x n_r, polytrope n = 1.5,
# seeded entropy perturbation.
SHELL_288_P3 = ShellConfig("shell_288_p3", 4, 3, 3, 0.75, 1.0, 1, 1e-3, 100,
                           make_phys(0.75, 1.5, 3.0, 1e-3))
SHELL_331776_P3 = ShellConfig("shell_331776_p3", 48, 24, 3, 0.75, 1.0, 2, 1e-3, 1000,
                              make_phys(0.75, 1.5, 3.0, 1e-3))
SHELL_786432_P4 = ShellConfig("shell_786432_p4", 64, 32, 4, 0.71, 1.0, 3, 1e-3, 100,
                              make_phys(0.71, 1.5, 4.0, 2.447e-3))

# a mid-size shell of the same family (state 126 MB in FP32, working set > L2) for profiling captures
SHELL_98304_P3 = ShellConfig("shell_98304_p3", 32, 16, 3, 0.75, 1.0, 2, 1e-3, 100,
                             make_phys(0.75, 1.5, 3.0, 1e-3))

# learned-closure workload: the 98,304-element shell at p = 2 (coarse) and p = 5 (fine, pair source)
SHELL_98304_P2 = ShellConfig("shell_98304_p2", 32, 16, 2, 0.75, 1.0, 5, 1e-3, 2000,
                             make_phys(0.75, 1.5, 3.0, 1e-3))
SHELL_98304_P5 = ShellConfig("shell_98304_p5", 32, 16, 5, 0.75, 1.0, 5, 1e-3, 2000,
                             make_phys(0.75, 1.5, 3.0, 1e-3))

CONFIGS = {c.name: c for c in (SHELL_288_P3, SHELL_331776_P3, SHELL_786432_P4, SHELL_98304_P3, SHELL_98304_P2,
                               SHELL_98304_P5)}


def small_shell(n: int, n_r: int, p: int, seed: int = 7, amp: float = 1e-3, beta: float = 0.75,
                N_rho: float = 3.0) -> ShellConfig:
    """A small shell of the same family for tests."""
    return ShellConfig(f"shell_{n}x{n_r}_p{p}", n, n_r, p, beta, 1.0, seed, amp, 10,
                       make_phys(beta, 1.5, N_rho, 1e-3))


def _splitmix64_next(state: int):
    """One step of SplitMix64 (Steele, Lea and Flood 2014): returns (new state, output)."""
    m = (1 << 64) - 1
    state = (state + 0x9E3779B97F4A7C15) & m
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return state, z ^ (z >> 31)


@dataclasses.dataclass(frozen=True)
class BatchConfig:
    """Independent shells advanced together: shell i draws its lateral cells per panel edge
    n in [n_lo, n_hi], radial layers n_r in [nr_lo, nr_hi] and order p in `orders` from a SplitMix64
    stream seeded with seed * 1000 + i, which is also its perturbation seed.  All shells share the
    radii and the physics of `phys`."""

    name: str
    n_shells: int
    seed: int
    n_lo: int
    n_hi: int
    nr_lo: int
    nr_hi: int
    orders: tuple
    r_inner: float
    r_outer: float
    entropy_amp: float
    phys: PhysParams

    def shells(self):
        out = []
        for i in range(self.n_shells):
            s = self.seed * 1000 + i
            st, a = _splitmix64_next(s)
            st, b = _splitmix64_next(st)
            st, c = _splitmix64_next(st)
            n = self.n_lo + a % (self.n_hi - self.n_lo + 1)
            n_r = self.nr_lo + b % (self.nr_hi - self.nr_lo + 1)
            p = self.orders[c % len(self.orders)]
            out.append(ShellConfig(f"{self.name}_{i}", n, n_r, p, self.r_inner, self.r_outer, s, self.entropy_amp,
                                   10, self.phys))
        return out


# 64 shells of the shell_288_p3 family (beta 0.75, 3 density scale heights), n 8-32, n_r 4-16, p 2-5
BATCH_64 = BatchConfig("batch_64", 64, 4, 8, 32, 4, 16, (2, 3, 4, 5), 0.75, 1.0, 1e-3,
                       make_phys(0.75, 1.5, 3.0, 1e-3))
# the same family at a quarter of the size (16 shells, 8-16 cells per panel edge, 4-8 layers): a
# batch whose kernels a profiler captures in seconds
BATCH_16 = BatchConfig("batch_16", 16, 4, 8, 16, 4, 8, (2, 3, 4, 5), 0.75, 1.0, 1e-3,
                       make_phys(0.75, 1.5, 3.0, 1e-3))


def small_batch() -> BatchConfig:
    """A small batch of the same family for tests (every order, ragged sizes)."""
    return BatchConfig("batch_small", 6, 9, 1, 3, 1, 3, (2, 3, 4, 5), 0.75, 1.0, 1e-3,
                       make_phys(0.75, 1.5, 3.0, 1e-3))


# ---- the paper's benchmark parameter sets (Tables 1 and 2), in this package's units
# Units: length R_o, GM = 1 (time sqrt(R_o^3 / GM)), density rho_c = the polytrope's mid-layer density
# (rho_i / chi_i^n), gas constant 1.  A dimensional kinematic coefficient k becomes k t_u / R_o^2,
# a rate W becomes W t_u, a luminosity L becomes L t_u^3 / (rho_c R_o^5).
_G_CGS = 6.67e-8
PAPER_CASES = {
    # Table 1 (Jupiter benchmark): kappa_r = 0
    "jupiter": dict(beta=0.35, n=2.0, N_rho=5.0, R_o=7.0e9, Omega=1.76e-4, M=1.9e30, rho_i=1.1, nu=3.64364e12,
                    kappa=3.64364e12, L=7.014464e32),
    # Table 2 (solar benchmark) with the radiative diffusivity of Section 7.2:
    # kappa_r = lambda (c0 + c1 w + c2 w^2), w = r / 1e10 cm, lambda such that the radiative flux
    # carries L at the bottom
    "sun": dict(beta=0.736762, n=1.5, N_rho=3.0, R_o=6.61e10, Omega=8.1e-5, M=1.98891e33, rho_i=0.21, nu=6.0e13,
                kappa=6.0e13, L=3.846e36, kappa_r_poly=(1.5600975e8, -4.5631718e7, 3.3370368e6)),
}


def paper_case_phys(name: str) -> tuple:
    """(beta, PhysParams) of a Table 1/2 case; bottom_flux = L / (4 pi r_i^2), T_top left NaN (the
    caller sets it from the stratification it uses); the solar case carries its kappa_r(r)."""
    c = PAPER_CASES[name]
    beta, n = c["beta"], c["n"]
    t_u = math.sqrt(c["R_o"] ** 3 / (_G_CGS * c["M"]))
    chi_o = (beta + 1.0) / (beta * math.exp(c["N_rho"] / n) + 1.0)
    chi_i = (1.0 + beta - chi_o) / beta
    rho_c = c["rho_i"] / chi_i ** n
    L = c["L"] * t_u ** 3 / (rho_c * c["R_o"] ** 5)
    nu = c["nu"] * t_u / c["R_o"] ** 2
    kappa = c["kappa"] * t_u / c["R_o"] ** 2
    gamma = 1.0 + 1.0 / n
    kr = (0.0, 0.0, 0.0)
    if "kappa_r_poly" in c:
        # lambda from F_r = -kappa_r rho_a C_p dT_a/dr = L / (4 pi r_i^2) at r_i = beta, with the
        # polytrope of Section 4.2 in these units (rho_c = 1, gas constant 1, GM = 1)
        d = 1.0 - beta
        alpha = (1.0 + beta) * (1.0 - chi_o) / d ** 2
        T_c = 1.0 / ((n + 1.0) * alpha * d)
        dTdr_i = -T_c * alpha * d / beta ** 2
        Cp = gamma / (gamma - 1.0)
        kr_i = L / (4.0 * math.pi * beta ** 2) / (chi_i ** n * Cp * -dTdr_i)
        s = c["R_o"] * 1e-10  # w = s r
        c0, c1, c2 = c["kappa_r_poly"]
        lam = kr_i / (c0 + c1 * s * beta + c2 * (s * beta) ** 2)
        kr = (lam * c0, lam * c1 * s, lam * c2 * s * s)
    phys = PhysParams(gamma=gamma, R_gas=1.0, GM=1.0, Omega=c["Omega"] * t_u, nu=nu, kappa=kappa, kappa_r=kr[0],
                      poly_n=n, N_rho=c["N_rho"], rho_c=1.0, bottom_flux=L / (4.0 * math.pi * beta * beta),
                      T_top=float("nan"), kappa_r1=kr[1], kappa_r2=kr[2])
    return beta, phys
