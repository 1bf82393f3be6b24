"""Oracle: initial state, background and time step (Section 4; Section 7.1 CFL remark).

Test infrastructure only (see the package docstring).

Background Q0: the polytropic adiabatic stratification of Eqs. 25-27 at rest,
evaluated at the solution points (rho_a, p_a, u = 0).  Initial state: the
background with a seeded random entropy perturbation S'/C_p = A xi, where
xi in [-1, 1) is drawn per global solution point g = e N^3 + (i + N j + N^2 k)
from SplitMix64 (Steele, Lea & Flood 2014) seeded with (seed XOR g):
    z = x + 0x9E3779B97F4A7C15;  z = (z ^ z>>30) * 0xBF58476D1CE4E5B9;
    z = (z ^ z>>27) * 0x94D049BB133111EB;  out = z ^ z>>31 ;
    xi = 2 (out >> 11) 2^-53 - 1.
The pressure is kept (p = p_a) and the density follows from S = C_p ln(p^(1/gamma)/rho)
(Eq. 23): rho = rho_a exp(-A xi); u = 0.
"""
from __future__ import annotations

import numpy as np

from .physics import Physics

_M64 = (1 << 64) - 1


def splitmix64(x: np.ndarray) -> np.ndarray:
    """One SplitMix64 output for each 64-bit input state (vectorised, wrapping uint64)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, index: np.ndarray) -> np.ndarray:
    z = splitmix64(np.uint64(seed) ^ np.asarray(index, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


def background(ph: Physics, x: np.ndarray) -> np.ndarray:
    """Q0 [E,5,N,N,N] from solution-point coordinates x [E,3,N,N,N]."""
    r = np.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2 + x[:, 2] ** 2)
    Q0 = np.zeros((x.shape[0], 5) + x.shape[2:])
    Q0[:, 0] = ph.rho_a(r)
    Q0[:, 4] = ph.p_a(r) / (ph.gamma - 1.0)
    return Q0


def initial_state(ph: Physics, x: np.ndarray, seed: int, amp: float, elems=None, Q0=None) -> np.ndarray:
    """Initial state at the solution points x [E,3,N,N,N] of elements `elems` (default 0..E-1), on
    the polytropic background or on the given background Q0 (same shape as the state)."""
    E = x.shape[0]
    N = x.shape[2]
    elems = np.arange(E) if elems is None else np.asarray(elems)
    g = (elems.astype(np.uint64)[:, None, None, None] * np.uint64(N ** 3)
         + np.arange(N ** 3, dtype=np.uint64).reshape(N, N, N)[None])
    xi = uniform_pm1(seed, g)
    Q = background(ph, x) if Q0 is None else np.array(Q0, dtype=np.float64)
    Q[:, 0] = Q[:, 0] * np.exp(-amp * xi)
    return Q


def min_edge_chord(node_xyz: np.ndarray, hex20: np.ndarray) -> float:
    """Shortest straight distance between the two corner nodes of any element edge."""
    edges = [(0, 1), (1, 2), (2, 3), (3, 0), (4, 5), (5, 6), (6, 7), (7, 4), (0, 4), (1, 5), (2, 6), (3, 7)]
    c = node_xyz[hex20[:, :8]]
    return float(min(np.min(np.linalg.norm(c[:, a] - c[:, b], axis=-1)) for a, b in edges))


def time_step(ph: Physics, p: int, h_min: float, Q: np.ndarray) -> float:
    """Fixed explicit step: 0.25 h/((2p+1) max(|u|+c)), capped by 0.25 h^2/((2p+1)^2 max(nu, kappa)).

    The paper states only a CFL condition (Section 7); h/((2p+1) c) is the one-dimensional limit,
    shared among the three directions of an element with comparable edges (factor 0.25 < 1/3)."""
    rho = Q[:, 0]
    u2 = (Q[:, 1] ** 2 + Q[:, 2] ** 2 + Q[:, 3] ** 2) / rho ** 2
    pres = (ph.gamma - 1.0) * (Q[:, 4] - 0.5 * rho * u2)
    wave = float(np.max(np.sqrt(u2) + np.sqrt(ph.gamma * pres / rho)))
    dt = 0.25 * h_min / ((2 * p + 1) * wave)
    diff = max(ph.nu, ph.kappa)
    if diff > 0:
        dt = min(dt, 0.25 * h_min * h_min / ((2 * p + 1) ** 2 * diff))
    return dt
