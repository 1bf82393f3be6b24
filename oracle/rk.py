"""Oracle: explicit SSP Runge-Kutta stepping of the semi-discrete system.

Test infrastructure only (see the package docstring).

The paper integrates with a five-stage fourth-order SSP scheme (Section 7.4,
coefficients in a reference that is not reproduced in the paper).  The shell
workloads use the three-stage third-order SSP scheme in Shu-Osher form:
    u1      = u + dt L(u)
    u2      = 3/4 u + 1/4 (u1 + dt L(u1))
    u^{n+1} = 1/3 u + 2/3 (u2 + dt L(u2))
"""
from __future__ import annotations

import numpy as np

from .residual import residual

SSPRK3 = ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))


def ssprk3_step(disc, ph, Q: np.ndarray, dt: float) -> np.ndarray:
    u = Q
    s = Q
    for a, b in SSPRK3:
        s = a * u + b * (s + dt * residual(disc, ph, s))
    return s


def run(disc, ph, Q: np.ndarray, dt: float, n_steps: int) -> np.ndarray:
    for _ in range(n_steps):
        Q = ssprk3_step(disc, ph, Q, dt)
    return Q
