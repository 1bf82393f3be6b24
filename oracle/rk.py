"""Oracle: explicit SSP Runge-Kutta stepping of the semi-discrete system.

Test infrastructure only (see the package docstring).

The shell workloads use the three-stage third-order SSP scheme in Shu-Osher form:
    u1      = u + dt L(u)
    u2      = 3/4 u + 1/4 (u1 + dt L(u1))
    u^{n+1} = 1/3 u + 2/3 (u2 + dt L(u2))
The paper integrates with the five-stage fourth-order SSP scheme of Spiteri and Ruuth (Section 7.4);
its coefficients are not printed in the paper.  `ssprk54_step` uses the published Shu-Osher form
of that scheme:
    u1 = u + b10 dt L(u)
    u2 = a20 u + a21 u1 + b21 dt L(u1)
    u3 = a30 u + a32 u2 + b32 dt L(u2)
    u4 = a40 u + a43 u3 + b43 dt L(u3)
    u^{n+1} = a52 u2 + a53 u3 + b53 dt L(u3) + a54 u4 + b54 dt L(u4)
"""
from __future__ import annotations

import numpy as np

from .residual import residual

SSPRK3 = ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))

# SSP-RK(5,4) Shu-Osher coefficients (Spiteri and Ruuth 2002)
RK54 = dict(
    b10=0.391752226571890,
    a20=0.444370493651235, a21=0.555629506348765, b21=0.368410593050371,
    a30=0.620101851488403, a32=0.379898148511597, b32=0.251891774271694,
    a40=0.178079954393132, a43=0.821920045606868, b43=0.544974750228521,
    a52=0.517231671970585, a53=0.096059710526147, b53=0.063692468666290,
    a54=0.386708617503269, b54=0.226007483236906,
)


def ssprk3_step(disc, ph, Q: np.ndarray, dt: float) -> np.ndarray:
    u = Q
    s = Q
    for a, b in SSPRK3:
        s = a * u + b * (s + dt * residual(disc, ph, s))
    return s


def ssprk54_step(disc, ph, Q: np.ndarray, dt: float) -> np.ndarray:
    c = RK54
    u = Q
    u1 = u + c["b10"] * dt * residual(disc, ph, u)
    u2 = c["a20"] * u + c["a21"] * u1 + c["b21"] * dt * residual(disc, ph, u1)
    u3 = c["a30"] * u + c["a32"] * u2 + c["b32"] * dt * residual(disc, ph, u2)
    L3 = residual(disc, ph, u3)
    u4 = c["a40"] * u + c["a43"] * u3 + c["b43"] * dt * L3
    return c["a52"] * u2 + c["a53"] * u3 + c["b53"] * dt * L3 + c["a54"] * u4 + c["b54"] * dt * residual(disc, ph, u4)


def run(disc, ph, Q: np.ndarray, dt: float, n_steps: int, scheme: str = "ssprk3") -> np.ndarray:
    step = ssprk3_step if scheme == "ssprk3" else ssprk54_step
    for _ in range(n_steps):
        Q = step(disc, ph, Q, dt)
    return Q
