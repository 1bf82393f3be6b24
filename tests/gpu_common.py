"""Shared helpers of the GPU parity tests: build the same shell for the oracle and the library,
and the relative error norm used to compare them.

Error norm (per conserved variable v, quadrature-weighted L2 over the compared points):
    e_v = sqrt(sum w|J| (A_v - B_v)^2) / sqrt(sum w|J| B_v^2),   reported as max over v.
States after time steps are compared on their departure from the background, q' = Q - Q0, so that
the O(1) background does not hide errors.
"""
import numpy as np

from chorus_inputs import cubed_sphere_hex20
from oracle import state as ostate
from oracle.physics import Physics
from oracle.residual import Discretization


class OracleShell:
    def __init__(self, cfg):
        self.cfg = cfg
        self.xyz, self.h20 = cubed_sphere_hex20(cfg.n, cfg.n_r, cfg.r_inner, cfg.r_outer)
        self.disc = Discretization(self.xyz, self.h20, cfg.p, cfg.r_inner, cfg.r_outer)
        self.ph = Physics.from_params(cfg.phys, cfg.r_inner, cfg.r_outer)
        self.N = cfg.p + 1

    def geometry(self, elems=None):
        elems = np.arange(self.disc.n_elem) if elems is None else np.asarray(elems)
        return self.disc.geometry(elems)

    def weights(self, elems=None):
        g = self.geometry(elems)
        w = self.disc.ops.w
        return w[None, :, None, None] * w[None, None, :, None] * w[None, None, None, :] * g["detJ"]

    def background(self, elems=None):
        return ostate.background(self.ph, self.geometry(elems)["x"])

    def initial_state(self, elems=None):
        """Seeded initial state of the given elements (the global point index is the element's own)."""
        cfg = self.cfg
        E = self.disc.n_elem
        elems = np.arange(E) if elems is None else np.asarray(elems)
        x = self.geometry(elems)["x"]
        N = self.N
        g = (elems[:, None, None, None].astype(np.uint64) * np.uint64(N ** 3)
             + np.arange(N ** 3, dtype=np.uint64).reshape(N, N, N)[None])
        xi = ostate.uniform_pm1(cfg.seed, g)
        Q = ostate.background(self.ph, x)
        Q[:, 0] = Q[:, 0] * np.exp(-cfg.entropy_amp * xi)
        return Q


def rel_err(A, B, W):
    """max over variables of the weighted relative L2 error of A against B ([E,5,N,N,N], W [E,N,N,N])."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    num = np.sqrt(np.sum(W[:, None] * (A - B) ** 2, axis=(0, 2, 3, 4)))
    den = np.sqrt(np.sum(W[:, None] * B ** 2, axis=(0, 2, 3, 4)))
    e = num / np.where(den > 0, den, 1.0)
    return float(e.max()), e


def to5(t, N):
    """GPU tensor [E,5,N^3] -> numpy [E,5,N,N,N] (axes k, j, i)."""
    a = t.detach().cpu().numpy().astype(np.float64)
    return a.reshape(a.shape[0], 5, N, N, N)
