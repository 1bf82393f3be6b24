"""GB300 spectral-difference residual and SSP-RK3 stepping for rotating stratified spherical shells.

The compute path is libchorus.so (hand-written sm_103a CUDA kernels behind the C ABI of
include/chorus.h); this package is its thin Python binding plus a shell helper that builds the
cubed-sphere inputs.
"""
from __future__ import annotations

from .native import FP32_PERT, FP64, Batch, ChorusError, Mesh, Params, load, stable_dt  # noqa: F401


class Shell:
    """A shell workload on the GPU: mesh handle, parameters and the stable time step."""

    def __init__(self, cfg, metric_mode: int = 0, stream=None):
        from chorus_inputs import cubed_sphere_hex20

        self.cfg = cfg
        xyz, h20 = cubed_sphere_hex20(cfg.n, cfg.n_r, cfg.r_inner, cfg.r_outer)
        self.mesh = Mesh(xyz, h20, cfg.p, cfg.r_inner, cfg.r_outer, metric_mode, stream)
        self.params = Params.from_phys(cfg.phys)
        info = self.mesh.info()
        self.h_min = info["h_min"]
        self.dt = self.mesh.stable_dt(self.params)


class Shells:
    """A batch of independent shells on the GPU (see chorus_batch_create) with one common stable
    time step: the smallest of the orders' steps by the single-shell rule."""

    def __init__(self, bcfg, stream=None):
        from chorus_inputs import cubed_sphere_hex20

        self.bcfg = bcfg
        self.cfgs = bcfg.shells()
        shells = []
        for c in self.cfgs:
            xyz, h20 = cubed_sphere_hex20(c.n, c.n_r, c.r_inner, c.r_outer)
            shells.append((xyz, h20, c.p, c.seed, c.entropy_amp))
        self.params = Params.from_phys(bcfg.phys)
        self.batch = Batch(shells, bcfg.r_inner, bcfg.r_outer, self.params, stream)
        self.dt = min(stable_dt(p, h, bcfg.r_inner, bcfg.r_outer, self.params)
                      for p, h in self.batch.group_h_min.items())
