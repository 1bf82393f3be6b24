"""GB300 spectral-difference residual and SSP-RK3 stepping for rotating stratified spherical shells.

The compute path is libchorus.so (hand-written sm_103a CUDA kernels behind the C ABI of
include/chorus.h); this package is its thin Python binding plus a shell helper that builds the
cubed-sphere inputs.
"""
from __future__ import annotations

from .native import FP32_PERT, FP64, ChorusError, Mesh, Params, load, max_sound_speed, stable_dt  # noqa: F401


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
        ph = cfg.phys
        self.dt = stable_dt(cfg.p, self.h_min, max_sound_speed(ph, cfg.r_inner, cfg.r_outer), max(ph.nu, ph.kappa))
