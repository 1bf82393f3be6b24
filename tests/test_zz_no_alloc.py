"""chorus_residual_noalloc: the residual for callers that cannot allocate device memory.

Such callers (for example an application whose device memory belongs to its own pool allocator,
or a loop that must not call cudaMalloc because it can synchronise the device) pass only Q and R;
the library keeps its scratch (traces, viscous face fluxes, gradient record) in a fixed static device
array.  This test calls the
entry point through the C ABI twice in a row, on two different states, and checks each result
against chorus_residual with a caller-provided workspace, within the parity tolerances the other
GPU tests use (1e-12 relative for FP64, 1e-5 for the FP32 perturbation path).  It also checks that a
mesh too large for the scratch is refused before any launch.  The file name makes pytest collect it
last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(a, b):
    a = a.double().cpu().numpy().reshape(a.shape[0], 5, -1)
    b = b.double().cpu().numpy().reshape(b.shape[0], 5, -1)
    num = np.sqrt(np.sum((a - b) ** 2, axis=(0, 2)))
    den = np.sqrt(np.sum(b ** 2, axis=(0, 2)))
    return float(np.max(num / den))


def _noalloc(lib, sh, prec, Q, R):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.chorus_residual_noalloc(sh.mesh.handle, ctypes.byref(sh.params), prec, ctypes.c_void_p(Q.data_ptr()),
                                       ctypes.c_void_p(R.data_ptr()), stream)


def test_noalloc_residual_matches_workspace_residual():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from chorus_inputs import SHELL_288_P3 as cfg
    from paper_1503_00834_gb300 import FP32_PERT, FP64, Shell, build, load

    build.build()
    lib = load()
    sh = Shell(cfg)
    for prec, dtype, tol in ((FP64, torch.float64, 1e-12), (FP32_PERT, torch.float32, 1e-5)):
        shape = sh.mesh.state_shape()
        QA = torch.empty(shape, dtype=dtype, device="cuda")
        sh.mesh.state_init(sh.params, cfg.seed, cfg.entropy_amp, prec, QA)
        ws = torch.empty(sh.mesh.workspace_bytes(prec), dtype=torch.uint8, device="cuda")
        QB = QA.clone()
        sh.mesh.rk_step(sh.params, prec, QB, ws, sh.dt, 2)  # a second, different state
        for Q in (QA, QB):  # two calls in a row share the static scratch
            R_ref = torch.empty_like(Q)
            sh.mesh.residual(sh.params, prec, Q, R_ref, ws)
            R = torch.full_like(Q, float("nan"))
            assert _noalloc(lib, sh, prec, Q, R) == 0
            sh.mesh.check()
            assert _rel(R, R_ref) <= tol


def test_noalloc_refuses_meshes_beyond_the_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from chorus_inputs import small_shell
    from paper_1503_00834_gb300 import FP32_PERT, FP64, Shell, load

    lib = load()
    cfg = small_shell(12, 5, 3)  # 4,320 elements: 56.4 MB of FP64 scratch, 28.2 MB in FP32 (limit 32 MiB)
    sh = Shell(cfg)
    Q = torch.zeros(sh.mesh.state_shape(), dtype=torch.float64, device="cuda")
    R = torch.zeros_like(Q)
    assert _noalloc(lib, sh, FP64, Q, R) == 1  # CHORUS_EINVAL, nothing launched
    assert not torch.any(R)
    sh.mesh.prepare(sh.params)
    q = torch.empty(sh.mesh.state_shape(), dtype=torch.float32, device="cuda")
    sh.mesh.state_init(sh.params, cfg.seed, cfg.entropy_amp, FP32_PERT, q)
    r = torch.empty_like(q)
    assert _noalloc(lib, sh, FP32_PERT, q, r) == 0
    sh.mesh.check()
    assert torch.isfinite(r).all()
