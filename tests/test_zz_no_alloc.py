"""chorus_residual_noalloc: the residual for callers that cannot allocate device memory.

Such callers (for example an application whose device memory belongs to its own pool allocator,
or a loop that must not call cudaMalloc because it can synchronise the device) pass only Q and R;
the library keeps its scratch (traces, viscous face fluxes, gradient record, common face fluxes) in a
fixed static device array.  This test calls the
entry point through the C ABI twice in a row, on two different states, and checks each result
against chorus_residual with a caller-provided workspace, within the parity tolerances the other
GPU tests use (1e-12 relative for FP64, 1e-5 for the FP32 perturbation path).  It also checks that a
mesh too large for the scratch is refused before any launch, that an attached learned closure is
added exactly as chorus_residual adds it, and that a radial radiative diffusivity whose flux-point
table has not been built is refused instead of allocated.  The file name makes pytest collect it
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
    cfg = small_shell(10, 5, 3)  # 3,000 elements: 50.7 MB of FP64 scratch, 25.3 MB in FP32 (limit 32 MiB)
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


def test_noalloc_adds_an_attached_closure():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from chorus_inputs import small_shell
    from paper_1503_00834_gb300 import FP32_PERT, FP64, Shell, build, load, native

    build.build()
    lib = load()
    cfg = small_shell(2, 2, 2)  # p = 2, the closure's order
    sh = Shell(cfg)
    sh.mesh.prepare(sh.params)
    w = native.closure_alloc(11, [1e-3] * 5, [2e-2] * 5)
    native.closure_attach(sh.mesh, w)
    try:
        for prec, dtype, tol in ((FP64, torch.float64, 1e-12), (FP32_PERT, torch.float32, 1e-5)):
            Q = torch.empty(sh.mesh.state_shape(), dtype=dtype, device="cuda")
            sh.mesh.state_init(sh.params, cfg.seed, 1e-2, prec, Q)
            ws = torch.empty(sh.mesh.workspace_bytes(prec), dtype=torch.uint8, device="cuda")
            R_ref = torch.empty_like(Q)
            sh.mesh.residual(sh.params, prec, Q, R_ref, ws)
            native.closure_attach(sh.mesh, None)
            R_plain = torch.empty_like(Q)
            sh.mesh.residual(sh.params, prec, Q, R_plain, ws)
            native.closure_attach(sh.mesh, w)
            assert _rel(R_plain, R_ref) > 10 * tol  # the closure changes the residual: the check is not vacuous
            for _ in range(2):
                R = torch.full_like(Q, float("nan"))
                assert _noalloc(lib, sh, prec, Q, R) == 0
                sh.mesh.check()
                assert _rel(R, R_ref) <= tol
    finally:
        native.closure_attach(sh.mesh, None)


def test_noalloc_radial_kappa_r_needs_its_table():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from chorus_inputs import SHELL_288_P3 as cfg
    from paper_1503_00834_gb300 import FP64, Shell, build, load

    build.build()
    lib = load()
    sh = Shell(cfg)
    sh.params.kappa_r1 = 2e-4  # kappa_r(r) = 2e-4 r: the flux-point table is needed
    Q = torch.empty(sh.mesh.state_shape(), dtype=torch.float64, device="cuda")
    R = torch.zeros_like(Q)
    # no table yet: refused before any launch, nothing allocated
    assert _noalloc(lib, sh, FP64, Q.fill_(1.0), R) == 1
    assert not torch.any(R)
    sh.mesh.state_init(sh.params, cfg.seed, cfg.entropy_amp, FP64, Q)  # prepares, building the table
    ws = torch.empty(sh.mesh.workspace_bytes(FP64), dtype=torch.uint8, device="cuda")
    R_ref = torch.empty_like(Q)
    sh.mesh.residual(sh.params, FP64, Q, R_ref, ws)
    for _ in range(2):
        R = torch.full_like(Q, float("nan"))
        assert _noalloc(lib, sh, FP64, Q, R) == 0
        sh.mesh.check()
        assert _rel(R, R_ref) <= 1e-12
