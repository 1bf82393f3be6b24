"""Failure paths of the library on the GPU, exercised without a fault.

  * A non-finite state: a NaN written into Q on the host makes chorus_reduce return CHORUS_ENAN.
  * A bounded device-side wait that runs out: with the mesh's wait limit set to zero polls the
    residual kernels give up their staging wait at once, wait for their bulk copies in flight, skip
    all computation and stores and set the error flag; chorus_check reports CHORUS_ETIMEOUT once and
    clears it, and the next residual with the default limit is correct.  Nothing spins unbounded.
"""
import numpy as np
import pytest

from chorus_inputs import SHELL_288_P3

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ENAN, ETIMEOUT = 5, 6


@pytest.fixture(scope="module")
def shell():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00834_gb300 import Shell, build

    build.build()
    sh = Shell(SHELL_288_P3)
    sh.mesh.prepare(sh.params)
    return sh


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_reduce_reports_nan(shell, prec):
    from paper_1503_00834_gb300 import ChorusError

    sh, cfg = shell, SHELL_288_P3
    dt = torch.float64 if prec == 0 else torch.float32
    Q = torch.empty(sh.mesh.state_shape(), dtype=dt, device="cuda")
    sh.mesh.state_init(sh.params, cfg.seed, cfg.entropy_amp, prec, Q)
    assert np.all(np.isfinite(sh.mesh.reduce(sh.params, prec, Q)))
    host = Q.cpu()
    host[17, 2, 5] = float("nan")  # one momentum value of one solution point
    Q.copy_(host)
    with pytest.raises(ChorusError) as e:
        sh.mesh.reduce(sh.params, prec, Q)
    assert e.value.status == ENAN


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_wait_timeout_is_reported_and_skips_the_outputs(shell, prec):
    from paper_1503_00834_gb300 import ChorusError

    sh, cfg = shell, SHELL_288_P3
    dt = torch.float64 if prec == 0 else torch.float32
    Q = torch.empty(sh.mesh.state_shape(), dtype=dt, device="cuda")
    sh.mesh.state_init(sh.params, cfg.seed, cfg.entropy_amp, prec, Q)
    ws = torch.empty(sh.mesh.workspace_bytes(prec), dtype=torch.uint8, device="cuda")
    R_ref = torch.empty_like(Q)
    sh.mesh.residual(sh.params, prec, Q, R_ref, ws)
    sh.mesh.check()
    try:
        sh.mesh.set_wait_limit(0)  # every staging wait gives up at once
        R = torch.full_like(Q, 12345.0)
        sh.mesh.residual(sh.params, prec, Q, R, ws)
        with pytest.raises(ChorusError) as e:
            sh.mesh.check()
        assert e.value.status == ETIMEOUT
        assert bool(torch.all(R == 12345.0))  # the kernel that gave up stored nothing
        sh.mesh.check()  # reported once, then cleared
    finally:
        sh.mesh.set_wait_limit(-1)  # the default limit
    R = torch.empty_like(Q)
    sh.mesh.residual(sh.params, prec, Q, R, ws)
    sh.mesh.check()
    assert torch.equal(R, R_ref)
