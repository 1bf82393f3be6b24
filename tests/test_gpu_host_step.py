"""chorus_rk_step_host, the end-to-end entry point (a host-resident state copied in, stepped, copied
back), against chorus_rk_step on the same state kept on the device.

In the FP32 form the last stage's residual runs in four element ranges whose new state is copied to
the host while the next range is computed; each element's arithmetic is the same, so the host state
must equal the device-stepped one bit for bit: for several orders, for element counts that do not
split evenly (state offsets of a range that are not 16-byte aligned at p = 2 take the kernels' plain
staging loads), with an attached learned closure (its correction shifted with the range), and in
the FP64 form (one copy each way).
"""
import pytest

from chorus_inputs import SHELL_288_P3, small_shell

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00834_gb300 import build

    build.build()


def _pair(cfg, prec, n_steps, closure=False):
    from paper_1503_00834_gb300 import FP64, Shell

    sh = Shell(cfg)
    m = sh.mesh
    m.prepare(sh.params)
    dt = torch.float64 if prec == FP64 else torch.float32
    Q = torch.empty(m.state_shape(), dtype=dt, device="cuda")
    m.state_init(sh.params, cfg.seed, cfg.entropy_amp, prec, Q)
    ws = torch.empty(m.workspace_bytes(prec), dtype=torch.uint8, device="cuda")
    from paper_1503_00834_gb300 import native

    w = native.closure_alloc(11, [1e-3] * 5, [2e-2] * 5) if closure else None
    if closure:
        native.closure_attach(m, w)
    try:
        host = torch.empty(Q.shape, dtype=dt, pin_memory=True)
        host.copy_(Q)
        Q_dev = torch.empty_like(Q)
        m.rk_step_host(sh.params, prec, host, Q_dev, ws, sh.dt, n_steps)
        m.rk_step(sh.params, prec, Q, ws, sh.dt, n_steps)
        torch.cuda.synchronize()
        m.check()
    finally:
        if closure:
            native.closure_attach(m, None)
    return host, Q.cpu()


@pytest.mark.parametrize("cfg", [SHELL_288_P3, small_shell(2, 1, 2), small_shell(1, 2, 5), small_shell(2, 1, 4)],
                         ids=lambda c: c.name)
def test_host_step_equals_device_step_fp32(cfg):
    from paper_1503_00834_gb300 import FP32_PERT

    host, dev = _pair(cfg, FP32_PERT, 2)
    assert bool(torch.isfinite(dev).all())
    assert torch.equal(host, dev)


def test_host_step_equals_device_step_fp64():
    from paper_1503_00834_gb300 import FP64

    host, dev = _pair(SHELL_288_P3, FP64, 1)
    assert bool(torch.isfinite(dev).all())
    assert torch.equal(host, dev)


def test_host_step_with_closure_attached():
    from paper_1503_00834_gb300 import FP32_PERT

    host, dev = _pair(small_shell(2, 1, 2), FP32_PERT, 2, closure=True)
    assert bool(torch.isfinite(dev).all())
    assert torch.equal(host, dev)
