"""GPU angular-momentum correction (Section 6, Eqs. 32-34) against the oracle.

Input on both sides: the seeded initial state plus a seeded random momentum field (energy left
unchanged), built independently by the oracle and on the device.  Tolerances: FP64 1e-12
relative; the FP32 perturbation path holds the momentum in FP32 (1e-6 relative).
"""
import numpy as np
import pytest

from chorus_inputs import SHELL_288_P3 as CFG
from gpu_common import OracleShell, rel_err, to5

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _momentum(cfg, dtype):
    rng = np.random.default_rng(2024)
    N = cfg.p + 1
    m = 0.01 * rng.standard_normal((cfg.n_elem, 3, N ** 3))
    return m.astype(dtype)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32pert"])
def test_am_correction_matches_oracle(prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle.am_correction import correct, momentum_and_inertia
    from paper_1503_00834_gb300 import Shell, build

    build.build()
    sh = Shell(CFG)
    N = CFG.p + 1
    dtype = np.float64 if prec == 0 else np.float32
    m = _momentum(CFG, dtype)
    Q = torch.empty(sh.mesh.state_shape(), dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
    sh.mesh.state_init(sh.params, CFG.seed, CFG.entropy_amp, prec, Q)
    Q[:, 1:4] = torch.from_numpy(m).to("cuda")
    dO_gpu = sh.mesh.am_correct(sh.params, prec, Q)

    osh = OracleShell(CFG)
    Qo = osh.initial_state()
    Qo[:, 1:4] = m.astype(np.float64).reshape(CFG.n_elem, 3, N, N, N)
    Qn, dO = correct(osh.disc, osh.ph, Qo)
    tol = 1e-12 if prec == 0 else 1e-6
    assert np.allclose(dO_gpu, dO, rtol=tol, atol=tol * np.abs(dO).max())
    got = to5(Q, N)
    Q0 = osh.background() if prec == 1 else 0.0
    e, ev = rel_err(got, Qn - Q0, osh.weights())
    print(f"am correction prec {prec}: dOmega {dO_gpu} vs {dO}, state rel err {ev}")
    assert e < tol
    # the corrected state carries (almost) no angular momentum
    L_after, _ = momentum_and_inertia(osh.disc, Qn)
    L_before, _ = momentum_and_inertia(osh.disc, Qo)
    assert np.linalg.norm(L_after) < 1e-2 * np.linalg.norm(L_before)
