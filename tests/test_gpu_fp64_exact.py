"""FP64 GPU path against an extended-precision run of the oracle.

The whole discretisation - 1D operators, geometry and metrics, residual - evaluated by the oracle in
numpy longdouble (80-bit extended on x86, IEEE binary128 on arm64) from the same FP64 node
coordinates and the same FP64 state (the oracle's seeded state is uploaded to the GPU, so both sides
see identical input bits) is the exact discrete result to far below FP64 rounding.  Against it the
FP64 oracle itself has an error: for a near-hydrostatic state the momentum residual is a difference
of O(rho g) terms that cancel to ~1e-3 of their size, so its relative FP64 floor is ~1e-12 - a few
1e-12 (measured per case and printed beside the GPU's).  The requirement, per conserved variable
(quadrature-weighted relative L2):
  * residuals: the GPU FP64 error is at most max(1e-12, 2 x the FP64 oracle's own error), on the
    polytrope shells of all orders and the almost-flux-balance stratifications of the paper's
    Jupiter and solar cases (the latter with the radial radiative diffusivity);
  * SSP-RK3 and SSP-RK(5,4) trajectories of every order, compared on q' = Q - Q0: the same bound
    (storing the total state in FP64 also rounds it by eps |Q0| every stage, on both sides alike).
"""
import dataclasses

import numpy as np
import pytest

from chorus_inputs import SHELL_288_P3, ShellConfig, paper_case_phys, small_shell
from gpu_common import OracleShell, to5
from oracle.residual import Discretization

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LD = np.longdouble


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if np.finfo(LD).eps > 1e-18:
        pytest.skip("no extended precision on this host")
    from paper_1503_00834_gb300 import build

    build.build()


def _rel(A, B, W):
    """Per-variable weighted relative L2 of A against B, evaluated in extended precision."""
    A = np.asarray(A, dtype=LD)
    B = np.asarray(B, dtype=LD)
    W = np.asarray(W, dtype=LD)[:, None]
    num = np.sqrt(np.sum(W * (A - B) ** 2, axis=(0, 2, 3, 4)))
    den = np.sqrt(np.sum(W * B ** 2, axis=(0, 2, 3, 4)))
    return np.asarray(num / np.where(den > 0, den, 1), dtype=np.float64)


def _extended(osh):
    """The same shell's discretisation evaluated in extended precision."""
    c = osh.cfg
    return Discretization(osh.xyz, osh.h20, c.p, c.r_inner, c.r_outer, dtype=LD)


def _upload(Q):
    E = Q.shape[0]
    return torch.tensor(np.ascontiguousarray(Q.reshape(E, 5, -1)), dtype=torch.float64, device="cuda")


def _afb_case(name):
    """The Table 1/2 parameter set on its almost-flux-balance background (2 x 2 x 2 x 2 shell, p = 3)."""
    from paper_1503_00834_gb300 import native

    beta, phys = paper_case_phys(name)
    prof = native.afb_profile(native.Params.from_phys(phys), beta, 1.0, 16385)
    r0, r1, rho, pr = prof
    phys = dataclasses.replace(phys, T_top=float(np.interp(1.0, np.linspace(r0, r1, rho.size), pr / (phys.R_gas * rho))))
    return ShellConfig(f"{name}_afb_2x2_p3", 2, 2, 3, beta, 1.0, 7, 1e-3, 10, phys)


CASES = [SHELL_288_P3, small_shell(2, 2, 2), small_shell(2, 2, 4), small_shell(1, 2, 5),
         small_shell(1, 1, 3, N_rho=0.5), "jupiter", "sun"]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c if isinstance(c, str) else c.name)
def test_fp64_residual_within_oracle_rounding_of_extended_precision(case):
    from oracle import afb
    from oracle import state as ostate
    from oracle.residual import residual
    from paper_1503_00834_gb300 import FP64, Shell

    cfg = _afb_case(case) if isinstance(case, str) else case
    osh = OracleShell(cfg)
    if isinstance(case, str):
        Q = ostate.initial_state(osh.ph, osh.geometry()["x"], cfg.seed, cfg.entropy_amp,
                                 Q0=afb.background(osh.ph, osh.geometry()["x"]))
    else:
        Q = osh.initial_state()
    W = osh.weights()
    sh = Shell(cfg)
    Qd = _upload(Q)
    R = torch.empty_like(Qd)
    ws = torch.empty(sh.mesh.workspace_bytes(FP64), dtype=torch.uint8, device="cuda")
    sh.mesh.residual(sh.params, FP64, Qd, R, ws)
    sh.mesh.check()
    Rx = residual(_extended(osh), osh.ph, Q.astype(LD))
    e_gpu = _rel(to5(R, cfg.p + 1), Rx, W)
    e_ora = _rel(residual(osh.disc, osh.ph, Q), Rx, W)
    print(f"{cfg.name}: FP64 residual vs extended precision: GPU {e_gpu}, FP64 oracle {e_ora}")
    assert np.all(e_gpu <= np.maximum(1e-12, 2.0 * e_ora)), (e_gpu, e_ora)


@pytest.mark.parametrize("scheme", [0, 1], ids=["ssprk3", "ssprk54"])
@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_fp64_steps_within_oracle_rounding_of_extended_precision(p, scheme):
    from oracle import rk
    from paper_1503_00834_gb300 import FP64, Shell

    cfg = small_shell(2, 1, p)
    n_steps = 6 if scheme == 0 else 4
    osh = OracleShell(cfg)
    Q = osh.initial_state()
    Q0 = osh.background().astype(LD)
    W = osh.weights()
    sh = Shell(cfg)
    Qd = _upload(Q)
    ws = torch.empty(sh.mesh.workspace_bytes(FP64), dtype=torch.uint8, device="cuda")
    sh.mesh.rk_step_scheme(sh.params, FP64, scheme, Qd, ws, sh.dt, n_steps)
    sh.mesh.check()
    name = "ssprk3" if scheme == 0 else "ssprk54"
    Qx = rk.run(_extended(osh), osh.ph, Q.astype(LD), sh.dt, n_steps, scheme=name)
    Q64 = rk.run(osh.disc, osh.ph, Q, sh.dt, n_steps, scheme=name)
    e_gpu = _rel(to5(Qd, p + 1) - Q0, Qx - Q0, W)
    e_ora = _rel(Q64 - Q0, Qx - Q0, W)
    print(f"p={p} {name} {n_steps} steps, q' vs extended precision: GPU {e_gpu}, FP64 oracle {e_ora}")
    assert np.all(e_gpu <= np.maximum(1e-12, 2.0 * e_ora)), (e_gpu, e_ora)
