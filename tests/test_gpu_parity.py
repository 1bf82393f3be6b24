"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances (see the module docstring of gpu_common for the norm):
  * FP64 residual: 1e-12 relative *backward* error.  The residual of a near-hydrostatic state is a
    difference of O(rho g) terms that cancel to the perturbation level, so its relative forward
    error is its condition number times the backward error.  The test measures the condition
    number kappa_v of each variable on the oracle (relative change of R_v under a random relative
    input change of 1e-10, divided by 1e-10) and requires e_v <= 1e-12 * max(1, kappa_v).
  * FP64 states after RK steps (compared on q' = Q - Q0): two error sources bound the agreement.
    (a) the residual's backward error, amplified by the same condition numbers kappa_v, enters
    each stage as dt R; summed over the run it is at most 1e-12 * kappa_v relative to q' as long as
    the run changes q' by no more than its own size; (b) FP64 storage of the total state Q rounds
    by eps |Q0| per stage, which is large relative to q' for density and energy; the test
    measures (b) by re-running the oracle with a relative 2^-53 perturbation of the state after
    every stage.  Tolerance: max(1e-12 * max(1, kappa_v), 10 x that spread).
  * FP32 perturbation path: 1e-5 relative L2 for the residual and for q' after steps.
"""
import numpy as np
import pytest

from chorus_inputs import SHELL_288_P3, small_shell
from gpu_common import OracleShell, rel_err, to5

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00834_gb300 import build

    build.build()


def _gpu(cfg):
    from paper_1503_00834_gb300 import Shell

    return Shell(cfg)


def _alloc(mesh, prec, n=1):
    dt = torch.float64 if prec == 0 else torch.float32
    return [torch.empty(mesh.state_shape(), dtype=dt, device="cuda") for _ in range(n)]


def _ws(mesh, prec):
    return torch.empty(mesh.workspace_bytes(prec), dtype=torch.uint8, device="cuda")


def _condition(osh, Q, R_ref, W, delta=1e-10):
    """Per-variable condition number of the oracle residual under a random relative input change."""
    from oracle.residual import residual

    rng = np.random.default_rng(123)
    Qp = Q * (1.0 + delta * rng.uniform(-1.0, 1.0, Q.shape))
    _, rel = rel_err(residual(osh.disc, osh.ph, Qp), R_ref, W)
    return rel / delta


# the one-element-thick shell uses a mild stratification so that its traces stay positive
CASES = [SHELL_288_P3, small_shell(2, 2, 2), small_shell(2, 2, 4), small_shell(1, 2, 5),
         small_shell(1, 1, 3, N_rho=0.5)]


@pytest.mark.parametrize("cfg", CASES, ids=lambda c: c.name)
def test_initial_state_matches_oracle(cfg):
    from paper_1503_00834_gb300 import FP32_PERT, FP64

    sh = _gpu(cfg)
    osh = OracleShell(cfg)
    Q64, q32 = _alloc(sh.mesh, FP64)[0], _alloc(sh.mesh, FP32_PERT)[0]
    sh.mesh.state_init(sh.params, cfg.seed, cfg.entropy_amp, FP64, Q64)
    sh.mesh.state_init(sh.params, cfg.seed, cfg.entropy_amp, FP32_PERT, q32)
    torch.cuda.synchronize()
    Qref = osh.initial_state()
    N = cfg.p + 1
    W = osh.weights()
    assert np.max(np.abs(to5(Q64, N) - Qref)) <= 1e-14 * np.max(np.abs(Qref))
    Q0 = osh.background()
    e, _ = rel_err(to5(q32, N), Qref - Q0, W)
    assert e < 1e-6  # FP32 rounding of the perturbation


@pytest.mark.parametrize("cfg", CASES, ids=lambda c: c.name)
def test_residual_fp64_and_fp32_match_oracle(cfg):
    from oracle.residual import residual
    from paper_1503_00834_gb300 import FP32_PERT, FP64

    sh = _gpu(cfg)
    osh = OracleShell(cfg)
    N = cfg.p + 1
    Q64, R64 = _alloc(sh.mesh, FP64, 2)
    q32, R32 = _alloc(sh.mesh, FP32_PERT, 2)
    sh.mesh.state_init(sh.params, cfg.seed, cfg.entropy_amp, FP64, Q64)
    sh.mesh.state_init(sh.params, cfg.seed, cfg.entropy_amp, FP32_PERT, q32)
    sh.mesh.residual(sh.params, FP64, Q64, R64, _ws(sh.mesh, FP64))
    sh.mesh.residual(sh.params, FP32_PERT, q32, R32, _ws(sh.mesh, FP32_PERT))
    sh.mesh.check()
    Q = osh.initial_state()
    Rref = residual(osh.disc, osh.ph, Q)
    W = osh.weights()
    _, e64 = rel_err(to5(R64, N), Rref, W)
    kappa = _condition(osh, Q, Rref, W)
    print(f"{cfg.name}: FP64 residual rel err {e64}, condition {kappa}")
    assert np.all(e64 <= 1e-12 * np.maximum(1.0, kappa))
    e32, ev = rel_err(to5(R32, N), Rref, W)
    print(f"{cfg.name}: FP32 residual rel err {ev}")
    assert e32 < 1e-5


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32pert"])
def test_rk_steps_match_oracle(prec):
    """The 288-element p=3 shell advanced by SSP-RK3 on both sides; compared on q' = Q - Q0."""
    from oracle import rk
    from paper_1503_00834_gb300 import FP64

    cfg = SHELL_288_P3
    n_steps = 100 if prec == FP64 else 20
    sh = _gpu(cfg)
    osh = OracleShell(cfg)
    N = cfg.p + 1
    Q = _alloc(sh.mesh, prec)[0]
    sh.mesh.state_init(sh.params, cfg.seed, cfg.entropy_amp, prec, Q)
    sh.mesh.rk_step(sh.params, prec, Q, _ws(sh.mesh, prec), sh.dt, n_steps)
    sh.mesh.check()
    Qinit = osh.initial_state()
    Qref = rk.run(osh.disc, osh.ph, Qinit, sh.dt, n_steps)
    Q0 = osh.background()
    W = osh.weights()
    got = to5(Q, N) - (Q0 if prec == FP64 else 0.0)
    e, ev = rel_err(got, Qref - Q0, W)
    print(f"rk {n_steps} steps prec {prec}: rel err on q' {ev}")
    if prec == FP64:
        from oracle.residual import residual

        noisy = _noisy_run(osh, Qinit, sh.dt, n_steps)
        _, spread = rel_err(noisy - Q0, Qref - Q0, W)
        kappa = _condition(osh, Qinit, residual(osh.disc, osh.ph, Qinit), W)
        print(f"oracle rounding spread {spread}, residual condition {kappa}")
        assert np.all(ev <= np.maximum(1e-12 * np.maximum(1.0, kappa), 10.0 * spread))
    else:
        assert e < 1e-5


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32pert"])
@pytest.mark.parametrize("p", [2, 4, 5])
def test_rk_steps_match_oracle_other_orders(p, prec):
    """RK mode (stage combination, next-stage traces) of the p = 2, 4, 5 kernels: 10 SSP-RK3 steps
    of a 24-element shell, same tolerances as the p = 3 trajectory test."""
    from oracle import rk
    from oracle.residual import residual
    from paper_1503_00834_gb300 import FP64

    cfg = small_shell(2, 1, p)
    n_steps = 10
    sh = _gpu(cfg)
    osh = OracleShell(cfg)
    Q = _alloc(sh.mesh, prec)[0]
    sh.mesh.state_init(sh.params, cfg.seed, cfg.entropy_amp, prec, Q)
    sh.mesh.rk_step(sh.params, prec, Q, _ws(sh.mesh, prec), sh.dt, n_steps)
    sh.mesh.check()
    Qinit = osh.initial_state()
    Qref = rk.run(osh.disc, osh.ph, Qinit, sh.dt, n_steps)
    Q0 = osh.background()
    W = osh.weights()
    got = to5(Q, p + 1) - (Q0 if prec == FP64 else 0.0)
    e, ev = rel_err(got, Qref - Q0, W)
    print(f"p={p} rk {n_steps} steps prec {prec}: rel err on q' {ev}")
    if prec == FP64:
        noisy = _noisy_run(osh, Qinit, sh.dt, n_steps)
        _, spread = rel_err(noisy - Q0, Qref - Q0, W)
        kappa = _condition(osh, Qinit, residual(osh.disc, osh.ph, Qinit), W)
        assert np.all(ev <= np.maximum(1e-12 * np.maximum(1.0, kappa), 10.0 * spread))
    else:
        assert e < 1e-5


def _noisy_run(osh, Q, dt, n_steps, scheme="ssprk3"):
    """The oracle's SSP-RK3 or SSP-RK(5,4) with a relative 2^-53 random perturbation of the state
    after every stage (the FP64 storage rounding of the total state, made explicit)."""
    from oracle.residual import residual
    from oracle.rk import RK54, SSPRK3

    rng = np.random.default_rng(7)
    eps = 2.0 ** -53

    def noise(a):
        return a * (1.0 + eps * rng.uniform(-1.0, 1.0, a.shape))

    def L(a):
        return dt * residual(osh.disc, osh.ph, a)

    u = noise(Q)
    for _ in range(n_steps):
        if scheme == "ssprk3":
            s = u
            for a, b in SSPRK3:
                s = noise(a * u + b * (s + L(s)))
            u = s
        else:
            c = RK54
            u1 = noise(u + c["b10"] * L(u))
            u2 = noise(c["a20"] * u + c["a21"] * u1 + c["b21"] * L(u1))
            u3 = noise(c["a30"] * u + c["a32"] * u2 + c["b32"] * L(u2))
            L3 = L(u3)
            u4 = noise(c["a40"] * u + c["a43"] * u3 + c["b43"] * L3)
            u = noise(c["a52"] * u2 + c["a53"] * u3 + c["b53"] * L3 + c["a54"] * u4 + c["b54"] * L(u4))
    return u


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32pert"])
def test_rk54_steps_match_oracle(prec):
    """The paper's SSP-RK(5,4) (scheme 1) on the 288-element shell against the oracle, on q'."""
    from oracle import rk
    from paper_1503_00834_gb300 import FP64

    cfg = SHELL_288_P3
    n_steps = 10
    sh = _gpu(cfg)
    osh = OracleShell(cfg)
    N = cfg.p + 1
    Q = _alloc(sh.mesh, prec)[0]
    sh.mesh.state_init(sh.params, cfg.seed, cfg.entropy_amp, prec, Q)
    sh.mesh.rk_step_scheme(sh.params, prec, 1, Q, _ws(sh.mesh, prec), sh.dt, n_steps)
    sh.mesh.check()
    Qinit = osh.initial_state()
    Qref = rk.run(osh.disc, osh.ph, Qinit, sh.dt, n_steps, scheme="ssprk54")
    Q0 = osh.background()
    W = osh.weights()
    got = to5(Q, N) - (Q0 if prec == FP64 else 0.0)
    e, ev = rel_err(got, Qref - Q0, W)
    print(f"rk54 {n_steps} steps prec {prec}: rel err on q' {ev}")
    if prec == FP64:
        from oracle.residual import residual

        noisy = _noisy_run(osh, Qinit, sh.dt, n_steps, scheme="ssprk54")
        _, spread = rel_err(noisy - Q0, Qref - Q0, W)
        kappa = _condition(osh, Qinit, residual(osh.disc, osh.ph, Qinit), W)
        print(f"oracle rounding spread {spread}, residual condition {kappa}")
        assert np.all(ev <= np.maximum(1e-12 * np.maximum(1.0, kappa), 10.0 * spread))
    else:
        assert e < 1e-5


def test_reductions_match_oracle():
    from oracle.diagnostics import integrals
    from paper_1503_00834_gb300 import FP32_PERT, FP64

    cfg = SHELL_288_P3
    sh = _gpu(cfg)
    osh = OracleShell(cfg)
    Q64, q32 = _alloc(sh.mesh, FP64)[0], _alloc(sh.mesh, FP32_PERT)[0]
    sh.mesh.state_init(sh.params, cfg.seed, cfg.entropy_amp, FP64, Q64)
    sh.mesh.state_init(sh.params, cfg.seed, cfg.entropy_amp, FP32_PERT, q32)
    Q = osh.initial_state()
    ref = integrals(osh.disc, Q)
    out64 = sh.mesh.reduce(sh.params, FP64, Q64)
    out32 = sh.mesh.reduce(sh.params, FP32_PERT, q32)
    for out, tol in ((out64, 1e-13), (out32, 1e-9)):
        assert abs(out[0] - ref["mass"]) < tol * ref["mass"]
        assert abs(out[1] - ref["energy"]) < tol * ref["energy"]
        assert abs(out[2] - ref["kinetic"]) < 1e-30 + tol
        assert abs(out[3] - np.linalg.norm(ref["L"])) < 1e-30 + tol
    info = sh.mesh.info()
    assert abs(info["volume"] - ref["volume"]) < 1e-13 * ref["volume"]
    assert info["n_dof"] == cfg.n_dof and info["n_faces"] == 768 + 192


def test_freestream_on_gpu():
    """A uniform flow with no gravity or rotation stays uniform away from the walls (FP64 path)."""
    import dataclasses

    from chorus_inputs import ShellConfig
    from paper_1503_00834_gb300 import FP64, Params, Shell

    base = small_shell(2, 5, 3)
    phys = dataclasses.replace(base.phys, GM=1e-30, Omega=0.0, nu=0.0, kappa=0.0)
    cfg = ShellConfig(base.name, base.n, base.n_r, base.p, base.r_inner, base.r_outer, 1, 0.0, 1, phys)
    sh = Shell(cfg)
    N = cfg.p + 1
    E = cfg.n_elem
    rho, u, p, gam = 1.3, np.array([0.3, -0.2, 0.1]), 0.9, phys.gamma
    Qh = np.zeros((E, 5, N ** 3))
    Qh[:, 0], Qh[:, 1:4] = rho, (rho * u)[None, :, None]
    Qh[:, 4] = p / (gam - 1) + 0.5 * rho * u @ u
    Q = torch.tensor(Qh, device="cuda")
    R = torch.empty_like(Q)
    sh.mesh.residual(Params.from_phys(phys), FP64, Q, R, _ws(sh.mesh, FP64))
    Rh = R.cpu().numpy().reshape(E, -1)
    k = np.arange(E) % cfg.n_r
    interior = (k >= 1) & (k < cfg.n_r - 1)
    assert np.abs(Rh[interior]).max() < 1e-13 * 1.3 * N * N / sh.h_min


@pytest.mark.parametrize("n,n_r,p", [(8, 4, 5), (8, 2, 5), (16, 8, 4)])
def test_time_step_rule_is_stable(n, n_r, p):
    """Near-isotropic elements at p = 4, 5: 150 SSP-RK3 steps at the package's step stay finite
    with bounded kinetic energy (with the factor 0.5 these shells went non-finite within 18-60
    steps, in the oracle as in the library)."""
    from paper_1503_00834_gb300 import FP32_PERT

    cfg = small_shell(n, n_r, p)
    sh = _gpu(cfg)
    sh.mesh.prepare(sh.params)
    Q = _alloc(sh.mesh, FP32_PERT)[0]
    sh.mesh.state_init(sh.params, cfg.seed, cfg.entropy_amp, FP32_PERT, Q)
    ws = _ws(sh.mesh, FP32_PERT)
    sh.mesh.rk_step(sh.params, FP32_PERT, Q, ws, sh.dt, 10)
    ke10 = sh.mesh.reduce(sh.params, FP32_PERT, Q)[2]
    sh.mesh.rk_step(sh.params, FP32_PERT, Q, ws, sh.dt, 140)
    ke150 = sh.mesh.reduce(sh.params, FP32_PERT, Q)[2]
    print(f"{cfg.name}: KE {ke10:.3e} -> {ke150:.3e}")
    assert np.isfinite(ke150) and ke150 <= 10.0 * ke10


def test_well_balanced_residual_leaves_out_the_background_residual():
    """With the option on, the residual of q' is R(Q0 + q') - R(Q0): zero for q' = 0 and the plain
    residual minus the plain residual of the background otherwise, both to FP32 rounding."""
    from paper_1503_00834_gb300 import FP32_PERT

    cfg = small_shell(2, 2, 3)
    sh = _gpu(cfg)
    sh.mesh.prepare(sh.params)
    q, zero, R, R0, Rw, Rw0 = _alloc(sh.mesh, FP32_PERT, 6)
    ws = _ws(sh.mesh, FP32_PERT)
    sh.mesh.state_init(sh.params, cfg.seed, 1e-2, FP32_PERT, q)
    zero.zero_()
    sh.mesh.residual(sh.params, FP32_PERT, q, R, ws)
    sh.mesh.residual(sh.params, FP32_PERT, zero, R0, ws)
    sh.mesh.set_well_balanced(True)
    sh.mesh.residual(sh.params, FP32_PERT, q, Rw, ws)
    sh.mesh.residual(sh.params, FP32_PERT, zero, Rw0, ws)
    sh.mesh.set_well_balanced(False)
    torch.cuda.synchronize()
    # q' = 0: only FP32 rounding of the perturbation-form differences remains
    assert R0.abs().max().item() > 0
    assert Rw0.abs().max().item() <= 1e-6 * R0.abs().max().item(), (Rw0.abs().max().item(), R0.abs().max().item())
    d = (Rw - (R - R0)).abs().max().item()
    assert d <= 1e-5 * R.abs().max().item(), d
