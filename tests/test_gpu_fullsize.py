"""Parity at the full workload sizes, in the launch configuration bench.py times.

The GPU evaluates the whole shell; the oracle evaluates sampled elements one neighbourhood at a
time (the residual of an element depends on its two-face-hop neighbourhood, one SSP-RK3 step on
its six-hop neighbourhood).  Samples cover wall layers, panel seams and interior elements.
Tolerances as in test_gpu_parity: FP32 perturbation path 1e-5 relative L2 over the sample, FP64
1e-12 relative backward error (the measured condition number of the sampled residual).
"""
import numpy as np
import pytest

from chorus_inputs import SHELL_331776_P3, SHELL_786432_P4, cubed_sphere_hex20
from gpu_common import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00834_gb300 import build

    build.build()


def _sample(cfg, count, seed):
    """Element indices: wall layers, both panel seams and random interior elements."""
    rng = np.random.default_rng(seed)
    n, n_r = cfg.n, cfg.n_r

    def eid(panel, j, i, k):
        return ((panel * n + j) * n + i) * n_r + k

    fixed = [eid(0, 0, 0, 0), eid(1, n - 1, n - 1, n_r - 1), eid(4, 0, n // 2, 0), eid(5, n // 2, n - 1, n_r - 1),
             eid(2, n // 2, 0, n_r // 2), eid(3, n - 1, n // 2, 1)]
    rand = rng.choice(cfg.n_elem, size=count - len(fixed), replace=False)
    return np.unique(np.concatenate([fixed, rand]))


class _Oracle:
    def __init__(self, cfg):
        from oracle.physics import Physics
        from oracle.residual import Discretization

        self.cfg = cfg
        xyz, h20 = cubed_sphere_hex20(cfg.n, cfg.n_r, cfg.r_inner, cfg.r_outer)
        self.disc = Discretization(xyz, h20, cfg.p, cfg.r_inner, cfg.r_outer)
        self.ph = Physics.from_params(cfg.phys, cfg.r_inner, cfg.r_outer)
        self.N = cfg.p + 1

    def closure(self, elems, hops):
        for _ in range(hops):
            elems = self.disc.conn.closure(elems)
        return elems

    def state(self, patch):
        from oracle import state as ostate

        cfg = self.cfg
        Q = np.zeros((self.disc.n_elem, 5) + (self.N,) * 3)
        x = self.disc.geometry(patch)["x"]
        Q[patch] = ostate.initial_state(self.ph, x, cfg.seed, cfg.entropy_amp, elems=patch)
        return Q

    def weights(self, elems):
        w = self.disc.ops.w
        g = self.disc.geometry(elems)
        return w[None, :, None, None] * w[None, None, :, None] * w[None, None, None, :] * g["detJ"]

    def background(self, elems):
        from oracle import state as ostate

        return ostate.background(self.ph, self.disc.geometry(elems)["x"])


def _gpu_state(cfg, prec):
    from paper_1503_00834_gb300 import Shell

    sh = Shell(cfg)
    dtype = torch.float64 if prec == 0 else torch.float32
    Q = torch.empty(sh.mesh.state_shape(), dtype=dtype, device="cuda")
    sh.mesh.state_init(sh.params, cfg.seed, cfg.entropy_amp, prec, Q)
    ws = torch.empty(sh.mesh.workspace_bytes(prec), dtype=torch.uint8, device="cuda")
    return sh, Q, ws


def _rows(t, elems, N):
    return t[torch.as_tensor(elems, device=t.device)].double().cpu().numpy().reshape(len(elems), 5, N, N, N)


@pytest.mark.parametrize("cfg", [SHELL_331776_P3, SHELL_786432_P4], ids=lambda c: c.name)
def test_fullsize_residual_sampled(cfg):
    from oracle.residual import residual
    from paper_1503_00834_gb300 import FP32_PERT, FP64

    orc = _Oracle(cfg)
    elems = _sample(cfg, 24, 5)
    patch = orc.closure(elems, 2)
    Q = orc.state(patch)
    Rref = residual(orc.disc, orc.ph, Q, elems)
    W = orc.weights(elems)
    N = cfg.p + 1
    precs = [FP32_PERT, FP64] if cfg is SHELL_331776_P3 else [FP32_PERT]
    for prec in precs:
        sh, q, ws = _gpu_state(cfg, prec)
        R = torch.empty_like(q)
        sh.mesh.residual(sh.params, prec, q, R, ws)
        sh.mesh.check()
        got = _rows(R, elems, N)
        e, ev = rel_err(got, Rref, W)
        print(f"{cfg.name} prec {prec}: sampled residual rel err {ev}")
        if prec == FP32_PERT:
            assert e < 1e-5
        else:
            rng = np.random.default_rng(1)
            Qp = Q.copy()
            Qp[patch] *= 1.0 + 1e-10 * rng.uniform(-1.0, 1.0, Qp[patch].shape)
            _, rel = rel_err(residual(orc.disc, orc.ph, Qp, elems), Rref, W)
            kappa = rel / 1e-10
            print(f"condition {kappa}")
            assert np.all(ev <= 1e-12 * np.maximum(1.0, kappa))
        del sh, q, ws, R
        torch.cuda.empty_cache()


def test_fullsize_rk_step_sampled():
    """One SSP-RK3 step of the 331,776-element shell, FP32 perturbation path, as bench.py runs it."""
    from oracle.residual import residual
    from oracle.rk import SSPRK3
    from paper_1503_00834_gb300 import FP32_PERT

    cfg = SHELL_331776_P3
    orc = _Oracle(cfg)
    elems = _sample(cfg, 12, 9)
    sh, q, ws = _gpu_state(cfg, FP32_PERT)
    dt = sh.dt
    sh.mesh.rk_step(sh.params, FP32_PERT, q, ws, dt, 1)
    sh.mesh.check()
    # stage k needs the residual on the (3-k)*2-hop neighbourhood of the sample
    patches = [orc.closure(elems, 4), orc.closure(elems, 2), elems]
    u = orc.state(orc.closure(elems, 6))
    s = u
    for (a, b), P in zip(SSPRK3, patches):
        s_new = np.zeros_like(u)
        s_new[P] = a * u[P] + b * (s[P] + dt * residual(orc.disc, orc.ph, s, P))
        s = s_new
    ref = s[elems] - orc.background(elems)
    got = _rows(q, elems, cfg.p + 1)
    e, ev = rel_err(got, ref, orc.weights(elems))
    print(f"rk step sampled rel err on q' {ev}")
    assert e < 1e-5


@pytest.mark.parametrize("cfg", [SHELL_786432_P4, SHELL_331776_P3], ids=lambda c: c.name)
def test_fullsize_runs_stay_bounded(cfg):
    """100 SSP-RK3 steps at the stable step (the solar shell's run length): finite, mass conserved to
    FP64 reduction round-off, kinetic energy bounded (the spurious flows of the discrete hydrostatic
    imbalance decay; an unstable step grows them exponentially and goes non-finite within ~30 steps)."""
    from paper_1503_00834_gb300 import FP32_PERT

    sh, q, ws = _gpu_state(cfg, FP32_PERT)
    sh.mesh.rk_step(sh.params, FP32_PERT, q, ws, sh.dt, 10)
    r10 = sh.mesh.reduce(sh.params, FP32_PERT, q)
    sh.mesh.rk_step(sh.params, FP32_PERT, q, ws, sh.dt, 90)
    r100 = sh.mesh.reduce(sh.params, FP32_PERT, q)
    print(f"{cfg.name}: KE after 10 steps {r10[2]:.3e}, after 100 steps {r100[2]:.3e}; mass {r10[0]!r} {r100[0]!r}")
    assert np.all(np.isfinite(r100))
    assert r100[2] <= 10.0 * r10[2]
    assert abs(r100[0] - r10[0]) <= 1e-6 * abs(r10[0])
    del sh, q, ws
    torch.cuda.empty_cache()
