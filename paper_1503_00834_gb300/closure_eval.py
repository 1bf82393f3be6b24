"""Evaluation of the learned subgrid closure on the 98,304-element shell (p = 2 coarse, p = 5 fine).

Procedure (every step runs in the library's kernels; this module only orders the calls and
computes the two error diagnostics on the host):
  1. A seeded p = 5 run with FP32 perturbation storage and SSP-RK3 at the common step
     dt = min(dt_5, dt_2).  Its projection to p = 2 (per-element L2 projection) at every checkpoint
     is the reference trajectory.  Both orders run well balanced (chorus_set_well_balanced): the
     discrete residual of the background is left out, so each run's perturbation evolves under its
     own dynamics and not under its order's hydrostatic truncation error.
  2. Training pairs from snapshots of the p = 5 run up to `train_until`: input the projected state,
     target (chorus_closure_make_pairs), scaled per variable by the RMS of the training data; Adam on
     the shuffled pairs.  Snapshots after `train_until` are held out.  Two targets:
       - "residual" (a priori): P R_5(Q_5) - R_2(P Q_5), the coarse residual's one-step defect;
       - "rollout" (multi-step, no adjoint of the residual needed): the projected fine state
         `horizon` steps later minus the plain coarse state after `horizon` steps from the same
         projected state, divided by horizon * dt - the mean tendency the coarse run misses over
         that window.
  3. Plain p = 2 and closure-corrected p = 2 runs (the correction also relaxed by factors below one)
     from the projected initial state, compared with the reference at the checkpoints by
       - the relative L2 error of the perturbation, per variable, maximum over variables, and
       - the kinetic-energy spectrum error: w = m / sqrt(rho) is expanded per element in the
         orthonormal Legendre basis of [0,1]^3 (degree <= 2 per direction); E(d) sums
         |w_hat_abc|^2 / 2 times the element volume over a + b + c = d; the error is
         sum_d |E(d) - E_ref(d)| / sum_d E_ref(d).

  python -m paper_1503_00834_gb300.closure_eval [--steps 2000] [--check-every 100] ...
prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np


def _solution_points(N: int) -> np.ndarray:
    """Chebyshev-Gauss points on [0,1] (Eq. 13)."""
    s = np.arange(N)
    return 0.5 * (1.0 - np.cos((2 * s + 1) * np.pi / (2 * N)))


def _legendre_inverse_vandermonde(N: int) -> np.ndarray:
    """Modal coefficients of the orthonormal Legendre basis from nodal values at the solution points."""
    X = _solution_points(N)
    t = 2.0 * X - 1.0
    P = [np.ones_like(t), t]
    for a in range(2, N):
        P.append(((2 * a - 1) * t * P[a - 1] - (a - 1) * P[a - 2]) / a)
    V = np.stack([math.sqrt(2 * a + 1) * P[a] for a in range(N)], axis=1)  # V[s, a]
    return np.linalg.inv(V)


def _element_volumes(xyz: np.ndarray, h20: np.ndarray) -> np.ndarray:
    """Volumes of the hexahedra spanned by the eight corners (five-tetrahedron split)."""
    c = xyz[h20[:, :8]]
    tets = ((0, 1, 3, 4), (1, 2, 3, 6), (1, 4, 5, 6), (3, 4, 6, 7), (1, 3, 4, 6))
    vol = np.zeros(h20.shape[0])
    for a, b, cc, d in tets:
        vol += np.abs(np.einsum("ei,ei->e", c[:, b] - c[:, a], np.cross(c[:, cc] - c[:, a], c[:, d] - c[:, a]))) / 6.0
    return vol


class Diagnostics:
    def __init__(self, xyz, h20, N, Q0):
        self.N = N
        self.vol = _element_volumes(xyz, h20)
        X = _solution_points(N)
        # interpolatory quadrature weights of the solution points (integrals of the Lagrange basis)
        V = np.vander(X, N, increasing=True)
        w = np.linalg.solve(V.T, 1.0 / np.arange(1, N + 1))
        self.w3 = (w[:, None, None] * w[None, :, None] * w[None, None, :])  # axes k, j, i
        self.Vinv = _legendre_inverse_vandermonde(N)
        self.rho0 = Q0[:, 0]  # [E, N, N, N]
        a = np.arange(N)
        self.deg = a[:, None, None] + a[None, :, None] + a[None, None, :]

    def l2(self, q, ref):
        W = self.vol[:, None, None, None] * self.w3[None]
        num = np.sqrt(np.sum(W[:, None] * (q - ref) ** 2, axis=(0, 2, 3, 4)))
        den = np.sqrt(np.sum(W[:, None] * ref ** 2, axis=(0, 2, 3, 4)))
        e = num / np.where(den > 0, den, 1.0)
        return float(e.max())

    def ke_spectrum(self, q):
        rho = self.rho0 + q[:, 0]
        wv = q[:, 1:4] / np.sqrt(rho)[:, None]  # [E, 3, k, j, i]
        V = self.Vinv
        wh = np.einsum("ak,bj,ci,exkji->exabc", V, V, V, wv)
        en = 0.5 * np.sum(wh ** 2, axis=1) * self.vol[:, None, None, None]  # [E, a, b, c]
        return np.array([en[:, self.deg == d].sum() for d in range(3 * (self.N - 1) + 1)])

    def ke_error(self, q, ref):
        Em, Er = self.ke_spectrum(q), self.ke_spectrum(ref)
        return float(np.abs(Em - Er).sum() / max(Er.sum(), 1e-300))


def evaluate(steps=2000, check_every=100, snap_every=50, train_until=1000, epochs=20, batch=1024, lr=1e-3,
             seed=11, relax=(1.0, 0.5, 0.25, 0.1), target="residual", horizon=50):
    """relax: factors applied to the trained closure's output (one coarse run each).  target:
    "residual" or "rollout" (horizon steps; a multiple of snap_every)."""
    if target == "rollout" and horizon % snap_every:
        raise ValueError("the rollout horizon must be a multiple of snap_every")
    import torch

    from chorus_inputs import SHELL_98304_P2, SHELL_98304_P5, cubed_sphere_hex20

    from . import FP32_PERT, FP64, Shell, native

    t_all = time.perf_counter()
    fine, coarse = Shell(SHELL_98304_P5), Shell(SHELL_98304_P2)
    fine.mesh.prepare(fine.params)
    coarse.mesh.prepare(coarse.params)
    # both orders well balanced: their background truncation residuals differ, and would otherwise
    # drive each run's perturbation (and the closure target) more than the dynamics compared
    fine.mesh.set_well_balanced(True)
    coarse.mesh.set_well_balanced(True)
    dt = min(fine.dt, coarse.dt)
    cfg = fine.cfg
    f32 = dict(dtype=torch.float32, device="cuda")
    qf = torch.empty(fine.mesh.state_shape(), **f32)
    fine.mesh.state_init(fine.params, cfg.seed, cfg.entropy_amp, FP32_PERT, qf)
    wsf = torch.empty(fine.mesh.workspace_bytes(FP32_PERT), dtype=torch.uint8, device="cuda")
    wsc = torch.empty(coarse.mesh.workspace_bytes(FP32_PERT), dtype=torch.uint8, device="cuda")
    cshape = coarse.mesh.state_shape()
    E, Nc = cshape[0], coarse.cfg.p + 1

    def project_and_pair(q):
        Rf = torch.empty_like(q)
        fine.mesh.residual(fine.params, FP32_PERT, q, Rf, wsf)
        qc, PRf, Rc = torch.empty(cshape, **f32), torch.empty(cshape, **f32), torch.empty(cshape, **f32)
        native.project(fine.mesh, coarse.mesh, FP32_PERT, 0, q, qc)
        native.project(fine.mesh, coarse.mesh, FP32_PERT, 1, Rf, PRf)
        coarse.mesh.residual(coarse.params, FP32_PERT, qc, Rc, wsc)
        return qc, PRf, Rc

    # ---- 1. fine run: reference checkpoints and snapshots
    t0 = time.perf_counter()
    ref, snaps = {}, []
    n = 0
    stride = math.gcd(check_every, snap_every)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fine_ms = 0.0
    while True:
        if n % check_every == 0 or n % snap_every == 0:
            qc, PRf, Rc = project_and_pair(qf)
            if n % check_every == 0:
                ref[n] = qc.cpu().numpy().astype(np.float64).reshape(E, 5, Nc, Nc, Nc)
            if n % snap_every == 0:
                snaps.append((n, qc, PRf, Rc))
        if n >= steps:
            break
        ev0.record()
        fine.mesh.rk_step(fine.params, FP32_PERT, qf, wsf, dt, stride)
        ev1.record()
        torch.cuda.synchronize()
        fine_ms += ev0.elapsed_time(ev1)
        n += stride
    fine_run_s = time.perf_counter() - t0

    # ---- rollout targets: (P Q_5(n + horizon) - coarse^horizon(P Q_5(n))) / (horizon dt), in the slot of
    # the projected fine residual, with a zero coarse residual (make_pairs forms their difference)
    if target == "rollout":
        by_step = {st: qc for st, qc, _, _ in snaps}
        zero = torch.zeros(cshape, **f32)
        rolled = []
        for st, qc, _, _ in snaps:
            if st + horizon not in by_step:
                continue
            q = qc.clone()
            coarse.mesh.rk_step(coarse.params, FP32_PERT, q, wsc, dt, horizon)
            rolled.append((st, qc, (by_step[st + horizon] - q) / (horizon * dt), zero))
        snaps = rolled

    # ---- 2. pairs, scales, training
    t0 = time.perf_counter()
    unit = native.closure_alloc(seed, [1.0] * 5, [1.0] * 5)
    X = torch.empty((E, 135), **f32)
    Y = torch.empty((E, 135), **f32)
    sx, sy, cnt = np.zeros(5), np.zeros(5), 0
    for step, qc, PRf, Rc in snaps:
        if step > train_until:
            continue
        native.closure_make_pairs(coarse.mesh, FP32_PERT, unit, qc, PRf, Rc, X, Y)
        sx += (X.view(E, 5, 27).double() ** 2).sum(dim=(0, 2)).cpu().numpy()
        sy += (Y.view(E, 5, 27).double() ** 2).sum(dim=(0, 2)).cpu().numpy()
        cnt += E * 27
    in_scale = [float(max(math.sqrt(v / cnt), 1e-12)) for v in sx]
    out_scale = [float(max(math.sqrt(v / cnt), 1e-12)) for v in sy]
    w = native.closure_alloc(seed, in_scale, out_scale)
    Xtr, Ytr, Xte, Yte = [], [], [], []
    for step, qc, PRf, Rc in snaps:
        Xs, Ys = torch.empty((E, 135), **f32), torch.empty((E, 135), **f32)
        native.closure_make_pairs(coarse.mesh, FP32_PERT, w, qc, PRf, Rc, Xs, Ys)
        (Xtr if step <= train_until else Xte).append(Xs)
        (Ytr if step <= train_until else Yte).append(Ys)
    Xtr, Ytr = torch.cat(Xtr), torch.cat(Ytr)
    g = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(Xtr.shape[0], generator=g).to("cuda")
    Xtr, Ytr = Xtr[perm].contiguous(), Ytr[perm].contiguous()
    te0 = time.perf_counter()
    losses = native.closure_train(Xtr, Ytr, w, epochs=epochs, batch=batch, lr=lr)
    train_s = time.perf_counter() - te0
    held = None
    if Xte:
        Xte, Yte = torch.cat(Xte), torch.cat(Yte)
        Yp = torch.empty_like(Xte)
        native.closure_forward(w, Xte, Yp)
        held = float(torch.linalg.norm(Yp - Yte).item() / max(torch.linalg.norm(Yte).item(), 1e-300))
    pairs_s = time.perf_counter() - t0
    del snaps

    # ---- 3. coarse runs from the projected initial state
    xyz, h20 = cubed_sphere_hex20(coarse.cfg.n, coarse.cfg.n_r, coarse.cfg.r_inner, coarse.cfg.r_outer)
    Q0 = torch.empty(cshape, dtype=torch.float64, device="cuda")
    coarse.mesh.state_init(coarse.params, 0, 0.0, FP64, Q0)  # amplitude 0: the background itself
    diag = Diagnostics(xyz, h20, Nc, Q0.cpu().numpy().reshape(E, 5, Nc, Nc, Nc))
    q_init = torch.tensor(ref[0].reshape(cshape), **f32)
    out = {}
    runs = [("plain", None, 1.0)] + [(f"closure_x{a:g}", w, a) for a in relax]
    for name, rec, a in runs:
        if rec is not None:
            native.closure_set_scales(rec, in_scale, [s * a for s in out_scale])
        native.closure_attach(coarse.mesh, rec)
        q = q_init.clone()
        l2, ke, ms, n = [], [], 0.0, 0
        while True:
            if n % check_every == 0:
                qa = q.cpu().numpy().astype(np.float64).reshape(E, 5, Nc, Nc, Nc)
                if not np.all(np.isfinite(qa)):
                    l2.append(float("nan"))
                    ke.append(float("nan"))
                    break
                l2.append(diag.l2(qa, ref[n]))
                ke.append(diag.ke_error(qa, ref[n]))
            if n >= steps:
                break
            ev0.record()
            coarse.mesh.rk_step(coarse.params, FP32_PERT, q, wsc, dt, check_every)
            ev1.record()
            torch.cuda.synchronize()
            ms += ev0.elapsed_time(ev1)
            n += check_every
        native.closure_attach(coarse.mesh, None)
        out[name] = dict(l2=l2, ke=ke, dof_stage_per_s=coarse.cfg.n_dof * 3 * n / max(ms / 1e3, 1e-12))
    ke_ref = diag.ke_spectrum(ref[max(ref)])
    return {
        "workload": "shell_98304: p=5 reference, p=2 plain and p=2 + learned closure",
        "dt": dt, "steps": steps, "checkpoints": list(range(0, steps + 1, check_every)),
        "l2": {k: v["l2"] for k, v in out.items()},
        "ke_err": {k: v["ke"] for k, v in out.items()},
        "ke_spectrum_ref_final": ke_ref.tolist(),
        "train": {"target": target, "horizon": horizon if target == "rollout" else 1,
                  "pairs": int(Xtr.shape[0]), "epochs": epochs, "batch": batch, "lr": lr,
                  "loss_first": losses[0], "loss_last": losses[-1], "held_out_ratio": held,
                  "in_scale": in_scale, "out_scale": out_scale, "train_until": train_until,
                  "snap_every": snap_every},
        "throughput": {"p5_dof_stage_per_s": cfg.n_dof * 3 * steps / max(fine_ms / 1e3, 1e-12),
                       "p2_plain_dof_stage_per_s": out["plain"]["dof_stage_per_s"],
                       "p2_closure_dof_stage_per_s": out[runs[1][0]]["dof_stage_per_s"]},
        "seconds": {"fine_run": fine_run_s, "pairs_and_training": pairs_s, "training": train_s,
                    "total": time.perf_counter() - t_all},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--check-every", type=int, default=100)
    ap.add_argument("--snap-every", type=int, default=50)
    ap.add_argument("--train-until", type=int, default=1000)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--target", default="residual", choices=["residual", "rollout"])
    ap.add_argument("--horizon", type=int, default=50)
    ap.add_argument("--relax", default="1,0.5,0.25,0.1")
    a = ap.parse_args()
    from . import build

    build.build()
    relax = tuple(float(x) for x in a.relax.split(","))
    print(json.dumps(evaluate(a.steps, a.check_every, a.snap_every, a.train_until, a.epochs, a.batch, a.lr,
                              relax=relax, target=a.target, horizon=a.horizon)))


if __name__ == "__main__":
    main()
