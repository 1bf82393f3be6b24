#!/usr/bin/env python
"""Benchmark: RK-stage DOF updates per second of the SD residual + SSP-RK3 update on a shell.

Default workload: the 331,776-element p=3 shell (6 x 48 x 48 x 24 cubed sphere, 21,233,664
solution points x 5 variables), FP32 perturbation path, SSP-RK3.  One bench step = one SSP-RK3
time step = 3 passes of the whole residual + stage update; the metric counts solution-point DOF
updates per stage (DOF = elements x N^3, Eq. 19).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl chorus|reference] [--prec fp32|fp64]
                  [--workload batch_64|batch_16] [--schedule auto|serial|concurrent|persistent]

--workload batch_64 times the batch of 64 independent shells (orders 2-5, uneven sizes, 176M
solution points) advanced together: per-order union meshes, a captured step graph (the orders one
after another or on forked streams) or one persistent launch per stage, tile shapes and schedule
from the autotuner (--schedule overrides the schedule); batch_16 is the same family at a quarter of
the size.

--impl reference times the plain FP64 CPU oracle (the only reference implementation: the paper
ships no code) on the host cores, on a bounded sample of the same workload.
Under torchrun each rank runs an independent replica (the path is not sharded); the value is the
total over ranks and the time the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RK-stage DOF updates/s (p=3 shell), FP32 vs FP64 GPU at stated L2 error"
UNIT = "DOF-stage/s"
# algorithmic bytes per RK-stage DOF update at p=3: FP32 state traffic (read u^(k), read u^n on two of
# three stages, write: 13.3 words) + FP32 stored metrics (|J|, grad xi at the solution points and
# one metric row per flux point: 21.25 words) = 34.6 words = 138 B
ALG_BYTES_PER_DOF_STAGE = {2: 141.0, 3: 138.0, 4: 137.0, 5: 135.0}
ALG_BYTES_PER_DOF_STAGE_FP64 = {2: 283.0, 3: 277.0, 4: 273.0, 5: 271.0}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms: float, world: int, device: str = "cuda") -> float:
    """The slowest rank's time (the job's time); a no-op for one rank."""
    if world <= 1:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput: every rank processes its own replica's units in the job's time."""
    return world * units_per_rank / seconds


def kernel_sources_digest() -> str:
    """SHA-256 of the residual kernels' sources (the stepping kernels, their headers and the build
    script with its per-source compiler options), comments and blank lines left out: the DRAM
    counters in profiles/traffic.json are reported only for the code they were taken on."""
    import hashlib
    import re

    csrc = os.path.join(ROOT, "paper_1503_00834_gb300", "csrc")
    names = ["internal.h", "sd_device.cuh", "sd_kernels.cuh", "kern_inst.cuh"] + [f"kern_p{p}.cu" for p in (2, 3, 4, 5)]
    names.append(os.path.join("..", "build.py"))
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(csrc, n)) as f:
            text = f.read()
        # drop C++ line comments (none of these files has "//" inside a string) and Python comments
        pat = r"#.*$" if n.endswith(".py") else r"//.*$"
        code = "\n".join(ln.rstrip() for ln in re.sub(pat, "", text, flags=re.M).splitlines() if ln.strip())
        h.update(n.encode() + b"\0" + code.encode())
    return h.hexdigest()


def lookup_traffic(path: str, kernel: str, workload: str, prec: str):
    """DRAM bytes per launch of `kernel` on `workload` from an ncu summary file, or None when the file
    is missing or its counters were taken on other kernel sources than the ones built here."""
    try:
        with open(path) as f:
            tr = json.load(f)
    except (OSError, ValueError):
        return None
    if tr.get("sources_sha256") != kernel_sources_digest():
        return None
    return tr.get(f"{kernel}:{workload}:{prec}")


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo) and architecture."""
    import platform

    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                name = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not name:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith(("model name", "cpu part")):
                        name = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return f"{name or platform.processor() or 'unknown'} ({platform.machine()})"


def _reference_sample(cfg_name: str, e0: int, n_sample: int):
    """The oracle's one-stage update (residual + stage combination) of elements [e0, e0 + n_sample) of
    a workload, with the seeded initial state on their two-face-hop patch."""
    import numpy as np

    from chorus_inputs import CONFIGS, BATCH_64, cubed_sphere_hex20
    from oracle.physics import Physics
    from oracle.residual import Discretization, residual
    from oracle import state as ostate

    cfg = CONFIGS.get(cfg_name) or next(c for c in BATCH_64.shells() if c.name == cfg_name)
    xyz, h20 = cubed_sphere_hex20(cfg.n, cfg.n_r, cfg.r_inner, cfg.r_outer)
    disc = Discretization(xyz, h20, cfg.p, cfg.r_inner, cfg.r_outer)
    ph = Physics.from_params(cfg.phys, cfg.r_inner, cfg.r_outer)
    N = cfg.p + 1
    e0 = min(e0, max(0, disc.n_elem - n_sample))
    elems = np.arange(e0, min(disc.n_elem, e0 + n_sample))
    patch = disc.conn.closure(disc.conn.closure(elems))
    Q = np.zeros((disc.n_elem, 5, N, N, N))
    Q[patch] = ostate.initial_state(ph, disc.geometry(patch)["x"], cfg.seed, cfg.entropy_amp, elems=patch)
    dt = 1e-3

    def one_stage():
        R = residual(disc, ph, Q, elems)
        return Q[elems] + dt * R

    return one_stage, len(elems) * N ** 3, int(elems[0]), len(elems)


def _timed_stages(one_stage, warmup: int, steps, seconds):
    """Run warm-up stages, then `steps` timed stages (or stages until `seconds` have passed)."""
    for _ in range(max(0, warmup)):
        one_stage()
    times = []
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        one_stage()
        times.append(time.perf_counter() - t0)
        if steps is not None and len(times) >= steps:
            break
        if steps is None and time.perf_counter() - t_start >= seconds:
            break
    return times


def _reference_worker(cfg_name, e0, n_sample, warmup, steps, seconds, barrier, queue):
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    try:
        one_stage, units, first, n = _reference_sample(cfg_name, e0, n_sample)
        barrier.wait(timeout=600)
        times = _timed_stages(one_stage, warmup, steps, seconds)
        queue.put((units, times, first, n))
    except Exception as exc:  # reported by the parent
        try:
            barrier.abort()
        except Exception:
            pass
        queue.put(repr(exc))


def run_reference(cfg_name: str, n_workers: int, n_sample: int, warmup: int, steps=None, seconds=None):
    """The plain FP64 oracle (numpy, one thread per process) timed on `n_workers` host cores, each
    worker on its own block of n_sample elements of the workload, started together.  Returns
    (DOF-stage/s over all workers, per-step seconds of the slowest worker, description)."""
    if n_workers <= 1:
        one_stage, units, first, n = _reference_sample(cfg_name, 0, n_sample)
        times = _timed_stages(one_stage, warmup, steps, seconds)
        desc = (f"{len(times)} x (residual + stage update) on elements {first}..{first + n - 1} of {cfg_name} "
                f"(numpy FP64, one process, one thread), {sum(times):.2f} s")
        return units * len(times) / sum(times), times, desc
    import multiprocessing as mp

    ctx = mp.get_context("spawn")  # never fork a process that may hold a CUDA context
    barrier, queue = ctx.Barrier(n_workers), ctx.Queue()
    procs = [ctx.Process(target=_reference_worker,
                         args=(cfg_name, w * n_sample, n_sample, warmup, steps, seconds, barrier, queue))
             for w in range(n_workers)]
    for pr in procs:
        pr.start()
    res = [queue.get(timeout=1200) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
    bad = [r for r in res if isinstance(r, str)]
    if bad:
        raise RuntimeError(f"reference worker failed: {bad[0]}")
    units = sum(u * len(t) for u, t, _, _ in res)
    slowest = max(res, key=lambda r: sum(r[1]))[1]
    span = max(sum(t) for _, t, _, _ in res)
    n_el = sum(n for _, _, _, n in res)
    desc = (f"{n_workers} processes (one thread each) started together, each timing (residual + stage update) "
            f"on its own {n_sample}-element block of {cfg_name} ({n_el} elements in all; numpy FP64), "
            f"{span:.2f} s")
    return units / span, slowest, desc


def cpu_baseline(cfg_name: str, n_sample: int, seconds: float) -> dict:
    """The oracle on the host cores: one core and all cores, about `seconds` of timed work each."""
    one, _, desc1 = run_reference(cfg_name, 1, n_sample, 1, seconds=seconds)
    cores = os.cpu_count() or 1
    allv, _, desc_all = run_reference(cfg_name, cores, n_sample, 1, seconds=seconds) if cores > 1 else (one, None,
                                                                                                        desc1)
    return {"value": allv, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc_all,
            "one_core": {"value": one, "cores": 1, "sample": desc1}, "nproc": cores, "cpu_model": cpu_model()}


def run_batch(args, rank, world, local):
    """Batched independent shells: K graph-replayed SSP-RK3 steps of the whole batch."""
    import torch

    from chorus_inputs import BATCH_16, BATCH_64

    bcfg = {"batch_64": BATCH_64, "batch_16": BATCH_16}[args.workload]
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_1503_00834_gb300 import Shells, build as _build

    _build.build()
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    sh = Shells(bcfg)
    b = sh.batch
    build_s = time.perf_counter() - t0
    Q = torch.empty(b.n_state, dtype=torch.float32, device="cuda")
    ws = torch.empty(b.workspace_bytes, dtype=torch.uint8, device="cuda")
    choice = b.autotune(Q, ws, sh.dt, n_trials=2)
    if args.schedule != "auto":  # the tiles stay the autotuner's
        b.schedule({"serial": b.SERIAL, "concurrent": b.CONCURRENT, "persistent": b.PERSISTENT}[args.schedule])
    b.init(Q)
    launches = b.rk_step(Q, ws, sh.dt, max(3, args.warmup))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    b.rk_step(Q, ws, sh.dt, args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    red = b.reduce(Q)  # also reports any device-side error flag
    n_dof = b.n_dof()
    stages = 3 * args.steps
    value = job_rate(world, n_dof * stages, ms / 1e3)
    alg = sum(e * (p + 1) ** 3 * ALG_BYTES_PER_DOF_STAGE[p] for e, p in zip(b.n_elem, b.orders))
    peak, peak_kind = _peaks()
    achieved = alg / (ms / stages / 1e3) / 1e9
    # end to end through chorus_batch_rk_step_host: every step copies each order's state in from
    # pinned host memory, steps it and copies it back, the orders pipelined
    host = torch.empty(Q.shape, dtype=Q.dtype, pin_memory=True)
    host.copy_(Q)
    if args.e2e_steps > 0:  # one untimed call: its copy streams and events are created on first use
        b.rk_step_host(host, Q, ws, sh.dt, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        b.rk_step_host(host, Q, ws, sh.dt, 1)
    e2e_s = max(time.perf_counter() - t0, 1e-9)
    e2e_value = world * n_dof * 3 * args.e2e_steps / e2e_s
    state_bytes = Q.numel() * Q.element_size()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cfg0 = next(c for c in sh.cfgs if c.p == 3)
        cpu = cpu_baseline(cfg0.name, args.ref_elems, args.cpu_seconds)
    if rank == 0:
        from collections import Counter

        print(json.dumps({
            "metric": "RK-stage DOF updates/s, batch of independent shells", "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": bcfg.name, "shells": len(sh.cfgs), "elements": sum(b.n_elem), "dof": n_dof,
                       "orders": dict(Counter(b.orders)), "precision": "FP32 perturbation + FP64 background",
                       "step": "one SSP-RK3 step of every shell (" + (
                           "one persistent launch per stage" if b.schedule() == b.PERSISTENT else
                           "captured graph, one launch per kernel and order") + ")",
                       "tiles_elements_per_cta_p2_to_p5": choice, "dt": sh.dt,
                       "orders_schedule": ("one after another", "concurrent streams", "one persistent launch per stage")[b.schedule()],
                       "l2": "inputs larger than L2 (state %.0f MB)" % (state_bytes / 1e6),
                       "build_s": build_s, "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "kernel": "whole step (all kernels of all orders)", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                         "peak_kind": peak_kind},
            "gpu_launches": int(launches * args.steps),
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                    "d2h_bytes_per_step": state_bytes, "call": "chorus_batch_rk_step_host (host state in and out)"},
            "cpu_baseline": cpu,
            "mass_total": float(red[:, 0].sum()),
        }))
    if world > 1:
        torch.distributed.destroy_process_group()


def stage_roofline(alg_bytes_per_dof: float, n_dof: int, stage_ms: float, peak: float, peak_kind: str,
                   kernels: dict, traffic: dict) -> dict:
    """The roofline of the whole RK stage (every kernel of the residual and the update): algorithmic
    bytes of one stage over its measured time, against the measured HBM copy bandwidth; per kernel
    its time, measured DRAM bytes (ncu, when taken on these sources) and their rate."""
    achieved = alg_bytes_per_dof * n_dof / (stage_ms / 1e3) / 1e9
    tr_stage = None
    if traffic and all(traffic.get(k) is not None for k in ("k_grad", "k_face", "k_resid")):
        tr_stage = traffic["k_grad"] + traffic["k_face"] + traffic["k_resid"]
    per = {}
    for name, ms in kernels.items():
        b = traffic.get(name) if traffic else None
        per[name] = {"launch_ms": ms, "dram_bytes": b,
                     "dram_gbs": (b / (ms / 1e3) / 1e9) if (b and ms) else None,
                     "dram_frac": (b / (ms / 1e3) / 1e9 / peak) if (b and ms) else None}
    return {"bound": "hbm", "kernel": "whole RK stage (k_grad + k_face + k_resid per stage; k_trace once per call)",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": tr_stage,
            "peak_kind": peak_kind, "alg_bytes_per_dof_stage": alg_bytes_per_dof, "stage_ms": stage_ms,
            "kernels": per}


def main():
    from chorus_inputs import CONFIGS

    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="chorus", choices=["chorus", "reference"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--config", default="shell_331776_p3", choices=sorted(CONFIGS))
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--ref-elems", type=int, default=256)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=None, choices=["batch_64", "batch_16"])
    ap.add_argument("--schedule", default="auto", choices=["auto", "serial", "concurrent", "persistent"],
                    help="batch workloads: the step schedule (auto: the autotuner's choice)")
    ap.add_argument("--closure", action="store_true",
                    help="attach a seeded learned-closure record (p = 2 shells): every stage adds the network")
    args = ap.parse_args()
    cfg = CONFIGS[args.config]
    rank, world, local = _dist()
    if args.workload in ("batch_64", "batch_16") and args.impl == "chorus":
        run_batch(args, rank, world, local)
        return

    if args.impl == "reference":
        if rank != 0:
            return
        if args.workload == "batch_64":
            from chorus_inputs import BATCH_64

            cfg = next(c for c in BATCH_64.shells() if c.p == 3)
        cores = os.cpu_count() or 1
        value, times, desc = run_reference(cfg.name, cores, args.ref_elems, args.warmup, steps=args.steps)
        line = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": cfg.name, "elements": cfg.n_elem, "p": cfg.p},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line))
        return

    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_1503_00834_gb300 import FP32_PERT, FP64, Shell, build as _build, native

    _build.build()
    prec = FP32_PERT if args.prec == "fp32" else FP64
    tdt = torch.float32 if prec == FP32_PERT else torch.float64
    stream = torch.cuda.current_stream()
    sh = Shell(cfg)
    mesh = sh.mesh
    shape = mesh.state_shape()
    Q = torch.empty(shape, dtype=tdt, device="cuda")
    ws = torch.empty(mesh.workspace_bytes(prec), dtype=torch.uint8, device="cuda")
    mesh.prepare(sh.params)
    mesh.state_init(sh.params, cfg.seed, cfg.entropy_amp, prec, Q)
    n_dof = cfg.n_dof
    closure_rec = None
    if args.closure:
        if cfg.p != 2:
            raise SystemExit("--closure needs a p = 2 shell (the closure's order)")
        closure_rec = native.closure_alloc(11, [1e-4] * 5, [1e-5] * 5)
        native.closure_attach(mesh, closure_rec)
    # measured arithmetic peaks of this GPU (the FP64 path is bound by its FP64 units)
    fma = {"fp64_tflops": native.fma_rate(FP64) / 1e12, "fp32_tflops": native.fma_rate(FP32_PERT) / 1e12}

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed_steps(prec_, Q_, ws_, n_steps):
        """n_steps timed SSP-RK3 steps with per-kernel event timing; (ms, kernel ms per launch)."""
        mesh.timing_enable(True)
        mesh.timing_read()  # clear
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        mesh.rk_step(sh.params, prec_, Q_, ws_, sh.dt, n_steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        kms, kcnt = mesh.timing_read()
        mesh.timing_enable(False)
        per = {nm: kms[c] / max(1, kcnt[c]) for c, nm in enumerate(("k_trace", "k_grad", "k_resid", "k_face"))}
        return ev0.elapsed_time(ev1), per, sum(kcnt)

    # ---- warm-up, then K timed steps (inputs far larger than L2: state 425 MB FP32)
    mesh.rk_step(sh.params, prec, Q, ws, sh.dt, max(3, args.warmup))
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    ms_local, kper, launches = timed_steps(prec, Q, ws, args.steps)
    barrier()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = max_over_ranks(ms_local, world)
    stages = 3 * args.steps
    value = job_rate(world, n_dof * stages, ms / 1e3)
    mesh.check()

    # ---- roofline of the whole stage
    alg = (ALG_BYTES_PER_DOF_STAGE if prec == FP32_PERT else ALG_BYTES_PER_DOF_STAGE_FP64)[cfg.p]
    peak, peak_kind = _peaks()
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    traffic = {k: lookup_traffic(tpath, k, cfg.name, args.prec) for k in ("k_grad", "k_face", "k_resid")}
    roof = stage_roofline(alg, n_dof, ms / stages, peak, peak_kind, kper, traffic)

    # ---- FP64 GPU path on the same workload (the metric compares both), with its FP64-unit roofline
    fp64 = None
    if prec == FP32_PERT and args.fp64_steps > 0:
        Q64 = torch.empty(shape, dtype=torch.float64, device="cuda")
        ws64 = torch.empty(mesh.workspace_bytes(FP64), dtype=torch.uint8, device="cuda")
        mesh.state_init(sh.params, cfg.seed, cfg.entropy_amp, FP64, Q64)
        mesh.rk_step(sh.params, FP64, Q64, ws64, sh.dt, 1)
        torch.cuda.synchronize()
        ms64, kper64, _ = timed_steps(FP64, Q64, ws64, args.fp64_steps)
        v64 = world * n_dof * 3 * args.fp64_steps / (ms64 / 1e3)
        fpath = os.path.join(ROOT, "profiles", "fp64_flops.json")
        fl = lookup_traffic(fpath, "stage", cfg.name, "fp64")  # FP64 flops per DOF-stage (ncu instruction counts)
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": ms64 / args.fp64_steps,
                "kernels_ms_per_launch": kper64,
                "roofline": {"bound": "alu", "unit": "TFLOP/s", "peak": fma["fp64_tflops"], "peak_kind": "measured",
                             "flops_per_dof_stage": fl,
                             "achieved": (fl * v64 / 1e12) if fl else None,
                             "frac": (fl * v64 / 1e12 / fma["fp64_tflops"]) if fl else None}}
        del Q64, ws64

    # ---- end to end through the public API with host buffers: each step copies the state in from
    # pinned host memory, steps, and copies it back (chorus_rk_step_host)
    host = torch.empty(shape, dtype=tdt, pin_memory=True)
    host.copy_(Q)
    if args.e2e_steps > 0:  # one untimed call: its copy stream and events are created on first use
        mesh.rk_step_host(sh.params, prec, host, Q, ws, sh.dt, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        mesh.rk_step_host(sh.params, prec, host, Q, ws, sh.dt, 1)
    e2e_s = time.perf_counter() - t0
    e2e_value = world * n_dof * 3 * args.e2e_steps / e2e_s
    state_bytes = Q.numel() * Q.element_size()

    # ---- CPU baseline: the oracle on a bounded sample, rank 0 at N=1 only
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cfg.name, args.ref_elems, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == FP32_PERT else "f64",
            "data": "synthetic",
            "config": {"workload": cfg.name, "elements": cfg.n_elem, "p": cfg.p, "dof": n_dof,
                       "precision": "FP32 perturbation + FP64 background" if prec == FP32_PERT else "FP64",
                       "step": "one SSP-RK3 step = 3 residual + stage-update passes"
                               + (" with the learned closure attached" if args.closure else ""),
                       "l2": "inputs larger than L2 (state %.0f MB)" % (state_bytes / 1e6),
                       "parallelism": f"replicas x{world}"},
            "roofline": roof,
            "fp64_gpu_value": fp64["value"] if fp64 else None,
            "fp64": fp64,
            "measured_fma_peaks": fma,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                    "d2h_bytes_per_step": state_bytes, "call": "chorus_rk_step_host (host state in and out)"},
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
