"""ctypes binding of libchorus.so (the C ABI declared in include/chorus.h).

Argument marshalling only: every step of the residual and the time stepping runs in the library's
CUDA kernels.  Device buffers are torch tensors (contiguous, on the current CUDA device); the
stream is torch's current stream unless one is given.  There is no CPU fallback: if the library is
missing the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libchorus.so")

FP64 = 0
FP32_PERT = 1

STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error", 4: "invalid mesh",
          5: "non-finite value", 6: "device wait timed out", 7: "unsupported"}

# every symbol declared in include/chorus.h
EXPORTS = ("chorus_mesh_create", "chorus_mesh_destroy", "chorus_mesh_info", "chorus_prepare", "chorus_state_init",
           "chorus_residual", "chorus_rk_workspace_bytes", "chorus_rk_step", "chorus_reduce", "chorus_check",
           "chorus_strerror", "chorus_timing_enable", "chorus_timing_read", "chorus_residual_noalloc",
           "chorus_am_correct", "chorus_rk_step_scheme", "chorus_closure_bytes", "chorus_closure_init",
           "chorus_project", "chorus_closure_forward", "chorus_closure_forward_tc", "chorus_closure_grad",
           "chorus_closure_make_pairs", "chorus_closure_train", "chorus_closure_apply", "chorus_closure_attach", "chorus_batch_create",
           "chorus_batch_destroy", "chorus_batch_layout", "chorus_batch_init", "chorus_batch_rk_step",
           "chorus_batch_reduce", "chorus_batch_autotune", "chorus_set_well_balanced", "chorus_prepare_profile",
           "chorus_afb_profile", "chorus_closure_set_scales", "chorus_stable_dt_rule", "chorus_stable_dt",
           "chorus_set_wait_limit", "chorus_fma_rate", "chorus_rk_step_host", "chorus_batch_schedule",
           "chorus_batch_set_wait_limit", "chorus_batch_rk_step_host")


class ChorusError(RuntimeError):
    def __init__(self, call: str, status: int):
        super().__init__(f"{call}: {STATUS.get(status, status)} (status {status})")
        self.status = status


class TrainCfg(ctypes.Structure):
    """chorus_train_cfg."""

    _fields_ = [("epochs", ctypes.c_int64), ("batch", ctypes.c_int64), ("lr", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class ShellDesc(ctypes.Structure):
    """chorus_shell_desc."""

    _fields_ = [("n_nodes", ctypes.c_int64), ("node_xyz", ctypes.POINTER(ctypes.c_double)),
                ("n_elem", ctypes.c_int64), ("hex20", ctypes.POINTER(ctypes.c_int64)), ("p", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("entropy_amp", ctypes.c_double)]


class Params(ctypes.Structure):
    """chorus_params (all doubles, in header order)."""

    _fields_ = [(n, ctypes.c_double) for n in ("gamma", "R_gas", "GM", "Omega", "nu", "kappa", "kappa_r", "poly_n",
                                                "N_rho", "rho_c", "bottom_flux", "T_top", "kappa_r1", "kappa_r2")]

    @classmethod
    def from_phys(cls, phys) -> "Params":
        return cls(*phys.as_tuple())


_lib = None


def load() -> ctypes.CDLL:
    """Load libchorus.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1503_00834_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, f64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    P = ctypes.POINTER
    sig = {
        "chorus_mesh_create": (i32, [i64, P(f64), i64, P(i64), i32, f64, f64, i32, vp, P(vp)]),
        "chorus_mesh_destroy": (i32, [vp]),
        "chorus_mesh_info": (i32, [vp, P(i64), P(i64), P(f64), P(f64)]),
        "chorus_prepare": (i32, [vp, P(Params), vp]),
        "chorus_state_init": (i32, [vp, P(Params), ctypes.c_uint64, f64, i32, vp, vp]),
        "chorus_residual": (i32, [vp, P(Params), i32, vp, vp, vp, vp]),
        "chorus_rk_workspace_bytes": (ctypes.c_size_t, [vp, i32]),
        "chorus_rk_step": (i32, [vp, P(Params), i32, vp, vp, f64, i64, vp]),
        "chorus_reduce": (i32, [vp, P(Params), i32, vp, P(f64), vp]),
        "chorus_check": (i32, [vp, vp]),
        "chorus_strerror": (ctypes.c_char_p, [i32]),
        "chorus_timing_enable": (i32, [vp, i32]),
        "chorus_timing_read": (i32, [vp, vp, P(f64), P(i64)]),
        "chorus_residual_noalloc": (i32, [vp, P(Params), i32, vp, vp, vp]),
        "chorus_am_correct": (i32, [vp, P(Params), i32, vp, P(f64), vp]),
        "chorus_rk_step_scheme": (i32, [vp, P(Params), i32, i32, vp, vp, f64, i64, vp]),
        "chorus_closure_bytes": (ctypes.c_size_t, []),
        "chorus_closure_init": (i32, [vp, ctypes.c_uint64, P(ctypes.c_float), P(ctypes.c_float), vp]),
        "chorus_closure_set_scales": (i32, [vp, P(ctypes.c_float), P(ctypes.c_float), vp]),
        "chorus_project": (i32, [vp, vp, i32, i32, vp, vp, vp]),
        "chorus_closure_forward": (i32, [vp, vp, vp, i64, vp]),
        "chorus_closure_forward_tc": (i32, [vp, vp, vp, i64, vp]),
        "chorus_closure_grad": (i32, [vp, vp, vp, i64, vp, P(f64), vp]),
        "chorus_closure_make_pairs": (i32, [vp, i32, vp, vp, vp, vp, vp, vp, vp]),
        "chorus_closure_train": (i32, [vp, vp, i64, vp, P(TrainCfg), P(f64), vp]),
        "chorus_closure_apply": (i32, [vp, i32, vp, vp, vp, vp]),
        "chorus_closure_attach": (i32, [vp, vp]),
        "chorus_set_well_balanced": (i32, [vp, i32]),
        "chorus_prepare_profile": (i32, [vp, P(Params), i64, f64, f64, P(f64), P(f64), vp]),
        "chorus_afb_profile": (i32, [P(Params), f64, f64, f64, f64, i64, P(f64), P(f64)]),
        "chorus_batch_create": (i32, [i32, P(ShellDesc), f64, f64, P(Params), vp, P(vp)]),
        "chorus_batch_destroy": (i32, [vp]),
        "chorus_batch_layout": (i32, [vp, P(i64), P(i64), P(ctypes.c_size_t), P(i32), P(i32), P(f64)]),
        "chorus_batch_init": (i32, [vp, vp, vp]),
        "chorus_batch_rk_step": (i32, [vp, vp, vp, f64, i64, vp, P(i64)]),
        "chorus_batch_reduce": (i32, [vp, vp, P(f64), vp]),
        "chorus_batch_autotune": (i32, [vp, vp, vp, f64, i32, vp, P(i32)]),
        "chorus_stable_dt_rule": (i32, [i32, f64, f64, f64, P(Params), P(f64)]),
        "chorus_stable_dt": (i32, [vp, P(Params), P(f64)]),
        "chorus_set_wait_limit": (i32, [vp, i64]),
        "chorus_fma_rate": (i32, [i32, vp, P(f64)]),
        "chorus_rk_step_host": (i32, [vp, P(Params), i32, vp, vp, vp, f64, i64, vp]),
        "chorus_batch_schedule": (i32, [vp, i32, P(i32)]),
        "chorus_batch_set_wait_limit": (i32, [vp, i64]),
        "chorus_batch_rk_step_host": (i32, [vp, vp, vp, vp, f64, i64, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ok(call: str, status: int) -> None:
    if status != 0:
        raise ChorusError(call, status)


def _stream(stream):
    if stream is None:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t) -> ctypes.c_void_p:
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Mesh:
    """A curved hexahedral shell mesh on the GPU (chorus_mesh handle)."""

    def __init__(self, node_xyz: np.ndarray, hex20: np.ndarray, p: int, r_inner: float, r_outer: float,
                 metric_mode: int = 0, stream=None):
        lib = load()
        xyz = np.ascontiguousarray(node_xyz, dtype=np.float64)
        h20 = np.ascontiguousarray(hex20, dtype=np.int64)
        self.p, self.N = p, p + 1
        self.n_elem = h20.shape[0]
        handle = ctypes.c_void_p()
        _ok("chorus_mesh_create", lib.chorus_mesh_create(
            xyz.shape[0], xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), h20.shape[0],
            h20.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), p, r_inner, r_outer, metric_mode, _stream(stream),
            ctypes.byref(handle)))
        self.handle = handle

    def close(self) -> None:
        if getattr(self, "handle", None) and self.handle.value:
            load().chorus_mesh_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        n_dof, n_faces = ctypes.c_int64(), ctypes.c_int64()
        h_min, vol = ctypes.c_double(), ctypes.c_double()
        _ok("chorus_mesh_info", load().chorus_mesh_info(self.handle, ctypes.byref(n_dof), ctypes.byref(n_faces),
                                                        ctypes.byref(h_min), ctypes.byref(vol)))
        return dict(n_dof=n_dof.value, n_faces=n_faces.value, h_min=h_min.value, volume=vol.value)

    def state_shape(self):
        return (self.n_elem, 5, self.N ** 3)

    def prepare(self, params: Params, stream=None) -> None:
        _ok("chorus_prepare", load().chorus_prepare(self.handle, ctypes.byref(params), _stream(stream)))

    def prepare_profile(self, params: Params, profile, stream=None) -> None:
        """Background from a radial profile (r0, r1, rho0, p0) on the uniform grid over [r0, r1]."""
        r0, r1, rho0, p0 = profile
        r = np.ascontiguousarray(rho0, dtype=np.float64)
        p = np.ascontiguousarray(p0, dtype=np.float64)
        dp = ctypes.POINTER(ctypes.c_double)
        _ok("chorus_prepare_profile", load().chorus_prepare_profile(self.handle, ctypes.byref(params), r.shape[0], r0,
                                                                    r1, r.ctypes.data_as(dp), p.ctypes.data_as(dp),
                                                                    _stream(stream)))

    def workspace_bytes(self, prec: int) -> int:
        return int(load().chorus_rk_workspace_bytes(self.handle, prec))

    def state_init(self, params: Params, seed: int, amp: float, prec: int, Q, stream=None) -> None:
        _ok("chorus_state_init", load().chorus_state_init(self.handle, ctypes.byref(params), seed, amp, prec, _ptr(Q),
                                                          _stream(stream)))

    def residual(self, params: Params, prec: int, Q, R, ws, stream=None) -> None:
        _ok("chorus_residual", load().chorus_residual(self.handle, ctypes.byref(params), prec, _ptr(Q), _ptr(R),
                                                      _ptr(ws), _stream(stream)))

    def rk_step(self, params: Params, prec: int, Q, ws, dt: float, n_steps: int, stream=None) -> None:
        _ok("chorus_rk_step", load().chorus_rk_step(self.handle, ctypes.byref(params), prec, _ptr(Q), _ptr(ws), dt,
                                                    n_steps, _stream(stream)))

    def rk_step_host(self, params: Params, prec: int, Q_host, Q_dev, ws, dt: float, n_steps: int,
                     stream=None) -> None:
        """n_steps SSP-RK3 steps of a host-resident state (Q_host: contiguous CPU tensor, pinned for full
        bandwidth): copied in, stepped on the device in Q_dev, copied back; synchronises."""
        if Q_host.is_cuda or not Q_host.is_contiguous():
            raise ValueError("Q_host must be a contiguous host tensor")
        _ok("chorus_rk_step_host", load().chorus_rk_step_host(self.handle, ctypes.byref(params), prec,
                                                              ctypes.c_void_p(Q_host.data_ptr()), _ptr(Q_dev),
                                                              _ptr(ws), dt, n_steps, _stream(stream)))

    def rk_step_scheme(self, params: Params, prec: int, scheme: int, Q, ws, dt: float, n_steps: int,
                       stream=None) -> None:
        """scheme 0: SSP-RK3, 1: SSP-RK(5,4)."""
        _ok("chorus_rk_step_scheme", load().chorus_rk_step_scheme(self.handle, ctypes.byref(params), prec, scheme,
                                                                  _ptr(Q), _ptr(ws), dt, n_steps, _stream(stream)))

    def reduce(self, params: Params, prec: int, Q, stream=None) -> np.ndarray:
        out = (ctypes.c_double * 4)()
        _ok("chorus_reduce", load().chorus_reduce(self.handle, ctypes.byref(params), prec, _ptr(Q), out,
                                                  _stream(stream)))
        return np.array(out[:])

    def am_correct(self, params: Params, prec: int, Q, stream=None) -> np.ndarray:
        """Angular-momentum correction in place; returns delta Omega (synchronises)."""
        out = (ctypes.c_double * 3)()
        _ok("chorus_am_correct", load().chorus_am_correct(self.handle, ctypes.byref(params), prec, _ptr(Q), out,
                                                          _stream(stream)))
        return np.array(out[:])

    def timing_enable(self, enable: bool) -> None:
        _ok("chorus_timing_enable", load().chorus_timing_enable(self.handle, 1 if enable else 0))

    def timing_read(self, stream=None):
        """(ms[4], counts[4]) per kernel class: 0 traces, 1 gradients (and wall fluxes), 2 residual/RK
        update, 3 interior-face common fluxes."""
        ms = (ctypes.c_double * 4)()
        cnt = (ctypes.c_int64 * 4)()
        _ok("chorus_timing_read", load().chorus_timing_read(self.handle, _stream(stream), ms, cnt))
        return list(ms), list(cnt)

    def set_well_balanced(self, enable: bool) -> None:
        """FP32 perturbation residual without R(Q0): the background becomes an exact steady state."""
        _ok("chorus_set_well_balanced", load().chorus_set_well_balanced(self.handle, 1 if enable else 0))

    def check(self, stream=None) -> None:
        _ok("chorus_check", load().chorus_check(self.handle, _stream(stream)))

    def stable_dt(self, params: Params) -> float:
        """The library's fixed explicit time step for this mesh (chorus_stable_dt)."""
        dt = ctypes.c_double()
        _ok("chorus_stable_dt", load().chorus_stable_dt(self.handle, ctypes.byref(params), ctypes.byref(dt)))
        return dt.value

    def set_wait_limit(self, polls: int) -> None:
        """Polls of the residual kernels' bounded staging waits (negative: the default; 0: give up at
        once)."""
        _ok("chorus_set_wait_limit", load().chorus_set_wait_limit(self.handle, polls))


# ---------------------------------------------------------------- batched independent shells


class Batch:
    """Independent shells of several orders advanced together (chorus_batch handle).

    shells: sequence of (node_xyz, hex20, p, seed, entropy_amp).  The FP32 perturbation state of
    every shell lives in one device array; `view(Q, s)` is shell s's [E][5][N^3] block.
    """

    def __init__(self, shells, r_inner: float, r_outer: float, params: Params, stream=None):
        lib = load()
        self._keep = []
        descs = (ShellDesc * len(shells))()
        self.orders, self.n_elem = [], []
        for i, (xyz, h20, p, seed, amp) in enumerate(shells):
            xyz = np.ascontiguousarray(xyz, dtype=np.float64)
            h20 = np.ascontiguousarray(h20, dtype=np.int64)
            self._keep += [xyz, h20]
            descs[i] = ShellDesc(xyz.shape[0], xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), h20.shape[0],
                                 h20.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), p, seed, amp)
            self.orders.append(p)
            self.n_elem.append(h20.shape[0])
        handle = ctypes.c_void_p()
        _ok("chorus_batch_create", lib.chorus_batch_create(len(shells), descs, r_inner, r_outer,
                                                           ctypes.byref(params), _stream(stream), ctypes.byref(handle)))
        self._keep = []
        self.handle = handle
        self.params = params
        off = (ctypes.c_int64 * len(shells))()
        n_state, ws, ng = ctypes.c_int64(), ctypes.c_size_t(), ctypes.c_int()
        gp, gh = (ctypes.c_int * 4)(), (ctypes.c_double * 4)()
        _ok("chorus_batch_layout", lib.chorus_batch_layout(handle, off, ctypes.byref(n_state), ctypes.byref(ws),
                                                           ctypes.byref(ng), gp, gh))
        self.offsets = list(off)
        self.n_state, self.workspace_bytes, self.n_groups = n_state.value, ws.value, ng.value
        self.group_h_min = {gp[g]: gh[g] for g in range(ng.value)}  # order -> shortest edge chord

    def close(self) -> None:
        if getattr(self, "handle", None) and self.handle.value:
            load().chorus_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def n_dof(self) -> int:
        return sum(e * (p + 1) ** 3 for e, p in zip(self.n_elem, self.orders))

    def view(self, Q, s: int):
        N3 = (self.orders[s] + 1) ** 3
        o = self.offsets[s]
        return Q[o:o + self.n_elem[s] * 5 * N3].view(self.n_elem[s], 5, N3)

    def init(self, Q, stream=None) -> None:
        _ok("chorus_batch_init", load().chorus_batch_init(self.handle, _ptr(Q), _stream(stream)))

    def rk_step(self, Q, ws, dt: float, n_steps: int, stream=None) -> int:
        """n_steps SSP-RK3 steps (graph replay); returns the kernel launches per step."""
        n = ctypes.c_int64()
        _ok("chorus_batch_rk_step", load().chorus_batch_rk_step(self.handle, _ptr(Q), _ptr(ws), dt, n_steps,
                                                                _stream(stream), ctypes.byref(n)))
        return n.value

    def rk_step_host(self, Q_host, Q_dev, ws, dt: float, n_steps: int, stream=None) -> None:
        """n_steps SSP-RK3 steps of a host-resident batch state (contiguous CPU tensor, pinned for full
        bandwidth), the orders' copies pipelined with their steps; synchronises."""
        if Q_host.is_cuda or not Q_host.is_contiguous():
            raise ValueError("Q_host must be a contiguous host tensor")
        _ok("chorus_batch_rk_step_host", load().chorus_batch_rk_step_host(
            self.handle, ctypes.c_void_p(Q_host.data_ptr()), _ptr(Q_dev), _ptr(ws), dt, n_steps, _stream(stream)))

    def reduce(self, Q, stream=None) -> np.ndarray:
        out = (ctypes.c_double * (4 * len(self.orders)))()
        _ok("chorus_batch_reduce", load().chorus_batch_reduce(self.handle, _ptr(Q), out, _stream(stream)))
        return np.array(out[:]).reshape(-1, 4)

    SERIAL, CONCURRENT, PERSISTENT = 0, 1, 2

    def set_wait_limit(self, polls: int) -> None:
        """Polls of the bounded staging waits and grid barriers of every mesh (negative: the default)."""
        _ok("chorus_batch_set_wait_limit", load().chorus_batch_set_wait_limit(self.handle, polls))

    def schedule(self, mode=None) -> int:
        """The schedule of a step: 0 the orders one after another, 1 on concurrent streams (a bool
        means 1 / 0), 2 one persistent launch per RK stage; sets it when given, returns the one in force."""
        out = ctypes.c_int()
        set_ = -1 if mode is None else int(mode)
        _ok("chorus_batch_schedule", load().chorus_batch_schedule(self.handle, set_, ctypes.byref(out)))
        return out.value

    def autotune(self, Q, ws, dt: float, n_trials: int = 3, stream=None):
        """Chosen elements per CTA for p = 2..5 (0 where absent)."""
        ch = (ctypes.c_int * 4)()
        _ok("chorus_batch_autotune", load().chorus_batch_autotune(self.handle, _ptr(Q), _ptr(ws), dt, n_trials,
                                                                  _stream(stream), ch))
        return list(ch)


# ---------------------------------------------------------------- learned closure

N_PARAMS = 128 * 135 + 128 * 128 + 135 * 128 + 128 + 128 + 135


def closure_alloc(seed: int, in_scale, out_scale, stream=None):
    """A seeded closure record on the device (uint8 tensor)."""
    import torch

    w = torch.empty(int(load().chorus_closure_bytes()), dtype=torch.uint8, device="cuda")
    a = (ctypes.c_float * 5)(*in_scale)
    b = (ctypes.c_float * 5)(*out_scale)
    _ok("chorus_closure_init", load().chorus_closure_init(_ptr(w), seed, a, b, _stream(stream)))
    return w


def closure_set_scales(w, in_scale, out_scale, stream=None) -> None:
    a = (ctypes.c_float * 5)(*in_scale)
    b = (ctypes.c_float * 5)(*out_scale)
    _ok("chorus_closure_set_scales", load().chorus_closure_set_scales(_ptr(w), a, b, _stream(stream)))


def project(fine: "Mesh", coarse: "Mesh", prec: int, kind: int, Qf, Qc, stream=None) -> None:
    _ok("chorus_project", load().chorus_project(fine.handle, coarse.handle, prec, kind, _ptr(Qf), _ptr(Qc),
                                                _stream(stream)))


def closure_forward(w, X, Y, stream=None) -> None:
    _ok("chorus_closure_forward", load().chorus_closure_forward(_ptr(w), _ptr(X), _ptr(Y), X.shape[0],
                                                                _stream(stream)))


def closure_forward_tc(w, X, Y, stream=None) -> None:
    """Tensor-core forward (BF16 layer inputs, FP32 accumulation)."""
    _ok("chorus_closure_forward_tc", load().chorus_closure_forward_tc(_ptr(w), _ptr(X), _ptr(Y), X.shape[0],
                                                                      _stream(stream)))


def closure_grad(w, X, Y, grad, stream=None) -> float:
    loss = ctypes.c_double()
    _ok("chorus_closure_grad", load().chorus_closure_grad(_ptr(w), _ptr(X), _ptr(Y), X.shape[0], _ptr(grad),
                                                          ctypes.byref(loss), _stream(stream)))
    return loss.value


def closure_make_pairs(coarse: "Mesh", prec: int, w, Qc, PRf, Rc, X, Y, stream=None) -> None:
    _ok("chorus_closure_make_pairs", load().chorus_closure_make_pairs(
        coarse.handle, prec, _ptr(w), _ptr(Qc), _ptr(PRf), _ptr(Rc), _ptr(X), _ptr(Y), _stream(stream)))


def closure_train(X, Y, w, epochs: int, batch: int, lr: float, stream=None):
    cfg = TrainCfg(epochs, batch, lr, 0.9, 0.999, 1e-8, 0)
    losses = (ctypes.c_double * epochs)()
    _ok("chorus_closure_train", load().chorus_closure_train(_ptr(X), _ptr(Y), X.shape[0], _ptr(w), ctypes.byref(cfg),
                                                            losses, _stream(stream)))
    return list(losses)


def closure_apply(coarse: "Mesh", prec: int, w, Q, R, stream=None) -> None:
    _ok("chorus_closure_apply", load().chorus_closure_apply(coarse.handle, prec, _ptr(w), _ptr(Q), _ptr(R),
                                                            _stream(stream)))


def closure_attach(coarse: "Mesh", w) -> None:
    """Attach the closure record w to the mesh (None detaches it); the mesh keeps a reference to w."""
    _ok("chorus_closure_attach", load().chorus_closure_attach(coarse.handle, None if w is None else _ptr(w)))
    coarse._closure_record = w


def afb_profile(params: Params, r_inner: float, r_outer: float, n: int = 16385, margin: float = 0.05):
    """Almost-flux-balance profile (r0, r1, rho0, p0) on n uniform radii spanning the shell plus
    `margin` of its thickness on both sides (host computation in the library)."""
    d = r_outer - r_inner
    r0, r1 = r_inner - margin * d, r_outer + margin * d
    rho = np.empty(n)
    p = np.empty(n)
    dp = ctypes.POINTER(ctypes.c_double)
    _ok("chorus_afb_profile", load().chorus_afb_profile(ctypes.byref(params), r_inner, r_outer, r0, r1, n,
                                                        rho.ctypes.data_as(dp), p.ctypes.data_as(dp)))
    return r0, r1, rho, p


def fma_rate(prec: int, stream=None) -> float:
    """Measured FMA throughput of the current GPU in flop/s (chorus_fma_rate; FP64 or FP32)."""
    r = ctypes.c_double()
    _ok("chorus_fma_rate", load().chorus_fma_rate(prec, _stream(stream), ctypes.byref(r)))
    return r.value


def stable_dt(p: int, h_min: float, r_inner: float, r_outer: float, params: Params) -> float:
    """The library's fixed explicit time step for order p and shortest element edge h_min
    (chorus_stable_dt_rule, a host computation)."""
    dt = ctypes.c_double()
    _ok("chorus_stable_dt_rule", load().chorus_stable_dt_rule(p, h_min, r_inner, r_outer, ctypes.byref(params),
                                                              ctypes.byref(dt)))
    return dt.value
