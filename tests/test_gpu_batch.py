"""Batched independent shells on the GPU.

A shell of the batch must compute what a single mesh of that shell computes: the batch puts the
shells of one order into one disjoint-union mesh and replays a captured multi-stream graph, none of
which may change a shell's arithmetic.  With the same tile shape the states agree bit for bit; a
shell's single-mesh result is itself parity-tested against the oracle (test_gpu_parity), and one
shell is compared with the oracle directly here.
"""
import numpy as np
import pytest

from chorus_inputs import small_batch
from gpu_common import OracleShell, rel_err, to5

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00834_gb300 import build

    build.build()


@pytest.fixture(scope="module")
def batch():
    from paper_1503_00834_gb300 import Shells

    return Shells(small_batch())


def _single(cfg, Q_init_only=False):
    from paper_1503_00834_gb300 import FP32_PERT, Shell

    sh = Shell(cfg)
    sh.mesh.prepare(sh.params)
    q = torch.empty(sh.mesh.state_shape(), dtype=torch.float32, device="cuda")
    sh.mesh.state_init(sh.params, cfg.seed, cfg.entropy_amp, FP32_PERT, q)
    ws = torch.empty(sh.mesh.workspace_bytes(FP32_PERT), dtype=torch.uint8, device="cuda")
    return sh, q, ws


def _alloc(b):
    Q = torch.empty(b.batch.n_state, dtype=torch.float32, device="cuda")
    ws = torch.empty(b.batch.workspace_bytes, dtype=torch.uint8, device="cuda")
    return Q, ws


def test_layout_covers_every_order(batch):
    b = batch.batch
    assert sorted(set(b.orders)) == [2, 3, 4, 5]
    assert b.n_groups == 4
    ends = sorted((o, o + e * 5 * (p + 1) ** 3) for o, e, p in zip(b.offsets, b.n_elem, b.orders))
    for (a0, a1), (b0, _) in zip(ends, ends[1:]):
        assert a1 <= b0  # shells do not overlap
    assert ends[-1][1] <= b.n_state


def test_init_and_steps_equal_single_meshes(batch):
    from paper_1503_00834_gb300 import FP32_PERT

    b = batch.batch
    Q, ws = _alloc(batch)
    b.init(Q)
    n_steps = 3
    launches = b.rk_step(Q, ws, batch.dt, n_steps)
    assert launches == 10 * 4  # per order: trace + 3 x (lifting, face, residual)
    b.rk_step(Q, ws, batch.dt, 0)
    torch.cuda.synchronize()
    red = b.reduce(Q)
    for s, cfg in enumerate(batch.cfgs):
        sh, q, w = _single(cfg)
        q0 = q.clone()
        sh.mesh.rk_step(sh.params, FP32_PERT, q, w, batch.dt, n_steps)
        torch.cuda.synchronize()
        got = b.view(Q, s)
        assert torch.equal(got, q), (s, cfg, (got - q).abs().max().item())
        assert not torch.equal(q, q0)
        r1 = sh.mesh.reduce(sh.params, FP32_PERT, q)
        assert np.allclose(red[s], r1, rtol=1e-13, atol=0), (s, red[s], r1)


def test_graph_replay_matches_a_fresh_capture(batch):
    """Two launches of n steps from one capture equal one call of 2n steps after a recapture."""
    b = batch.batch
    Q1, ws1 = _alloc(batch)
    b.init(Q1)
    b.rk_step(Q1, ws1, batch.dt, 2)
    b.rk_step(Q1, ws1, batch.dt, 2)
    Q2, ws2 = _alloc(batch)
    b.init(Q2)
    b.rk_step(Q2, ws2, batch.dt, 4)  # other pointers: captured again
    torch.cuda.synchronize()
    for s in range(len(batch.cfgs)):  # the alignment gaps between orders are not state
        assert torch.equal(b.view(Q1, s), b.view(Q2, s)), s


def test_one_shell_against_the_oracle(batch):
    from oracle import rk

    b = batch.batch
    s = next(i for i, c in enumerate(batch.cfgs) if c.p == 3)
    cfg = batch.cfgs[s]
    Q, ws = _alloc(batch)
    b.init(Q)
    b.rk_step(Q, ws, batch.dt, 2)
    torch.cuda.synchronize()
    osh = OracleShell(cfg)
    Qref = rk.run(osh.disc, osh.ph, osh.initial_state(), batch.dt, 2)
    Q0 = osh.background()
    e, ev = rel_err(to5(b.view(Q, s), cfg.p + 1), Qref - Q0, osh.weights())
    print(f"batch shell {s} ({cfg.n}x{cfg.n_r}, p={cfg.p}) after 2 steps: rel err on q' {ev}")
    assert e < 1e-5


def test_autotune_picks_a_built_tile_and_keeps_results(batch):
    b = batch.batch
    Q, ws = _alloc(batch)
    choice = b.autotune(Q, ws, batch.dt, n_trials=2)
    print(f"autotuned elements per CTA for p = 2..5: {choice}")
    built = {2: (14, 6), 3: (4, 8), 4: (5, 2), 5: (2, 4)}
    for p in (2, 3, 4, 5):
        assert choice[p - 2] in built[p]
    b.init(Q)
    b.rk_step(Q, ws, batch.dt, 2)
    torch.cuda.synchronize()
    from paper_1503_00834_gb300 import FP32_PERT

    for s, cfg in enumerate(batch.cfgs):
        sh, q, w = _single(cfg)
        sh.mesh.rk_step(sh.params, FP32_PERT, q, w, batch.dt, 2)
        torch.cuda.synchronize()
        got = b.view(Q, s)
        # another tile shape keeps each element's arithmetic; allow FP32 rounding in case the
        # compiler schedules the two instantiations differently
        d = (got - q).abs().max().item()
        scale = q.abs().max().item()
        print(f"shell {s}: max |batch - single| = {d:.3e} (scale {scale:.3e})")
        assert d <= 1e-6 * scale


def _persistent_or_skip(b):
    """Select the persistent schedule, or skip where the device offers no cooperative launch."""
    from paper_1503_00834_gb300 import ChorusError

    try:
        b.schedule(b.PERSISTENT)
    except ChorusError as e:
        if e.status == 7:  # CHORUS_EUNSUPPORTED
            pytest.skip("no cooperative launch on this device")
        raise


def test_all_schedules_give_the_same_shells(batch):
    """The orders one after another or on concurrent streams (the same kernels on disjoint data):
    every shell's state is bit-identical after three steps.  One persistent launch per RK stage runs
    the same per-element arithmetic compiled into another kernel (where the compiler may fuse other
    products into FMAs): within 1e-6 of the state's scale, and three launches a step."""
    b = batch.batch
    was = b.schedule()
    try:
        out = []
        for mode in (b.CONCURRENT, b.SERIAL, b.PERSISTENT):
            if mode == b.PERSISTENT:
                _persistent_or_skip(b)
            assert b.schedule(mode) == mode
            Q, ws = _alloc(batch)
            b.init(Q)
            launches = b.rk_step(Q, ws, batch.dt, 3)
            torch.cuda.synchronize()
            assert np.all(np.isfinite(b.reduce(Q)))  # also reports a flag a wait set
            assert launches == (3 if mode == b.PERSISTENT else 10 * len({c.p for c in batch.cfgs})), (mode, launches)
            out.append(Q)
        for s in range(len(batch.cfgs)):
            assert torch.equal(b.view(out[0], s), b.view(out[1], s)), s
            q, p = b.view(out[0], s), b.view(out[2], s)
            d, scale = (q - p).abs().max().item(), q.abs().max().item()
            print(f"shell {s}: max |persistent - serial| = {d:.3e} (scale {scale:.3e})")
            assert d <= 1e-6 * scale, s
    finally:
        b.schedule(was)


def test_persistent_barrier_timeout_is_reported_and_stores_nothing(batch):
    """The persistent schedule's bounded waits, made to run out: with a wait limit of zero polls the
    first grid barrier (or staging wait) of every launch gives up at once, the CTAs stop, nothing of
    the state is written, and the batch reduction reports CHORUS_ETIMEOUT once; with the default
    limit again the same step gives the normal result.  Nothing spins unbounded."""
    from paper_1503_00834_gb300 import ChorusError

    b = batch.batch
    was = b.schedule()
    try:
        _persistent_or_skip(b)
        Q, ws = _alloc(batch)
        b.init(Q)
        Q0 = Q.clone()
        try:
            b.set_wait_limit(0)
            b.rk_step(Q, ws, batch.dt, 1)
            torch.cuda.synchronize()
            with pytest.raises(ChorusError) as e:
                b.reduce(Q)
            assert e.value.status == 6  # CHORUS_ETIMEOUT
        finally:
            b.set_wait_limit(-1)
        assert torch.equal(Q, Q0)  # the launches that gave up wrote nothing of the state
        b.rk_step(Q, ws, batch.dt, 1)
        assert np.all(np.isfinite(b.reduce(Q)))  # reported once, then cleared
        Q1 = Q.clone()
        b.init(Q)
        b.rk_step(Q, ws, batch.dt, 1)
        assert torch.equal(Q, Q1) and not torch.equal(Q1, Q0)
    finally:
        b.schedule(was)


def test_host_step_equals_device_step(batch):
    """chorus_batch_rk_step_host (the orders' copies pipelined with their steps) against the graph
    step with the orders one after another, on the same initial state: every shell bit-identical."""
    b = batch.batch
    was = b.schedule()
    try:
        b.schedule(b.SERIAL)
        Q, ws = _alloc(batch)
        b.init(Q)
        host = torch.empty(Q.shape, dtype=Q.dtype, pin_memory=True)
        host.copy_(Q)
        Q_dev = torch.empty_like(Q)
        b.rk_step_host(host, Q_dev, ws, batch.dt, 2)
        b.rk_step(Q, ws, batch.dt, 2)
        torch.cuda.synchronize()
        assert np.all(np.isfinite(b.reduce(Q)))
        Qc = Q.cpu()
        for s in range(len(batch.cfgs)):
            assert torch.equal(b.view(host, s), b.view(Qc, s)), s
    finally:
        b.schedule(was)
