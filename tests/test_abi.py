"""The C-ABI library loads, exports every entry point of include/chorus.h, and rejects invalid
input on the host before touching the GPU (no device needed)."""
import ctypes
import re

import numpy as np
import pytest

from chorus_inputs import cubed_sphere_hex20


@pytest.fixture(scope="module")
def lib():
    from paper_1503_00834_gb300 import build, native

    build.build()
    return native.load()


def test_header_and_exports(lib):
    import os

    from paper_1503_00834_gb300 import native

    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "chorus.h")).read()
    declared = set(re.findall(r"\b(chorus_[a-z_]+)\s*\(", hdr))
    assert declared == set(native.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name
    assert lib.chorus_strerror(4) == b"invalid mesh"


def _create(lib, xyz, h20, p=3, ri=0.75, ro=1.0, mode=0):
    h = ctypes.c_void_p()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    h20 = np.ascontiguousarray(h20, dtype=np.int64)
    st = lib.chorus_mesh_create(xyz.shape[0], xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), h20.shape[0],
                                h20.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), p, ri, ro, mode, None,
                                ctypes.byref(h))
    return st, h


def test_invalid_meshes_rejected_on_host(lib):
    xyz, h20 = cubed_sphere_hex20(1, 1, 0.75, 1.0)
    assert _create(lib, xyz, h20, p=1)[0] == 7          # unsupported order
    assert _create(lib, xyz, h20, p=3, ri=1.0)[0] == 1  # r_inner >= r_outer
    assert _create(lib, xyz, h20, mode=5)[0] == 1
    bad = h20.copy()
    bad[0, 3] = xyz.shape[0] + 7
    assert _create(lib, xyz, bad)[0] == 4                # node index out of range
    bad = h20.copy()
    bad[0, 5] = bad[0, 4]
    assert _create(lib, xyz, bad)[0] == 4                # repeated node
    # a stray boundary: drop one element so its neighbours get faces on neither wall
    assert _create(lib, xyz, h20[1:])[0] == 4
    # an inverted element (mirror its reference axes) must fail the |J| > 0 check
    flip = h20.copy()
    perm = [1, 0, 3, 2, 5, 4, 7, 6, 8, 11, 10, 9, 12, 15, 14, 13, 17, 16, 19, 18]
    flip[0] = h20[0, perm]
    assert _create(lib, xyz, flip)[0] == 4


def test_null_arguments(lib):
    assert lib.chorus_mesh_destroy(None) == 1
    assert lib.chorus_check(None, None) == 1
    assert lib.chorus_rk_workspace_bytes(None, 0) == 0


def _params(phys):
    from paper_1503_00834_gb300 import native

    return native.Params.from_phys(phys)


@pytest.mark.parametrize("p,nu", [(2, 5e-4), (3, 5e-4), (5, 5e-4), (3, 0.5)])
def test_stable_dt_rule_matches_oracle(lib, p, nu):
    """The time-step rule behind the C ABI against the oracle's, evaluated on the polytrope at rest at
    the inner wall (where its sound speed peaks); nu = 0.5 takes the diffusive cap."""
    import dataclasses

    from chorus_inputs import make_phys
    from oracle import state
    from oracle.physics import Physics

    phys = dataclasses.replace(make_phys(0.75, 1.5, 3.0, 1e-3), nu=nu)
    ph = Physics.from_params(phys, 0.75, 1.0)
    Q = state.background(ph, np.array([0.75, 0.0, 0.0]).reshape(1, 3, 1, 1, 1))
    h = 0.0371
    want = state.time_step(ph, p, h, Q)
    got = ctypes.c_double()
    assert lib.chorus_stable_dt_rule(p, h, 0.75, 1.0, ctypes.byref(_params(phys)), ctypes.byref(got)) == 0
    assert abs(got.value - want) <= 1e-14 * want
    if nu == 0.5:
        assert abs(want - 0.25 * h * h / ((2 * p + 1) ** 2 * nu)) <= 1e-15 * want  # the cap is the branch taken


def test_stable_dt_rule_rejects_bad_input(lib):
    from chorus_inputs import make_phys

    P = _params(make_phys(0.75, 1.5, 3.0, 1e-3))
    dt = ctypes.c_double()
    assert lib.chorus_stable_dt_rule(1, 0.1, 0.75, 1.0, ctypes.byref(P), ctypes.byref(dt)) == 1  # order
    assert lib.chorus_stable_dt_rule(3, 0.0, 0.75, 1.0, ctypes.byref(P), ctypes.byref(dt)) == 1  # h_min
    assert lib.chorus_stable_dt_rule(3, 0.1, 1.0, 0.75, ctypes.byref(P), ctypes.byref(dt)) == 1  # radii
    assert lib.chorus_stable_dt_rule(3, 0.1, 0.75, 1.0, None, ctypes.byref(dt)) == 1
    assert lib.chorus_stable_dt(None, ctypes.byref(P), ctypes.byref(dt)) == 1
    assert lib.chorus_set_wait_limit(None, 5) == 1
