"""Pins of the oracle's angular-momentum correction (Section 6, Eqs. 32-34)."""
import numpy as np

from chorus_inputs import cubed_sphere_hex20, make_phys
from oracle import state
from oracle.am_correction import atan2_paper, correct, momentum_and_inertia
from oracle.physics import Physics
from oracle.residual import Discretization


def _setup(n=4, n_r=2, p=3):
    xyz, h20 = cubed_sphere_hex20(n, n_r, 0.75, 1.0)
    disc = Discretization(xyz, h20, p, 0.75, 1.0)
    ph = Physics.from_params(make_phys(0.75, 1.5, 3.0, 1e-3), 0.75, 1.0)
    g = disc.geometry(np.arange(disc.n_elem))
    return disc, ph, g


def test_atan2_identity_matches_library():
    rng = np.random.default_rng(0)
    m1 = rng.standard_normal(1000)
    m2 = rng.standard_normal(1000)
    ok = ~((m2 < 0) & (np.abs(m1) < 1e-3))
    assert np.allclose(atan2_paper(m1[ok], m2[ok]), np.arctan2(m1[ok], m2[ok]), atol=1e-12)


def test_eq32_equals_cartesian_angular_momentum():
    # the spherical-coordinate integrands of Eq. 32 are the components of x cross (rho u)
    disc, ph, g = _setup()
    Q = state.background(ph, g["x"])
    rng = np.random.default_rng(1)
    Q[:, 1:4] = 0.1 * Q[:, :1] * rng.standard_normal(Q[:, 1:4].shape)
    L, I = momentum_and_inertia(disc, Q)
    w = disc.ops.w
    W = w[None, :, None, None] * w[None, None, :, None] * w[None, None, None, :] * g["detJ"]
    x = np.moveaxis(g["x"], 1, -1)
    m = np.moveaxis(Q[:, 1:4], 1, -1)
    Lc = np.sum(W[..., None] * np.cross(x, m), axis=(0, 1, 2, 3))
    assert np.allclose(L, Lc, rtol=1e-12, atol=1e-14 * np.abs(Lc).max())
    r2 = np.sum(x * x, axis=-1)
    Ic = np.sum(W[..., None] * Q[:, 0, ..., None] * (r2[..., None] - x * x), axis=(0, 1, 2, 3))
    assert np.allclose(I, Ic, rtol=1e-13)


def test_correction_removes_a_rigid_rotation_exactly():
    # a solid-body rotation about any axis on the spherically symmetric background is removed
    # to round-off (the cubed sphere's reflection symmetries make the products of inertia vanish)
    disc, ph, g = _setup()
    Q = state.background(ph, g["x"])
    x = np.moveaxis(g["x"], 1, -1)
    Om = np.array([0.02, -0.03, 0.05])
    u = np.cross(Om, x)
    Q[:, 1:4] = np.moveaxis(Q[:, 0, ..., None] * u, -1, 1)
    Q[:, 4] += 0.5 * Q[:, 0] * np.sum(u * u, axis=-1)
    Qn, dO = correct(disc, ph, Q)
    assert np.allclose(dO, Om, rtol=1e-12)
    assert np.abs(Qn[:, 1:4]).max() < 1e-13 * np.abs(Q[:, 1:4]).max()
    L, _ = momentum_and_inertia(disc, Qn)
    L0, _ = momentum_and_inertia(disc, Q)
    assert np.abs(L).max() < 1e-13 * np.abs(L0).max()
    # density and pressure kept
    p0 = (ph.gamma - 1) * (Q[:, 4] - 0.5 * np.sum(Q[:, 1:4] ** 2, axis=1) / Q[:, 0])
    p1 = (ph.gamma - 1) * (Qn[:, 4] - 0.5 * np.sum(Qn[:, 1:4] ** 2, axis=1) / Qn[:, 0])
    assert np.array_equal(Qn[:, 0], Q[:, 0]) and np.allclose(p1, p0, rtol=1e-13)


def test_correction_leaves_zero_momentum_state_unchanged():
    disc, ph, g = _setup()
    Q = state.initial_state(ph, g["x"], seed=3, amp=1e-3)
    Qn, dO = correct(disc, ph, Q)
    assert np.all(dO == 0.0)
    assert np.allclose(Qn, Q, rtol=1e-15, atol=0.0)
