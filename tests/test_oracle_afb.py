"""Pins of the almost-flux-balance stratification (oracle/afb.py, Section 4.3)."""
import dataclasses
import math

import numpy as np

from chorus_inputs import make_phys
from oracle import afb
from oracle.physics import Physics


def _ph(bottom_flux=0.0, kappa_r=0.0, kappa=5e-4):
    base = make_phys(0.75, 1.5, 3.0, 1e-3, kappa=kappa)
    return Physics.from_params(dataclasses.replace(base, bottom_flux=bottom_flux, kappa_r=kappa_r), 0.75, 1.0)


def test_no_flux_gives_the_polytrope():
    ph = _ph()
    prof = afb.profile(ph)
    r = np.linspace(0.75, 1.0, 201)
    rho, p = prof(r)
    assert np.max(np.abs(rho / ph.rho_a(r) - 1.0)) < 1e-11
    assert np.max(np.abs(p / ph.p_a(r) - 1.0)) < 1e-11


def test_profile_is_hydrostatic_with_the_target_entropy_gradient():
    """Finite differences of the solution (independent of the integrator) reproduce dp/dr = -rho g
    and dS/dr = Gamma with S = C_p ln(p^(1/gamma) / rho)."""
    ph = _ph(bottom_flux=2e-5)
    prof = afb.profile(ph)
    r = np.linspace(0.76, 0.99, 47)
    h = 1e-5
    rho, p = prof(r)
    rp, pp = prof(r + h)
    rm, pm = prof(r - h)
    dp = (pp - pm) / (2 * h)
    assert np.max(np.abs(dp / (-rho * ph.GM / r ** 2) - 1.0)) < 1e-7

    def S(rho_, p_):
        return ph.Cp * (np.log(p_) / ph.gamma - np.log(rho_))

    dS = (S(rp, pp) - S(rm, pm)) / (2 * h)
    G = afb.target_entropy_gradient(ph, r)
    assert np.max(np.abs(dS - G)) < 1e-7 * np.max(np.abs(G))
    assert np.all(G < 0)  # outward luminosity through entropy diffusion: superadiabatic, dS/dr < 0


def test_target_gradient_closed_form_and_radiative_term():
    """Gamma = -L/(4 pi r^2 rho_a T_a kappa) - C_p kappa_r dT_a/dr / (T_a kappa); L = 4 pi r_i^2 f_b.
    And the thermal balance of Section 4.1 holds for the reference: the total flux
    -kappa rho_a T_a Gamma - kappa_r rho_a C_p dT_a/dr equals L / (4 pi r^2)."""
    ph = _ph(bottom_flux=3e-5, kappa_r=2e-4)
    r = np.array([0.8, 0.9])
    L = 4 * math.pi * 0.75 ** 2 * 3e-5
    pt = ph.polytrope
    dT = -pt["T_c"] * pt["alpha"] * pt["d"] / r ** 2
    want = -L / (4 * math.pi * r ** 2 * ph.rho_a(r) * ph.T_a(r) * 5e-4) - ph.Cp * 2e-4 * dT / (ph.T_a(r) * 5e-4)
    G = afb.target_entropy_gradient(ph, r)
    assert np.allclose(G, want, rtol=1e-14)
    flux = -5e-4 * ph.rho_a(r) * ph.T_a(r) * G - 2e-4 * ph.rho_a(r) * ph.Cp * dT
    assert np.allclose(flux, L / (4 * math.pi * r ** 2), rtol=1e-13)
    # dT_a/dr against a finite difference of T_a
    h = 1e-6
    assert np.allclose(afb.dT_a_dr(ph, r), (ph.T_a(r + h) - ph.T_a(r - h)) / (2 * h), rtol=1e-8)


def test_solar_radiative_profile_carries_the_luminosity_at_the_bottom():
    """The Section 7.2 choice of lambda: the radiative flux equals L/(4 pi r_i^2) at r_i, so the
    target entropy gradient vanishes there; above it the layer is superadiabatic."""
    from chorus_inputs import paper_case_phys

    beta, phys = paper_case_phys("sun")
    ph = Physics.from_params(phys, beta, 1.0)
    assert ph.kappa_r_varies
    G = afb.target_entropy_gradient(ph, np.array([beta, 0.8, 0.9, 1.0]))
    G_scale = abs(afb.luminosity(ph)) / (4 * math.pi * beta ** 2 * ph.rho_a(beta) * ph.T_a(beta) * ph.kappa)
    assert abs(G[0]) < 1e-10 * G_scale
    assert np.all(G[1:] < 0)
    r = np.linspace(beta, 1.0, 50)
    assert np.all(ph.kappa_r_at(r) > 0)
