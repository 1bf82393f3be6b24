"""Host-side diagnostics of the closure evaluation (no GPU)."""
import numpy as np

from paper_1503_00834_gb300.closure_eval import (Diagnostics, _element_volumes, _legendre_inverse_vandermonde,
                                                 _solution_points)


def _unit_cube():
    c = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], float)
    return c, np.arange(8)[None].repeat(1, 0)


def test_volume_of_cube_and_sheared_hex():
    c, h = _unit_cube()
    h20 = np.concatenate([h, np.zeros((1, 12), int)], axis=1)
    assert abs(_element_volumes(c, h20)[0] - 1.0) < 1e-14
    s = c * np.array([2.0, 3.0, 0.5]) + c[:, 2:3] * np.array([0.7, -0.2, 0.0])  # scaled and sheared
    assert abs(_element_volumes(s, h20)[0] - 3.0) < 1e-12


def test_legendre_modes_are_orthonormal_on_the_unit_interval():
    N = 3
    X = _solution_points(N)
    Vinv = _legendre_inverse_vandermonde(N)
    # nodal values of x^2 -> modal; the L2 norm on [0,1] of x^2 is 1/5
    m = Vinv @ X ** 2
    assert abs(np.sum(m ** 2) - 0.2) < 1e-14


def test_spectrum_of_constant_and_linear_fields():
    N = 3
    c, h = _unit_cube()
    h20 = np.concatenate([h, np.zeros((1, 12), int)], axis=1)
    Q0 = np.zeros((1, 5, N, N, N))
    Q0[:, 0] = 1.0
    d = Diagnostics(c, h20, N, Q0)
    q = np.zeros((1, 5, N, N, N))
    q[:, 1] = 2.0  # m_x = 2, rho = 1: kinetic energy 2 in degree 0 only
    E = d.ke_spectrum(q)
    assert abs(E[0] - 2.0) < 1e-13 and np.all(np.abs(E[1:]) < 1e-13)
    X = _solution_points(N)
    q[:, 1] = 0.0
    q[:, 2] = X[None, None, :]  # m_y = x (axis i): mean 1/2, linear mode sqrt(1/12)
    E = d.ke_spectrum(q)
    assert abs(E[0] - 0.125) < 1e-13 and abs(E[1] - 0.5 / 12) < 1e-13
    assert d.l2(q, q) == 0.0 and d.ke_error(q, q) == 0.0
