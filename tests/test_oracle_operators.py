"""Pins of the oracle's 1D points and Lagrange operators (Section 3, Eqs. 13-18).

Each check compares against something the oracle does not compute itself:
closed forms, library root finders and quadrature rules, or exactness on
polynomials, which a dropped term or transposed index breaks.
"""
import itertools
import math

import numpy as np
import pytest

from oracle.sd_points import flux_points, lagrange, lagrange_deriv, operators, solution_points

NS = [2, 3, 4, 5, 6]


@pytest.mark.parametrize("N", NS)
def test_solution_points_are_chebyshev_roots(N):
    # Eq. 13 points are the roots of T_N(2x - 1) (Chebyshev-Gauss points)
    c = np.zeros(N + 1)
    c[-1] = 1.0
    roots = np.sort(0.5 * (np.polynomial.chebyshev.chebroots(c) + 1.0))
    assert np.allclose(solution_points(N), roots, atol=1e-14)


@pytest.mark.parametrize("N", NS)
def test_flux_points_are_legendre_gauss_plus_ends(N):
    # Eq. 14: roots of P_{N-1} on [0,1] plus 0 and 1 (library Gauss-Legendre nodes)
    xf = flux_points(N)
    assert xf.size == N + 1 and xf[0] == 0.0 and xf[-1] == 1.0
    if N > 1:
        g, _ = np.polynomial.legendre.leggauss(N - 1)
        assert np.allclose(xf[1:-1], 0.5 * (np.sort(g) + 1.0), atol=1e-14)


def test_flux_points_N4_closed_form():
    s = math.sqrt(3.0 / 5.0)
    assert np.allclose(flux_points(4), [0.0, 0.5 - 0.5 * s, 0.5, 0.5 + 0.5 * s, 1.0], atol=1e-15)


@pytest.mark.parametrize("N", NS)
def test_lagrange_cardinal(N):
    for nodes in (solution_points(N), flux_points(N)):
        M = np.array([[lagrange(nodes, i, nodes[j]) for j in range(len(nodes))] for i in range(len(nodes))])
        assert np.allclose(M, np.eye(len(nodes)), atol=1e-13)


@pytest.mark.parametrize("N", NS)
def test_interpolation_and_derivative_exact_on_polynomials(N):
    ops = operators(N)
    Xs, Xf = ops.Xs, ops.Xf
    for k in range(N):  # degree <= N-1 is reproduced by I
        assert np.allclose(ops.I @ Xs ** k, Xf ** k, atol=1e-13)
    for k in range(N + 1):  # degree <= N is differentiated exactly by D and Dff, evaluated by Lfs
        dk = k * Xs ** (k - 1) if k else np.zeros(N)
        assert np.allclose(ops.D @ Xf ** k, dk, atol=1e-11)
        assert np.allclose(ops.Lfs @ Xf ** k, Xs ** k, atol=1e-13)
        assert np.allclose(ops.Dfs @ Xf ** k, dk, atol=1e-11)
        dkf = k * Xf ** (k - 1) if k else np.zeros(N + 1)
        assert np.allclose(ops.Dff @ Xf ** k, dkf, atol=1e-11)


@pytest.mark.parametrize("N", NS)
def test_quadrature_weights(N):
    ops = operators(N)
    # interpolatory weights integrate every polynomial of degree < N exactly
    for k in range(N):
        assert abs(np.sum(ops.w * ops.Xs ** k) - 1.0 / (k + 1)) < 1e-14
    assert np.allclose(ops.w, ops.w[::-1], atol=1e-15)
    # discrete divergence theorem: sum_s w_s (D f)_s = f(1) - f(0) for any flux-point data
    rng = np.random.default_rng(N)
    f = rng.standard_normal(N + 1)
    assert abs(ops.w @ (ops.D @ f) - (f[-1] - f[0])) < 1e-13


def test_weights_p2_closed_form():
    assert np.allclose(operators(3).w, [2.0 / 9.0, 5.0 / 9.0, 2.0 / 9.0], atol=1e-15)


@pytest.mark.parametrize("N", [3, 4])
def test_tensor_product_against_brute_force(N):
    """Eqs. 17-18 on one element: the oracle's sweeps equal per-point triple Lagrange sums."""
    from oracle.residual import derivative, interp_to_flux

    ops = operators(N)
    Xs, Xf = ops.Xs, ops.Xf
    rng = np.random.default_rng(3)
    q = rng.standard_normal((N, N, N))  # [k, j, i]
    a_xi, a_eta, a_zeta = interp_to_flux(ops, q)
    for f, j, k in itertools.product(range(N + 1), range(N), range(N)):
        bf = sum(q[kk, jj, ii] * lagrange(Xs, ii, Xf[f]) * lagrange(Xs, jj, Xs[j]) * lagrange(Xs, kk, Xs[k])
                 for ii, jj, kk in itertools.product(range(N), repeat=3))
        assert abs(a_xi[k, j, f] - bf) < 1e-12
        bf = sum(q[kk, jj, ii] * lagrange(Xs, ii, Xs[j]) * lagrange(Xs, jj, Xf[f]) * lagrange(Xs, kk, Xs[k])
                 for ii, jj, kk in itertools.product(range(N), repeat=3))
        assert abs(a_eta[k, f, j] - bf) < 1e-12
        bf = sum(q[kk, jj, ii] * lagrange(Xs, ii, Xs[j]) * lagrange(Xs, jj, Xs[k]) * lagrange(Xs, kk, Xf[f])
                 for ii, jj, kk in itertools.product(range(N), repeat=3))
        assert abs(a_zeta[f, k, j] - bf) < 1e-12
    # Eq. 18: derivative of F~ = sum F_{i+1/2} l(xi) h(eta) h(zeta) at the solution points
    F = rng.standard_normal((N, N, N + 1))
    dxi = derivative(ops, (F, np.zeros((N, N + 1, N)), np.zeros((N + 1, N, N))))[0]
    for i, j, k in itertools.product(range(N), repeat=3):
        bf = sum(F[k, j, f] * lagrange_deriv(Xf, f, Xs[i]) for f in range(N + 1))
        assert abs(dxi[k, j, i] - bf) < 1e-11


def test_splitmix64_published_value():
    # first output of SplitMix64 from state 0 (Vigna's reference generator)
    from oracle.state import splitmix64

    assert int(splitmix64(np.uint64(0))) == 0xE220A8397B1DCDAF
