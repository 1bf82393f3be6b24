"""Pins of the oracle's closure pieces: order projection and network backpropagation."""
import numpy as np
import pytest

from oracle.closure import adam_step, forward, init_params, loss_and_grad, project, projection_matrix, silu, \
    silu_grad
from oracle.sd_points import solution_points


@pytest.mark.parametrize("Nf,Nc", [(6, 3), (5, 3), (4, 2)])
def test_projection_exact_on_coarse_polynomials_and_orthogonal(Nf, Nc):
    P = projection_matrix(Nf, Nc)
    xf, xc = solution_points(Nf), solution_points(Nc)
    for k in range(Nc):  # degree < Nc is kept exactly
        assert np.allclose(P @ xf ** k, xc ** k, atol=1e-13)
    # the projection error of a higher-degree function is orthogonal to the coarse polynomials
    gx, gw = np.polynomial.legendre.leggauss(12)
    gx, gw = 0.5 * (gx + 1), 0.5 * gw
    from oracle.sd_points import lagrange

    f = xf ** (Nf - 1)
    fine = sum(f[s] * lagrange(xf, s, gx) for s in range(Nf))
    coarse = sum((P @ f)[a] * lagrange(xc, a, gx) for a in range(Nc))
    for k in range(Nc):
        assert abs(np.sum(gw * (fine - coarse) * gx ** k)) < 1e-13


def test_projection_tensor_product():
    P = projection_matrix(6, 3)
    xf = solution_points(6)
    Z, Y, X = np.meshgrid(xf, xf, xf, indexing="ij")
    Q = 1.0 + 2.0 * X - Y * Z + 0.5 * X * Y * Z  # degree <= 2 per axis
    xc = solution_points(3)
    Zc, Yc, Xc = np.meshgrid(xc, xc, xc, indexing="ij")
    assert np.allclose(project(Q[None], P)[0], 1.0 + 2.0 * Xc - Yc * Zc + 0.5 * Xc * Yc * Zc, atol=1e-13)


def test_silu_derivative():
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    assert np.allclose((silu(z + h) - silu(z - h)) / (2 * h), silu_grad(z), atol=1e-8)


def test_backprop_against_finite_differences():
    rng = np.random.default_rng(0)
    p = init_params(1, n_in=7, n_hidden=5, n_out=6, scale_out=1.0)
    X = rng.standard_normal((9, 7))
    T = rng.standard_normal((9, 6))
    _, g = loss_and_grad(p, X, T)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = loss_and_grad(p, X, T)
            flat[idx] = old - h
            lm, _ = loss_and_grad(p, X, T)
            flat[idx] = old
            assert abs((lp - lm) / (2 * h) - g[k].reshape(-1)[idx]) < 1e-7 * max(1.0, abs(g[k].reshape(-1)[idx]))


def test_adam_reduces_loss_on_a_fit():
    rng = np.random.default_rng(3)
    p = init_params(2, n_in=8, n_hidden=16, n_out=4)
    X = rng.standard_normal((64, 8))
    T = np.tanh(X[:, :4]) * 0.3
    st = {}
    l0, _ = loss_and_grad(p, X, T)
    for _ in range(300):
        _, g = loss_and_grad(p, X, T)
        adam_step(p, g, st, 3e-3)
    l1, _ = loss_and_grad(p, X, T)
    assert l1 < 0.2 * l0


def test_round_bf16_against_exact_values():
    from oracle.closure import round_bf16

    # exactly representable values stay; 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even keeps 1;
    # 1 + 3 * 2^-8 ties between 1 + 2^-7 (odd) and 1 + 2^-6 (even); above a tie rounds up
    x = np.array([1.0, -2.5, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -20, 3.0e-39, 0.0])
    want = np.array([1.0, -2.5, 1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7, None, 0.0], dtype=object)
    got = round_bf16(x)
    for g, w in zip(got, want):
        if w is not None:
            assert g == w
    # relative rounding error at most 2^-8 for normal numbers
    rng = np.random.default_rng(3)
    v = rng.standard_normal(10000) * 10.0 ** rng.uniform(-5, 5, 10000)
    assert np.all(np.abs(round_bf16(v) - v.astype(np.float32)) <= 2.0 ** -8 * np.abs(v.astype(np.float32)))


def test_forward_bf16_inputs_close_to_forward():
    from oracle.closure import forward, forward_bf16_inputs, init_params

    p = init_params(4)
    X = np.random.default_rng(5).standard_normal((64, 135))
    Y, _ = forward(p, X)
    Yb = forward_bf16_inputs(p, X)
    rel = np.linalg.norm(Yb - Y) / np.linalg.norm(Y)
    assert 1e-5 < rel < 1e-2  # BF16 inputs perturb the result at the 2^-9 level, no more
