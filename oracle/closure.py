"""Oracle: pieces of the learned subgrid closure (test infrastructure only).

The paper motivates large-eddy / subgrid-scale modelling as future work (Section 8); the closure
itself is defined by the workload, not by the paper:
  * coarse state: per-element L2 projection of a fine-order state onto the coarse-order basis.
    Reading: the projection is taken in the reference cube (unweighted by |J|), one direction at a
    time, Pi = P x P x P with P = M_c^{-1} B, M_c[a][b] = int_0^1 h^c_a h^c_b, B[a][s] =
    int_0^1 h^c_a h^f_s (h^c, h^f the Lagrange bases through the coarse / fine solution points,
    Eq. 15), integrals exact with Gauss-Legendre quadrature;
  * network: per element, x (27 x 5 = 135) -> SiLU(W1 x + b1) (128) -> SiLU(W2 h1 + b2) (128) ->
    W3 h2 + b3 (135), SiLU(z) = z / (1 + exp(-z));
  * loss: mean over samples and outputs of (y - target)^2 / 2.
"""
from __future__ import annotations

import numpy as np

from .sd_points import lagrange, solution_points


def projection_matrix(Nf: int, Nc: int) -> np.ndarray:
    """P [Nc, Nf] mapping fine solution-point values to coarse ones (1D L2 projection)."""
    xs_f, xs_c = solution_points(Nf), solution_points(Nc)
    gx, gw = np.polynomial.legendre.leggauss(Nf + Nc)
    gx, gw = 0.5 * (gx + 1.0), 0.5 * gw
    hc = np.array([lagrange(xs_c, a, gx) for a in range(Nc)])  # [Nc, G]
    hf = np.array([lagrange(xs_f, s, gx) for s in range(Nf)])  # [Nf, G]
    M = (hc * gw) @ hc.T
    B = (hc * gw) @ hf.T
    return np.linalg.solve(M, B)


def project(Q: np.ndarray, P: np.ndarray) -> np.ndarray:
    """Apply P along the three axes of [..., Nf, Nf, Nf] (k, j, i) -> [..., Nc, Nc, Nc]."""
    return np.einsum("ck,bj,ai,...kji->...cba", P, P, P, Q)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init_params(seed: int, n_in: int = 135, n_hidden: int = 128, n_out: int = 135, scale_out: float = 0.1):
    """Seeded initial weights (uniform, fan-in scaled); the output layer starts small."""
    rng = np.random.default_rng(seed)

    def u(n_o, n_i, s=1.0):
        lim = s * np.sqrt(3.0 / n_i)
        return rng.uniform(-lim, lim, size=(n_o, n_i))

    return dict(W1=u(n_hidden, n_in), b1=np.zeros(n_hidden), W2=u(n_hidden, n_hidden), b2=np.zeros(n_hidden),
                W3=u(n_out, n_hidden, scale_out), b3=np.zeros(n_out))


def forward(params, X):
    """X [B, 135] -> (Y [B, 135], cache)."""
    z1 = X @ params["W1"].T + params["b1"]
    h1 = silu(z1)
    z2 = h1 @ params["W2"].T + params["b2"]
    h2 = silu(z2)
    Y = h2 @ params["W3"].T + params["b3"]
    return Y, dict(X=X, z1=z1, h1=h1, z2=z2, h2=h2)


def round_bf16(x):
    """Round to the nearest bfloat16 value (8-bit significand, ties to even), returned as float64.

    bfloat16 keeps the sign, the 8 exponent bits and the top 7 fraction bits of an IEEE binary32.
    The value is first rounded to binary32, then the low 16 bits are rounded off: add 0x7FFF plus
    the lowest kept bit and truncate (round half to even on the dropped 16 bits)."""
    b = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    keep = (b >> np.uint64(16)) & np.uint64(1)
    r = ((b + np.uint64(0x7FFF) + keep) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16_inputs(params, X):
    """The forward pass with every layer's input rounded to bfloat16 (the tensor-core arithmetic:
    BF16 operands, sums in a wider format)."""
    z1 = round_bf16(X) @ params["W1"].T + params["b1"]
    z2 = round_bf16(silu(z1)) @ params["W2"].T + params["b2"]
    return round_bf16(silu(z2)) @ params["W3"].T + params["b3"]


def loss_and_grad(params, X, T):
    """Mean squared error / 2 and its gradient with respect to every parameter (backpropagation)."""
    Y, c = forward(params, X)
    n = Y.size
    dY = (Y - T) / n
    loss = 0.5 * np.sum((Y - T) ** 2) / n
    g = {}
    g["W3"] = dY.T @ c["h2"]
    g["b3"] = dY.sum(0)
    dz2 = (dY @ params["W3"]) * silu_grad(c["z2"])
    g["W2"] = dz2.T @ c["h1"]
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ params["W2"]) * silu_grad(c["z1"])
    g["W1"] = dz1.T @ c["X"]
    g["b1"] = dz1.sum(0)
    return loss, g


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015) in place; state holds m, v and the step count."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = beta1 * m + (1 - beta1) * grads[k]
        v[...] = beta2 * v + (1 - beta2) * grads[k] ** 2
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params
