"""Oracle: 1D point sets and Lagrange operators of the SD method (Section 3).

Test infrastructure only (see the package docstring).

Reference element [0, 1].  N = p + 1 solution points per direction.
  solution points  Eq. 13: X_s = (1 - cos((2s-1) pi / (2N))) / 2, s = 1..N
  flux points      Eq. 14: the N-1 roots of the shifted Legendre polynomial
                   P_{N-1} (built by the three-term recurrence) plus the end
                   points 0 and 1, N + 1 points in total.
  h_i              Eq. 15: degree N-1 Lagrange basis through the solution points
  l_{i+1/2}        Eq. 16: degree N Lagrange basis through the flux points; the
                   product runs over s = 0..N, s != i (the printed index is
                   garbled; this is the only reading that gives a cardinal basis).
"""
from __future__ import annotations

import functools

import numpy as np


def solution_points(N: int, dtype=np.float64) -> np.ndarray:
    s = np.arange(1, N + 1).astype(dtype)
    pi = np.arccos(dtype(-1))  # pi to the working precision
    return 0.5 * (1.0 - np.cos((2.0 * s - 1.0) / (2.0 * N) * pi))


def shifted_legendre(n: int, x):
    """P_n on [0,1] from the recurrence of Eq. 14 (P_{-1} = 0, P_0 = 1)."""
    x = np.asarray(x)
    if x.dtype.kind != "f":
        x = x.astype(np.float64)
    p_prev = np.zeros_like(x)
    p = np.ones_like(x)
    for m in range(1, n + 1):
        p_prev, p = p, ((2.0 * m - 1.0) / m) * (2.0 * x - 1.0) * p - ((m - 1.0) / m) * p_prev
    return p


def flux_points(N: int, dtype=np.float64) -> np.ndarray:
    """End points plus the roots of P_{N-1}; roots bracketed on a fine grid, then bisected."""
    n = N - 1
    roots = []
    if n >= 1:
        grid = np.linspace(dtype(0), dtype(1), 200 * N + 1, dtype=dtype)
        vals = shifted_legendre(n, grid)
        for a, b, fa, fb in zip(grid[:-1], grid[1:], vals[:-1], vals[1:]):
            if fa == 0.0:
                roots.append(a)
                continue
            if fa * fb < 0.0:
                lo, hi, flo = a, b, fa
                for _ in range(200):
                    mid = 0.5 * (lo + hi)
                    fm = shifted_legendre(n, mid)
                    if fm == 0.0 or mid == lo or mid == hi:
                        break
                    if (fm < 0.0) == (flo < 0.0):
                        lo, flo = mid, fm
                    else:
                        hi = mid
                roots.append(0.5 * (lo + hi))
    assert len(roots) == n, (N, roots)
    return np.array([dtype(0)] + sorted(roots) + [dtype(1)], dtype=dtype)


def lagrange(nodes: np.ndarray, i: int, x):
    """Lagrange cardinal polynomial through `nodes`, index i, at x (Eqs. 15, 16)."""
    x = np.asarray(x, dtype=nodes.dtype)
    out = np.ones_like(x)
    for s in range(len(nodes)):
        if s != i:
            out = out * (x - nodes[s]) / (nodes[i] - nodes[s])
    return out


def lagrange_deriv(nodes: np.ndarray, i: int, x):
    """d/dx of the Lagrange cardinal polynomial: product rule over the factors."""
    x = np.asarray(x, dtype=nodes.dtype)
    total = np.zeros_like(x)
    for m in range(len(nodes)):
        if m == i:
            continue
        term = np.full_like(x, 1.0 / (nodes[i] - nodes[m]))
        for s in range(len(nodes)):
            if s != i and s != m:
                term = term * (x - nodes[s]) / (nodes[i] - nodes[s])
        total = total + term
    return total


class Operators:
    """1D matrices of one order N.

    I[f, s]   = h_s(Xf_f)        solution -> flux points          (N+1, N)
    D[s, f]   = l'_f(X_s)        flux-point values -> d/dX at solution points (N, N+1)
    Lfs[s, a] = l_a(X_s)         flux-point polynomial evaluated at solution points (N, N+1)
    Dff[a, b] = l'_b(Xf_a)       derivative on the flux-point grid (N+1, N+1)
    Dfs[s, a] = l'_a(X_s)        derivative of flux-point polynomials at solution points (N, N+1)
    w[s]      = int_0^1 h_s dX   interpolatory quadrature weights at the solution points

    dtype: the working precision of the points and matrices (float64; np.longdouble for extended-
    precision runs of the oracle).  The weights are computed in float64 (they enter only integrals).
    """

    def __init__(self, N: int, dtype=np.float64):
        self.N = N
        self.Xs = solution_points(N, dtype)
        self.Xf = flux_points(N, dtype)
        Xs, Xf = self.Xs, self.Xf
        self.I = np.array([[lagrange(Xs, s, Xf[f]) for s in range(N)] for f in range(N + 1)])
        self.D = np.array([[lagrange_deriv(Xf, f, Xs[s]) for f in range(N + 1)] for s in range(N)])
        self.Lfs = np.array([[lagrange(Xf, a, Xs[s]) for a in range(N + 1)] for s in range(N)])
        self.Dff = np.array([[lagrange_deriv(Xf, b, Xf[a]) for b in range(N + 1)] for a in range(N + 1)])
        self.Dfs = np.array([[lagrange_deriv(Xf, a, Xs[s]) for a in range(N + 1)] for s in range(N)])
        # exact integral of h_s over [0,1] with an N-point Gauss-Legendre rule (degree N-1 integrand)
        gx, gw = np.polynomial.legendre.leggauss(N)
        gx = 0.5 * (gx + 1.0)
        gw = 0.5 * gw
        Xs64 = Xs.astype(np.float64)
        self.w = np.array([np.sum(gw * lagrange(Xs64, s, gx)) for s in range(N)])


@functools.lru_cache(maxsize=None)
def operators(N: int, dtype=np.float64) -> Operators:
    return Operators(N, dtype)
