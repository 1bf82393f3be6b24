"""Oracle: iso-parametric 20-node geometry and metrics (Section 3, Eqs. 10-12; Section 5).

Test infrastructure only (see the package docstring).

The physical element is the image of the unit cube under the quadratic
serendipity map of its 20 nodes (8 corners + 12 mid-edge nodes, Section 5).
The Jacobian matrix is Eq. 10; the transformed fluxes of Eq. 12 need the rows
of |J| J^{-1}, i.e. S^d_n = |J| d xi_d / d x_n.

Metric evaluation (the paper only states Eq. 12): conservative curl form
    S^d_n = -[ curl_xi  I^N( X_l grad_xi X_m ) ]_d ,  (n, m, l) cyclic,
where I^N interpolates on the (N+1)^3 tensor grid of flux-point coordinates
(end points included) and X_m is itself first interpolated on that grid.  The
curl is taken exactly.  This makes the discrete metric identities hold, so a
uniform flow is preserved on curved elements for every N, and the metric on a
face depends only on that face's geometry.  The check variant
`analytic_cofactors` evaluates x_eta x x_zeta etc. directly.

Rounding: the Jacobian matrix and the curl-form products are formed from the node coordinates
measured from the element's node centroid.  Eqs. 10-12 are invariant under a translation of x
(d x / d xi is unchanged; curl I^N(c grad X_m) = 0 for the polynomial map), so the discrete metrics
are the same, but the products X_l grad X_m are then of size h^2 instead of h, which removes the
cancellation that otherwise costs a factor ~1/h of FP64 accuracy in the metrics.

All geometry follows the dtype of the node coordinates (float64; np.longdouble for extended-
precision runs of the oracle).
"""
from __future__ import annotations

import numpy as np

from .sd_points import operators

# node reference coordinates in units of 1/2 (same order as the mesh inputs)
_REF2 = np.array(
    [
        [0, 0, 0], [2, 0, 0], [2, 2, 0], [0, 2, 0],
        [0, 0, 2], [2, 0, 2], [2, 2, 2], [0, 2, 2],
        [1, 0, 0], [2, 1, 0], [1, 2, 0], [0, 1, 0],
        [1, 0, 2], [2, 1, 2], [1, 2, 2], [0, 1, 2],
        [0, 0, 1], [2, 0, 1], [2, 2, 1], [0, 2, 1],
    ],
    dtype=np.float64,
)
# natural coordinates in {-1, 0, 1}
_NAT = _REF2 - 1.0


def shape_functions(xi, eta, zeta):
    """Serendipity 20-node shape functions N_a and d N_a / d(xi, eta, zeta) on [0,1]^3.

    Returns (N [...,20], dN [...,20,3]).  With natural coordinates
    a = 2 xi - 1 etc. and node coordinates (a_i, b_i, c_i):
      corner:      (1/8)(1+a a_i)(1+b b_i)(1+c c_i)(a a_i + b b_i + c c_i - 2)
      mid-edge with a_i = 0: (1/4)(1-a^2)(1+b b_i)(1+c c_i), and likewise.
    """
    dt = np.result_type(np.asarray(xi), np.asarray(eta), np.asarray(zeta), np.float64)
    a = 2.0 * np.asarray(xi, dtype=dt) - 1.0
    b = 2.0 * np.asarray(eta, dtype=dt) - 1.0
    c = 2.0 * np.asarray(zeta, dtype=dt) - 1.0
    a, b, c = np.broadcast_arrays(a, b, c)
    shp = a.shape + (20,)
    Nv = np.zeros(shp, dtype=dt)
    dN = np.zeros(shp + (3,), dtype=dt)
    for i in range(20):
        ai, bi, ci = _NAT[i]
        if ai != 0 and bi != 0 and ci != 0:
            fa, fb, fc = 1 + a * ai, 1 + b * bi, 1 + c * ci
            s = a * ai + b * bi + c * ci - 2.0
            Nv[..., i] = 0.125 * fa * fb * fc * s
            da = 0.125 * (ai * fb * fc * s + fa * fb * fc * ai)
            db = 0.125 * (bi * fa * fc * s + fa * fb * fc * bi)
            dc = 0.125 * (ci * fa * fb * s + fa * fb * fc * ci)
        elif ai == 0:
            fb, fc = 1 + b * bi, 1 + c * ci
            Nv[..., i] = 0.25 * (1 - a * a) * fb * fc
            da = 0.25 * (-2 * a) * fb * fc
            db = 0.25 * (1 - a * a) * bi * fc
            dc = 0.25 * (1 - a * a) * fb * ci
        elif bi == 0:
            fa, fc = 1 + a * ai, 1 + c * ci
            Nv[..., i] = 0.25 * (1 - b * b) * fa * fc
            da = 0.25 * (1 - b * b) * ai * fc
            db = 0.25 * (-2 * b) * fa * fc
            dc = 0.25 * (1 - b * b) * fa * ci
        else:
            fa, fb = 1 + a * ai, 1 + b * bi
            Nv[..., i] = 0.25 * (1 - c * c) * fa * fb
            da = 0.25 * (1 - c * c) * ai * fb
            db = 0.25 * (1 - c * c) * fa * bi
            dc = 0.25 * (-2 * c) * fa * fb
        # chain rule d/dxi = 2 d/da
        dN[..., i, 0] = 2.0 * da
        dN[..., i, 1] = 2.0 * db
        dN[..., i, 2] = 2.0 * dc
    return Nv, dN


def map_points(nodes: np.ndarray, xi, eta, zeta) -> np.ndarray:
    """x(xi) for elements nodes [E,20,3] at reference points (broadcast shape P) -> [E, *P, 3]."""
    Nv, _ = shape_functions(xi, eta, zeta)
    return np.einsum("...a,ean->e...n", Nv, nodes)


def jacobian_matrix(nodes: np.ndarray, xi, eta, zeta) -> np.ndarray:
    """Eq. 10: Jm[e, ..., n, d] = d x_n / d xi_d."""
    _, dN = shape_functions(xi, eta, zeta)
    return np.einsum("...ad,ean->e...nd", dN, nodes)


def _grid(ops):
    """Solution-point grid (k, j, i) order: returns xi, eta, zeta broadcastable [N,N,N]."""
    X = ops.Xs
    return X[None, None, :], X[None, :, None], X[:, None, None]


def centred(nodes: np.ndarray) -> np.ndarray:
    """Node coordinates measured from each element's node centroid (a translation: same metrics)."""
    return nodes - nodes.mean(axis=1, keepdims=True)


def det3(J: np.ndarray) -> np.ndarray:
    """Determinant of [..., 3, 3] matrices by cofactor expansion along the first row."""
    return (J[..., 0, 0] * (J[..., 1, 1] * J[..., 2, 2] - J[..., 1, 2] * J[..., 2, 1])
            - J[..., 0, 1] * (J[..., 1, 0] * J[..., 2, 2] - J[..., 1, 2] * J[..., 2, 0])
            + J[..., 0, 2] * (J[..., 1, 0] * J[..., 2, 1] - J[..., 1, 1] * J[..., 2, 0]))


def solution_geometry(nodes: np.ndarray, N: int):
    """x [E,3,N,N,N] and |J| [E,N,N,N] at the solution points (axes k, j, i)."""
    ops = operators(N, nodes.dtype.type)
    xi, eta, zeta = _grid(ops)
    x = map_points(nodes, xi, eta, zeta)  # [E,k,j,i,3]
    Jm = jacobian_matrix(centred(nodes), xi, eta, zeta)  # [E,k,j,i,3,3]
    detJ = det3(Jm)
    return np.moveaxis(x, -1, 1), detJ


def curl_metrics(nodes: np.ndarray, N: int):
    """Conservative curl-form metrics.

    Returns
      S_xi   [E,3(n),N(k),N(j),N+1(f)]   S^xi_n   at the xi-flux points
      S_eta  [E,3(n),N(k),N+1(f),N(i)]   S^eta_n  at the eta-flux points
      S_zeta [E,3(n),N+1(f),N(j),N(i)]   S^zeta_n at the zeta-flux points
      S_sol  [E,3(d),3(n),N,N,N]         S^d_n    at the solution points
    """
    ops = operators(N, nodes.dtype.type)
    Xf = ops.Xf
    dt = nodes.dtype
    # geometry on the (N+1)^3 flux-point grid, axes (c, b, a) = (zeta, eta, xi), from the centroid
    X = map_points(centred(nodes), Xf[None, None, :], Xf[:, None][None], Xf[:, None, None])  # [E,c,b,a,3]
    Dff = ops.Dff
    # derivatives of the grid interpolant of each coordinate: dX[e,c,b,a,m,dir]
    dX = np.stack(
        [
            np.einsum("ax,ecbxm->ecbam", Dff, X),
            np.einsum("by,ecyam->ecbam", Dff, X),
            np.einsum("cz,ezbam->ecbam", Dff, X),
        ],
        axis=-1,
    )
    E = nodes.shape[0]
    Lfs, Dfs = ops.Lfs, ops.Dfs
    S_xi = np.zeros((E, 3, N, N, N + 1), dtype=dt)
    S_eta = np.zeros((E, 3, N, N + 1, N), dtype=dt)
    S_zeta = np.zeros((E, 3, N + 1, N, N), dtype=dt)
    S_sol = np.zeros((E, 3, 3, N, N, N), dtype=dt)
    for n in range(3):
        m, l = (n + 1) % 3, (n + 2) % 3
        V = X[..., l, None] * dX[..., m, :]  # [E,c,b,a,dir] = X_l * d X_m / d xi_dir
        Vxi, Veta, Vzeta = V[..., 0], V[..., 1], V[..., 2]
        # S^xi_n = -(d_eta V_zeta - d_zeta V_eta), evaluated at (Xf_f, X_j, X_k)
        S_xi[:, n] = -(
            np.einsum("jb,kc,ecbf->ekjf", Dfs, Lfs, Vzeta) - np.einsum("jb,kc,ecbf->ekjf", Lfs, Dfs, Veta)
        )
        # S^eta_n = -(d_zeta V_xi - d_xi V_zeta), at (X_i, Xf_f, X_k)
        S_eta[:, n] = -(
            np.einsum("kc,ia,ecfa->ekfi", Dfs, Lfs, Vxi) - np.einsum("kc,ia,ecfa->ekfi", Lfs, Dfs, Vzeta)
        )
        # S^zeta_n = -(d_xi V_eta - d_eta V_xi), at (X_i, X_j, Xf_f)
        S_zeta[:, n] = -(
            np.einsum("ia,jb,efba->efji", Dfs, Lfs, Veta) - np.einsum("ia,jb,efba->efji", Lfs, Dfs, Vxi)
        )
        # the same three polynomials at the solution points
        S_sol[:, 0, n] = -(
            np.einsum("ia,jb,kc,ecba->ekji", Lfs, Dfs, Lfs, Vzeta)
            - np.einsum("ia,jb,kc,ecba->ekji", Lfs, Lfs, Dfs, Veta)
        )
        S_sol[:, 1, n] = -(
            np.einsum("ia,jb,kc,ecba->ekji", Lfs, Lfs, Dfs, Vxi)
            - np.einsum("ia,jb,kc,ecba->ekji", Dfs, Lfs, Lfs, Vzeta)
        )
        S_sol[:, 2, n] = -(
            np.einsum("ia,jb,kc,ecba->ekji", Dfs, Lfs, Lfs, Veta)
            - np.einsum("ia,jb,kc,ecba->ekji", Lfs, Dfs, Lfs, Vxi)
        )
    return S_xi, S_eta, S_zeta, S_sol


def analytic_cofactors(nodes: np.ndarray, xi, eta, zeta) -> np.ndarray:
    """S[e,...,d,n] = rows of the cofactor matrix |J| J^{-1} from x_xi, x_eta, x_zeta directly."""
    Jm = jacobian_matrix(nodes, xi, eta, zeta)  # [..., n, d]
    a = [Jm[..., :, d] for d in range(3)]  # covariant basis vectors a_d = dx/dxi_d
    return np.stack([np.cross(a[1], a[2]), np.cross(a[2], a[0]), np.cross(a[0], a[1])], axis=-2)
