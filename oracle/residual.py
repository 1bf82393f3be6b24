"""Oracle: the semi-discrete spectral-difference residual (Sections 3 and 5).

Test infrastructure only (see the package docstring).

State layout: Q[e, v, k, j, i] (v = rho, rho u, rho v, rho w, E; i along xi,
j along eta, k along zeta), physical conserved variables at the solution
points.  The residual returned is dQ/dt at the solution points.  The paper
advances Q~ = |J| Q (Eq. 11); on a static mesh that is the same ODE divided by
|J|.

Steps, in the paper's order (Eqs. 11-18 and the interface treatment):
  1. interpolate Q from the solution points to the flux points of each
     direction with h_i (Eq. 17);
  2. viscous part, BR1-like "simple averaging" (reading of the one-sentence
     description): the common solution on a face point is the average of the
     two one-sided traces; the conserved variables are lifted, i.e. dQ/dxi_d
     at the solution points is the derivative of the degree-N polynomial
     through the flux-point values (Eq. 18 basis l) with the face values
     replaced by the common solution; grad Q follows by the chain rule with
     grad xi_d = S^d / |J|; primitive gradients by the quotient rule; they are
     interpolated to the flux points with h_i;
  3. transformed fluxes at the flux points (Eq. 12): F~ = S^xi . (F, G, H);
  4. common fluxes on faces: Rusanov for the inviscid part with the face
     normal taken in physical form n = sigma S^d / |S^d|, and the average of
     the two one-sided normal viscous fluxes; F~ = sigma |S^d| F_n;
  5. walls (Section 5): exact inviscid flux (0, p n, 0) since V_r = 0;
     stress-free: only the normal viscous traction (n.tau.n) n is kept and
     u.tau.n = 0; energy flux f.n = -L/(4 pi R_i^2) at the bottom (prescribed)
     and from the lifted gradient with T fixed at the top.  In the lifting the
     wall common state has zero normal velocity, the interior density, and
     the interior pressure (bottom) or p = R rho T_top (top);
  6. divergence with the derivative of l (Eq. 18) along each direction;
  7. dQ/dt = -(div)/|J| - M (Eqs. 4, 11).
"""
from __future__ import annotations

import numpy as np

from .geometry import curl_metrics, solution_geometry
from .mesh import Connectivity
from .physics import (Physics, grad_primitives, heat_flux, inviscid_flux, primitives, rusanov,
                      source, stress, viscous_flux)
from .sd_points import operators


class Discretization:
    """Mesh, operators and per-element geometry of one shell at order p.

    dtype: working precision of the operators and the geometry (float64; np.longdouble evaluates the
    whole discretisation in extended precision from the same float64 node coordinates)."""

    def __init__(self, node_xyz: np.ndarray, hex20: np.ndarray, p: int, r_inner: float, r_outer: float,
                 dtype=np.float64):
        self.p = p
        self.N = p + 1
        self.dtype = dtype
        self.ops = operators(self.N, dtype)
        self.node_xyz = np.asarray(node_xyz, dtype=np.float64)
        self.hex20 = np.asarray(hex20, dtype=np.int64)
        self.n_elem = self.hex20.shape[0]
        self.r_inner, self.r_outer = r_inner, r_outer
        self.conn = Connectivity(self.node_xyz, self.hex20, self.N, r_inner, r_outer)
        self._geom = {}

    def geometry(self, elems: np.ndarray) -> dict:
        """x, |J|, metrics at flux points and grad xi at solution points for `elems`."""
        key = elems.tobytes()
        if key not in self._geom:
            nodes = self.node_xyz[self.hex20[elems]].astype(self.dtype)
            x, detJ = solution_geometry(nodes, self.N)
            S_xi, S_eta, S_zeta, S_sol = curl_metrics(nodes, self.N)
            self._geom = {key: dict(x=x, detJ=detJ, S=(S_xi, S_eta, S_zeta),
                                    gradxi=S_sol / detJ[:, None, None])}
        return self._geom[key]


# ---------------------------------------------------------------- face helpers

def face_values(arr3, face: int) -> np.ndarray:
    """Values at the N^2 points of a local face, flattened t = t1 + N t2.

    arr3 = (a_xi [..., k, j, f], a_eta [..., k, f, i], a_zeta [..., f, j, i]).
    """
    d, side = face // 2, face % 2
    a = arr3[d]
    if d == 0:
        v = a[..., -1] if side else a[..., 0]  # [..., k, j]
    elif d == 1:
        v = a[..., -1, :] if side else a[..., 0, :]  # [..., k, i]
    else:
        v = a[..., -1, :, :] if side else a[..., 0, :, :]  # [..., j, i]
    return v.reshape(v.shape[:-2] + (-1,))


def set_face_values(arr3, face: int, vals: np.ndarray) -> None:
    d, side = face // 2, face % 2
    a = arr3[d]
    f = -1 if side else 0
    if d == 0:
        a[..., f] = vals.reshape(vals.shape[:-1] + (a.shape[-3], a.shape[-2]))
    elif d == 1:
        a[..., f, :] = vals.reshape(vals.shape[:-1] + (a.shape[-3], a.shape[-1]))
    else:
        a[..., f, :, :] = vals.reshape(vals.shape[:-1] + (a.shape[-2], a.shape[-1]))


def interp_to_flux(ops, u: np.ndarray):
    """Eq. 17: values at the solution points [..., k, j, i] -> the three flux-point sets."""
    I = ops.I
    return (np.einsum("fi,...kji->...kjf", I, u),
            np.einsum("fj,...kji->...kfi", I, u),
            np.einsum("fk,...kji->...fji", I, u))


def derivative(ops, a3):
    """d/dxi_d of the degree-N flux-point polynomials at the solution points (Eq. 18)."""
    D = ops.D
    return (np.einsum("if,...kjf->...kji", D, a3[0]),
            np.einsum("jf,...kfi->...kji", D, a3[1]),
            np.einsum("kf,...fji->...kji", D, a3[2]))


def _last(a, axis):
    return np.moveaxis(a, axis, -1)


# ---------------------------------------------------------------- residual

def residual(disc: Discretization, ph: Physics, Q: np.ndarray, elems=None) -> np.ndarray:
    """dQ/dt at the solution points of `elems` (all elements if None).

    Q: full state [E, 5, N, N, N].  Returns [len(elems), 5, N, N, N].
    Only the two-face-hop neighbourhood of `elems` is evaluated.
    """
    N, ops, conn = disc.N, disc.ops, disc.conn
    E = disc.n_elem
    if elems is None:
        elems = np.arange(E)
    elems = np.asarray(elems, dtype=np.int64)
    S1 = conn.closure(elems)
    S2 = conn.closure(S1)
    conn.ensure_perm(S2)
    loc = np.full(E, -1, dtype=np.int64)
    loc[S2] = np.arange(S2.size)
    gamma = ph.gamma

    # ---- step 1: traces of Q on every face of the patch S2
    Q2 = Q[S2]
    Qf2 = interp_to_flux(ops, Q2)
    trace = np.stack([face_values(Qf2, F) for F in range(6)], axis=1)  # [S2,6,5,N2]

    # ---- step 2: lifted gradients for S1
    g1 = disc.geometry(S1)
    # a radial radiative-diffusivity profile enters like the solution: its values at the solution
    # points, interpolated to the flux points (Eq. 17); each face side uses its own interpolant
    krf1 = krface = None
    if ph.kappa_r_varies:
        x1 = g1["x"]
        krf1 = interp_to_flux(ops, ph.kappa_r_at(np.sqrt(x1[:, 0] ** 2 + x1[:, 1] ** 2 + x1[:, 2] ** 2)))
        krface = np.stack([face_values(krf1, F) for F in range(6)], axis=1)  # [S1,6,N2]
    i1 = loc[S1]
    Qf1 = tuple(a[i1].copy() for a in Qf2)
    Qc_all = []
    for F in range(6):
        own = trace[i1, F]  # [S1,5,N2]
        Qc = np.empty_like(own)
        nb = conn.nbr[S1, F]
        inner = nb >= 0
        nbl = loc[nb[inner]]
        pidx = conn.perm[S1[inner], F]
        nb_tr = trace[nbl[:, None], conn.nbr_face[S1[inner], F][:, None], :, pidx]  # [S,N2,5]
        Qc[inner] = 0.5 * (own[inner] + np.moveaxis(nb_tr, -1, 1))
        wall = ~inner
        if np.any(wall):
            Sf = face_values(g1["S"], F)[wall]  # [W,3,N2]
            sigma = 1.0 if F % 2 else -1.0
            nhat = _last(sigma * Sf / np.linalg.norm(Sf, axis=1, keepdims=True), 1)  # [W,N2,3]
            qo = _last(own[wall], 1)  # [W,N2,5]
            rho, u, p = primitives(qo, ph)
            u_c = u - np.sum(u * nhat, axis=-1, keepdims=True) * nhat
            top = (conn.wall[S1[wall], F] == 2)[:, None]
            p_c = np.where(top, ph.R_gas * rho * ph.T_wall_top, p)
            qc = np.empty_like(qo)
            qc[..., 0] = rho
            qc[..., 1:4] = rho[..., None] * u_c
            qc[..., 4] = p_c / (gamma - 1.0) + 0.5 * rho * np.sum(u_c * u_c, axis=-1)
            Qc[wall] = np.moveaxis(qc, -1, 1)
        Qc_all.append(Qc)
        set_face_values(Qf1, F, Qc)
    dQ = derivative(ops, Qf1)  # 3 x [S1,5,k,j,i]
    gradQ = sum(dQ[d][:, :, None] * g1["gradxi"][:, d][:, None] for d in range(3))  # [S1,5,3(n),k,j,i]
    Qs1 = Q[S1]
    gradW = grad_primitives(_last(Qs1, 1), np.moveaxis(gradQ, (1, 2), (-2, -1)), ph)  # [S1,k,j,i,5,3]
    gradW = np.moveaxis(gradW, (-2, -1), (1, 2))  # [S1,5,3,k,j,i]
    gWf1 = interp_to_flux(ops, gradW)  # three [S1,5,3,...]
    gface = np.stack([face_values(gWf1, F) for F in range(6)], axis=1)  # [S1,6,5,3,N2]
    loc1 = np.full(E, -1, dtype=np.int64)
    loc1[S1] = np.arange(S1.size)

    # ---- steps 3-7 for the requested elements
    ie = loc1[elems]
    g0 = {"S": tuple(s[ie] for s in g1["S"]), "detJ": g1["detJ"][ie], "x": g1["x"][ie]}
    Qf = tuple(a[loc[elems]] for a in Qf2)  # uncorrected interpolated state
    gWf = tuple(a[ie] for a in gWf1)
    Ftil = []
    for d in range(3):
        Qd = _last(Qf[d], 1)  # [..., 5]
        gd = np.moveaxis(gWf[d], (1, 2), (-2, -1))  # [..., 5, 3]
        krd = None if krf1 is None else krf1[d][ie]
        Ftot = inviscid_flux(Qd, ph) - viscous_flux(Qd, gd, ph, krd)  # [..., 3(n), 5]
        Sd = _last(g0["S"][d], 1)  # [..., 3(n)]
        Ftil.append(np.moveaxis(np.einsum("...n,...nv->...v", Sd, Ftot), -1, 1))  # [e,5,...]

    for F in range(6):
        sigma = 1.0 if F % 2 else -1.0
        Sf = _last(face_values(g0["S"], F), 1)  # [e,N2,3]
        mag = np.linalg.norm(Sf, axis=-1)
        nhat = sigma * Sf / mag[..., None]
        q_own = _last(trace[loc[elems], F], 1)  # [e,N2,5]
        gw_own = np.moveaxis(gface[ie, F], -1, 1)  # [e,N2,5,3]
        kr_own = None if krface is None else krface[ie, F]  # [e,N2]
        Fn = np.zeros_like(q_own)
        nb = conn.nbr[elems, F]
        inner = nb >= 0
        if np.any(inner):
            pidx = conn.perm[elems[inner], F]
            nf = conn.nbr_face[elems[inner], F][:, None]
            q_nb = trace[loc[nb[inner]][:, None], nf, :, pidx]  # [S,N2,5]
            gw_nb = gface[loc1[nb[inner]][:, None], nf, :, :, pidx]  # [S,N2,5,3]
            nh = nhat[inner]
            kr_i = None if kr_own is None else kr_own[inner]
            kr_nb = None if krface is None else krface[loc1[nb[inner]][:, None], nf, pidx]  # [S,N2]
            Fv_own = np.einsum("...n,...nv->...v", nh, viscous_flux(q_own[inner], gw_own[inner], ph, kr_i))
            Fv_nb = np.einsum("...n,...nv->...v", nh, viscous_flux(q_nb, gw_nb, ph, kr_nb))
            Fn[inner] = rusanov(q_own[inner], q_nb, nh, ph) - 0.5 * (Fv_own + Fv_nb)
        wall = ~inner
        if np.any(wall):
            nh = nhat[wall]
            qo = q_own[wall]
            gwo = gw_own[wall]
            rho, u, p = primitives(qo, ph)
            tau = stress(qo, gwo, ph)
            trac = np.einsum("...a,...ab,...b->...", nh, tau, nh)
            top = (conn.wall[elems[wall], F] == 2)[:, None]
            p_top = ph.R_gas * rho * ph.T_wall_top
            f_top = heat_flux(rho, p_top, gwo[..., 0, :], gwo[..., 4, :], ph, None if kr_own is None else kr_own[wall])
            fn = np.where(top, np.sum(f_top * nh, axis=-1), -ph.bottom_flux)
            Fw = np.zeros_like(qo)
            Fw[..., 1:4] = (p - trac)[..., None] * nh
            Fw[..., 4] = fn  # inviscid 0, minus viscous (u.tau.n - f.n) = f.n
            Fn[wall] = Fw
        set_face_values(Ftil, F, np.moveaxis(sigma * mag[..., None] * Fn, -1, 1))

    div = sum(derivative(ops, Ftil))  # [e,5,k,j,i]
    M = source(_last(Q[elems], 1), _last(g0["x"], 1), ph)  # [e,k,j,i,5]
    return -div / g0["detJ"][:, None] - np.moveaxis(M, -1, 1)
