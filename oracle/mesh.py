"""Oracle: element faces, face pairing and face-point correspondence.

Test infrastructure only (see the package docstring).

Local faces of the reference cube: 0: xi=0, 1: xi=1, 2: eta=0, 3: eta=1,
4: zeta=0, 5: zeta=1 (normal direction d = face // 2, side = face % 2).
The N^2 flux points of a face are numbered t = t1 + N*t2, where (t1, t2) are
the solution-point indices along the two tangential directions in increasing
axis order (xi-face: (j, k); eta-face: (i, k); zeta-face: (i, j)).

Two elements share a face when the face has the same four corner nodes.  The
point correspondence across a shared face is found here from physical
coordinates: each face point of one side is matched with the face point of
the other side at the same location (the flux-point sets are symmetric under
the eight square symmetries, so every point has an exact partner).
Unshared faces are walls (Section 5), tagged 1 (inner sphere r = R_i) or 2
(outer sphere r = R_o) from the radius of their corner nodes.
"""
from __future__ import annotations

import numpy as np

from .geometry import map_points
from .sd_points import operators

# corner nodes of each local face (reference-cube corner numbering)
FACE_CORNERS = np.array(
    [
        [0, 3, 4, 7],  # xi = 0
        [1, 2, 5, 6],  # xi = 1
        [0, 1, 4, 5],  # eta = 0
        [3, 2, 7, 6],  # eta = 1
        [0, 1, 2, 3],  # zeta = 0
        [4, 5, 6, 7],  # zeta = 1
    ]
)


def face_point_coords(N: int, face: int):
    """Reference coordinates (xi, eta, zeta) of the N^2 face points, t = t1 + N t2."""
    ops = operators(N)
    X = ops.Xs
    t1 = np.tile(np.arange(N), N)
    t2 = np.repeat(np.arange(N), N)
    d, side = face // 2, face % 2
    fixed = np.full(N * N, float(side))
    if d == 0:
        return fixed, X[t1], X[t2]
    if d == 1:
        return X[t1], fixed, X[t2]
    return X[t1], X[t2], fixed


class Connectivity:
    """nbr[e,f]   neighbour element (-1 for walls)
    nbr_face[e,f] neighbour's local face
    perm[e,f,t]   neighbour face-point index matching own face point t
    wall[e,f]     0 interior, 1 inner wall, 2 outer wall
    """

    def __init__(self, node_xyz: np.ndarray, hex20: np.ndarray, N: int, r_inner: float, r_outer: float):
        E = hex20.shape[0]
        self.N = N
        self.nbr = np.full((E, 6), -1, dtype=np.int64)
        self.nbr_face = np.full((E, 6), -1, dtype=np.int64)
        self.wall = np.zeros((E, 6), dtype=np.int64)
        self.perm = np.full((E, 6, N * N), -1, dtype=np.int64)

        corners = hex20[:, :8]
        keys = np.sort(corners[:, FACE_CORNERS], axis=-1)  # [E,6,4]
        flat = keys.reshape(-1, 4)
        order = np.lexsort(flat.T[::-1])
        sf = flat[order]
        same = np.all(sf[1:] == sf[:-1], axis=1)
        if np.any(same[1:] & same[:-1]):
            raise ValueError("a face is shared by more than two elements")
        first = order[:-1][same]
        second = order[1:][same]
        ea, fa = first // 6, first % 6
        eb, fb = second // 6, second % 6
        self.nbr[ea, fa], self.nbr_face[ea, fa] = eb, fb
        self.nbr[eb, fb], self.nbr_face[eb, fb] = ea, fa

        # walls by radius of the face's corner nodes
        bnd_e, bnd_f = np.nonzero(self.nbr < 0)
        rad = np.linalg.norm(node_xyz[corners[bnd_e][np.arange(len(bnd_e))[:, None], FACE_CORNERS[bnd_f]]], axis=-1)
        tol = 1e-6 * (r_outer - r_inner)
        inner = np.all(np.abs(rad - r_inner) < tol, axis=1)
        outer = np.all(np.abs(rad - r_outer) < tol, axis=1)
        if not np.all(inner | outer):
            raise ValueError("boundary face that lies on neither shell wall")
        self.wall[bnd_e[inner], bnd_f[inner]] = 1
        self.wall[bnd_e[outer], bnd_f[outer]] = 2

        self._node_xyz, self._hex20 = node_xyz, hex20
        self._r_outer = r_outer
        self._have_perm = np.zeros(E, dtype=bool)

    def ensure_perm(self, elems: np.ndarray) -> None:
        """Fill perm[e] for the given elements from physical coordinates (computed on first use)."""
        elems = np.asarray(elems, dtype=np.int64)
        todo = elems[~self._have_perm[elems]]
        if todo.size == 0:
            return
        N = self.N
        xyz, h20 = self._node_xyz, self._hex20
        for fa_ in range(6):
            for fb_ in range(6):
                sel = todo[(self.nbr[todo, fa_] >= 0) & (self.nbr_face[todo, fa_] == fb_)]
                for c0 in range(0, sel.size, 8192):
                    s = sel[c0:c0 + 8192]
                    pa = _face_points(xyz[h20[s]], N, fa_)  # [S,N2,3]
                    pb = _face_points(xyz[h20[self.nbr[s, fa_]]], N, fb_)
                    dist = np.linalg.norm(pa[:, :, None, :] - pb[:, None, :, :], axis=-1)
                    match = np.argmin(dist, axis=2)
                    if np.max(np.min(dist, axis=2)) > 1e-9 * self._r_outer:
                        raise ValueError("face points of paired faces do not coincide")
                    self.perm[s, fa_] = match
        self._have_perm[todo] = True

    def closure(self, elems: np.ndarray) -> np.ndarray:
        """elems plus all their face neighbours (sorted, unique)."""
        nb = self.nbr[elems].reshape(-1)
        return np.unique(np.concatenate([elems, nb[nb >= 0]]))


def _face_points(nodes: np.ndarray, N: int, face: int) -> np.ndarray:
    xi, eta, zeta = face_point_coords(N, face)
    return map_points(nodes, xi, eta, zeta)
