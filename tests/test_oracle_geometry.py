"""Pins of the oracle's geometry: 20-node map, Jacobian, curl-form metrics, mesh.

(Section 3 Eqs. 10-12, Section 5 20-node elements.)
"""
import math

import numpy as np
import pytest

from chorus_inputs import HEX20_REF2, cubed_sphere_hex20
from oracle.geometry import analytic_cofactors, curl_metrics, jacobian_matrix, map_points, shape_functions, \
    solution_geometry
from oracle.mesh import Connectivity
from oracle.sd_points import operators


def test_shape_functions_partition_and_nodal():
    ref = HEX20_REF2 / 2.0
    Nv, dN = shape_functions(ref[:, 0], ref[:, 1], ref[:, 2])
    assert np.allclose(Nv, np.eye(20), atol=1e-15)
    rng = np.random.default_rng(0)
    p = rng.random((50, 3))
    Nv, dN = shape_functions(p[:, 0], p[:, 1], p[:, 2])
    assert np.allclose(Nv.sum(-1), 1.0, atol=1e-14)
    assert np.allclose(dN.sum(-2), 0.0, atol=1e-13)
    # derivatives against central differences
    h = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        Np, _ = shape_functions(*(p + e).T)
        Nm, _ = shape_functions(*(p - e).T)
        assert np.allclose((Np - Nm) / (2 * h), dN[..., d], atol=1e-8)


def test_serendipity_reproduces_quadratics():
    # complete quadratic fields are interpolated exactly by the 20-node element
    rng = np.random.default_rng(1)
    ref = HEX20_REF2 / 2.0
    c = rng.standard_normal(10)

    def f(x, y, z):
        return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * x + c[5] * y * y + c[6] * z * z
                + c[7] * x * y + c[8] * y * z + c[9] * x * z)

    nodal = f(ref[:, 0], ref[:, 1], ref[:, 2])
    p = rng.random((40, 3))
    Nv, _ = shape_functions(*p.T)
    assert np.allclose(Nv @ nodal, f(*p.T), atol=1e-13)


def _affine_element(rng):
    A = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
    b = rng.standard_normal(3)
    ref = HEX20_REF2 / 2.0
    return (ref @ A.T + b)[None], A


@pytest.mark.parametrize("N", [3, 4])
def test_metrics_affine_element(N):
    rng = np.random.default_rng(2)
    nodes, A = _affine_element(rng)
    cof = np.linalg.det(A) * np.linalg.inv(A)  # |J| J^{-1}: row d is S^d
    S_xi, S_eta, S_zeta, S_sol = curl_metrics(nodes, N)
    for d, S in enumerate((S_xi, S_eta, S_zeta)):
        assert np.allclose(np.moveaxis(S[0], 0, -1), cof[d], atol=1e-12)
    assert np.allclose(np.moveaxis(S_sol[0], (0, 1), (-2, -1)), cof, atol=1e-12)
    _, detJ = solution_geometry(nodes, N)
    assert np.allclose(detJ, np.linalg.det(A), atol=1e-13)


def _shell(n=2, n_r=2, ri=0.75, ro=1.0):
    xyz, h20 = cubed_sphere_hex20(n, n_r, ri, ro)
    return xyz, h20, xyz[h20]


@pytest.mark.parametrize("N", [4, 5])
def test_curl_metrics_equal_analytic_cofactors_for_N_ge_4(N):
    # the 20-node map has cofactors of degree <= 4 per direction: the curl form is exact for N >= 4
    _, _, nodes = _shell()
    nodes = nodes[:12]
    ops = operators(N)
    Xs, Xf = ops.Xs, ops.Xf
    S_xi, S_eta, S_zeta, S_sol = curl_metrics(nodes, N)
    ref = analytic_cofactors(nodes, Xf[None, None, :], Xs[None, :, None], Xs[:, None, None])  # xi-flux points
    assert np.allclose(np.moveaxis(S_xi, 1, -1), ref[..., 0, :], atol=1e-13)
    ref = analytic_cofactors(nodes, Xs[None, None, :], Xf[None, :, None], Xs[:, None, None])
    assert np.allclose(np.moveaxis(S_eta, 1, -1), ref[..., 1, :], atol=1e-13)
    ref = analytic_cofactors(nodes, Xs[None, None, :], Xs[None, :, None], Xf[:, None, None])
    assert np.allclose(np.moveaxis(S_zeta, 1, -1), ref[..., 2, :], atol=1e-13)
    ref = analytic_cofactors(nodes, Xs[None, None, :], Xs[None, :, None], Xs[:, None, None])
    assert np.allclose(np.moveaxis(S_sol, (1, 2), (-2, -1)), ref, atol=1e-13)


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_discrete_metric_identity(N):
    # sum_d d/dxi_d S^d = 0 discretely (what makes a uniform flow a steady solution)
    from oracle.residual import derivative

    _, _, nodes = _shell()
    ops = operators(N)
    S = curl_metrics(nodes[:24], N)[:3]
    div = sum(derivative(ops, S))
    scale = max(np.abs(s).max() for s in S)
    assert np.abs(div).max() < 1e-13 * scale * N * N


def test_shell_volume_converges():
    exact = 4.0 * math.pi / 3.0 * (1.0 - 0.75 ** 3)
    errs = []
    for n in (2, 4, 8):
        _, _, nodes = _shell(n, 1)
        ops = operators(4)
        _, detJ = solution_geometry(nodes, 4)
        w = ops.w
        vol = np.sum(w[None, :, None, None] * w[None, None, :, None] * w[None, None, None, :] * detJ)
        errs.append(abs(vol - exact))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 1e-4 * exact
    assert min(rates) > 2.8  # quadratic geometry: O(h^3) or better


@pytest.mark.parametrize("n,n_r", [(2, 1), (4, 3)])
def test_cubed_sphere_connectivity(n, n_r):
    xyz, h20, nodes = _shell(n, n_r)
    E = 6 * n * n * n_r
    conn = Connectivity(xyz, h20, 4, 0.75, 1.0)
    conn.ensure_perm(np.arange(E))
    assert np.sum(conn.wall == 1) == 6 * n * n and np.sum(conn.wall == 2) == 6 * n * n
    assert np.sum(conn.nbr >= 0) == 6 * E - 12 * n * n
    # pairing is symmetric and the point map is a bijection
    e, f = np.nonzero(conn.nbr >= 0)
    nb, nf = conn.nbr[e, f], conn.nbr_face[e, f]
    assert np.all(conn.nbr[nb, nf] == e) and np.all(conn.nbr_face[nb, nf] == f)
    back = np.take_along_axis(conn.perm[nb, nf], conn.perm[e, f], axis=1)
    assert np.all(back == np.arange(16)[None])
    # every element is right-handed
    _, detJ = solution_geometry(nodes, 4)
    assert detJ.min() > 0
    # corners sit on spheres: radius of node positions
    r = np.linalg.norm(xyz, axis=1)
    assert r.min() > 0.75 - 1e-14 and r.max() < 1.0 + 1e-14


def test_config_sizes_and_dof_formula():
    # Eq. 19 DOF count (N = p + 1) and the paper's performance-table element counts
    from chorus_inputs import CONFIGS

    assert CONFIGS["shell_288_p3"].n_dof == 18432
    assert CONFIGS["shell_331776_p3"].n_dof == 21233664
    assert CONFIGS["shell_786432_p4"].n_dof == 98304000
    assert 294912 * 4 ** 3 == 18874368 and 307200 * 4 ** 3 == 19660800 and 1105920 * 4 ** 3 == 70778880
