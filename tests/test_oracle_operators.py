"""Pins of the oracle's spatial operators.

Against geometry closed forms (areas, volumes, closed-wall area vectors) and
against a dense brute-force assembly written independently (tests/brute_dense.py)
on 1-4 element meshes: mass matrix, weak Laplacian with the wetting wall term
(Eq. weak), nodal force average, and the force-split streaming right-hand side
with flux bounce-back (Eq. spetrum, Sec. 3.3, Sec. 2.2).
"""
import math

import numpy as np
import pytest
from scipy.integrate import dblquad

from paper_2609_00535_b300 import inputs
from oracle import lattice, method
from tests.brute_dense import Dense
from tests.helpers import oracle_mesh


def tiny_meshes():
    return {
        "box2d": inputs.box((2, 2), (0, 0), (1.0, 0.7), 4, face_tags={2: 0, 3: 1}),
        "box2d_periodic": inputs.box((2, 1), (0, 0), (1.0, 0.5), 3, periodic=(True, False),
                                     face_tags={2: 0}),
        "cyl2d_rot": inputs.rotate_elements(inputs.cylinder_ogrid(5, n_theta=4, n_r=1), 7),
        "box3d_rot": inputs.rotate_elements(
            inputs.box((2, 1, 1), (0, 0, 0), (1.0, 0.5, 0.6), 3, face_tags={4: 0, 1: 1}), 11),
        "sphere3d": inputs.sphere_cap_box(3, ne=(2, 2, 1)),
    }


def smooth_field(xyz, k, periodic_L=None):
    """A smooth, element-continuous test field (function of position only)."""
    x = xyz[..., 0]
    y = xyz[..., 1]
    z = xyz[..., 2] if xyz.shape[-1] == 3 else 0.0 * x
    if periodic_L is not None:
        x = 2 * math.pi * x / periodic_L
        return 0.55 + 0.2 * np.sin(x + 0.3 * k) * np.cos(1.3 * y + k) + 0.05 * np.cos(2 * z + k)
    return 0.55 + 0.2 * np.sin(2.1 * x + 0.3 * k) * np.cos(1.3 * y + k) + 0.05 * np.cos(2 * z + k)


def build(name, mesh, beta=2e-3, delta=0.2, thetas=(math.radians(60), math.radians(125))):
    lat = lattice.d2q9() if mesh.dim == 2 else lattice.d3q13()
    p = method.Params(beta=beta, delta=delta, dt=0.01, tau=0.7, theta_w=thetas[0],
                      theta_tag=thetas[1:],
                      wall_velocity={1: [0.03, -0.02, 0.01][:mesh.dim]})   # tag 1 slides
    om = oracle_mesh(mesh)
    return om, method.SemLbm(om, lat, p), Dense(mesh)


@pytest.mark.parametrize("name", list(tiny_meshes()))
def test_mass_matrix_dense(name):
    mesh = tiny_meshes()[name]
    om, s, dn = build(name, mesh)
    M = dn.mass()
    np.testing.assert_allclose(M - np.diag(np.diag(M)), 0, atol=1e-15)
    np.testing.assert_allclose(dn.to_local(np.diag(M)).reshape(om.Mg.shape), om.Mg, rtol=1e-12)


@pytest.mark.parametrize("name", list(tiny_meshes()))
def test_weak_laplacian_with_wetting_dense(name):
    mesh = tiny_meshes()[name]
    om, s, dn = build(name, mesh)
    per = 1.0 if name == "box2d_periodic" else None
    rho = smooth_field(mesh.node_xyz, 0, per).reshape(om.shape)
    lap = s.laplacian(rho)
    rg = dn.to_global(rho)
    p = s.p

    def wet(e, sel, nrm, tag):
        r = rg[dn.gmap[e][sel]]
        return p.cos_theta(tag) * math.sqrt(2 * p.beta / p.kappa) * (p.rho_l - r) * (r - p.rho_v)

    b = dn.wall_vector(wet)
    K = dn.stiffness()
    M = np.diag(dn.mass())
    ref = (b - K @ rg) / M
    scale = np.abs(ref).max()
    np.testing.assert_allclose(lap.reshape(-1), dn.to_local(ref).reshape(-1), atol=1e-12 * scale)
    # stiffness: symmetric, positive semidefinite, constants in the null space
    np.testing.assert_allclose(K, K.T, atol=1e-12 * np.abs(K).max())
    assert np.linalg.eigvalsh(0.5 * (K + K.T)).min() > -1e-10 * np.abs(K).max()
    np.testing.assert_allclose(K @ np.ones(dn.G), 0, atol=1e-12 * np.abs(K).max())


@pytest.mark.parametrize("name", list(tiny_meshes()))
def test_force_average_dense(name):
    mesh = tiny_meshes()[name]
    om, s, dn = build(name, mesh)
    per = 1.0 if name == "box2d_periodic" else None
    rho = smooth_field(mesh.node_xyz, 0, per).reshape(om.shape)
    mu = (0.01 * smooth_field(mesh.node_xyz, 2, per)).reshape(om.shape)
    F = s.force(rho, mu)
    rg, mg = dn.to_global(rho), dn.to_global(mu)
    M = np.diag(dn.mass())
    for a in range(mesh.dim):
        ea = np.eye(mesh.dim)[a]
        ref = (s.cs2 * dn.convection(ea) @ rg - dn.convection(ea, weight=rg) @ mg) / M
        np.testing.assert_allclose(F[..., a].reshape(-1), dn.to_local(ref).reshape(-1),
                                   atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("name", list(tiny_meshes()))
def test_streaming_rhs_dense(name):
    mesh = tiny_meshes()[name]
    om, s, dn = build(name, mesh)
    lat, cs2 = s.lat, s.cs2
    per = 1.0 if name == "box2d_periodic" else None
    g = np.stack([lat.t[a] * smooth_field(mesh.node_xyz, a + 1, per) for a in range(lat.Q)])
    g = g.reshape((lat.Q,) + om.shape)
    rho = s.density(g)
    mu = s.chemical_potential(rho)
    L = s.streaming_rhs(g, rho, mu)
    rg, mg = dn.to_global(rho), dn.to_global(mu)
    M = np.diag(dn.mass())
    for a in range(lat.Q):
        e, t = lat.e[a], lat.t[a]
        ga = dn.to_global(g[a])
        gb = dn.to_global(g[lat.opp[a]])

        def bb(el, sel, nrm, tag):
            ne = nrm @ e
            idx = dn.gmap[el][sel]
            ub = s.p.u_b(tag, mesh.dim)
            jump = ga[idx] - gb[idx] - 2 * t / cs2 * rg[idx] * (e @ ub)
            return np.where(ne < -1e-12, ne * jump, 0.0)

        rhs = -dn.convection(e) @ (ga - t * rg) - (t / cs2) * dn.convection(e, weight=rg) @ mg
        rhs = rhs + dn.wall_vector(bb)
        ref = rhs / M
        scale = max(np.abs(ref).max(), 1e-30)
        np.testing.assert_allclose(L[a].reshape(-1), dn.to_local(ref).reshape(-1),
                                   atol=2e-12 * scale)


def test_area_vector_is_cofactor_row():
    mesh = tiny_meshes()["sphere3d"]
    om = oracle_mesh(mesh)
    cof = om.detJ[..., None, None] * om.Jinv        # row b: detJ d xi_b / dx
    flat = cof.reshape(om.E, -1, 3, 3)
    n = om.n
    for k in np.nonzero(om.wall_tag == 0)[0]:
        e, node = om.wall_elem[k], om.wall_node[k]
        # tag 0 is the sphere, face 4 (xi_3 = -1): outward area = -(cofactor row 3)
        i, j = node % n, (node // n) % n
        ref = -flat[e, node, 2] * om.w[i] * om.w[j]
        np.testing.assert_allclose(om.wall_area[k], ref, atol=1e-15)


def test_areas_and_volumes():
    m = inputs.box((3, 2), (0, 0), (1.5, 0.7), 4)
    assert abs(oracle_mesh(m).Me.sum() - 1.5 * 0.7) < 1e-14
    m = inputs.box((2, 2, 1), (0, 0, 0), (1.0, 0.5, 0.3), 3)
    assert abs(oracle_mesh(m).Me.sum() - 0.15) < 1e-15
    # curved O-grid: area of the square minus the disc, converging spectrally
    errs = []
    for N in (2, 4, 8):
        A = oracle_mesh(inputs.cylinder_ogrid(N, n_theta=16, n_r=2)).Me.sum()
        errs.append(abs(A - (1 - math.pi * 0.01)))
    assert errs[2] < 1e-9 and errs[2] < 1e-3 * errs[0]
    # sphere-cap box: volume against a 2D quadrature of the lid height
    vol, _ = dblquad(lambda y, x: 0.25 - (-0.7 + math.sqrt(0.49 - (x - .25) ** 2 - (y - .25) ** 2)),
                     0, 0.5, 0, 0.5, epsabs=1e-13)
    V = oracle_mesh(inputs.sphere_cap_box(6, ne=(4, 4, 2))).Me.sum()
    assert abs(V - vol) < 1e-9


def test_closed_wall_area_vectors_sum_to_zero():
    om = oracle_mesh(inputs.rotate_elements(inputs.cylinder_ogrid(5, n_theta=8, n_r=2), 3))
    inner = om.wall_tag == 0
    np.testing.assert_allclose(om.wall_area[inner].sum(0), 0, atol=1e-15)
    np.testing.assert_allclose(om.wall_area[~inner].sum(0), 0, atol=1e-15)
    # circle perimeter from the surface weights (spectral convergence)
    assert abs(np.linalg.norm(om.wall_area[inner], axis=1).sum() - 2 * math.pi * 0.1) < 1e-6
    om3 = oracle_mesh(inputs.rotate_elements(inputs.box((2, 2, 1), (0, 0, 0), (1, 1, 1), 3), 5))
    np.testing.assert_allclose(om3.wall_area.sum(0), 0, atol=1e-15)


def test_wall_nodes_on_curved_walls():
    m = inputs.cylinder_ogrid(6, n_theta=16, n_r=2)
    om = oracle_mesh(m)
    x = m.node_xyz.reshape(om.E, -1, 2)[om.wall_elem, om.wall_node]
    r = np.linalg.norm(x - 0.5, axis=1)
    inner = om.wall_tag == 0
    np.testing.assert_allclose(r[inner], 0.1, atol=1e-15)
    m3 = inputs.sphere_cap_box(4, ne=(3, 3, 2))
    om3 = oracle_mesh(m3)
    x = m3.node_xyz.reshape(om3.E, -1, 3)[om3.wall_elem, om3.wall_node]
    sph = om3.wall_tag == 0
    np.testing.assert_allclose(np.linalg.norm(x[sph] - [0.25, 0.25, -0.7], axis=1), 0.7, atol=1e-15)


def test_dss_counts_shared_copies():
    m = inputs.box((3, 3), (0, 0), (1, 1), 4, periodic=(True, True))
    om = oracle_mesh(m)
    assert om.G == (3 * 4) ** 2
    ones = np.ones(om.shape)
    copies = om.gather(om.assemble(ones))
    n = om.n
    c = copies[0]
    assert c[0, 0] == 4 and c[0, 2] == 2 and c[2, 2] == 1 and c[n - 1, n - 1] == 4
