"""Shared test helpers: build the oracle for a Case (test-only)."""
import numpy as np

from oracle import geometry, lattice, method


def oracle_mesh(mesh):
    return geometry.Mesh(mesh.dim, mesh.N, mesh.node_xyz, mesh.global_id, mesh.face_kind,
                         mesh.face_tag)


def oracle_of(case, **over):
    om = oracle_mesh(case.mesh)
    lat = lattice.by_name(case.lattice)
    kw = dict(rho_l=case.rho_l, rho_v=case.rho_v, beta=case.beta, kappa=case.kappa,
              tau=case.tau, dt=case.dt, theta_w=case.theta_w, theta_tag=case.theta_tag,
              wall_velocity=case.wall_velocity, force_split=case.force_split)
    kw.update(over)
    return om, method.SemLbm(om, lat, method.Params(**kw))


def local_shape(case):
    return (case.mesh.n_elem,) + (case.mesh.N + 1,) * case.mesh.dim


def make_case(name, mesh, lattice, beta, delta, tau, theta_w, theta_tag=(), rho0=None,
              rho_l=1.0, rho_v=0.1, cfl=0.4, wall_velocity=None):
    """A Case with kappa from the interface width and the stable default dt."""
    from paper_2609_00535_b300 import inputs
    kappa = inputs.kappa_from_width(beta, delta, rho_l, rho_v)
    dt = inputs.cfl_dt(mesh, lattice, cfl, kappa, rho_l)
    return inputs.Case(name, mesh, lattice, rho_l, rho_v, beta, kappa, tau, dt, theta_w,
                       tuple(theta_tag), rho0, wall_velocity=dict(wall_velocity or {}))
