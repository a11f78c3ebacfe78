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


def oracle_state(case, steps):
    """fbar [Q, V] after `steps` oracle steps from the case's initial density."""
    om, orc = oracle_of(case)
    f = orc.initial_state(case.rho0.reshape(om.shape))
    f = orc.run(f, steps)
    return f.reshape(f.shape[0], -1)


def assert_matches_oracle(case, f_gpu, steps, tol=1e-12):
    """max |f_gpu - f_oracle| / max |f_oracle| <= tol, for fbar and rho."""
    f_ref = oracle_state(case, steps)
    f_gpu = np.asarray(f_gpu).reshape(f_ref.shape)
    err = np.abs(f_gpu - f_ref).max() / np.abs(f_ref).max()
    rho_ref = f_ref.sum(0)
    err_rho = np.abs(f_gpu.sum(0) - rho_ref).max() / np.abs(rho_ref).max()
    assert err <= tol and err_rho <= tol, (case.name, err, err_rho)
    return err
