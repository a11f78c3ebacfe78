"""Linear stability of the oracle's time step about a drop at rest (test and
analysis infrastructure only; nothing in the library uses it).

A drop at rest, fbar = t_a rho_eq with a discrete equilibrium density rho_eq
(the chemical potential of Eq. chemi constant at every node), is a fixed point
of the step of Sec. 2.1 / Sec. 3.3 under either force reading: the collision's
F** is proportional to u, and the force-split streaming term rho e.grad(mu)
vanishes with grad(mu).  Whether small disturbances of that state die out or
grow is decided by the spectrum of the Jacobian of one step there.

Linearising F** = (t_a / c_s^2) [ (e_a.u)(e_a.F) / c_s^2 - u.F ] about u = 0
gives (t_a / c_s^2) [ (e_a.du)(e_a.F_eq) / c_s^2 - du.F_eq ]: the disturbance
of the force drops out (it multiplies u = 0), and what remains is the velocity
disturbance du coupled to the force of the equilibrium, F_eq.  Under the
printed reading F = c_s^2 grad(rho) - rho grad(mu), F_eq = c_s^2 grad(rho_eq),
which is large across the interface; under the potential-part reading
(force_split = 1) F_eq = -rho grad(mu_eq) = 0 and the linearised collision is
plain BGK relaxation.  This module measures what that coupling does to the
spectrum.

The Jacobian acts on continuous states (one value per global node and
velocity; the copies of a shared node are equal before and after a step), so
its columns are built from perturbations of whole global nodes, by central
differences of the oracle's own step.
"""
import numpy as np


def global_index(mesh):
    """For every global node, the element-local flat index of one of its copies."""
    _, first = np.unique(mesh.inv.ravel(), return_index=True)
    return first


def to_global(mesh, f):
    """[Q, E, n..] state with equal copies -> [Q, G] values."""
    Q = f.shape[0]
    return f.reshape(Q, -1)[:, global_index(mesh)]


def to_local(mesh, fg):
    """[Q, G] -> [Q, E, n..] with every copy of a node set to its value."""
    return fg[:, mesh.inv]


def equilibrate(orc, f, steps, every=1000):
    """Advance f by `steps` oracle steps; returns f and the KE_max history."""
    hist = []
    done = 0
    while done < steps:
        k = min(every, steps - done)
        f = orc.run(f, k)
        done += k
        hist.append((done, orc.diagnostics(f)["ke_max"]))
    return f, hist


def jacobian(orc, f_eq, eps=1e-7):
    """Dense Jacobian of one step at f_eq, on the continuous state space [Q * G]."""
    mesh = orc.mesh
    base = to_global(mesh, f_eq)
    Q, G = base.shape
    n = Q * G
    J = np.empty((n, n))
    scale = np.abs(base).max()
    h = eps * scale
    for col in range(n):
        q, g = divmod(col, G)
        plus = base.copy()
        plus[q, g] += h
        minus = base.copy()
        minus[q, g] -= h
        fp = to_global(mesh, orc.step(to_local(mesh, plus)))
        fm = to_global(mesh, orc.step(to_local(mesh, minus)))
        J[:, col] = ((fp - fm) / (2 * h)).reshape(-1)
    return J


def mode_summary(orc, vec):
    """Where an eigenvector lives: its density and momentum parts per node, and
    how much of it alternates in sign from node to node (odd-even content)."""
    mesh, lat = orc.mesh, orc.lat
    Q = lat.Q
    v = np.real_if_close(vec).reshape(Q, -1)
    v = np.real(v) if np.iscomplexobj(v) else v
    drho = v.sum(0)
    dm = v.T @ lat.e                     # [G, d] momentum disturbance
    return {"rho_part": float(np.linalg.norm(drho)), "mom_part": float(np.linalg.norm(dm)),
            "nonhydro_part": float(np.linalg.norm(v)), "drho": drho, "dm": dm}


def _build(ne, N, D, Cn, beta, tau, cfl, force_split):
    """Oracle of the periodic drop of Sec. 3.3 (2D, ne x ne elements of order N)."""
    from paper_2609_00535_b300 import inputs
    from . import geometry, lattice, method
    case = inputs.periodic_droplet(dim=2, ne=ne, N=N, D=D, Cn=Cn, beta=beta, tau=tau, cfl=cfl)
    m = case.mesh
    mesh = geometry.Mesh(m.dim, m.N, m.node_xyz, m.global_id, m.face_kind, m.face_tag)
    p = method.Params(rho_l=case.rho_l, rho_v=case.rho_v, beta=case.beta, kappa=case.kappa,
                      tau=case.tau, dt=case.dt, theta_w=case.theta_w, force_split=force_split)
    return case, method.SemLbm(mesh, lattice.by_name(case.lattice), p)


def main(argv=None):
    """Relax a periodic drop under force_split = 1, then print, for each force
    reading, the spectral radius of one step about the state reached."""
    import argparse
    import json
    import math
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--ne", type=int, default=3)
    ap.add_argument("--N", type=int, default=4)
    ap.add_argument("--D", type=float, default=0.6)
    ap.add_argument("--Cn", type=float, default=0.15)
    ap.add_argument("--beta", type=float, default=0.1)
    ap.add_argument("--tau", type=float, default=1.0)
    ap.add_argument("--cfl", type=float, default=0.4)
    ap.add_argument("--relax-steps", type=int, default=4000)
    ap.add_argument("--relax-cfl", type=float, default=None,
                    help="CFL number of the relaxation (default --cfl); the state at rest "
                         "does not depend on the time step, so one relaxation serves every dt")
    a = ap.parse_args(argv)
    rcfl = a.relax_cfl if a.relax_cfl is not None else a.cfl
    rcase, rorc = _build(a.ne, a.N, a.D, a.Cn, a.beta, a.tau, rcfl, 1)
    f = rorc.initial_state(rcase.rho0.reshape(rorc.mesh.shape))
    f, hist = equilibrate(rorc, f, a.relax_steps, every=max(1, a.relax_steps // 5))
    case, _ = _build(a.ne, a.N, a.D, a.Cn, a.beta, a.tau, a.cfl, 1)
    out = {"case": vars(a), "dt": case.dt, "relax_ke_max": ["%d:%.1e" % h for h in hist]}
    for fs in (0, 1):
        _, o = _build(a.ne, a.N, a.D, a.Cn, a.beta, a.tau, a.cfl, fs)
        w = np.linalg.eigvals(jacobian(o, f))
        r = float(np.abs(w).max())
        out["force_split_%d" % fs] = {"spectral_radius": r, "n_above_1": int(np.sum(np.abs(w) > 1 + 1e-8)),
                                      "ln_radius_over_dt2": math.log(r) / case.dt ** 2}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
