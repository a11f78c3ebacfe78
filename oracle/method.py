"""The SEM-LBM time step, written out in the paper's order (test infrastructure only).

State: the modified distributions fbar[alpha, e, nodes] on element-local GLL
nodes (shared nodes duplicated and kept equal by the gather-scatter).

One step from fbar^n (Sec. 2.1-2.2, Sec. 3.3, Sec. 4):
 1. macros: rho = sum_a fbar_a (Eq. density), rho u = sum_a fbar_a e_a (Eq. momentum);
 2. chemical potential mu = mu0(rho) - kappa lap(rho) (Eq. chemi), with lap from
    the weak form Eq. (weak) whose wall integral carries the wetting gradient
    n.grad(rho) = cos(theta) sqrt(2 e0 / kappa) (Sec. 2.2, mechanism 1);
 3. collision with the higher-order force F** (collision equation of Sec. 2.1,
    modified distributions of Appendix A);
 4. streaming of the post-collision state by SSP-RK3 (Sec. 2.1) using the
    force-split form of Sec. 3.3 and the flux bounce-back wall flux J (Sec. 2.2);
    rho, mu and grad(mu) are recomputed from every Runge-Kutta stage state
    (Sec. 4: the force is added consistently at each stage).

Readings where the paper is silent or inconsistent (each is configurable or
stated; they are the same readings the CUDA library implements):
 * mu0 = 2 beta (rho-rho_l)(rho-rho_v)(2rho-rho_l-rho_v) = d e0/d rho; Eq. chemi
   prints the factor without the 2, but kappa and gamma of Appendix A follow only
   with it (``mu0_factor``, default 2).
 * The force-split streaming equation is used with +(t/c_s^2) rho e.grad(mu) on
   its left side, the sign that follows from F* = t/c_s^2 e.F with
   F = c_s^2 grad(rho) - rho grad(mu); Sec. 3.3 prints a minus.
 * Outward wall normal; theta measured through the liquid (theta < 90 deg wets).
 * sqrt(2 e0/kappa) is evaluated as the signed polynomial
   sqrt(2 beta/kappa)(rho_l - rho)(rho - rho_v) (equal inside [rho_v, rho_l]).
 * The nodal force used in collision is the mass-weighted gather-scatter average
   of the element-local collocated F (collocated gradients jump across faces).
 * Stage 1 uses rho and mu of fbar^n: collision conserves mass exactly, so they
   equal those of the post-collision state.
 * SSP-RK3 is the three-stage Shu-Osher form.
 * Wall velocity u_b per wall tag (static, u_b = 0, unless given); tags < 0
   are static neutral walls.

Pinned by tests/test_oracle_operators.py (dense brute-force assembly of
tests/brute_dense.py on 1-4 element meshes: weak Laplacian with the wetting
term, force average, streaming right-hand side with bounce-back),
tests/test_oracle_physics.py (stationarity, mass conservation, the tanh
interface, tilted-interface wetting residual, collision moments, Couette flow),
tests/test_oracle_tables.py (equilibrium and force moments, mu0 = de0/drho,
RK3 on a linear ODE), tests/test_oracle_equilibria.py (Laplace law, static
angle) and tests/test_oracle_wetting.py (wetting moments).
"""
import numpy as np

from .geometry import Mesh, deriv


class Params:
    def __init__(self, rho_l=1.0, rho_v=0.1, beta=1e-3, kappa=None, delta=None, tau=0.5,
                 dt=None, theta_w=np.pi / 2, theta_tag=(), mu0_factor=2.0, wall_velocity=None,
                 force_split=0):
        self.rho_l, self.rho_v, self.beta, self.tau = rho_l, rho_v, beta, tau
        if kappa is None:
            # Appendix A: kappa = beta delta^2 (rho_l - rho_v)^2 / 8
            kappa = beta * delta ** 2 * (rho_l - rho_v) ** 2 / 8
        self.kappa = kappa
        if dt is None:
            raise ValueError("the oracle takes an explicit time step")
        self.dt = dt
        self.theta_w = theta_w
        self.theta_tag = tuple(theta_tag)
        self.mu0_factor = mu0_factor
        self.wall_velocity = dict(wall_velocity or {})   # tag -> u_b
        # force entering F** of the collision: 0 = F = c_s^2 grad rho - rho grad mu
        # as printed (Sec. 2.1); 1 = its potential part -rho grad mu alone
        if force_split not in (0, 1):
            raise ValueError("force_split must be 0 or 1")
        self.force_split = force_split

    def u_b(self, tag, dim):
        """Velocity of the walls with this tag (zero unless given; tags < 0 are static)."""
        if tag < 0 or tag not in self.wall_velocity:
            return np.zeros(dim)
        return np.asarray(self.wall_velocity[tag], dtype=np.float64)

    def cos_theta(self, tag):
        """tag < 0: neutral wall (90 deg); 0: theta_w; k >= 1: theta_tag[k-1]."""
        if tag < 0:
            return 0.0
        if tag == 0:
            return np.cos(self.theta_w)
        return np.cos(self.theta_tag[tag - 1])

    def surface_tension(self):
        """gamma = (rho_l - rho_v)^3 sqrt(2 kappa beta) / 6 (Appendix A)."""
        return (self.rho_l - self.rho_v) ** 3 * np.sqrt(2 * self.kappa * self.beta) / 6


class SemLbm:
    def __init__(self, mesh: Mesh, lattice, params: Params):
        if mesh.dim != lattice.dim:
            raise ValueError("lattice dimension does not match the mesh")
        self.mesh, self.lat, self.p = mesh, lattice, params
        self.cs2 = lattice.cs2
        self.wall_cos = np.array([params.cos_theta(int(t)) for t in mesh.wall_tag])
        self.wall_ub = np.array([params.u_b(int(t), mesh.dim) for t in mesh.wall_tag]).reshape(-1, mesh.dim)
        # G_bc = M_e sum_a Jinv[b,a] Jinv[c,a]: metric of the stiffness integral
        self.Gstiff = mesh.Me[..., None, None] * np.einsum("...ba,...ca->...bc", mesh.Jinv, mesh.Jinv)

    # --- Eq. density / Eq. momentum -----------------------------------------
    def density(self, f):
        return f.sum(axis=0)

    def velocity(self, f, rho):
        m = np.einsum("q...,qa->...a", f, self.lat.e)
        return m / rho[..., None]

    # --- Appendix A / Eq. chemi -------------------------------------------------
    def bulk_energy(self, rho):
        p = self.p
        return p.beta * (rho - p.rho_l) ** 2 * (rho - p.rho_v) ** 2

    def mu0(self, rho):
        p = self.p
        return p.mu0_factor * p.beta * (rho - p.rho_l) * (rho - p.rho_v) * (2 * rho - p.rho_l - p.rho_v)

    def wetting_gradient(self, rho_wall):
        """n.grad(rho) = cos(theta) sqrt(2 e0/kappa), signed-polynomial form (Sec. 2.2)."""
        p = self.p
        return self.wall_cos * np.sqrt(2 * p.beta / p.kappa) * (p.rho_l - rho_wall) * (rho_wall - p.rho_v)

    def laplacian(self, rho, wall_gradient=None):
        """Eq. (weak): M^-1 ( wall integral of phi n.grad(rho) - int grad(rho).grad(phi) )."""
        m = self.mesh
        gxi = [deriv(rho, m.D, b, m.dim) for b in range(m.dim)]
        r = np.zeros_like(rho)
        for b in range(m.dim):
            tb = sum(self.Gstiff[..., b, c] * gxi[c] for c in range(m.dim))
            r -= deriv(tb, m.D, b, m.dim, transpose=True)
        if wall_gradient is None:
            wall_gradient = self.wetting_gradient(m.at_wall(rho))
        ws = np.linalg.norm(m.wall_area, axis=-1)    # surface quadrature weight
        r = m.add_wall_nodes(r, ws * wall_gradient)
        return m.dss_average(r)

    def chemical_potential(self, rho):
        return self.mu0(rho) - self.p.kappa * self.laplacian(rho)

    # --- forcing (Sec. 2.1) --------------------------------------------------
    def force(self, rho, mu):
        """Nodal F = c_s^2 grad(rho) - rho grad(mu) (or -rho grad(mu) alone when
        force_split = 1), gather-scatter averaged; it enters only F**."""
        m = self.mesh
        Fe = -rho[..., None] * m.grad(mu)
        if self.p.force_split == 0:
            Fe = self.cs2 * m.grad(rho) + Fe
        return np.stack([m.dss_average(m.Me * Fe[..., a]) for a in range(m.dim)], axis=-1)

    def equilibrium(self, rho, u):
        """Eq. (geq_s)."""
        cs2 = self.cs2
        eu = np.einsum("qa,...a->q...", self.lat.e, u)
        uu = np.einsum("...a,...a->...", u, u)
        t = self.lat.t.reshape((-1,) + (1,) * rho.ndim)
        return rho[None] * t * (1 + eu / cs2 + eu ** 2 / (2 * cs2 ** 2) - uu[None] / (2 * cs2))

    def force_terms(self, u, F):
        """Leading-order F*_a = t/c_s^2 e.F and higher-order F**_a (Sec. 2.1)."""
        cs2 = self.cs2
        t = self.lat.t.reshape((-1,) + (1,) * (u.ndim - 1))
        eF = np.einsum("qa,...a->q...", self.lat.e, F)
        eu = np.einsum("qa,...a->q...", self.lat.e, u)
        uF = np.einsum("...a,...a->...", u, F)
        Fstar = t / cs2 * eF
        Fss = t / cs2 * (eu * eF / cs2 - uF[None])
        return Fstar, Fss

    def collide(self, f, rho, mu):
        """f* = fbar - (fbar - fbar_eq)/(tau + 1/2) + dt F** (Sec. 2.1, Appendix A)."""
        p = self.p
        u = self.velocity(f, rho)
        F = self.force(rho, mu)
        feq = self.equilibrium(rho, u)
        _, Fss = self.force_terms(u, F)
        fbar_eq = feq - 0.5 * p.dt * Fss
        return f - (f - fbar_eq) / (p.tau + 0.5) + p.dt * Fss

    # --- streaming (Eq. advection / spetrum, Sec. 3.3, Sec. 2.2) -------------
    def streaming_rhs(self, g, rho, mu):
        """L_a(g) = M^-1 DSS[ M_e s_a + wall flux ], the force-split weak form."""
        m, lat, cs2 = self.mesh, self.lat, self.cs2
        grad_rho = m.grad(rho)
        grad_mu = m.grad(mu)
        r = np.empty_like(g)
        for a in range(lat.Q):
            e, t = lat.e[a], lat.t[a]
            grad_g = m.grad(g[a])
            s = -np.einsum("...c,c->...", grad_g - t * grad_rho, e) \
                - (t / cs2) * rho * np.einsum("...c,c->...", grad_mu, e)
            r[a] = m.Me * s
        # flux bounce-back: J_a = n.e_a [fbar_a]_bc on incoming directions (n.e_a < 0)
        if len(m.wall_elem):
            gw = m.at_wall(g)                    # [Q, W]
            rw = m.at_wall(rho)
            flux = np.zeros_like(gw)
            for a in range(lat.Q):
                ae = m.wall_area @ lat.e[a]       # w_face * |a| * n.e_a
                inc = ae < 0
                bc = gw[a] - gw[lat.opp[a]] - 2 * lat.t[a] / cs2 * rw * (self.wall_ub @ lat.e[a])
                flux[a] = np.where(inc, ae * bc, 0.0)
            r = m.add_wall_nodes(r, flux)
        return np.stack([m.dss_average(r[a]) for a in range(lat.Q)])

    @staticmethod
    def ssp_rk3(U0, L, dt):
        """Three-stage SSP Runge-Kutta (Shu-Osher form); L(g, stage)."""
        U1 = U0 + dt * L(U0, 0)
        U2 = 0.75 * U0 + 0.25 * (U1 + dt * L(U1, 1))
        return U0 / 3 + 2.0 / 3.0 * (U2 + dt * L(U2, 2))

    # --- one full time step ---------------------------------------------------
    def step(self, f):
        rho = self.density(f)
        mu = self.chemical_potential(rho)
        fs = self.collide(f, rho, mu)

        def L(g, stage):
            if stage == 0:
                return self.streaming_rhs(g, rho, mu)
            r = self.density(g)
            return self.streaming_rhs(g, r, self.chemical_potential(r))

        return self.ssp_rk3(fs, L, self.p.dt)

    def run(self, f, n_steps):
        for _ in range(n_steps):
            f = self.step(f)
        return f

    # --- initial state and diagnostics (Appendix A, Sec. 3.3) ----------------
    def initial_state(self, rho):
        """fbar = f^eq(rho, u = 0) (u = 0 makes F** vanish)."""
        return self.equilibrium(rho, np.zeros(rho.shape + (self.mesh.dim,)))

    def wetting_moments(self, f, tag=0, rho_v=None, rho_l=None):
        """Integrals for measuring the static contact angle of Sec. 3.1 / 3.2 from
        the state: with the liquid fraction phi = (rho - rho_v)/(rho_l - rho_v)
        (reference densities given, or else measured: phi on the state's density
        range [min, max], then the mass-weighted mean density of the nodes with
        phi < 0.02 for rho_v and phi > 0.98 for rho_l),
        volume = int phi dV, centroid = int phi x dV / volume, and over the wall
        faces of the given tag (all walls for tag < 0), wall = int dS,
        wetted = int phi dS, wet_centroid = int phi x dS / wetted.  The volume
        integral uses the GLL quadrature of the mass matrix, the wall integrals
        the face quadrature of the wetting term (weight w |a| per face-node)."""
        m = self.mesh
        rho = self.density(f)
        if rho_v is None or rho_l is None:
            lo, hi = float(rho.min()), float(rho.max())
            phi0 = (rho - lo) / (hi - lo)
            vap, liq = phi0 < 0.02, phi0 > 0.98
            rho_v = float(np.sum(m.Me[vap] * rho[vap]) / np.sum(m.Me[vap]))
            rho_l = float(np.sum(m.Me[liq] * rho[liq]) / np.sum(m.Me[liq]))
        phi = (rho - rho_v) / (rho_l - rho_v)
        X = m.X
        vol = float(np.sum(m.Me * phi))
        cen = [float(np.sum(m.Me * phi * X[..., a])) / vol for a in range(m.dim)]
        sel = (m.wall_tag == tag) if tag >= 0 else np.ones(len(m.wall_tag), dtype=bool)
        ws = np.linalg.norm(m.wall_area, axis=-1)[sel]
        phw = m.at_wall(phi)[sel]
        wall = float(np.sum(ws))
        wet = float(np.sum(ws * phw))
        wcen = [float(np.sum(ws * phw * m.at_wall(X[..., a])[sel])) / wet if wet else 0.0
                for a in range(m.dim)]
        return {"volume": vol, "centroid": cen, "wall": wall, "wetted": wet,
                "wet_centroid": wcen, "rho_v_ref": rho_v, "rho_l_ref": rho_l}

    def diagnostics(self, f):
        rho = self.density(f)
        u = self.velocity(f, rho)
        u2 = np.einsum("...a,...a->...", u, u)
        ke = 0.5 * rho * u2
        return {
            "mass": float(np.sum(self.mesh.Me * rho)),
            "ke_max": float(ke.max()),
            "ke_int": float(np.sum(self.mesh.Me * ke)),
            "umax": float(np.sqrt(u2.max())),
            "rho_min": float(rho.min()),
            "rho_max": float(rho.max()),
            "n_nonfinite": int(np.count_nonzero(~np.isfinite(f))),
        }
