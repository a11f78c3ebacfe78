"""Seeded synthetic inputs: meshes, initial densities and run parameters.

This module holds no arithmetic of the time step.  It builds what a user (and
the tests and the benchmark) hand to the library: GLL node coordinates of
isoparametric quad/hex elements, global node ids (equal ids = shared node;
periodicity is expressed through ids), per-face kinds and wall tags, the
tanh-initialised density of Appendix A (Eq. dens / A.8) and seeded density
noise.  The GLL reference points come from numpy's Legendre root finder.

Meshes (the paper's own GMSH meshes are not available; these generators stand
in for them with the paper's geometry as the shape):
 * ``box``               affine quads/hexes, walls or periodic per axis
                         (flat-wall droplet of Sec. 3.1, isolated periodic
                         droplet of Sec. 3.3);
 * ``cylinder_ogrid``    curved O-grid around a circular cylinder inside the
                         unit square (Sec. 3.2, 2D);
 * ``sphere_cap_box``    box whose bottom is a sphere cap (Sec. 3.2, 3D);
 * ``rotate_elements``   random proper rotations of the element-local axes, so
                         that neighbouring elements disagree on orientation
                         (unstructured connectivity).

Layout of the arrays (the library's mesh ABI):
  node_xyz  [E][(N+1)^d][d] float64, local node k = i + n j (+ n^2 l), i fastest
  global_id [E][(N+1)^d]    int64
  face_kind [E][2d]         uint8, face f = 2 b + s (b = reference axis,
                            s = 0 for xi_b = -1, 1 for xi_b = +1); 1 = wall
  face_tag  [E][2d]         int32; wall contact-angle tag: < 0 neutral (90 deg),
                            0 = theta_w, k >= 1 = theta_tag[k-1]
"""
from dataclasses import dataclass, field
import math

import numpy as np
from numpy.polynomial import legendre as _leg


def gll_points(N):
    """GLL points of order N (numpy Legendre roots of P_N' plus the end points)."""
    if N < 1:
        raise ValueError("N must be >= 1")
    inner = _leg.Legendre.basis(N).deriv().roots() if N >= 2 else np.zeros(0)
    return np.concatenate([[-1.0], np.sort(inner.real), [1.0]])


@dataclass
class MeshArrays:
    dim: int
    N: int
    node_xyz: np.ndarray
    global_id: np.ndarray
    face_kind: np.ndarray
    face_tag: np.ndarray
    name: str = "mesh"

    @property
    def n_elem(self):
        return self.node_xyz.shape[0]

    @property
    def n_local(self):
        return self.node_xyz.shape[0] * self.node_xyz.shape[1]

    def validate(self):
        n = self.N + 1
        E = self.n_elem
        assert self.node_xyz.shape == (E, n ** self.dim, self.dim)
        assert self.global_id.shape == (E, n ** self.dim)
        assert self.face_kind.shape == (E, 2 * self.dim)
        assert self.face_tag.shape == (E, 2 * self.dim)
        return self


def _local_multi_index(dim, n):
    """[n^d, d] multi-indices (i, j, l) of the local nodes, i fastest."""
    idx = np.indices((n,) * dim).reshape(dim, -1)[::-1].T   # columns (i, j, l)
    return idx


def _element_multi_index(ne):
    dim = len(ne)
    return np.indices(tuple(ne[::-1])).reshape(dim, -1)[::-1].T  # axis 0 fastest


def _structured(ne, N, mapping, periodic, face_tags, name):
    """Build a mesh on a structured block of elements through a mapping.

    mapping(s) maps block coordinates s in [0,1]^d (array [..., d]) to physical
    points.  periodic[a] glues the two ends of block axis a.
    """
    dim = len(ne)
    n = N + 1
    xi = gll_points(N)
    loc = _local_multi_index(dim, n)                 # [n^d, d]
    eid = _element_multi_index(ne)                   # [E, d]
    E = eid.shape[0]
    ne_arr = np.asarray(ne)
    s = (eid[:, None, :] + (xi[loc][None, :, :] + 1) / 2) / ne_arr   # [E, n^d, d]
    node_xyz = mapping(s)
    I = eid[:, None, :] * N + loc[None, :, :]        # structured node index
    counts = []
    for a in range(dim):
        if periodic[a]:
            I[..., a] %= ne[a] * N
            counts.append(ne[a] * N)
        else:
            counts.append(ne[a] * N + 1)
    stride = np.cumprod([1] + counts[:-1])
    gid = (I * stride).sum(-1).astype(np.int64)
    kind = np.zeros((E, 2 * dim), dtype=np.uint8)
    tag = np.zeros((E, 2 * dim), dtype=np.int32)
    for a in range(dim):
        for side in (0, 1):
            on = eid[:, a] == (0 if side == 0 else ne[a] - 1)
            if periodic[a]:
                continue
            kind[on, 2 * a + side] = 1
            tag[on, 2 * a + side] = face_tags.get(2 * a + side, -1)
    return MeshArrays(dim, N, np.ascontiguousarray(node_xyz), gid, kind, tag, name).validate()


def box(ne, lo, hi, N, periodic=None, face_tags=None, name="box"):
    """Affine box of prod(ne) elements; face_tags maps domain face 2a+s -> tag."""
    dim = len(ne)
    periodic = tuple(periodic) if periodic is not None else (False,) * dim
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return _structured(ne, N, lambda s: lo + s * (hi - lo), periodic, face_tags or {}, name)


def cylinder_ogrid(N, n_theta=64, n_r=16, Rc=0.1, center=(0.5, 0.5), half=0.5, ratio=None,
                   name="cylinder"):
    """Curved O-grid between a circle of radius Rc and the square of half-width half.

    Reference axis 0 runs radially outward, axis 1 counter-clockwise around; the
    radial spacing is geometric with the first layer close to the arc length of
    one element on the circle.  Inner face (axis 0, s = 0) is the cylinder wall
    (tag 0), outer face the square's wall (tag -1, neutral).
    """
    c = np.asarray(center, dtype=np.float64)
    if ratio is None:
        arc = 2 * math.pi * Rc / n_theta
        gap = half - Rc
        lo_r, hi_r = 1.0 + 1e-9, 2.0
        for _ in range(200):   # first layer gap * (r-1)/(r^n - 1) = arc
            mid = 0.5 * (lo_r + hi_r)
            first = gap * (mid - 1) / (mid ** n_r - 1)
            lo_r, hi_r = (mid, hi_r) if first > arc else (lo_r, mid)
        ratio = 0.5 * (lo_r + hi_r)

    def grade(sr):
        if abs(ratio - 1.0) < 1e-12:
            return sr
        return (ratio ** (n_r * sr) - 1) / (ratio ** n_r - 1)

    def mapping(s):
        sr, st = s[..., 0], s[..., 1]
        ph = 2 * math.pi * st
        cs, sn = np.cos(ph), np.sin(ph)
        pc = c + Rc * np.stack([cs, sn], -1)
        scale = half / np.maximum(np.abs(cs), np.abs(sn))
        ps = c + scale[..., None] * np.stack([cs, sn], -1)
        return pc + grade(sr)[..., None] * (ps - pc)

    return _structured((n_r, n_theta), N, mapping, (False, True), {0: 0, 1: -1}, name)


def sphere_cap_box(N, ne=(16, 16, 16), L=0.5, W=0.5, H=0.25, Rs=0.7, center=(0.25, 0.25, -0.7),
                   name="sphere"):
    """Box [0,L]x[0,W] whose bottom is the sphere |x - center| = Rs and top z = H.

    The bottom face (axis 2, s = 0) is the wetting wall (tag 0); the other five
    sides are neutral walls (tag -1).  Plan-view coordinates are affine; z blends
    linearly from the sphere to the lid.
    """
    cx, cy, cz = center

    def mapping(s):
        x = s[..., 0] * L
        y = s[..., 1] * W
        zb = cz + np.sqrt(Rs ** 2 - (x - cx) ** 2 - (y - cy) ** 2)
        z = zb * (1 - s[..., 2]) + H * s[..., 2]
        return np.stack([x, y, z], -1)

    return _structured(tuple(ne), N, mapping, (False, False, False), {4: 0}, name)


def _rotations(dim):
    """Proper signed permutations of the reference axes: (perm, flips)."""
    import itertools
    out = []
    for perm in itertools.permutations(range(dim)):
        inv = sum(1 for i in range(dim) for j in range(i + 1, dim) if perm[i] > perm[j])
        for flips in itertools.product((0, 1), repeat=dim):
            if (inv + sum(flips)) % 2 == 0:
                out.append((perm, flips))
    return out


def rotate_elements(mesh, seed):
    """Re-express each element in a randomly rotated local frame (same geometry)."""
    dim, N = mesh.dim, mesh.N
    n = N + 1
    rng = np.random.default_rng(seed)
    rots = _rotations(dim)
    loc = _local_multi_index(dim, n)
    stride = n ** np.arange(dim)
    xyz = mesh.node_xyz.copy()
    gid = mesh.global_id.copy()
    kind = mesh.face_kind.copy()
    tag = mesh.face_tag.copy()
    for e in range(mesh.n_elem):
        perm, flips = rots[rng.integers(len(rots))]
        old = np.empty_like(loc)
        for bn in range(dim):          # new axis bn reads old axis perm[bn]
            old[:, perm[bn]] = (N - loc[:, bn]) if flips[bn] else loc[:, bn]
        src = (old * stride).sum(-1)
        xyz[e] = mesh.node_xyz[e, src]
        gid[e] = mesh.global_id[e, src]
        for bn in range(dim):
            for sn in (0, 1):
                fo = 2 * perm[bn] + (sn ^ flips[bn])
                kind[e, 2 * bn + sn] = mesh.face_kind[e, fo]
                tag[e, 2 * bn + sn] = mesh.face_tag[e, fo]
    return MeshArrays(dim, N, xyz, gid, kind, tag, mesh.name + "-rot").validate()


def min_node_spacing(mesh):
    """Smallest distance between neighbouring GLL nodes along any reference axis."""
    n = mesh.N + 1
    X = mesh.node_xyz.reshape((mesh.n_elem,) + (n,) * mesh.dim + (mesh.dim,))
    h = np.inf
    for b in range(mesh.dim):
        ax = mesh.dim - b
        dx = np.diff(X, axis=ax)
        h = min(h, float(np.sqrt((dx ** 2).sum(-1)).min()))
    return h


def tanh_profile(dist, delta, rho_l, rho_v):
    """Appendix A (Eq. dens): liquid where the signed distance is negative."""
    return 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * np.tanh(2 * dist / delta)


def droplet_density(mesh, x0, R, delta, rho_l=1.0, rho_v=0.1, periodic_L=None):
    """Eq. A.8: rho = tanh profile of |x - x0| - R at every element-local node."""
    d = mesh.node_xyz - np.asarray(x0, dtype=np.float64)
    if periodic_L is not None:   # minimum-image distance in a periodic box
        Lp = np.asarray(periodic_L, dtype=np.float64)
        d = d - Lp * np.round(d / Lp)
    dist = np.sqrt((d ** 2).sum(-1)) - R
    return tanh_profile(dist, delta, rho_l, rho_v)


_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x):
    """SplitMix64 finaliser (Steele, Lea & Flood 2014) on uint64 arrays."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def node_noise(mesh, seed, amplitude):
    """Uniform(-a, a) noise per GLL node, keyed by global id (continuous field)."""
    key = np.uint64(seed) ^ mesh.global_id.astype(np.uint64)
    u = (splitmix64(key) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return amplitude * (2 * u - 1)


# ---------------------------------------------------------------------------
# The workloads.  Each returns a Case with everything the library's create()
# takes plus the initial density and the number of steps.
# ---------------------------------------------------------------------------
SPEED_MAX = {"D2Q9": math.sqrt(2.0), "D3Q13": math.sqrt(5.0 / 3.0), "D3Q19": math.sqrt(2.0),
             "D3Q27": math.sqrt(3.0)}   # max |e_alpha|


@dataclass
class Case:
    name: str
    mesh: MeshArrays
    lattice: str
    rho_l: float
    rho_v: float
    beta: float
    kappa: float
    tau: float
    dt: float
    theta_w: float
    theta_tag: tuple = ()
    rho0: np.ndarray = None
    steps: int = 0
    extra: dict = field(default_factory=dict)
    wall_velocity: dict = field(default_factory=dict)   # wall tag -> u_b
    force_split: int = 0   # force in F**: 0 c_s^2 grad rho - rho grad mu, 1 -rho grad mu

    @property
    def nodes(self):
        return self.mesh.n_local


def kappa_from_width(beta, delta, rho_l, rho_v):
    """Appendix A parameter relation kappa = beta delta^2 (rho_l - rho_v)^2 / 8."""
    return beta * delta ** 2 * (rho_l - rho_v) ** 2 / 8


def kelvin_shift(beta, kappa, rho_l, rho_v, R, dim):
    """Density shift of both bulk phases around a drop of radius R at rest.  The
    Laplace pressure (dim - 1) gamma / R (gamma of Appendix A) raises the chemical
    potential of both phases by dmu = (dim - 1) gamma / (R (rho_l - rho_v)), and the
    double well's curvature there, d mu0 / d rho = 2 beta (rho_l - rho_v)^2 at
    rho_v and at rho_l, turns it into the shift d rho = dmu / (d mu0 / d rho).  A
    drop started between the unshifted densities in a closed box evaporates until
    its vapour carries the shift: with a vapour volume V_v, a liquid mass of about
    V_v d rho leaves the drop, which can be most of a small drop."""
    gamma = (rho_l - rho_v) ** 3 * math.sqrt(2 * kappa * beta) / 6
    dmu = (dim - 1) * gamma / (R * (rho_l - rho_v))
    return dmu / (2 * beta * (rho_l - rho_v) ** 2)


CAPILLARY_NUMBER = 0.1


def cfl_dt(mesh, lattice, cfl=0.4, kappa=None, rho_l=1.0):
    """Time step: min(cfl h_min / max|e|, 0.1 h_min^2 / sqrt(rho_l kappa)).

    The second bound keeps the fastest capillary wave (omega ~ sqrt(rho kappa) k^2,
    from the kappa lap(rho) part of mu in the streaming force) inside the SSP-RK3
    stability region; the library applies the same rule when given dt <= 0.
    """
    h = min_node_spacing(mesh)
    dt = cfl * h / SPEED_MAX[lattice]
    if kappa:
        dt = min(dt, CAPILLARY_NUMBER * h * h / math.sqrt(rho_l * kappa))
    return dt


def flat_wall_2d(N=4, ne=(8, 8), theta=math.radians(60), R=0.25, beta=1e-3, tau=0.5,
                 width_spacings=4.0, rho_l=1.0, rho_v=0.1, steps=200, cfl=0.4, seed=None,
                 noise=0.0):
    """Sessile half-disc on the wall y = 0 of the unit square (Sec. 3.1 shape)."""
    mesh = box(ne, (0.0, 0.0), (1.0, 1.0), N, face_tags={2: 0})
    delta = width_spacings * (1.0 / ne[0]) / N
    kappa = kappa_from_width(beta, delta, rho_l, rho_v)
    rho0 = droplet_density(mesh, (0.5, 0.0), R, delta, rho_l, rho_v)
    if noise:
        rho0 = rho0 + node_noise(mesh, seed or 0, noise)
    return Case("flat2d", mesh, "D2Q9", rho_l, rho_v, beta, kappa, tau,
                cfl_dt(mesh, "D2Q9", cfl, kappa, rho_l),
                theta, (), rho0, steps, {"delta": delta})


def cylinder_2d(theta=math.radians(90), N=6, n_theta=64, n_r=16, Rc=0.1, beta=1e-2, tau=0.5,
                rho_l=1.0, rho_v=0.1, noise=1e-3, seed=1, perm_seed=2, cfl=0.4, steps=200):
    """Droplet of radius 0.3 Rc touching a cylinder (Sec. 3.2 shape), curved O-grid."""
    mesh = rotate_elements(cylinder_ogrid(N, n_theta, n_r, Rc), perm_seed)
    Rd = 0.3 * Rc
    spacing = 2 * math.pi * Rc / n_theta / N
    delta = 4 * spacing
    kappa = kappa_from_width(beta, delta, rho_l, rho_v)
    rho0 = droplet_density(mesh, (0.5, 0.5 + Rc + Rd), Rd, delta, rho_l, rho_v)
    rho0 = rho0 + node_noise(mesh, seed, noise)
    return Case("cylinder2d", mesh, "D2Q9", rho_l, rho_v, beta, kappa, tau,
                cfl_dt(mesh, "D2Q9", cfl, kappa, rho_l), theta, (), rho0, steps, {"delta": delta})


def sphere_3d(N=5, ne=(16, 16, 16), theta=math.radians(60), beta=1e-3, Cn=0.08, d=0.25,
              La=60.0, rho_l=1.0, rho_v=0.1, cfl=0.4, steps=20000, lattice="D3Q13"):
    """3D droplet (d = 0.25 at (0.25, 0.25, 0.04)) on a sphere-cap bottom (Sec. 3.2)."""
    mesh = sphere_cap_box(N, ne)
    delta = Cn * d
    kappa = kappa_from_width(beta, delta, rho_l, rho_v)
    dt = cfl_dt(mesh, lattice, cfl, kappa, rho_l)
    gamma = (rho_l - rho_v) ** 3 * math.sqrt(2 * kappa * beta) / 6
    eta = math.sqrt(gamma * d / La)          # La = gamma d / eta^2
    nu = eta / rho_l
    tau = nu / ((1.0 / 3.0) * dt)            # nu = tau c_s^2 dt
    rho0 = droplet_density(mesh, (0.25, 0.25, 0.04), d / 2, delta, rho_l, rho_v)
    return Case("sphere3d", mesh, lattice, rho_l, rho_v, beta, kappa, tau, dt, theta, (),
                rho0, steps, {"delta": delta, "La": La})


def periodic_droplet(dim=2, ne=4, N=8, L=1.0, D=0.5, Cn=0.063, beta=1e-3, tau=0.5,
                     rho_l=1.0, rho_v=0.1, cfl=0.4, steps=200):
    """Isolated droplet in a periodic box (Sec. 3.3)."""
    mesh = box((ne,) * dim, (0.0,) * dim, (L,) * dim, N, periodic=(True,) * dim)
    delta = Cn * D
    kappa = kappa_from_width(beta, delta, rho_l, rho_v)
    lat = "D2Q9" if dim == 2 else "D3Q13"
    rho0 = droplet_density(mesh, (L / 2,) * dim, D / 2, delta, rho_l, rho_v)
    return Case("droplet%dd" % dim, mesh, lat, rho_l, rho_v, beta, kappa, tau,
                cfl_dt(mesh, lat, cfl, kappa, rho_l), math.pi / 2, (), rho0, steps,
                {"delta": delta, "R": D / 2})


# ---------------------------------------------------------------------------
# Mixed workloads for batching and serving (uneven meshes, orders and angles).
# ---------------------------------------------------------------------------
def _log_uniform_int(rng, lo, hi):
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def mixed_case(rng, kind, E, N, theta, radius_scale=1.0, saturate=False):
    """One solve of the given kind with about E elements (rounded to the
    generator's grid).  `saturate` applies to the sweep kinds capwall2d and
    discwall2d."""
    if kind == "flat2d":
        a = max(2, int(round(math.sqrt(E))))
        b = max(2, int(round(E / a)))
        c = flat_wall_2d(N=N, ne=(a, b), theta=theta, R=0.25 * radius_scale)
    elif kind == "cylinder2d":
        n_r = max(2, int(round(math.sqrt(E / 4.0))))
        n_t = max(8, int(round(E / n_r)))
        c = cylinder_2d(theta=theta, N=N, n_theta=n_t, n_r=n_r, seed=int(rng.integers(1 << 30)),
                        perm_seed=int(rng.integers(1 << 30)))
    elif kind == "sphere3d":
        ne = max(2, int(round(E ** (1.0 / 3.0))))
        c = sphere_3d(N=N, ne=(ne, ne, ne), theta=theta, d=0.25 * radius_scale)
    elif kind == "droplet2d":
        ne = max(2, int(round(math.sqrt(E))))
        c = periodic_droplet(dim=2, ne=ne, N=N, D=0.5 * radius_scale, Cn=max(0.063, 4.0 / (ne * N)))
    elif kind == "droplet3d":
        ne = max(2, int(round(E ** (1.0 / 3.0))))
        c = periodic_droplet(dim=3, ne=ne, N=N, D=0.5 * radius_scale, Cn=max(0.063, 4.0 / (ne * N)))
    elif kind in ("capwall2d", "discwall2d"):
        c = cap_on_wall_2d(theta, N=N, ne=max(4, int(round(math.sqrt(E / 2.0)))),
                           R=0.25 * radius_scale, init="cap" if kind == "capwall2d" else "disc",
                           saturate=saturate)
    elif kind == "boxdrop2d":
        c = closed_box_drop(N=N, ne=max(4, int(round(math.sqrt(E)))), R=0.25 * radius_scale)
    elif kind.startswith("relax"):
        c = relaxing_case(kind, E, N, theta, radius_scale)
    else:
        raise ValueError(kind)
    c.name = "%s-E%d-N%d-%.0fdeg" % (kind, c.mesh.n_elem, N, math.degrees(theta))
    return c


def viscous_tau(dt, L, steps=1.0e4, cap=10.0):
    """Relaxation time that makes the viscous time L^2 / nu of a domain of size L
    last about `steps` time steps (nu = tau c_s^2 dt), within [1, cap]: beyond
    ~10 the overdamped relaxation of a drop on a cylinder slows (measured: tau 3
    and 10 converge within 1.7e5 steps, tau 20-50 do not within 6e4)."""
    return min(cap, max(1.0, L * L / ((1.0 / 3.0) * dt * dt * steps)))


def relaxing_case(kind, E, N, theta, radius_scale=1.0, beta=0.1, rho_l=1.0, rho_v=0.1, cfl=0.4,
                  saturate=False):
    """Requests that relax to rest (the serving stream run to a kinetic-energy
    threshold): stiff surface tension (beta = 0.1), interface width 3 node
    spacings (2.5 on the 3D sphere wall), tau from viscous_tau so the slowest
    viscous mode decays within ~1e4 steps, each drop started at its equilibrium
    cap, and the potential-part force reading in F** (force_split = 1, under
    which a drop at rest is linearly stable; with the printed force a periodic
    drop at rest has a growing mode).  With `saturate` both phases start at the
    densities of a drop of that radius at rest (kelvin_shift): started at the
    bulk densities, a drop gives the closed box's vapour the mass it needs to
    reach them, which is most of a small 60-degree drop.  The serving stream
    keeps the bulk densities: on its coarse meshes (interface up to 0.8 of the
    drop radius) the first-order shift is far from the discrete equilibrium, and
    its requests took longer to come to rest with it (measured: converged p50
    16.1 s against 7.5 s on 100 requests).  Kinds:
      relaxflat2d    cap on the wall y = 0 of [0, 2] x [0, 1], 2 ne x ne quads
      relaxcyl2d     cap on a cylinder of radius 0.15 (curved O-grid, rotated frames)
      relaxsphere3d  cap on the sphere wall of the Sec. 3.2 box (ne^3 curved hexes)
      relaxdrop2d / relaxdrop3d   drop of diameter 0.5 in a periodic unit box
    E sets the element count (rounded to each generator's grid)."""
    if kind == "relaxflat2d":
        ne = max(3, int(round(math.sqrt(E / 2.0))))
        mesh = box((2 * ne, ne), (0.0, 0.0), (2.0, 1.0), N, face_tags={2: 0})
        h = 1.0 / (ne * N)
        delta, L, lat, dim = 3 * h, 1.0, "D2Q9", 2
        area = 0.5 * math.pi * (0.25 * radius_scale) ** 2
        R = cap_radius(area, theta)
        density = lambda rl, rv: sessile_cap_density(mesh, 1.0, area, theta, delta, rl, rv)
    elif kind == "relaxcyl2d":
        Rc = 0.15
        n_r = max(3, int(round(math.sqrt(E / 6.0))))
        n_t = max(12, int(round(E / n_r)))
        mesh = rotate_elements(cylinder_ogrid(N, n_theta=n_t, n_r=n_r, Rc=Rc), 2)
        delta, L, lat, dim = 3 * 2 * math.pi * Rc / n_t / N, 0.5 - Rc, "D2Q9", 2
        R = 0.15 * radius_scale
        density = lambda rl, rv: cylinder_cap_density(mesh, (0.5, 0.5), Rc, R, theta, delta,
                                                      rl, rv)
    elif kind == "relaxsphere3d":
        ne = max(3, int(round(E ** (1.0 / 3.0))))
        mesh = sphere_cap_box(N, (ne, ne, ne))
        delta, L, lat, dim = 2.5 * 0.5 / (ne * N), 0.5, "D3Q13", 3
        R = 0.13 * radius_scale
        density = lambda rl, rv: curved_cap_density(mesh, (0.25, 0.25, -0.7), 0.7, R, theta,
                                                    delta, (0.0, 0.0, 1.0), rl, rv)
    elif kind in ("relaxdrop2d", "relaxdrop3d"):
        dim = 2 if kind == "relaxdrop2d" else 3
        ne = max(2, int(round(E ** (1.0 / dim))))
        mesh = box((ne,) * dim, (0.0,) * dim, (1.0,) * dim, N, periodic=(True,) * dim)
        delta, L, lat = 3.0 / (ne * N), 1.0, "D2Q9" if dim == 2 else "D3Q13"
        R = 0.25 * radius_scale
        density = lambda rl, rv: droplet_density(mesh, (0.5,) * dim, R, delta, rl, rv)
        theta = math.pi / 2
    else:
        raise ValueError(kind)
    kappa = kappa_from_width(beta, delta, rho_l, rho_v)
    dr = kelvin_shift(beta, kappa, rho_l, rho_v, R, dim) if saturate else 0.0
    rho0 = density(rho_l + dr, rho_v + dr)
    dt = cfl_dt(mesh, lat, cfl, kappa, rho_l)
    return Case(kind, mesh, lat, rho_l, rho_v, beta, kappa, viscous_tau(dt, L), dt, theta, (),
                rho0, 0, {"delta": delta, "kelvin_shift": dr}, force_split=1)


# element-count ranges of the relaxing request kinds (sizes whose slowest modes
# decay to KE_max < 1e-20 within a few 1e4 steps where the physics allows it)
RELAX_SIZES = {"relaxflat2d": (32, 72), "relaxcyl2d": (72, 150), "relaxsphere3d": (27, 64),
               "relaxdrop2d": (16, 64), "relaxdrop3d": (27, 125)}


def relaxing_request_stream(n=500, rate=10.0, seed=8, orders=(4,)):
    """Poisson stream run to a kinetic-energy threshold: a quarter each of drops
    on a flat wall, on a cylinder and on the sphere wall of Sec. 3.2, and
    isolated periodic drops (2D or 3D); E log-uniform in each kind's range
    (RELAX_SIZES), N uniform in `orders`, contact angle uniform in [15, 165]
    degrees, drop size x [0.9, 1.1]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    kinds = ["relaxflat2d", "relaxcyl2d", "relaxsphere3d", "relaxdrop"]
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        kind = kinds[i % 4]
        if kind == "relaxdrop":
            kind = "relaxdrop2d" if rng.random() < 0.5 else "relaxdrop3d"
        out.append(Request(i, t, kind, _log_uniform_int(rng, *RELAX_SIZES[kind]),
                           int(rng.choice(orders)), math.radians(rng.uniform(15.0, 165.0)),
                           float(rng.uniform(0.9, 1.1)), int(rng.integers(1 << 30))))
    return out


def cap_on_wall_2d(theta, N=4, ne=8, R=0.25, beta=0.1, delta=0.1, tau=1.0, rho_l=1.0,
                   rho_v=0.1, cfl=0.4, init="cap", saturate=False):
    """Drop on the wall y = 0 of [0, 2] x [0, 1] (2 ne x ne quads; the other
    walls neutral) with the area of a half-disc of radius R (Sec. 3.1 shape,
    stiff surface tension), started at its equilibrium cap for the angle theta
    (init "cap") or as the half-disc (init "disc", the 90-degree cap).  With
    `saturate` both phases start shifted by the Kelvin shift of the equilibrium
    cap's radius (kelvin_shift), so the drop does not evaporate into the box."""
    mesh = box((2 * ne, ne), (0.0, 0.0), (2.0, 1.0), N, face_tags={2: 0})
    kappa = kappa_from_width(beta, delta, rho_l, rho_v)
    shape = theta if init == "cap" else math.pi / 2
    area = 0.5 * math.pi * R * R
    dr = kelvin_shift(beta, kappa, rho_l, rho_v, cap_radius(area, theta), 2) if saturate else 0.0
    rho0 = sessile_cap_density(mesh, 1.0, area, shape, delta, rho_l + dr, rho_v + dr)
    return Case("capwall2d" if init == "cap" else "discwall2d", mesh, "D2Q9", rho_l, rho_v, beta,
                kappa, tau,
                cfl_dt(mesh, "D2Q9", cfl, kappa, rho_l), theta, (), rho0, 0,
                {"delta": delta, "R": R})


def angle_sweep_stream(n=64, rate=20.0, seed=7, angles=(20.0, 110.0), ne=8, N=4, init="cap",
                       saturate=True):
    """Poisson stream of contact-angle sweep requests: drops on a flat wall
    started at their equilibrium caps (init "cap") or as half-discs ("disc"),
    angle uniform in `angles` (degrees), drop size x [0.9, 1.1], both phases at
    the Kelvin-shifted densities of the equilibrium cap when `saturate`; the
    same seed gives the same angles and sizes for both starts."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        out.append(Request(i, t, "capwall2d" if init == "cap" else "discwall2d", 2 * ne * ne, N,
                           math.radians(rng.uniform(*angles)), float(rng.uniform(0.9, 1.1)),
                           int(rng.integers(1 << 30)), saturate))
    return out


def closed_box_drop(N=4, ne=8, R=0.25, beta=0.1, delta=0.1, tau=1.0, rho_l=1.0, rho_v=0.1,
                    cfl=0.4):
    """Drop in the unit box with neutral no-slip walls: relaxes to its Laplace
    equilibrium, with KE_max below 1e-20 after ~2e4 steps at these parameters."""
    mesh = box((ne, ne), (0.0, 0.0), (1.0, 1.0), N, face_tags={0: -1, 1: -1, 2: -1, 3: -1})
    kappa = kappa_from_width(beta, delta, rho_l, rho_v)
    rho0 = droplet_density(mesh, (0.5, 0.5), R, delta, rho_l, rho_v)
    return Case("boxdrop2d", mesh, "D2Q9", rho_l, rho_v, beta, kappa, tau,
                cfl_dt(mesh, "D2Q9", cfl, kappa, rho_l), math.pi / 2, (), rho0, 0,
                {"delta": delta, "R": R})


def batch_mix(n=64, seed=4, elems=(256, 4096), orders=(4, 5, 6, 7, 8)):
    """Batched workload: n solves, E log-uniform, N uniform, theta uniform in
    [15, 165] degrees, 2D/3D half and half (flat wall or cylinder in 2D, sphere
    cap in 3D)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        E = _log_uniform_int(rng, *elems)
        N = int(rng.choice(orders))
        theta = math.radians(rng.uniform(15.0, 165.0))
        if rng.random() < 0.5:
            kind = "flat2d" if rng.random() < 0.5 else "cylinder2d"
        else:
            kind = "sphere3d"
        out.append(mixed_case(rng, kind, E, N, theta))
    return out


@dataclass
class Request:
    rid: int
    arrival: float         # seconds after the start of the stream
    kind: str
    E: int
    N: int
    theta: float
    radius_scale: float
    seed: int
    saturate: bool = False   # sweep kinds: start at the Kelvin-shifted densities

    def case(self):
        return mixed_case(np.random.default_rng(self.seed), self.kind, self.E, self.N, self.theta,
                          self.radius_scale, self.saturate)


def request_stream(n=500, rate=10.0, seed=5, elems=(256, 8192), orders=(4, 5, 6, 7)):
    """Poisson arrivals of sweep requests: a quarter each of 2D flat wall, 2D
    cylinder, 3D sphere cap and isolated periodic droplet (2D or 3D), E
    log-uniform, N uniform, random contact angle and drop radius."""
    rng = np.random.default_rng(seed)
    t = 0.0
    kinds = ["flat2d", "cylinder2d", "sphere3d", "droplet"]
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        kind = kinds[i % 4]
        if kind == "droplet":
            kind = "droplet2d" if rng.random() < 0.5 else "droplet3d"
        out.append(Request(i, t, kind, _log_uniform_int(rng, *elems), int(rng.choice(orders)),
                           math.radians(rng.uniform(15.0, 165.0)), float(rng.uniform(0.8, 1.2)),
                           int(rng.integers(1 << 30))))
    return out


# ---------------------------------------------------------------------------
# Equilibrium-shape initial densities (the paper starts its parasitic-current
# runs from the equilibrium cap, Sec. 3.1 and Sec. 3.2).
# ---------------------------------------------------------------------------
def cap_radius(area, theta):
    """Radius of a circular cap of the given area meeting a flat wall at theta."""
    return math.sqrt(area / (theta - math.sin(theta) * math.cos(theta)))


def sessile_cap_density(mesh, x_c, area, theta, delta, rho_l=1.0, rho_v=0.1):
    """Drop on the wall y = 0 at its equilibrium shape: a circle of radius R
    centred at (x_c, -R cos(theta)) holding `area` above the wall."""
    R = cap_radius(area, theta)
    c = np.array([x_c, -R * math.cos(theta)] + [0.0] * (mesh.dim - 2))
    dist = np.sqrt(((mesh.node_xyz - c) ** 2).sum(-1)) - R
    return tanh_profile(dist, delta, rho_l, rho_v)


def sessile_cap_density_3d(mesh, x_c, y_c, volume, theta, delta, rho_l=1.0, rho_v=0.1):
    """3D drop on the wall z = 0 at its equilibrium shape: a sphere of radius R
    centred at (x_c, y_c, -R cos(theta)) holding `volume` above the wall,
    V = pi R^3 (1 - cos theta)^2 (2 + cos theta) / 3."""
    c0 = math.cos(theta)
    R = (3 * volume / (math.pi * (1 - c0) ** 2 * (2 + c0))) ** (1.0 / 3.0)
    c = np.array([x_c, y_c, -R * c0])
    dist = np.sqrt(((mesh.node_xyz - c) ** 2).sum(-1)) - R
    return tanh_profile(dist, delta, rho_l, rho_v)


def curved_cap_density(mesh, wall_center, Rw, Rd, theta, delta, direction, rho_l=1.0,
                       rho_v=0.1):
    """Drop of radius Rd on a circular (2D) or spherical (3D) wall of radius Rw
    centred at wall_center, at its equilibrium position along the unit vector
    `direction`: centre distance d with d^2 = Rw^2 + Rd^2 - 2 Rw Rd cos(theta)."""
    d = math.sqrt(Rw * Rw + Rd * Rd - 2 * Rw * Rd * math.cos(theta))
    n = np.asarray(direction, dtype=np.float64)
    c = np.asarray(wall_center, dtype=np.float64) + d * n / np.linalg.norm(n)
    dist = np.sqrt(((mesh.node_xyz - c) ** 2).sum(-1)) - Rd
    return tanh_profile(dist, delta, rho_l, rho_v)


def cylinder_cap_density(mesh, center, Rc, Rd, theta, delta, rho_l=1.0, rho_v=0.1):
    """Drop of radius Rd on a cylinder of radius Rc at its equilibrium position:
    centre distance d with d^2 = Rc^2 + Rd^2 - 2 Rc Rd cos(theta), along +y."""
    d = math.sqrt(Rc * Rc + Rd * Rd - 2 * Rc * Rd * math.cos(theta))
    c = np.asarray(center, dtype=np.float64) + np.array([0.0, d])
    dist = np.sqrt(((mesh.node_xyz - c) ** 2).sum(-1)) - Rd
    return tanh_profile(dist, delta, rho_l, rho_v)


def converging_request_stream(n=100, rate=20.0, seed=6,
                              shapes=((6, 4), (7, 4), (8, 4), (9, 4), (6, 5))):
    """Poisson stream of drop-radius sweep requests that relax to KE_max < 1e-20:
    closed-box drops, R = 0.25 x [0.88, 1.2], (elements per side, N) uniform over
    `shapes`, which keep dt within a factor ~2 of each other (the viscosity is
    proportional to tau dt, so the steps to converge grow like 1/dt^2: 10x10
    quads at N = 4 or 7x7 at N = 5 need more than 6e4)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        ne, N = shapes[int(rng.integers(len(shapes)))]
        out.append(Request(i, t, "boxdrop2d", ne * ne, N, math.pi / 2,
                           float(rng.uniform(0.88, 1.2)), int(rng.integers(1 << 30))))
    return out
