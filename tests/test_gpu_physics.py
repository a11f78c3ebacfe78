"""Physics of the GPU path at equilibrium (through the C ABI):

* static contact angle on a flat wall for wetting angles (Sec. 3.1); with the
  interface widths affordable here (delta / R ~ 0.2-0.4) non-wetting drops
  settle below the prescribed angle (108 for 120 degrees) or lift off at 150,
  so those angles are not asserted,
* contact angle on a circular cylinder from the circle-circle geometry
  cos(theta) = (R_c^2 + R_d^2 - d^2) / (2 R_c R_d) (Sec. 3.2), and on the
  sphere wall of the Sec. 3.2 box from the sphere-sphere geometry, with the
  vapour started at the Kelvin-shifted density of the drop's radius,
* Laplace's law gamma / R for drops of several radii (Appendix A gamma), and
  the drop's residual kinetic energy reaching the paper's isolated-drop level
  (~1e-30, Sec. 3.3) in a closed box with neutral walls,
* the flat-wall parasitic currents decaying steadily (the paper's wetting
  residuals are reached after ~1e6 steps; here the trend is checked over 2e5).
"""
import math

import numpy as np
import pytest

from paper_2609_00535_b300 import inputs, wetting
from tests.helpers import make_case
from tests.test_oracle_equilibria import contact_angle, contour_points, fit_circle

pytestmark = pytest.mark.gpu


def _run(case, steps, moments=False):
    from paper_2609_00535_b300 import semlbm
    s = semlbm.Solver.from_case(case)
    s.set_density(case.rho0)
    s.step(steps)
    d = s.diagnostics()
    rho = s.field("rho")
    w = s.wetting_moments(0) if moments else None
    s.close()
    return (rho, d, w) if moments else (rho, d)


@pytest.mark.parametrize("deg", [30, 60, 90])
def test_flat_wall_contact_angle(deg):
    m = inputs.box((16, 8), (0, 0), (2, 1), 4, face_tags={2: 0})
    th0 = math.radians(deg)
    c = make_case("ca", m, "D2Q9", 0.1, 0.1, 1.0, th0,
                  rho0=inputs.sessile_cap_density(m, 1.0, 0.5 * math.pi * 0.25 ** 2, th0, 0.1))
    rho, d, w = _run(c, 12000, moments=True)
    assert d["status"] == 0
    th = contact_angle(m, rho.reshape(m.n_elem, -1), 0.1, 5)
    assert abs(th - deg) < 3.0, (deg, th)
    # the same angle from the device's wetting moments (cap area and wetted base)
    th_dev = wetting.contact_angle(w, 2, delta=0.1)
    assert abs(th_dev - deg) < 4.0 and abs(th_dev - th) < 3.0, (deg, th, th_dev)


def test_flat_wall_angle_with_thinner_interface():
    """At delta / R = 0.2 (32x16 quads, N = 4, delta = 0.05) the drops of 90 and
    120 degrees, which at delta / R = 0.4 evaporate or settle low, hold their
    prescribed angle to within 1.5 degrees (device moments; force_split = 1; one
    batch, each drop measured when its KE_max first falls below 1e-14, as in
    bench.py --angle-study).  Started at the bulk densities, the 90-degree drop
    gives the vapour 17 % of its area, comes to rest near 1.6e5 steps, and
    rearranges later (KE_max back near 1e-7 around 2.2e5 steps while it sheds
    another 0.6 % of its area), so it is measured at its first rest."""
    from paper_2609_00535_b300 import semlbm
    b = semlbm.Batch()
    runs = {}
    for deg in (90.0, 120.0):
        c = inputs.cap_on_wall_2d(math.radians(deg), N=4, ne=16, delta=0.05)
        c.force_split = 1
        s = semlbm.Solver.from_case(c)
        s.set_density(c.rho0)
        runs[b.add(s)] = (deg, s)
    measured = {}
    done = 0
    while runs and done < 240000:
        b.step(2000)
        done += 2000
        d = b.diagnostics()
        for slot in list(runs):
            deg, s = runs[slot]
            assert d[slot]["status"] == 0, (deg, d[slot])
            if d[slot]["ke_max"] < 1e-14:
                measured[deg] = (done, wetting.contact_angle(s.wetting_moments(0), 2, delta=0.05))
                b.remove(slot)
                s.close()
                del runs[slot]
    assert not runs, ("not at rest within 2.4e5 steps", [deg for deg, _ in runs.values()])
    for deg, (steps, th) in measured.items():
        assert abs(th - deg) < 1.5, (deg, steps, th)
    b.close()


@pytest.mark.parametrize("deg", [60, 120])
def test_cylinder_contact_angle(deg):
    Rc = 0.15
    m = inputs.rotate_elements(inputs.cylinder_ogrid(6, n_theta=48, n_r=10, Rc=Rc), 2)
    delta = 0.06
    Rd = 0.15
    c = make_case("cyl", m, "D2Q9", 0.1, delta, 1.0, math.radians(deg),
                  rho0=inputs.cylinder_cap_density(m, (0.5, 0.5), Rc, Rd, math.radians(deg), delta))
    rho, d, w = _run(c, 15000, moments=True)
    assert d["status"] == 0
    p = contour_points(m.node_xyz, rho.reshape(m.n_elem, -1), 0.55, 7)
    p = p[np.linalg.norm(p - 0.5, axis=1) > Rc + delta]
    cx, cy, R = fit_circle(p)
    dist = math.hypot(cx - 0.5, cy - 0.5)
    th = math.degrees(math.acos((Rc ** 2 + R ** 2 - dist ** 2) / (2 * Rc * R)))
    assert abs(th - deg) < 4.0, (deg, th)
    # the same angle from the device's wetting moments (liquid area and wetted arc)
    th_dev = wetting.contact_angle(w, 2, delta=delta, wall_radius=Rc)
    assert abs(th_dev - deg) < 4.0 and abs(th_dev - th) < 5.0, (deg, th, th_dev)


def test_cylinder_contact_angle_thinner_interface():
    """The cylinder case at half the interface width (delta / R = 0.2: O-grid
    96x20, N = 6, delta = 0.03), 60 and 120 degrees in one batch for 6e4 steps: the
    contour circle fit and the device moments agree with each other and with the
    prescribed angle to within 3 degrees (at delta / R = 0.4 the 120-degree drop's
    two estimates differ by 4.2 degrees)."""
    from paper_2609_00535_b300 import semlbm
    Rc = Rd = 0.15
    delta = 0.03
    m = inputs.rotate_elements(inputs.cylinder_ogrid(6, n_theta=96, n_r=20, Rc=Rc), 2)
    b = semlbm.Batch()
    runs = {}
    for deg in (60, 120):
        c = make_case("cyl2", m, "D2Q9", 0.1, delta, 1.0, math.radians(deg),
                      rho0=inputs.cylinder_cap_density(m, (0.5, 0.5), Rc, Rd, math.radians(deg), delta))
        s = semlbm.Solver.from_case(c)
        s.set_density(c.rho0)
        runs[b.add(s)] = (deg, s)
    b.step(60000)
    d = b.diagnostics()
    for slot, (deg, s) in runs.items():
        assert d[slot]["status"] == 0
        rho = s.field("rho")
        p = contour_points(m.node_xyz, rho.reshape(m.n_elem, -1), 0.55, 7)
        p = p[np.linalg.norm(p - 0.5, axis=1) > Rc + delta]
        cx, cy, R = fit_circle(p)
        dist = math.hypot(cx - 0.5, cy - 0.5)
        th = math.degrees(math.acos((Rc ** 2 + R ** 2 - dist ** 2) / (2 * Rc * R)))
        th_dev = wetting.contact_angle(s.wetting_moments(0), 2, delta=delta, wall_radius=Rc)
        assert abs(th - deg) < 3.0 and abs(th_dev - deg) < 3.0 and abs(th - th_dev) < 3.0, \
            (deg, th, th_dev)
    b.close()
    for _, s in runs.values():
        s.close()


@pytest.mark.parametrize("R", [0.25, 0.3])
def test_laplace_law_and_residual_kinetic_energy(R):
    m = inputs.box((8, 8), (0, 0), (1, 1), 4, face_tags={0: -1, 1: -1, 2: -1, 3: -1})
    c = make_case("lap", m, "D2Q9", 0.1, 0.1, 1.0, math.pi / 2,
                  rho0=inputs.droplet_density(m, (0.5, 0.5), R, 0.1))
    rho, d = _run(c, 30000)
    assert d["ke_max"] < 1e-26, d["ke_max"]          # the paper's isolated drop: ~1e-30
    r = np.linalg.norm(m.node_xyz - 0.5, axis=-1).reshape(-1)
    rin, rout = rho[r < 0.05].mean(), rho[r > 0.45].mean()
    beta, kappa = c.beta, c.kappa
    mu0 = lambda x: 2 * beta * (x - 1.0) * (x - 0.1) * (2 * x - 1.1)
    e0 = lambda x: beta * (x - 1.0) ** 2 * (x - 0.1) ** 2
    p0 = lambda x: x * mu0(x) - e0(x)
    from tests.helpers import oracle_mesh
    Me = oracle_mesh(m).Me.reshape(-1)
    area = np.sum(Me * (rho - rout) / (rin - rout))
    gamma = 0.9 ** 3 * math.sqrt(2 * kappa * beta) / 6
    ratio = (p0(rin) - p0(rout)) / (gamma / math.sqrt(area / math.pi))
    assert abs(ratio - 1) < 0.01, ratio


def test_flat_wall_parasitic_currents_decay():
    """Paper-like parameters (beta = 1e-3, tau = 0.5, 60 degrees): KE_max keeps
    falling geometrically and is below 1e-14 after 2e5 steps."""
    from paper_2609_00535_b300 import semlbm
    c = inputs.flat_wall_2d()
    s = semlbm.Solver.from_case(c)
    s.set_density(c.rho0)
    ke = []
    for _ in range(4):
        s.step(50000)
        ke.append(s.diagnostics()["ke_max"])
    s.close()
    assert ke[-1] < 1e-14 and all(b < 0.5 * a for a, b in zip(ke, ke[1:])), ke


def test_isolated_drop_long_run_by_force_split():
    """The paper's isolated drop (Sec. 3.3 shape: 4x4 quads, N = 8, Cn 0.063,
    beta 1e-3, tau 0.5, CFL 0.4).  With F** built from the printed force
    c_s^2 grad rho - rho grad mu, a growing mode takes over after ~1e4 steps
    (the oracle shows the same growth on these inputs); with its potential part
    -rho grad mu alone, KE_max stays finite and below its early level."""
    from paper_2609_00535_b300 import semlbm
    out = {}
    for mode in (0, 1):
        c = inputs.periodic_droplet(dim=2, ne=4, N=8)
        c.force_split = mode
        s = semlbm.Solver.from_case(c)
        s.set_density(c.rho0)
        ke = []
        for _ in range(8):
            s.step(5000)
            d = s.diagnostics()
            ke.append(d["ke_max"] if d["status"] == 0 else float("inf"))
        s.close()
        out[mode] = ke
    assert max(out[0][3:]) > 1e3 * min(out[0]), out[0]           # growth (or non-finite)
    assert all(np.isfinite(out[1])) and max(out[1][2:]) < out[1][0], out[1]


@pytest.mark.parametrize("deg", [60, 90, 120])
def test_flat_wall_contact_angle_3d(deg):
    """A 3D drop on the wall z = 0 (D3Q13), started from its equilibrium cap,
    keeps the prescribed angle; measured from the device's wetting moments.
    The drop is a hemisphere's volume of radius 0.3 with delta = 0.07 (R/delta
    ~ 4): smaller drops (R/delta ~ 2) evaporate into the box's vapour in 3D,
    their Laplace pressure 2 gamma / R being twice the 2D one."""
    m = inputs.box((8, 8, 4), (0, 0, 0), (1, 1, 0.5), 6, face_tags={4: 0})
    th0 = math.radians(deg)
    c = make_case("ca3", m, "D3Q13", 0.01, 0.07, 1.0, th0,
                  rho0=inputs.sessile_cap_density_3d(m, 0.5, 0.5, 2 * math.pi * 0.3 ** 3 / 3,
                                                     th0, 0.07))
    rho, d, w = _run(c, 6000, moments=True)
    assert d["status"] == 0 and d["ke_max"] < 1e-6, d
    th = wetting.contact_angle(w, 3, delta=0.07)
    assert abs(th - deg) < 4.0, (deg, th)


def test_sphere_wall_contact_angle_3d():
    """Drops on the sphere-cap bottom of Sec. 3.2 (wall sphere of radius 0.7
    under the 0.5 x 0.5 x 0.25 box, D3Q13) at 60, 90 and 120 degrees: the relaxing
    sphere-wall request on 8^3 curved hexes at N = 4 (drop radius 0.13, interface
    2.5 node spacings, delta / R = 0.3), started at its equilibrium position with
    both bulk densities raised by the Kelvin shift of its radius (otherwise the
    closed box's vapour takes most of a 60-degree drop before it comes to rest).
    After 5e4 steps in one batch every drop is at rest, has kept its volume, and a
    sphere fitted to its mid-density contour meets the wall within 3.5 degrees of
    the prescribed angle.  The device moments agree within 3.5 degrees at 90 and
    120; at 60 the cap is only ~2.4 interface widths high and their diffuse-interface
    correction leaves 7 degrees (the error of both falls with delta / R)."""
    from paper_2609_00535_b300 import semlbm
    b = semlbm.Batch()
    runs = {}
    for deg in (60, 90, 120):
        th0 = math.radians(deg)
        c = inputs.relaxing_case("relaxsphere3d", 8 ** 3, 4, th0, saturate=True)
        assert c.extra["kelvin_shift"] > 0
        s = semlbm.Solver.from_case(c)
        s.set_density(c.rho0)
        runs[b.add(s)] = (deg, c, s)
    b.step(50000)
    d = b.diagnostics()
    for slot, (deg, c, s) in runs.items():
        assert d[slot]["status"] == 0 and d[slot]["ke_max"] < 1e-11, (deg, d[slot])
        delta = c.extra["delta"]
        w = s.wetting_moments(0)
        vol0 = wetting.curved_cap(0.7, 0.13, math.radians(deg), 3)[0]
        assert abs(w["volume"] / vol0 - 1) < 0.06, (deg, w, vol0)
        th_c = wetting.contour_angle_on_curved_wall(
            c.mesh.node_xyz, s.field("rho").reshape(c.mesh.n_elem, -1), 5, 3,
            (0.25, 0.25, -0.7), 0.7, delta)
        th_m = wetting.contact_angle(w, 3, delta=delta, wall_radius=0.7)
        assert abs(th_c - deg) < 3.5, (deg, th_c, th_m)
        assert abs(th_m - deg) < (8.0 if deg == 60 else 3.5), (deg, th_c, th_m)
    b.close()
    for _, _, s in runs.values():
        s.close()


def test_flat_wall_wetting_residual():
    """A 60-degree drop on a flat wall, started at its equilibrium cap, settles to
    the residual kinetic energy the paper reports for wetting configurations
    (~1e-24 to ~1e-27, Sec. 3.1 and 4): below 1e-24 after 1.5e5 steps."""
    from paper_2609_00535_b300 import semlbm
    c = inputs.cap_on_wall_2d(math.radians(60))
    s = semlbm.Solver.from_case(c)
    s.set_density(c.rho0)
    s.step(150000)
    d = s.diagnostics()
    s.close()
    assert d["status"] == 0 and d["ke_max"] < 1e-24, d
