"""Pins of the oracle's wetting moments and of the contact-angle inversion.

The liquid fraction of the tanh profile (Appendix A) is the Fermi function
phi = 1/(1 + exp(4 s / delta)) of the signed distance s, whose integrals across
a curved interface follow the Sommerfeld expansion with no odd terms:
  disc of radius R:      int phi dA = pi R^2 + pi^3 delta^2 / 48
  ball of radius R:      int phi dV = 4 pi R^3 / 3 + pi^3 delta^2 R / 12
  a line through a disc: int phi dx = 2 R   (exactly, up to exp(-4R/delta) terms)
Halves of these sit on a wall through the centre.  The oracle's quadratures
converge to them spectrally; the contact-angle inversion recovers sharp caps
exactly and the equilibrium-cap initial densities to within two degrees on flat
walls (2.5 on cylinders and spheres).
"""
import math

import numpy as np
import pytest

from paper_2609_00535_b300 import inputs, wetting
from tests.helpers import make_case, oracle_of


def _moments(mesh, lattice, rho0, tag=0):
    c = make_case("w", mesh, lattice, 1e-3, 0.1, 0.5, math.pi / 2, theta_tag=(math.pi / 2,),
                  rho0=rho0)
    om, o = oracle_of(c)
    return o.wetting_moments(o.initial_state(rho0.reshape(om.shape)), tag, 0.1, 1.0)


def test_half_disc_on_a_wall():
    R, d = 0.4, 0.1
    m = inputs.box((16, 8), (0, 0), (2, 1), 8, face_tags={2: 0})
    rho0 = inputs.tanh_profile(np.sqrt(((m.node_xyz - [1.0, 0.0]) ** 2).sum(-1)) - R, d, 1.0, 0.1)
    w = _moments(m, "D2Q9", rho0)
    assert w["volume"] == pytest.approx(0.5 * math.pi * (R * R + math.pi ** 2 * d * d / 48), rel=1e-7)
    assert w["wetted"] == pytest.approx(2 * R, rel=1e-7)
    assert w["wall"] == pytest.approx(2.0, rel=1e-13)              # the tag-0 wall y = 0
    assert w["wet_centroid"][0] == pytest.approx(1.0, abs=1e-12)
    assert w["centroid"][0] == pytest.approx(1.0, abs=1e-12)
    every = _moments(m, "D2Q9", rho0, tag=-1)                       # all four walls
    assert every["wall"] == pytest.approx(6.0, rel=1e-13)
    assert every["volume"] == w["volume"]


def test_half_ball_on_a_wall():
    R, d = 0.3, 0.1
    m = inputs.box((8, 8, 4), (0, 0, 0), (1.6, 1.6, 0.8), 8, face_tags={4: 0})
    rho0 = inputs.tanh_profile(np.sqrt(((m.node_xyz - [0.8, 0.8, 0.0]) ** 2).sum(-1)) - R, d, 1.0, 0.1)
    w = _moments(m, "D3Q13", rho0)
    assert w["volume"] == pytest.approx(0.5 * (4 * math.pi * R ** 3 / 3
                                               + math.pi ** 3 * d * d * R / 12), rel=5e-6)
    assert w["wetted"] == pytest.approx(math.pi * R * R + math.pi ** 3 * d * d / 48, rel=5e-6)
    assert w["wall"] == pytest.approx(1.6 * 1.6, rel=1e-13)
    assert w["wet_centroid"][:2] == pytest.approx([0.8, 0.8], abs=1e-12)


def test_liquid_everywhere():
    m = inputs.box((3, 2), (0, 0), (1.5, 1.0), 5, face_tags={0: 1, 2: 0})
    w = _moments(m, "D2Q9", np.ones(m.global_id.shape))
    assert w["volume"] == pytest.approx(1.5, rel=1e-13)
    assert w["wetted"] == pytest.approx(w["wall"], rel=1e-13) and w["wall"] == pytest.approx(1.5)
    assert _moments(m, "D2Q9", np.ones(m.global_id.shape), tag=1)["wall"] == pytest.approx(1.0)


@pytest.mark.parametrize("deg", [15, 45, 90, 135, 170])
def test_sharp_caps_invert_exactly(deg):
    t, R = math.radians(deg), 0.37
    area = R * R * (t - math.sin(t) * math.cos(t))
    vol = math.pi * R ** 3 * (1 - math.cos(t)) ** 2 * (2 + math.cos(t)) / 3
    b = R * math.sin(t)
    assert math.degrees(wetting.cap_angle_2d(area, 2 * b)) == pytest.approx(deg, abs=1e-9)
    assert math.degrees(wetting.cap_angle_3d(vol, math.pi * b * b)) == pytest.approx(deg, abs=1e-9)


@pytest.mark.parametrize("deg", [30, 60, 90, 120, 150])
def test_diffuse_caps_on_a_flat_wall(deg):
    d = 0.1
    m = inputs.box((16, 8), (0, 0), (2, 1), 8, face_tags={2: 0})
    rho0 = inputs.sessile_cap_density(m, 1.0, 0.5 * math.pi * 0.3 ** 2, math.radians(deg), d)
    w = _moments(m, "D2Q9", rho0)
    assert wetting.contact_angle(w, 2, delta=d) == pytest.approx(deg, abs=2.0)


@pytest.mark.parametrize("deg", [60, 90, 120])
def test_diffuse_caps_on_a_flat_wall_3d(deg):
    d = 0.1
    m = inputs.box((8, 8, 4), (0, 0, 0), (1, 1, 0.5), 6, face_tags={4: 0})
    rho0 = inputs.sessile_cap_density_3d(m, 0.5, 0.5, 2 * math.pi * 0.25 ** 3 / 3, math.radians(deg), d)
    w = _moments(m, "D3Q13", rho0)
    assert wetting.contact_angle(w, 3, delta=d) == pytest.approx(deg, abs=2.0)


def test_measured_reference_densities():
    """With phases off the nominal rho_v, rho_l (as a drop in a closed box
    settles), the measured references find the bulk densities (to the few 1e-3
    that the tanh tails inside the 2 % bands add) and the moments follow."""
    R, d, rv, rl = 0.4, 0.1, 0.12, 1.01
    m = inputs.box((16, 8), (0, 0), (2, 1), 8, face_tags={2: 0})
    rho0 = inputs.tanh_profile(np.sqrt(((m.node_xyz - [1.0, 0.0]) ** 2).sum(-1)) - R, d, rl, rv)
    c = make_case("w", m, "D2Q9", 1e-3, 0.1, 0.5, math.pi / 2, rho0=rho0)
    om, o = oracle_of(c)
    f = o.initial_state(rho0.reshape(om.shape))
    w = o.wetting_moments(f, 0)
    assert w["rho_v_ref"] == pytest.approx(rv, rel=5e-3) and w["rho_l_ref"] == pytest.approx(rl, rel=5e-3)
    assert w["volume"] == pytest.approx(0.5 * math.pi * (R * R + math.pi ** 2 * d * d / 48), rel=5e-3)
    assert w["wetted"] == pytest.approx(2 * R, rel=5e-3)
    nominal = o.wetting_moments(f, 0, 0.1, 1.0)                 # vapour counted as liquid
    assert nominal["volume"] > w["volume"] + 0.02


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("deg", [25, 60, 90, 135, 165])
def test_curved_caps_invert_exactly(dim, deg):
    v, w = wetting.curved_cap(0.15, 0.11, math.radians(deg), dim)
    assert math.degrees(wetting.cap_angle_on_curved_wall(v, w, 0.15, dim)) == pytest.approx(deg, abs=1e-7)


def test_curved_cap_geometry():
    """The lens formulas against brute force (2D: a fine grid of the drop disc
    outside the wall disc, the wall arc by angular sampling) and against the
    flat-wall caps as the wall radius grows."""
    Rw, Rd, t = 0.2, 0.15, math.radians(70)
    area, arc = wetting.curved_cap(Rw, Rd, t, 2)
    d = math.sqrt(Rw * Rw + Rd * Rd - 2 * Rw * Rd * math.cos(t))
    n = 2000
    x, y = np.meshgrid(np.linspace(-0.4, 0.4, n), np.linspace(-0.3, 0.5, n))
    h = 0.8 / (n - 1)
    inside = ((x ** 2 + (y - d) ** 2) < Rd * Rd) & ((x ** 2 + y ** 2) >= Rw * Rw)
    assert area == pytest.approx(inside.sum() * h * h, rel=2e-3)
    phi = np.linspace(0, 2 * np.pi, 200001)
    on = (Rw * np.cos(phi)) ** 2 + (Rw * np.sin(phi) - d) ** 2 < Rd * Rd
    assert arc == pytest.approx(on.mean() * 2 * np.pi * Rw, rel=1e-4)
    for dim in (2, 3):
        v, w = wetting.curved_cap(1e4, 0.3, t, dim)     # larger radii lose digits to cancellation
        hc = 0.3 * (1 - math.cos(t))
        vf = 0.09 * (t - math.sin(t) * math.cos(t)) if dim == 2 else math.pi * hc * hc * (0.9 - hc) / 3
        wf = 0.6 * math.sin(t) if dim == 2 else math.pi * (0.3 * math.sin(t)) ** 2
        assert v == pytest.approx(vf, rel=1e-4) and w == pytest.approx(wf, rel=1e-4)


@pytest.mark.parametrize("deg", [60, 90, 120])
def test_diffuse_caps_on_a_cylinder(deg):
    Rc, Rd, d = 0.15, 0.15, 0.06
    m = inputs.cylinder_ogrid(8, n_theta=48, n_r=10, Rc=Rc)
    rho0 = inputs.cylinder_cap_density(m, (0.5, 0.5), Rc, Rd, math.radians(deg), d)
    w = _moments(m, "D2Q9", rho0)
    assert wetting.contact_angle(w, 2, delta=d, wall_radius=Rc) == pytest.approx(deg, abs=2.5)


@pytest.mark.parametrize("deg", [60, 90, 120])
def test_diffuse_caps_on_a_sphere(deg):
    """The sphere-cap box of Sec. 3.2 (wall sphere of radius 0.7 under the box)."""
    m = inputs.sphere_cap_box(5, (8, 8, 6))
    rho0 = inputs.curved_cap_density(m, (0.25, 0.25, -0.7), 0.7, 0.14, math.radians(deg), 0.04,
                                     (0.0, 0.0, 1.0))
    w = _moments(m, "D3Q13", rho0)
    assert wetting.contact_angle(w, 3, delta=0.04, wall_radius=0.7) == pytest.approx(deg, abs=2.5)


@pytest.mark.parametrize("deg", [60, 90, 120])
def test_contour_sphere_fit_on_a_sphere(deg):
    """The contour estimate recovers the angle of the equilibrium-cap initial
    density on the sphere wall of Sec. 3.2 (the tanh profile is centred on the
    drop's sphere, so the mid-density contour is that sphere up to the
    interpolation between nodes)."""
    m = inputs.sphere_cap_box(5, (8, 8, 6))
    rho0 = inputs.curved_cap_density(m, (0.25, 0.25, -0.7), 0.7, 0.14, math.radians(deg), 0.04,
                                     (0.0, 0.0, 1.0))
    th = wetting.contour_angle_on_curved_wall(m.node_xyz, rho0.reshape(m.n_elem, -1), 6, 3,
                                              (0.25, 0.25, -0.7), 0.7, 0.04, level=0.55)
    assert th == pytest.approx(deg, abs=0.5)


def test_contour_circle_fit_on_a_cylinder():
    """The same estimate in 2D, on the cylinder cap, and the least-squares fit
    itself on exact points of a circle."""
    t = np.linspace(0.3, 2.5, 40)
    c, R = wetting.fit_sphere(np.c_[0.2 + 0.7 * np.cos(t), -0.1 + 0.7 * np.sin(t)])
    assert np.allclose(c, [0.2, -0.1], atol=1e-12) and R == pytest.approx(0.7, abs=1e-12)
    m = inputs.cylinder_ogrid(8, n_theta=48, n_r=10, Rc=0.15)
    rho0 = inputs.cylinder_cap_density(m, (0.5, 0.5), 0.15, 0.15, math.radians(60), 0.06)
    th = wetting.contour_angle_on_curved_wall(m.node_xyz, rho0.reshape(m.n_elem, -1), 9, 2,
                                              (0.5, 0.5), 0.15, 0.06, level=0.55)
    assert th == pytest.approx(60, abs=0.5)

