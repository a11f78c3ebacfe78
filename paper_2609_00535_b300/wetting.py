"""Static contact angle of a sessile drop from the wetting moments that the
library integrates on the device (sem_lbm_wetting_moments): on a flat wall (the
cap relations below) or on a circular cylinder / sphere (the lens geometry of
curved_cap, further down).

A drop at equilibrium on a flat wall is a circular cap (2D) or a spherical cap
(3D) meeting the wall at the contact angle theta measured through the liquid
(Sec. 3.1).  The moments give the cap's size two ways: the liquid area/volume
int phi dV and the wetted wall measure int_wall phi dS (the cap's base: length
2b in 2D, area pi b^2 in 3D).  Their scale-free ratio is a monotone function of
theta alone, inverted here by bisection:

  2D  area / b^2      = (theta - sin theta cos theta) / sin^2 theta
  3D  V / A_w^(3/2)   = (1 - cos theta)^2 (2 + cos theta) / (3 sqrt(pi) sin^3 theta)

Diffuse interfaces: for the tanh profile of width delta (Appendix A) the
liquid fraction phi = 1/(1 + exp(4 s / delta)) (s the signed distance) integrates
across a curved interface to the sharp value plus (pi^2/6)(delta/4)^2 times the
integral of the summed principal curvatures over the interface (the Sommerfeld
expansion; no odd terms, since phi - 1/2 is odd in s).  For a cap of radius R
that adds pi^2 delta^2 theta / 48 to the 2D area, pi^3 delta^2 R (1 - cos theta) / 24
to the 3D volume, and pi^3 (delta / sin theta)^2 / 48 to the 3D wetted area (the
contact circle, crossed at angle theta); the 2D wetted length has no correction.
With delta > 0 these are removed by a fixed-point iteration.

A second, independent estimate on curved walls fits a circle (2D) or sphere (3D)
to the density contour halfway between the phases, away from the wall, and takes
the angle between it and the wall (contour_angle_on_curved_wall).
"""
import math

import numpy as np


def _bisect(fn, target, lo=1e-9, hi=math.pi - 1e-9, iters=200):
    """theta in (lo, hi) with fn(theta) = target, fn increasing."""
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if fn(mid) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _g2(t):
    return (t - math.sin(t) * math.cos(t)) / math.sin(t) ** 2


def _g3(t):
    c, s = math.cos(t), math.sin(t)
    return (1 - c) ** 2 * (2 + c) / (3 * math.sqrt(math.pi) * s ** 3)


def cap_angle_2d(area, wetted, delta=0.0, iters=20):
    """Contact angle (radians) of a 2D circular cap from its liquid area and its
    wetted wall length 2b."""
    b = 0.5 * wetted
    theta = _bisect(_g2, area / b ** 2)
    for _ in range(iters if delta > 0 else 0):
        theta = _bisect(_g2, (area - math.pi ** 2 * delta ** 2 * theta / 48) / b ** 2)
    return theta


def cap_angle_3d(volume, wetted, delta=0.0, iters=20):
    """Contact angle (radians) of a 3D spherical cap from its liquid volume and its
    wetted wall area pi b^2."""
    theta = _bisect(_g3, volume / wetted ** 1.5)
    for _ in range(iters if delta > 0 else 0):
        s = math.sin(theta)
        aw = wetted - math.pi ** 3 * (delta / s) ** 2 / 48
        if aw <= 0:      # contact circle no wider than the interface: no correction
            return _bisect(_g3, volume / wetted ** 1.5)
        R = math.sqrt(aw / math.pi) / s
        v = volume - math.pi ** 3 * delta ** 2 * R * (1 - math.cos(theta)) / 24
        theta = _bisect(_g3, v / aw ** 1.5)
    return theta


# ---------------------------------------------------------------------------
# Curved walls: a drop of radius Rd on a cylinder (2D) or sphere (3D) of radius
# Rw, centres a distance d apart with d^2 = Rw^2 + Rd^2 - 2 Rw Rd cos(theta)
# (the equilibrium position used by inputs.cylinder_cap_density).  The liquid
# volume is the drop's disc/ball minus the lens it shares with the wall body;
# the wetted measure is the wall's arc/cap inside the drop.
# ---------------------------------------------------------------------------
def _half_angles(Rw, Rd, d):
    ca = max(-1.0, min(1.0, (Rw * Rw + d * d - Rd * Rd) / (2 * Rw * d)))
    cb = max(-1.0, min(1.0, (Rd * Rd + d * d - Rw * Rw) / (2 * Rd * d)))
    return math.acos(ca), math.acos(cb)


def curved_cap(Rw, Rd, theta, dim):
    """(liquid volume, wetted measure) of a sharp drop of radius Rd meeting a
    wall of radius Rw at the angle theta."""
    d = math.sqrt(Rw * Rw + Rd * Rd - 2 * Rw * Rd * math.cos(theta))
    a, b = _half_angles(Rw, Rd, d)
    if dim == 2:
        lens = Rw * Rw * a + Rd * Rd * b - d * Rw * math.sin(a)
        return math.pi * Rd * Rd - lens, 2 * Rw * a
    hw, hd = Rw * (1 - math.cos(a)), Rd * (1 - math.cos(b))
    lens = math.pi * hw * hw * (3 * Rw - hw) / 3 + math.pi * hd * hd * (3 * Rd - hd) / 3
    return 4 * math.pi * Rd ** 3 / 3 - lens, 2 * math.pi * Rw * hw


def _excess(Rw, Rd, theta, dim, delta):
    """Diffuse-interface excess of the volume and of the wetted measure (the
    Sommerfeld term over the drop's free surface; the contact line as on a flat
    wall)."""
    if delta <= 0:
        return 0.0, 0.0
    d = math.sqrt(Rw * Rw + Rd * Rd - 2 * Rw * Rd * math.cos(theta))
    _, b = _half_angles(Rw, Rd, d)
    if dim == 2:
        return math.pi ** 2 * delta ** 2 * 2 * (math.pi - b) / 96, 0.0
    hd = Rd * (1 - math.cos(b))
    dv = math.pi ** 2 * delta ** 2 * (8 * math.pi * Rd - 4 * math.pi * hd) / 96
    return dv, math.pi ** 3 * (delta / math.sin(theta)) ** 2 / 48


def cap_angle_on_curved_wall(volume, wetted, Rw, dim, delta=0.0, iters=20):
    """Contact angle (radians) of a drop on a circular cylinder (2D) or a sphere
    (3D) of radius Rw from its liquid volume and wetted measure: for each trial
    angle the drop radius that holds the volume is found by bisection, and the
    angle is bisected on the wetted measure (which falls as theta grows)."""
    def size_for(theta, vol):
        lo, hi = 1e-9, 1e3 * (Rw + vol)
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if curved_cap(Rw, mid, theta, dim)[0] < vol:
                lo = mid
            else:
                hi = mid
        return 0.5 * (lo + hi)

    vol, wet = volume, wetted
    theta = math.pi / 2
    for _ in range(iters if delta > 0 else 1):
        lo, hi = 1e-6, math.pi - 1e-6
        for _ in range(100):
            mid = 0.5 * (lo + hi)
            if curved_cap(Rw, size_for(mid, vol), mid, dim)[1] > wet:
                lo = mid
            else:
                hi = mid
        theta = 0.5 * (lo + hi)
        dv, dw = _excess(Rw, size_for(theta, vol), theta, dim, delta)
        vol, wet = volume - dv, wetted - dw
    return theta


def _check(volume, base):
    if not (volume > 0 and base > 0):
        raise ValueError("no drop on the wall (volume %g, wetted %g)" % (volume, base))


def contact_angle(moments, dim, delta=0.0, wall_radius=None):
    """Degrees, from the liquid volume and wetted measure of Solver.wetting_moments:
    a flat wall, or with wall_radius a cylinder (2D) or sphere (3D) of that
    radius."""
    if wall_radius is not None:
        _check(moments["volume"], moments["wetted"])
        return math.degrees(cap_angle_on_curved_wall(moments["volume"], moments["wetted"],
                                                     wall_radius, dim, delta))
    _check(moments["volume"], moments["wetted"])
    f = cap_angle_2d if dim == 2 else cap_angle_3d
    return math.degrees(f(moments["volume"], moments["wetted"], delta))


def contour_points(xyz, rho, level, n, dim):
    """Crossings of rho = level along the element-local GLL lines of every
    element, by linear interpolation between neighbouring nodes.  xyz is
    [E, n^dim, dim] and rho [E, n^dim] (nodes i fastest); returns [P, dim]."""
    E = rho.shape[0]
    R = np.asarray(rho).reshape((E,) + (n,) * dim)
    X = np.asarray(xyz).reshape((E,) + (n,) * dim + (dim,))
    pts = []
    for ax in range(1, dim + 1):
        a = np.moveaxis(R, ax, -1)
        xa = np.moveaxis(X, ax, -2)
        at = np.nonzero((a[..., :-1] - level) * (a[..., 1:] - level) < 0)
        nxt = at[:-1] + (at[-1] + 1,)
        t = (level - a[at]) / (a[nxt] - a[at])
        pts.append(xa[at] + t[:, None] * (xa[nxt] - xa[at]))
    return np.vstack(pts)


def fit_sphere(p):
    """Least-squares circle (2D) or sphere (3D) through the points p [P, dim]:
    |x|^2 = 2 c.x + (R^2 - |c|^2) is linear in c and the constant.  Returns
    (centre, radius)."""
    A = np.c_[2 * p, np.ones(len(p))]
    sol = np.linalg.lstsq(A, (p ** 2).sum(1), rcond=None)[0]
    c = sol[:-1]
    return c, math.sqrt(sol[-1] + c @ c)


def contour_angle_on_curved_wall(xyz, rho, n, dim, wall_center, Rw, exclude, level=None):
    """Contact angle (degrees) of a drop on a circular (2D) or spherical (3D) wall
    of radius Rw from the contour rho = level (default: halfway between the
    smallest and largest density): the points farther than Rw + exclude from the
    wall centre are fitted with a circle/sphere of centre c and radius Rd, and
    cos(theta) = (Rw^2 + Rd^2 - |c - wall_center|^2) / (2 Rw Rd)."""
    rho = np.asarray(rho)
    if level is None:
        level = 0.5 * (float(rho.min()) + float(rho.max()))
    p = contour_points(xyz, rho, level, n, dim)
    wc = np.asarray(wall_center, dtype=np.float64)
    p = p[np.linalg.norm(p - wc, axis=1) > Rw + exclude]
    if len(p) < dim + 1:
        raise ValueError("no drop contour away from the wall")
    c, Rd = fit_sphere(p)
    d2 = float((c - wc) @ (c - wc))
    return math.degrees(math.acos(max(-1.0, min(1.0, (Rw * Rw + Rd * Rd - d2) / (2 * Rw * Rd)))))

