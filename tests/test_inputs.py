"""Checks of the seeded input generators (meshes, densities, noise)."""
import math

import numpy as np
import pytest

from paper_2609_00535_b300 import inputs


def _check_ids(mesh, periodic_L=None):
    x = mesh.node_xyz.reshape(-1, mesh.dim)
    g = mesh.global_id.ravel()
    order = np.argsort(g, kind="stable")
    gs, xs = g[order], x[order]
    same = gs[1:] == gs[:-1]
    d = xs[1:][same] - xs[:-1][same]
    if periodic_L is not None:
        L = np.asarray(periodic_L)
        d = d - L * np.round(d / L)
    assert np.abs(d).max(initial=0) < 1e-13
    # distinct ids are distinct points (no unglued copies)
    uniq = np.unique(g)
    first = xs[np.r_[True, ~same]]
    if periodic_L is None:
        key = np.round(first / 1e-9).astype(np.int64)
        assert len(np.unique(key, axis=0)) == len(uniq)


@pytest.mark.parametrize("mk", [
    lambda: inputs.box((3, 2), (0, 0), (1, 1), 4),
    lambda: inputs.rotate_elements(inputs.box((2, 2, 2), (0, 0, 0), (1, 1, 1), 3), 1),
    lambda: inputs.cylinder_ogrid(4, n_theta=8, n_r=2),
    lambda: inputs.rotate_elements(inputs.cylinder_ogrid(5, n_theta=8, n_r=2), 3),
    lambda: inputs.sphere_cap_box(3, ne=(2, 3, 2)),
])
def test_shared_ids_are_shared_points(mk):
    _check_ids(mk())


def test_periodic_ids():
    m = inputs.box((3, 2), (0, 0), (1.5, 1.0), 4, periodic=(True, True))
    _check_ids(m, periodic_L=(1.5, 1.0))
    assert len(np.unique(m.global_id)) == 12 * 8
    assert m.face_kind.sum() == 0


def test_rotation_preserves_geometry_and_walls():
    m = inputs.box((2, 2), (0, 0), (1, 1), 4, face_tags={2: 0})
    r = inputs.rotate_elements(m, 5)
    for e in range(m.n_elem):
        a = np.sort(m.node_xyz[e].round(12).view("f8,f8").ravel())
        b = np.sort(r.node_xyz[e].round(12).view("f8,f8").ravel())
        assert (a == b).all()
        # same multiset of (kind, tag) over the faces
        assert sorted(zip(m.face_kind[e], m.face_tag[e])) == sorted(zip(r.face_kind[e], r.face_tag[e]))


def test_noise_is_seeded_and_keyed_by_global_id():
    m = inputs.box((2, 2), (0, 0), (1, 1), 4)
    a = inputs.node_noise(m, 7, 1e-3)
    b = inputs.node_noise(m, 7, 1e-3)
    c = inputs.node_noise(m, 8, 1e-3)
    assert (a == b).all() and not (a == c).all()
    assert np.abs(a).max() <= 1e-3
    g = m.global_id.ravel()
    av = a.ravel()
    for gid in np.unique(g)[:50]:
        assert np.ptp(av[g == gid]) == 0.0
    # SplitMix64 reference value: state 0 -> 0xE220A8397B1DCDAF (first output, seed 0)
    assert int(inputs.splitmix64(np.array([0], dtype=np.uint64))[0]) == 0xE220A8397B1DCDAF


def test_configs_shapes():
    c1 = inputs.flat_wall_2d()
    assert c1.nodes == 1600 and c1.mesh.n_elem == 64
    c2 = inputs.cylinder_2d()
    assert c2.mesh.n_elem == 1024 and c2.nodes == 1024 * 49
    assert abs(c1.kappa - 1e-3 * 0.125 ** 2 * 0.81 / 8) < 1e-18


def test_equilibrium_cap_shapes():
    import math
    m = inputs.box((8, 4), (0, 0), (2, 1), 6)
    area = 0.5 * math.pi * 0.25 ** 2
    for deg in (30, 90, 150):
        th = math.radians(deg)
        R = inputs.cap_radius(area, th)
        # the cap holds the requested area above the wall
        assert abs(R * R * (th - math.sin(th) * math.cos(th)) - area) < 1e-15
        rho = inputs.sessile_cap_density(m, 1.0, area, th, 0.02)
        assert rho.max() > 0.99 and rho.min() < 0.11
    assert abs(inputs.cap_radius(area, math.pi / 2) - 0.25) < 1e-15     # half disc
    # on a cylinder at 90 degrees the drop circle is orthogonal to the wall
    mc = inputs.cylinder_ogrid(4, n_theta=16, n_r=2)
    r = inputs.cylinder_cap_density(mc, (0.5, 0.5), 0.1, 0.05, math.pi / 2, 0.01)
    assert r.shape == mc.global_id.shape


def test_converging_request_stream():
    reqs = inputs.converging_request_stream(n=20, rate=10.0, seed=3)
    assert [r.rid for r in reqs] == list(range(20))
    assert all(b.arrival > a.arrival for a, b in zip(reqs, reqs[1:]))
    for r in reqs[:4]:
        c = r.case()
        assert c.name.startswith("boxdrop2d") and c.lattice == "D2Q9" and c.theta_tag == ()
        assert (c.mesh.face_kind == 1).sum() == 4 * int(round(math.sqrt(r.E))) and c.dt > 1e-3
        assert abs(c.rho0.max() - c.rho_l) < 1e-3 and abs(c.rho0.min() - c.rho_v) < 1e-3


def test_generator_defaults_match_the_paper():
    """The workload generators default to the parameters the paper prints
    (tests/golden/paper_values.json, each entry with its citation)."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    iso, sph = gold["isolated_droplet"], gold["sphere"]
    c = inputs.periodic_droplet()
    assert (c.rho_l, c.rho_v) == (gold["densities"]["rho_l"], gold["densities"]["rho_v"])
    assert c.tau == iso["tau"] and c.beta == iso["beta"] and c.mesh.N != 0
    assert c.extra["R"] * 2 == iso["D"] and c.extra["delta"] == pytest.approx(iso["Cn"] * iso["D"])
    assert np.ptp(c.mesh.node_xyz[..., 0]) == pytest.approx(iso["L"])
    s = inputs.sphere_3d(ne=(2, 2, 2))
    assert s.extra["La"] == sph["La"] and s.extra["delta"] == pytest.approx(sph["Cn"] * sph["drop_d"])
    x = s.mesh.node_xyz.reshape(-1, 3)
    assert np.ptp(x[:, 0]) == pytest.approx(sph["box"][0]) and np.ptp(x[:, 1]) == pytest.approx(sph["box"][1])
    assert x[:, 2].max() == pytest.approx(sph["box"][2])
    top = x[np.argmin(np.hypot(x[:, 0] - 0.25, x[:, 1] - 0.25))]          # sphere top under the drop
    assert top[2] == pytest.approx(0.0, abs=1e-12)
    n = s.mesh.N + 1
    wall = s.mesh.node_xyz[s.mesh.face_kind[:, 4] == 1][:, :n * n].reshape(-1, 3)   # l = 0 face nodes
    r = np.linalg.norm(wall - [0.25, 0.25, -sph["sphere_D"] / 2], axis=1)
    assert len(wall) > 0 and np.allclose(r, sph["sphere_D"] / 2, atol=1e-12)


def test_relaxing_request_stream():
    """The serving stream run to a KE threshold: a quarter each of flat-wall,
    cylinder and sphere-wall caps and periodic drops, sizes in each kind's
    range, the potential-part force reading, and tau from the viscous-time rule."""
    reqs = inputs.relaxing_request_stream(n=40, rate=10.0, seed=8)
    assert all(b.arrival > a.arrival for a, b in zip(reqs, reqs[1:]))
    kinds = [r.kind for r in reqs]
    assert kinds.count("relaxflat2d") == kinds.count("relaxcyl2d") == kinds.count("relaxsphere3d") == 10
    assert kinds.count("relaxdrop2d") + kinds.count("relaxdrop3d") == 10
    for r in reqs[:8]:
        lo, hi = inputs.RELAX_SIZES[r.kind]
        assert lo <= r.E <= hi
        c = r.case()
        assert c.force_split == 1 and c.beta == 0.1 and c.tau >= 1.0
        assert c.lattice == ("D3Q13" if r.kind.endswith("3d") else "D2Q9")
        assert c.tau == pytest.approx(max(1.0, inputs.viscous_tau(c.dt, 1.0 if "flat" in r.kind or "drop" in r.kind
                                                                  else (0.35 if "cyl" in r.kind else 0.5))))
        assert c.rho0.max() > 0.85 and abs(c.rho0.min() - c.rho_v) < 2e-3   # a drop in vapour
    assert inputs.viscous_tau(0.01, 1.0, steps=1e4) == pytest.approx(3.0)
    assert inputs.viscous_tau(0.1, 1.0) == 1.0
    assert inputs.viscous_tau(1e-3, 1.0) == 10.0          # capped


def test_kelvin_shifted_starts():
    """Saturated starts put both bulk phases at the Kelvin shift of the drop's
    radius: the equilibrium cap's circle for the flat-wall drop, the drop radius
    for the relaxing kinds."""
    import math
    c0 = inputs.cap_on_wall_2d(math.radians(60))
    c1 = inputs.cap_on_wall_2d(math.radians(60), saturate=True)
    R = inputs.cap_radius(0.5 * math.pi * 0.25 ** 2, math.radians(60))
    dr = inputs.kelvin_shift(c1.beta, c1.kappa, c1.rho_l, c1.rho_v, R, 2)
    assert dr > 0
    assert np.allclose(c1.rho0 - dr, c0.rho0, atol=1e-14)
    c = inputs.relaxing_case("relaxsphere3d", 27, 4, math.radians(90), saturate=True)
    assert c.extra["kelvin_shift"] == pytest.approx(
        inputs.kelvin_shift(c.beta, c.kappa, c.rho_l, c.rho_v, 0.13, 3))
    assert inputs.relaxing_case("relaxsphere3d", 27, 4, math.radians(90)).extra["kelvin_shift"] == 0
    req = inputs.angle_sweep_stream(n=2)[0]
    assert req.saturate and req.case().rho0.min() > req.case().rho_v + 1e-3

