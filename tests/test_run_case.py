"""Argument handling of the long-run command (run_case): each --case builds the
workload its options describe; bad options are rejected before any GPU work."""
import math

import pytest

from paper_2609_00535_b300 import run_case


def _case(*argv):
    args = run_case.parse_args(list(argv))
    c = run_case.make(args)
    c.force_split = args.force_split
    return c


def test_defaults_are_the_flat_wall_drop():
    c = _case()
    assert c.lattice == "D2Q9" and c.mesh.N == 4 and c.mesh.n_elem == 64
    assert c.theta_w == pytest.approx(math.radians(60)) and c.force_split == 0


@pytest.mark.parametrize("argv,dim,lattice,N,E", [
    (("--case", "flat2d", "--ne", "6", "--N", "5"), 2, "D2Q9", 5, 36),
    (("--case", "capwall2d", "--ne", "5", "--theta", "30"), 2, "D2Q9", 4, 50),
    (("--case", "droplet2d", "--ne", "3", "--N", "6"), 2, "D2Q9", 6, 9),
    (("--case", "droplet3d", "--ne", "2", "--N", "3"), 3, "D3Q13", 3, 8),
    (("--case", "sphere3d", "--ne", "2", "--N", "3"), 3, "D3Q13", 3, 8),
    (("--case", "cylinder2d", "--N", "3"), 2, "D2Q9", 3, 1024),
])
def test_each_case_builds_its_mesh(argv, dim, lattice, N, E):
    c = _case(*argv)
    assert (c.mesh.dim, c.lattice, c.mesh.N, c.mesh.n_elem) == (dim, lattice, N, E)
    assert c.rho0.shape == c.mesh.global_id.shape


def test_droplet_options_reach_the_case():
    c = _case("--case", "droplet2d", "--ne", "4", "--N", "8", "--beta", "0.01", "--tau", "0.8",
              "--Cn", "0.1", "--cfl", "0.2", "--force-split", "1")
    assert c.beta == 0.01 and c.tau == 0.8 and c.force_split == 1
    ref = _case("--case", "droplet2d", "--ne", "4", "--N", "8", "--beta", "0.01", "--tau", "0.8",
                "--Cn", "0.1", "--cfl", "0.4")
    assert c.dt < ref.dt                  # the smaller CFL number gives the smaller step


@pytest.mark.parametrize("argv", [("--case", "nosuch"), ("--force-split", "2"), ("--steps", "0"),
                                  ("--every", "-5")])
def test_bad_options_are_rejected(argv):
    with pytest.raises(SystemExit):
        run_case.parse_args(list(argv))
