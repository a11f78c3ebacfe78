"""Linear stability of a periodic drop at rest under the two force readings of
the collision's F** (Sec. 2.1), from the Jacobian of one oracle step.

A drop at rest is a fixed point of the step under both readings (F** is
proportional to u).  Linearised there, F** couples the velocity disturbance to
the equilibrium force F_eq: c_s^2 grad(rho_eq) under the printed force, zero
under its potential part -rho grad(mu) (force_split = 1).  On a small drop the
printed reading has eigenvalues above 1 (the disturbance grows), and the
growth per step scales like dt^2 (so per unit time like dt: a splitting effect
of collision and streaming that vanishes as dt -> 0); the potential-part
reading has spectral radius 1 (the conserved mass and momentum), so the drop
relaxes to its equilibrium.
"""
import math

import numpy as np
import pytest

from oracle import linear_stability as ls
from paper_2609_00535_b300 import inputs
from tests.helpers import oracle_of


def _drop(cfl):
    # 2x2 elements at N = 4 (an 8x8-node periodic box), drop diameter 0.6
    return inputs.periodic_droplet(dim=2, ne=2, N=4, D=0.6, Cn=0.2, beta=0.1, tau=1.0, cfl=cfl)


@pytest.fixture(scope="module")
def drop_at_rest():
    case = _drop(0.4)
    om, orc = oracle_of(case, force_split=1)
    f = orc.initial_state(case.rho0.reshape(om.shape))
    f = orc.run(f, 1500)
    assert orc.diagnostics(f)["ke_max"] < 1e-15
    return f


def _spectral_radius(cfl, force_split, f):
    om, orc = oracle_of(_drop(cfl), force_split=force_split)
    J = ls.jacobian(orc, f)
    return np.abs(np.linalg.eigvals(J)).max(), orc.p.dt


def test_global_state_round_trip(drop_at_rest):
    om, _ = oracle_of(_drop(0.4))
    f = drop_at_rest
    assert np.array_equal(ls.to_local(om, ls.to_global(om, f)), f)


def test_potential_part_reading_is_neutrally_stable(drop_at_rest):
    rho1, _ = _spectral_radius(0.4, 1, drop_at_rest)
    assert abs(rho1 - 1.0) < 1e-8, rho1


def test_printed_force_grows_like_dt_squared(drop_at_rest):
    rho_a, dt_a = _spectral_radius(0.4, 0, drop_at_rest)
    rho_b, dt_b = _spectral_radius(0.2, 0, drop_at_rest)
    assert rho_a > 1.01 and rho_b > 1.0, (rho_a, rho_b)
    ratio = math.log(rho_b) / math.log(rho_a)
    assert abs(ratio / (dt_b / dt_a) ** 2 - 1.0) < 0.3, ratio
