"""Batched stepping: many solves of uneven meshes, orders and angles in one
batch give exactly the same bits as each solve alone (batch invariance), also
when members join and leave mid-run and across autotuning."""
import math

import numpy as np
import pytest

from paper_2609_00535_b300 import inputs
from tests.helpers import assert_matches_oracle, make_case

pytestmark = pytest.mark.gpu


def mix():
    cases = [
        inputs.flat_wall_2d(N=4, ne=(8, 8), theta=math.radians(30)),
        inputs.flat_wall_2d(N=4, ne=(5, 3), theta=math.radians(150)),
        inputs.flat_wall_2d(N=6, ne=(4, 4), theta=math.radians(75)),
        inputs.sphere_3d(N=4, ne=(3, 3, 2), Cn=0.3, theta=math.radians(45)),
        inputs.sphere_3d(N=5, ne=(2, 2, 2), Cn=0.35, theta=math.radians(120)),
        inputs.periodic_droplet(dim=2, ne=3, N=8, Cn=0.25),
    ]
    m = inputs.rotate_elements(inputs.cylinder_ogrid(5, n_theta=12, n_r=2), 3)
    cases.append(make_case("cyl", m, "D2Q9", 1e-2, 0.05, 0.5, math.radians(20),
                           rho0=inputs.droplet_density(m, (0.5, 0.63), 0.04, 0.05)
                           + inputs.node_noise(m, 2, 1e-3)))
    return cases


def _solver(case):
    from paper_2609_00535_b300 import semlbm
    s = semlbm.Solver.from_case(case)
    s.set_density(case.rho0)
    return s


def alone(case, steps):
    s = _solver(case)
    s.step(steps)
    f, k = s.get_state()
    s.close()
    return f


def test_batch_matches_alone_bitwise():
    from paper_2609_00535_b300 import semlbm
    cases = mix()
    b = semlbm.Batch()
    solvers = [_solver(c) for c in cases]
    slots = [b.add(s) for s in solvers]
    assert len(b.info()) == 6            # (D2Q9, 4 5 6 8), (D3Q13, 4 5)
    b.step(25)
    for c, s in zip(cases, solvers):
        f, k = s.get_state()
        assert k == 25
        assert np.array_equal(f, alone(c, 25)), c.name
    d = b.diagnostics()
    for slot, s in zip(slots, solvers):
        assert d[slot]["status"] == 0 and d[slot]["step"] == 25
    b.close()
    for s in solvers:
        s.close()


def test_batch_members_match_oracle():
    """Members of four (velocity set, N) groups, advanced only by the batched
    persistent kernels, element by element against the oracle."""
    from paper_2609_00535_b300 import semlbm
    cases = [inputs.flat_wall_2d(N=6, ne=(4, 4), theta=math.radians(75)),
             inputs.sphere_3d(N=4, ne=(3, 3, 2), Cn=0.3, theta=math.radians(45)),
             inputs.sphere_3d(N=5, ne=(2, 2, 2), Cn=0.35, theta=math.radians(120)),
             inputs.periodic_droplet(dim=2, ne=3, N=8, Cn=0.25)]
    b = semlbm.Batch()
    solvers = [_solver(c) for c in cases]
    for s in solvers:
        b.add(s)
    b.step(60)
    for c, s in zip(cases, solvers):
        f, k = s.get_state()
        assert k == 60
        assert_matches_oracle(c, f, 60)
    b.close()
    for s in solvers:
        s.close()


def test_members_join_and_leave_mid_run():
    from paper_2609_00535_b300 import semlbm
    cases = mix()[:4]
    b = semlbm.Batch()
    s0, s1, s2, s3 = [_solver(c) for c in cases]
    a0 = b.add(s0)
    a1 = b.add(s1)
    b.step(10)
    a2 = b.add(s2)                      # joins an existing group (D2Q9, N=4) ... or a new one
    b.step(10)
    b.remove(a0)                        # leaves after 20 steps
    a3 = b.add(s3)
    b.step(10)
    assert np.array_equal(s0.get_state()[0], alone(cases[0], 20))
    assert np.array_equal(s1.get_state()[0], alone(cases[1], 30))
    assert np.array_equal(s2.get_state()[0], alone(cases[2], 20))
    assert np.array_equal(s3.get_state()[0], alone(cases[3], 10))
    # a removed solver steps on its own again
    s0.step(5)
    assert np.array_equal(s0.get_state()[0], alone(cases[0], 25))
    b.close()
    for s in (s0, s1, s2, s3):
        s.close()


def test_autotune_keeps_results_and_picks_a_candidate():
    from paper_2609_00535_b300 import semlbm
    cases = mix()[:3]
    b = semlbm.Batch()
    solvers = [_solver(c) for c in cases]
    for s in solvers:
        b.add(s)
    b.tune(3)                            # every candidate: 1 + 2 x 2 real steps
    info = b.info()
    total = {}
    for g in info:
        assert g["epb"] in [e for e, _ in g["candidates"]]
        assert all(ms > 0 for _, ms in g["candidates"])
    b.step(4)
    for c, s in zip(cases, solvers):
        f, k = s.get_state()
        assert np.array_equal(f, alone(c, k))
    b.close()
    for s in solvers:
        s.close()


def test_batched_solver_rejects_single_steps_and_large_orders():
    from paper_2609_00535_b300 import semlbm
    b = semlbm.Batch()
    s = _solver(mix()[0])
    b.add(s)
    with pytest.raises(semlbm.SemLbmError):
        s.step(1)
    big = _solver(make_case("n10", inputs.box((2, 2), (0, 0), (1, 1), 10), "D2Q9", 1e-2, 0.3, 0.5,
                            math.pi / 2, rho0=np.full((4, 121), 0.5)))
    with pytest.raises(semlbm.SemLbmError) as ei:
        b.add(big)
    assert ei.value.code == -6
    s.close()                            # destroying a member removes it from its batch
    assert b.info() == []
    b.step(3)                            # empty batch: nothing to do
    big.close()
    b.close()


def test_batch_with_all_3d_sets():
    from paper_2609_00535_b300 import semlbm
    cases = [inputs.sphere_3d(N=4, ne=(2, 2, 2), Cn=0.35, lattice=l)
             for l in ("D3Q13", "D3Q19", "D3Q27")]
    b = semlbm.Batch()
    solvers = [_solver(c) for c in cases]
    for s in solvers:
        b.add(s)
    b.step(12)
    for c, s in zip(cases, solvers):
        assert np.array_equal(s.get_state()[0], alone(c, 12)), c.lattice
    b.close()
    for s in solvers:
        s.close()


def test_batch_with_moving_wall_member():
    from paper_2609_00535_b300 import semlbm
    m = inputs.box((4, 3), (0, 0), (1, 0.8), 4, face_tags={2: 0, 3: 1})
    moving = make_case("lid", m, "D2Q9", 1e-2, 0.25, 0.7, math.radians(60), (math.pi / 2,),
                       rho0=inputs.droplet_density(m, (0.5, 0.0), 0.35, 0.25),
                       wall_velocity={1: (0.02, 0.0)})
    cases = [moving, mix()[0]]            # same (D2Q9, N=4) group, one static
    b = semlbm.Batch()
    solvers = [_solver(c) for c in cases]
    for s in solvers:
        b.add(s)
    b.step(15)
    for c, s in zip(cases, solvers):
        assert np.array_equal(s.get_state()[0], alone(c, 15))
    b.close()
    for s in solvers:
        s.close()


def test_batch_stream_is_not_shared_with_solvers():
    """A batch captures its step on its stream; solvers created meanwhile (on
    other threads, from torch's stream pool, which repeats) never get that stream."""
    import torch
    from paper_2609_00535_b300 import semlbm
    b = semlbm.Batch()
    pooled = {torch.cuda.Stream().cuda_stream for _ in range(80)}
    assert b.stream.cuda_stream not in pooled
    s = _solver(inputs.flat_wall_2d())
    b.add(s)
    b.step(3)
    b.synchronize()
    f, k = s.get_state()
    assert k == 3 and np.array_equal(f, alone(inputs.flat_wall_2d(), 3))
    b.close()
    s.close()
