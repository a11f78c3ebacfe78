"""Serving: requests admitted while others run produce exactly the results
they produce alone."""
import math

import numpy as np
import pytest

from paper_2609_00535_b300 import inputs
from paper_2609_00535_b300.serve import Server
from tests.helpers import assert_matches_oracle

pytestmark = pytest.mark.gpu


def test_continuous_batching_equals_alone():
    from paper_2609_00535_b300 import semlbm
    kinds = ["flat2d", "cylinder2d", "sphere3d", "droplet2d", "droplet3d", "flat2d"]
    # arrivals 20 ms apart, each request 600 steps: several are on the GPU at once
    reqs = [inputs.Request(i, 0.02 * i, k, 64 if "3d" in k else 96, 4 + i % 3,
                           math.radians(20 + 25 * i), 1.0, 1000 + i) for i, k in enumerate(kinds)]
    srv = Server(hbm_budget_bytes=4 << 30, epoch_steps=20, ke_tol=0.0, max_steps=600,
                 min_steps=20, keep_state=True, workers=3)
    st = srv.run(reqs)
    summ = st.summary()
    assert summ["completed"] == len(reqs) and summ["failed"] == 0
    assert summ["max_slots"] >= 2 and summ["overlapped_admissions"] >= 1
    for req, rec in zip(reqs, st.records):
        assert rec.steps >= 600 and rec.state is not None
        case = req.case()
        s = semlbm.Solver.from_case(case)
        s.set_density(case.rho0)
        s.step(rec.steps)
        assert np.array_equal(s.get_state()[0], rec.state), rec.name
        s.close()


def test_served_requests_match_oracle():
    """Requests served side by side (three kinds, three orders), each result
    element by element against the oracle run of the same request."""
    kinds = ["flat2d", "sphere3d", "droplet2d"]
    reqs = [inputs.Request(i, 0.02 * i, k, 27 if "3d" in k else 36, 4 + i, math.radians(40 + 35 * i),
                           1.0, 77 + i) for i, k in enumerate(kinds)]
    srv = Server(hbm_budget_bytes=2 << 30, epoch_steps=20, ke_tol=0.0, max_steps=80,
                 min_steps=20, keep_state=True, workers=3)
    st = srv.run(reqs)
    assert st.summary()["completed"] == len(reqs)
    for req, rec in zip(reqs, st.records):
        assert rec.steps >= 80 and rec.state is not None
        assert_matches_oracle(req.case(), rec.state, rec.steps)


def test_budget_limits_concurrent_slots():
    reqs = [inputs.Request(i, 0.0, "flat2d", 64, 4, math.radians(60), 1.0, i) for i in range(4)]
    from paper_2609_00535_b300 import semlbm
    one = semlbm.workspace_bytes(reqs[0].case().mesh, 4, "D2Q9")
    st = Server(hbm_budget_bytes=int(1.5 * one), epoch_steps=10, ke_tol=0.0, max_steps=30,
                min_steps=10).run(reqs)
    assert st.summary()["completed"] == 4 and st.max_slots == 1


def test_requests_run_to_convergence():
    """Closed-box drops relax to KE_max < 1e-20; each retires on convergence,
    not on the step cap, and its final state is the one it reaches alone."""
    from paper_2609_00535_b300 import semlbm
    reqs = inputs.converging_request_stream(n=4, rate=50.0, seed=9, shapes=((6, 4),))
    st = Server(hbm_budget_bytes=2 << 30, epoch_steps=500, ke_tol=1e-20, max_steps=60000,
                min_steps=1000, keep_state=True).run(reqs)
    summ = st.summary()
    assert summ["completed"] == 4 and summ["converged"] == 4, summ
    for req, rec in zip(reqs, st.records):
        assert rec.ke_max < 1e-20 and rec.steps < 60000
        case = req.case()
        s = semlbm.Solver.from_case(case)
        s.set_density(case.rho0)
        s.step(rec.steps)
        assert np.array_equal(s.get_state()[0], rec.state), rec.name
        assert s.diagnostics()["ke_max"] < 1e-20
        s.close()


def test_relaxing_requests_converge():
    """One request of each relaxing kind (flat wall, cylinder, sphere wall,
    periodic drop 2D and 3D), served together, each retires on KE_max < 1e-20
    within its step budget; the served state of the first equals its solo run."""
    from paper_2609_00535_b300 import semlbm
    kinds = [("relaxflat2d", 32), ("relaxcyl2d", 72), ("relaxsphere3d", 27), ("relaxdrop2d", 16),
             ("relaxdrop3d", 27)]
    reqs = [inputs.Request(i, 0.01 * i, k, E, 4, math.radians(60 + 20 * i), 1.0, 300 + i)
            for i, (k, E) in enumerate(kinds)]
    st = Server(hbm_budget_bytes=2 << 30, epoch_steps=1000, ke_tol=1e-20, max_steps=200000,
                min_steps=1000, keep_state=True).run(reqs)
    summ = st.summary()
    assert summ["completed"] == 5 and summ["converged"] == 5, [(r.name, r.steps, r.ke_max)
                                                               for r in st.records]
    rec = st.records[0]
    case = reqs[0].case()
    s = semlbm.Solver.from_case(case)
    s.set_density(case.rho0)
    s.step(rec.steps)
    assert np.array_equal(s.get_state()[0], rec.state)
    assert s.diagnostics()["ke_max"] < 1e-20
    s.close()
