"""Failure detection without a GPU fault: the failures are made on the host.

A NaN planted in a solve's host-written initial density must surface as the
solve's status SEMLBM_ENONFINITE (set by the gather-scatter/RK kernel's
non-finite flag, not by a trap), leave the CUDA context usable, and stay
confined to its own slot in a batch and to its own request in the server.  A
request that cannot be built (an order the library does not compile) fails
alone at admission.
"""
import math

import numpy as np
import pytest

from paper_2609_00535_b300 import inputs
from paper_2609_00535_b300.serve import Server

pytestmark = pytest.mark.gpu

ENONFINITE = -4


def _poison(case):
    case.rho0 = np.array(case.rho0, dtype=np.float64, copy=True)
    case.rho0.reshape(-1)[case.rho0.size // 2] = np.nan
    return case


def _solver(case):
    from paper_2609_00535_b300 import semlbm
    s = semlbm.Solver.from_case(case)
    s.set_density(case.rho0)
    return s


def test_nonfinite_state_is_reported_and_the_context_survives():
    s = _solver(_poison(inputs.flat_wall_2d()))
    s.step(5)
    d = s.diagnostics()
    assert d["status"] == ENONFINITE and d["n_nonfinite"] > 0
    s.close()
    ok = _solver(inputs.flat_wall_2d())        # the context still runs a healthy solve
    ok.step(5)
    assert ok.diagnostics()["status"] == 0
    ok.close()


def test_nonfinite_member_is_confined_to_its_slot():
    from paper_2609_00535_b300 import semlbm
    cases = [inputs.flat_wall_2d(), _poison(inputs.flat_wall_2d(theta=math.radians(45))),
             inputs.sphere_3d(N=4, ne=(3, 3, 2), Cn=0.3)]
    solvers = [_solver(c) for c in cases]
    b = semlbm.Batch()
    slots = [b.add(s) for s in solvers]
    b.step(6)
    diag = b.diagnostics()
    assert diag[slots[1]]["status"] == ENONFINITE
    for i in (0, 2):
        assert diag[slots[i]]["status"] == 0
        alone = _solver(cases[i])
        alone.step(6)
        assert np.array_equal(alone.get_state()[0], solvers[i].get_state()[0])
        alone.close()
    b.close()
    for s in solvers:
        s.close()


class _PoisonedRequest(inputs.Request):
    def case(self):
        return _poison(super().case())


def test_server_fails_only_the_broken_requests():
    reqs = [inputs.Request(0, 0.0, "flat2d", 64, 4, math.radians(60), 1.0, 1),
            _PoisonedRequest(1, 0.0, "flat2d", 64, 4, math.radians(60), 1.0, 2),
            inputs.Request(2, 0.0, "flat2d", 64, 20, math.radians(60), 1.0, 3),   # N not built
            inputs.Request(3, 0.01, "droplet2d", 16, 5, math.radians(90), 1.0, 4)]
    st = Server(hbm_budget_bytes=1 << 30, epoch_steps=10, ke_tol=0.0, max_steps=30,
                min_steps=10).run(reqs)
    by = {r.rid: r for r in st.records}
    summ = st.summary()
    assert summ["completed"] == 4 and summ["failed"] == 2, summ
    assert by[1].failed and "status %d" % ENONFINITE in by[1].error
    assert by[2].failed and by[2].steps == 0 and by[2].error
    assert not by[0].failed and not by[3].failed and by[0].steps >= 30 and by[3].steps >= 30


def test_cancelled_requests_leave_the_others_unchanged():
    """One request withdrawn before it arrives (never built), one withdrawn while
    it runs (retired at the next epoch); the rest run as they would alone."""
    import threading
    from paper_2609_00535_b300 import semlbm
    reqs = [inputs.Request(i, 0.3 if i == 1 else 0.0, "flat2d", 64, 4, math.radians(40 + 10 * i),
                           1.0, 10 + i) for i in range(4)]
    srv = Server(hbm_budget_bytes=1 << 30, epoch_steps=500, ke_tol=0.0, max_steps=40000,
                 min_steps=500, keep_state=True)
    srv.cancel(1)
    timer = threading.Timer(0.5, srv.cancel, args=(2,))
    timer.start()
    st = srv.run(reqs)
    timer.join()
    by = {r.rid: r for r in st.records}
    assert st.summary()["cancelled"] == 2 and st.summary()["failed"] == 0
    assert by[1].cancelled and by[1].steps == 0
    assert by[2].cancelled and 0 < by[2].steps < 40000
    for rid in (0, 3):
        r = by[rid]
        assert not r.cancelled and r.steps >= 40000
        case = reqs[rid].case()
        s = semlbm.Solver.from_case(case)
        s.set_density(case.rho0)
        s.step(r.steps)
        assert np.array_equal(s.get_state()[0], r.state)
        s.close()
