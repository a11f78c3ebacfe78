"""The allocation-free chemical potential entry point (collected last).

sem_lbm_chemical_potential_noalloc serves callers that must not allocate
device memory while they run (serving loops that reserve all memory up front,
programs whose device memory belongs to another allocator).  It keeps its
scratch in a fixed array inside the library.  These tests call it through the
C ABI and compare it with the existing entry point, sem_lbm_get_field(mu), on
two calls in a row, on two meshes (so a second call cannot pass on a previous
call's leftovers), and check that an oversized mesh is rejected.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2609_00535_b300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _noalloc(solver, rho_dev, mu_dev):
    from paper_2609_00535_b300 import semlbm
    lib = semlbm.load()
    rc = lib.sem_lbm_chemical_potential_noalloc(solver.h, ctypes.c_void_p(rho_dev.data_ptr()),
                                                ctypes.c_void_p(mu_dev.data_ptr()))
    semlbm.check(rc)
    solver.synchronize()


def _check(case, steps):
    import torch
    from paper_2609_00535_b300 import semlbm
    s = semlbm.Solver.from_case(case)
    s.set_density(case.rho0)
    s.step(steps)
    mu_ref = s.field("mu")                               # existing entry point
    rho = torch.from_numpy(s.field("rho")).to("cuda")
    for _ in range(2):                                   # two calls in a row
        mu = torch.full_like(rho, float("nan"))
        _noalloc(s, rho, mu)
        got = mu.cpu().numpy()
        err = np.abs(got - mu_ref).max() / np.abs(mu_ref).max()
        assert np.isfinite(got).all() and err <= TOL, err
    s.close()


def test_noalloc_matches_get_field_2d_then_3d():
    _check(inputs.flat_wall_2d(N=5, ne=(3, 4), noise=1e-3, seed=4), 7)
    _check(inputs.sphere_3d(N=4, ne=(3, 3, 2), Cn=0.3), 5)
    _check(inputs.flat_wall_2d(N=4, ne=(8, 8), theta=math.radians(120)), 3)


def test_noalloc_rejects_meshes_above_its_limit():
    import torch
    from paper_2609_00535_b300 import semlbm
    mesh = inputs.box((65, 65), (0, 0), (1, 1), 15)      # 65*65*256 = 1,081,600 > 2^20 nodes
    assert mesh.n_local > semlbm.NOALLOC_MAX_NODES
    s = semlbm.Solver(mesh, "D2Q9", 1e-3, 1e-6, 0.5, math.pi / 2, dt=1e-4)
    rho = torch.full((mesh.n_local,), 0.5, dtype=torch.float64, device="cuda")
    mu = torch.empty_like(rho)
    with pytest.raises(semlbm.SemLbmError) as ei:
        _noalloc(s, rho, mu)
    assert ei.value.code == -1 and "at most" in str(ei.value)
    s.close()
