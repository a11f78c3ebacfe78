"""The allocation-free chemical potential entry point (collected last).

sem_lbm_chemical_potential_noalloc serves callers that must not allocate
device memory while they run (serving loops that reserve all memory up front,
programs whose device memory belongs to another allocator).  It keeps its
scratch in a fixed array inside the library.  These tests call it through the
C ABI and compare it with the existing entry point, sem_lbm_get_field(mu), on
two calls in a row, on three meshes (so a later call cannot pass on an earlier
call's leftovers).  Both paths run the same Laplacian and gather-scatter
kernels on the same density, so the results must agree bit for bit.  They
also check that, once the library is loaded on the device, a call changes the
device's free memory by nothing, and that an oversized mesh is rejected.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2609_00535_b300 import inputs

pytestmark = pytest.mark.gpu


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
    outs = [torch.full_like(rho, float("nan")) for _ in range(2)]
    _noalloc(s, rho, outs[0])                            # loads the library's array on first use
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for mu in outs:                                      # two calls in a row
        mu.fill_(float("nan"))
        _noalloc(s, rho, mu)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0         # no device memory taken
    for mu in outs:
        got = mu.cpu().numpy()
        assert np.isfinite(got).all() and np.array_equal(got, mu_ref)
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
