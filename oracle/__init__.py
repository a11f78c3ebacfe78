"""Plain, slow FP64 CPU oracle of the SEM-LBM wetting step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It restates, step by step and in the paper's order, the method of
"Spectral element lattice Boltzmann method for non-ideal gases with partial
wetting boundary condition" (Zhao, Patel, Lee):

* ``gll``       Gauss-Lobatto-Legendre nodes, weights and the Lagrange
                derivative matrix (the discretisation that Sec. 2.1 defers
                to Deville et al.).
* ``lattice``   D2Q9 (Sec. 2.1) and the 13-velocity 3D set (Sec. 3.2).
* ``geometry``  isoparametric metrics, mass, wall-face area vectors and the
                direct-stiffness (gather-scatter) sum, by global node id.
* ``method``    Eq. (chemi), Eq. (weak), the forcing and its split
                (Sec. 2.1), collision, the force-split streaming equation
                (Sec. 3.3), flux bounce-back (Sec. 2.2, Eq. 9), SSP-RK3 and
                the diagnostics of Sec. 3.3.

It shares no code with the CUDA library: it recomputes every table, metric and
gather-scatter map from the raw mesh arrays by its own route.  Only the seeded
input generators (mesh + initial density) are shared, and those hold none of
the method's arithmetic.

Parity status per function is recorded in each module's header; every function
is pinned by a ``-m "not gpu"`` test except where a header says
"parity unpinned".
"""
