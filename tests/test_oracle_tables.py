"""Pins of the oracle's tables and pointwise formulas against closed forms.

GLL tables (Deville-Fischer-Mund closed forms), the velocity-set moments, the
free-energy relations of Appendix A, the equilibrium and force moments of
Sec. 2.1 / Appendix A, and SSP-RK3 on a linear ODE.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as L

from oracle import gll, lattice, method


def test_gll_closed_forms():
    x, w, _ = gll.tables(2)
    np.testing.assert_allclose(x, [-1, 0, 1], atol=1e-16)
    np.testing.assert_allclose(w, [1 / 3, 4 / 3, 1 / 3], rtol=1e-15)
    x, w, _ = gll.tables(4)
    r = math.sqrt(3 / 7)
    np.testing.assert_allclose(x, [-1, -r, 0, r, 1], atol=1e-16)
    np.testing.assert_allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], rtol=1e-15)


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 8, 11, 16])
def test_gll_nodes_match_numpy_roots(N):
    x, _, _ = gll.tables(N)
    ref = np.sort(L.Legendre.basis(N).deriv().roots().real)
    np.testing.assert_allclose(x[1:-1], ref, atol=1e-13)


@pytest.mark.parametrize("N", [2, 4, 5, 8, 16])
def test_gll_quadrature_exact_to_degree_2N_minus_1(N):
    x, w, _ = gll.tables(N)
    for k in range(2 * N):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14 * max(1, N)
    # degree 2N is NOT integrated exactly (GLL is exact only to 2N-1)
    assert abs(np.dot(w, x ** (2 * N)) - 2.0 / (2 * N + 1)) > 1e-11


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 8, 12, 16])
def test_gll_derivative_exact_on_polynomials(N):
    x, _, D = gll.tables(N)
    for k in range(N + 1):
        np.testing.assert_allclose(D @ x ** k, k * x ** max(k - 1, 0) if k else 0 * x,
                                   atol=2e-13 * N * N)
    # GLL structure: D_00 = -N(N+1)/4, D_NN = N(N+1)/4, centro-antisymmetric
    assert abs(D[0, 0] + N * (N + 1) / 4) < 1e-12 * N * N
    np.testing.assert_allclose(D, -D[::-1, ::-1], atol=1e-12 * N * N)


@pytest.mark.parametrize("name", ["D2Q9", "D3Q13", "D3Q19", "D3Q27"])
def test_velocity_set_moments(name):
    lat = lattice.by_name(name)
    e, t, cs2, d = lat.e, lat.t, lat.cs2, lat.dim
    I = np.eye(d)
    assert abs(t.sum() - 1) < 1e-15
    np.testing.assert_allclose(np.einsum("q,qa->a", t, e), 0, atol=1e-15)
    np.testing.assert_allclose(np.einsum("q,qa,qb->ab", t, e, e), cs2 * I, atol=1e-15)
    np.testing.assert_allclose(np.einsum("q,qa,qb,qc->abc", t, e, e, e), 0, atol=1e-15)
    iso4 = cs2 ** 2 * (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
                       + np.einsum("ad,bc->abcd", I, I))
    np.testing.assert_allclose(np.einsum("q,qa,qb,qc,qd->abcd", t, e, e, e, e), iso4, atol=1e-15)
    np.testing.assert_allclose(np.einsum("q,qa,qb,qc,qd,qf->abcdf", t, e, e, e, e, e), 0,
                               atol=1e-15)
    np.testing.assert_allclose(e[lat.opp], -e, atol=1e-15)
    assert lat.Q == {"D2Q9": 9, "D3Q13": 13, "D3Q19": 19, "D3Q27": 27}[name]


def test_d3q13_speed():
    lat = lattice.d3q13()
    np.testing.assert_allclose(np.linalg.norm(lat.e[1:], axis=1), math.sqrt(5 / 3), rtol=1e-15)
    np.testing.assert_allclose(lat.t, [2 / 5] + [1 / 20] * 12, rtol=1e-15)


def _bare(dim=2):
    class _M:   # a stand-in mesh for the pointwise formulas only
        pass
    m = _M()
    m.dim = dim
    m.wall_tag = np.zeros(0, dtype=int)
    m.Me = np.ones((1, 1))
    m.Jinv = np.ones((1, 1, dim, dim))
    return m


def _solver(dim=2, **kw):
    lat = lattice.d2q9() if dim == 2 else lattice.d3q13()
    p = method.Params(dt=0.01, **({"delta": 0.1} | kw))
    return method.SemLbm(_bare(dim), lat, p)


def test_mu0_is_derivative_of_bulk_energy():
    s = _solver(beta=1e-3)
    rho = np.linspace(0.05, 1.1, 41)
    h = 1e-6
    fd = (s.bulk_energy(rho + h) - s.bulk_energy(rho - h)) / (2 * h)
    np.testing.assert_allclose(s.mu0(rho), fd, rtol=1e-8, atol=1e-14)


def test_surface_tension_and_kappa_relations():
    """Appendix A: the tanh profile of width delta solves mu = 0 in 1D for
    kappa = beta delta^2 (rho_l-rho_v)^2/8, and its excess energy equals gamma."""
    from scipy.integrate import quad
    beta, delta, rl, rv = 1e-3, 0.07, 1.0, 0.1
    s = _solver(beta=beta, delta=delta, rho_l=rl, rho_v=rv)
    kappa = s.p.kappa
    amp = (rl - rv) / 2
    rho = lambda x: (rl + rv) / 2 - amp * np.tanh(2 * x / delta)
    drho = lambda x: -amp * (2 / delta) / np.cosh(2 * x / delta) ** 2
    d2rho = lambda x: amp * (8 / delta ** 2) * np.tanh(2 * x / delta) / np.cosh(2 * x / delta) ** 2
    xs = np.linspace(-5 * delta, 5 * delta, 101)
    # 1D Euler-Lagrange: mu0(rho) - kappa rho'' = 0 for the planar profile
    np.testing.assert_allclose(s.mu0(rho(xs)) - kappa * d2rho(xs), 0, atol=1e-17)
    # first integral kappa rho'^2 / 2 = e0(rho)
    np.testing.assert_allclose(0.5 * kappa * drho(xs) ** 2, s.bulk_energy(rho(xs)), rtol=1e-10,
                               atol=1e-20)
    gamma_num, _ = quad(lambda x: kappa * drho(x) ** 2, -40 * delta, 40 * delta, limit=400)
    assert abs(gamma_num - s.p.surface_tension()) < 1e-9 * s.p.surface_tension()


@pytest.mark.parametrize("dim", [2, 3])
def test_equilibrium_and_force_moments(dim):
    s = _solver(dim)
    lat, cs2 = s.lat, s.cs2
    rng = np.random.default_rng(3)
    rho = rng.uniform(0.1, 1.0, 7)
    u = rng.uniform(-0.05, 0.05, (7, dim))
    F = rng.uniform(-1e-3, 1e-3, (7, dim))
    feq = s.equilibrium(rho, u)
    np.testing.assert_allclose(feq.sum(0), rho, rtol=1e-14)
    np.testing.assert_allclose(np.einsum("q...,qa->...a", feq, lat.e), rho[:, None] * u, atol=1e-16)
    P = np.einsum("q...,qa,qb->...ab", feq, lat.e, lat.e)
    Pex = rho[:, None, None] * (cs2 * np.eye(dim) + np.einsum("ia,ib->iab", u, u))
    np.testing.assert_allclose(P, Pex, atol=1e-15)
    Fs, Fss = s.force_terms(u, F)
    np.testing.assert_allclose(Fs.sum(0), 0, atol=1e-19)
    np.testing.assert_allclose(np.einsum("q...,qa->...a", Fs, lat.e), F, atol=1e-18)
    np.testing.assert_allclose(Fss.sum(0), 0, atol=1e-19)
    np.testing.assert_allclose(np.einsum("q...,qa->...a", Fss, lat.e), 0, atol=1e-19)
    # F* + F** is the full forcing term of Sec. 2.1
    eu = np.einsum("qa,ia->qi", lat.e, u)
    full = lat.t[:, None] / cs2 * np.einsum(
        "qia,ia->qi", lat.e[:, None, :] - u[None] + eu[..., None] * lat.e[:, None, :] / cs2, F)
    np.testing.assert_allclose(Fs + Fss, full, atol=1e-19)
    # its second moment is u F + F u
    S2 = np.einsum("q...,qa,qb->...ab", Fss, lat.e, lat.e)
    np.testing.assert_allclose(S2, np.einsum("ia,ib->iab", u, F) + np.einsum("ia,ib->iab", F, u),
                               atol=1e-18)


def test_ssp_rk3_on_linear_ode():
    for z in [-0.3, -1.0, -2.4, 0.2, 1j * 1.5, -0.5 + 1.0j]:
        lam, dt = z / 0.1, 0.1
        y = method.SemLbm.ssp_rk3(np.array([1.0 + 0j]), lambda g, k: lam * g, dt)
        assert abs(y[0] - (1 + z + z * z / 2 + z ** 3 / 6)) < 1e-14
