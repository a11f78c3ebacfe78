"""Gauss-Lobatto-Legendre tables for the oracle (test infrastructure only).

The paper (Sec. 2.1, after Eq. momentum) defers the spectral element operators
to Deville, Fischer & Mund; what they need is the GLL point set of order N, its
quadrature weights and the derivative matrix of the nodal Lagrange basis.

Route taken here (deliberately different from the CUDA library's host tables):
* nodes: -1, +1 and the roots of P_N', found by Newton iteration in long double
  from the Chebyshev-Gauss-Lobatto points;
* weights: w_i = 2 / (N (N+1) P_N(x_i)^2);
* derivative matrix: D_ij = l_j'(x_i) from the generic product formula for the
  derivative of a Lagrange polynomial (no GLL-specific closed form).

Pinned by tests/test_oracle_tables.py (test_gll_*): closed forms for N = 2 and
N = 4, exactness of the quadrature to degree 2N-1 and of D on polynomials of
degree <= N, and a cross-check of the nodes against numpy's Legendre root finder.
"""
import numpy as np

_LD = np.longdouble


def legendre(N, x):
    """P_N(x) and P_N'(x) by the three-term recurrence (long double)."""
    x = np.asarray(x, dtype=_LD)
    p_prev = np.ones_like(x)
    if N == 0:
        return p_prev, np.zeros_like(x)
    p = x.copy()
    dp_prev = np.zeros_like(x)
    dp = np.ones_like(x)
    for k in range(1, N):
        p_next = ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
        # derivative recurrence: P'_{k+1} = P'_{k-1} + (2k+1) P_k
        dp_next = dp_prev + (2 * k + 1) * p
        p_prev, p = p, p_next
        dp_prev, dp = dp, dp_next
    return p, dp


def gll_nodes(N):
    """The N+1 GLL points on [-1, 1], ascending."""
    if N < 1:
        raise ValueError("GLL order N must be >= 1")
    j = np.arange(N + 1, dtype=_LD)
    x = -np.cos(np.pi * j / N).astype(_LD)
    inner = x[1:-1].copy()
    for _ in range(100):
        p, dp = legendre(N, inner)
        # Legendre ODE: (1 - x^2) P'' = 2 x P' - N (N+1) P
        d2p = (2 * inner * dp - N * (N + 1) * p) / (1 - inner * inner)
        step = dp / d2p
        inner = inner - step
        if np.all(np.abs(step) < 1e-30):
            break
    x[1:-1] = inner
    x[0], x[-1] = -1, 1
    return x


def gll_weights(N, x=None):
    if x is None:
        x = gll_nodes(N)
    p, _ = legendre(N, x)
    return _LD(2) / (N * (N + 1) * p * p)


def lagrange_derivative_matrix(x):
    """D[i, j] = d l_j / dx evaluated at x_i for the Lagrange basis on points x."""
    x = np.asarray(x, dtype=_LD)
    n = len(x)
    D = np.zeros((n, n), dtype=_LD)
    for j in range(n):
        denom = _LD(1)
        for m in range(n):
            if m != j:
                denom *= x[j] - x[m]
        for i in range(n):
            if i == j:
                s = _LD(0)
                for m in range(n):
                    if m != j:
                        s += 1 / (x[j] - x[m])
                D[i, j] = s
            else:
                num = _LD(1)
                for m in range(n):
                    if m != j and m != i:
                        num *= x[i] - x[m]
                D[i, j] = num / denom
    return D


def tables(N):
    """(nodes, weights, D) in float64."""
    x = gll_nodes(N)
    w = gll_weights(N, x)
    D = lagrange_derivative_matrix(x)
    return x.astype(np.float64), w.astype(np.float64), D.astype(np.float64)
