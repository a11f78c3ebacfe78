"""Algorithmic FP64 work per element-local node of each kernel of the step.

The count is that of the formulation the kernels evaluate (minimal work for
the method, not the instructions a compiler emits): a fused multiply-add is
2 flops and 1 FP64 pipe operation; an add or a multiply is 1 of each.  Let
n = N+1, d the dimension, M = Q-1 moving velocities.

k_rhs (force-split streaming right-hand side, per element-local node):
  reference derivatives of mu               d derivatives (those of rho are
                                            stored by k_lap of the same stage)
  v_b = d_b rho - (rho/c_s^2) d_b mu        1 mul + d fma
  M_e * |e| scale                           1 mul
  per velocity pair, c = J^-1 C_alpha       D2Q9: 0 (axis) or d adds (diagonal);
                                            D3Q13: d fma
  per moving velocity                       d derivatives, d fma (t v - dg),
                                            1 mul + (d-1) fma (dot), 1 mul (M_e)
  wall records, per moving velocity         1 sub + 1 fma
A derivative along one axis is 1 mul + (n-1) fma.
"""


def _deriv(n):
    return {"ops": n, "flops": 2 * n - 1}


# non-zero components of each representative velocity (one per opposite pair)
_REP_NONZERO = {
    "D2Q9": [1, 1, 2, 2],
    "D3Q13": [2] * 6,                       # (0, 1, phi) and its cyclic images
    "D3Q19": [1] * 3 + [2] * 6,
    "D3Q27": [1] * 3 + [2] * 6 + [3] * 4,
}
_DIM = {"D2Q9": 2, "D3Q13": 3, "D3Q19": 3, "D3Q27": 3}


def _pair_coeff_work(lattice, d):
    """c_b = (J^-1 C)_b for every pair: adds for unit components, an fma for phi."""
    ops = flops = 0
    for k in _REP_NONZERO[lattice]:
        if lattice == "D3Q13":
            ops += d          # one fma per reference direction
            flops += 2 * d
        else:
            ops += (k - 1) * d
            flops += (k - 1) * d
    return ops, flops


def rhs_work_per_node(lattice, N):
    n, d = N + 1, _DIM[lattice]
    M = 2 * len(_REP_NONZERO[lattice])   # moving velocities
    dv = _deriv(n)
    ops = d * dv["ops"] + 1 + d + 1
    flops = d * dv["flops"] + 1 + 2 * d + 1
    po, pf = _pair_coeff_work(lattice, d)
    ops += po
    flops += pf
    per_v_ops = d * dv["ops"] + d + d + 1
    per_v_flops = d * dv["flops"] + 2 * d + (1 + 2 * (d - 1)) + 1
    return {"ops": ops + M * per_v_ops, "flops": flops + M * per_v_flops}


def rhs_work(lattice, N, n_local, n_wall_nodes):
    """FP64 ops and flops of one k_rhs launch over the whole mesh."""
    Q = 2 * len(_REP_NONZERO[lattice]) + 1
    w = rhs_work_per_node(lattice, N)
    return {"ops": w["ops"] * n_local + 2 * (Q - 1) * n_wall_nodes,
            "flops": w["flops"] * n_local + 3 * (Q - 1) * n_wall_nodes}


def rhs_bytes_per_node(lattice, N):
    """Minimum DRAM bytes of k_rhs per node: read g (Q-1), rho, mu, grad rho (d),
    J^-1 (d^2), M_e, wall slot (4 B); write r (Q-1)."""
    d = _DIM[lattice]
    Q = 2 * len(_REP_NONZERO[lattice]) + 1
    return 8 * ((Q - 1) + 2 + d + d * d + 1 + (Q - 1)) + 4
