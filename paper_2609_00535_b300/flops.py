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


def rhs_work_per_node(lattice, N):
    n, d = N + 1, (2 if lattice == "D2Q9" else 3)
    Q = 9 if lattice == "D2Q9" else 13
    M = Q - 1
    dv = _deriv(n)
    ops = d * dv["ops"] + 1 + d + 1
    flops = d * dv["flops"] + 1 + 2 * d + 1
    if lattice == "D2Q9":
        ops += 2 * d            # two diagonal pairs: d adds each
        flops += 2 * d
    else:
        ops += 6 * d            # six pairs: d fma each
        flops += 6 * 2 * d
    per_v_ops = d * dv["ops"] + d + d + 1
    per_v_flops = d * dv["flops"] + 2 * d + (1 + 2 * (d - 1)) + 1
    return {"ops": ops + M * per_v_ops, "flops": flops + M * per_v_flops}


def rhs_work(lattice, N, n_local, n_wall_nodes):
    """FP64 ops and flops of one k_rhs launch over the whole mesh."""
    Q = 9 if lattice == "D2Q9" else 13
    w = rhs_work_per_node(lattice, N)
    return {"ops": w["ops"] * n_local + 2 * (Q - 1) * n_wall_nodes,
            "flops": w["flops"] * n_local + 3 * (Q - 1) * n_wall_nodes}


def rhs_bytes_per_node(lattice, N):
    """Minimum DRAM bytes of k_rhs per node: read g (Q-1), rho, mu, grad rho (d),
    J^-1 (d^2), M_e, wall slot (4 B); write r (Q-1)."""
    d = 2 if lattice == "D2Q9" else 3
    Q = 9 if lattice == "D2Q9" else 13
    return 8 * ((Q - 1) + 2 + d + d * d + 1 + (Q - 1)) + 4
