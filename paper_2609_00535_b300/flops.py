"""Algorithmic FP64 work per element-local node of each kernel of the step.

The count is that of the formulation the kernels evaluate (minimal work for
the method, not the instructions a compiler emits): a fused multiply-add is
2 flops and 1 FP64 pipe operation; an add or a multiply is 1 of each.  Let
n = N+1, d the dimension, M = Q-1 moving velocities.

k_rhs (force-split streaming right-hand side, per element-local node; the
metric array holds M_e S J^-1, so the mass and the speed scale cost nothing):
  reference derivatives of mu               d derivatives (those of rho are
                                            stored by k_lap of the same stage)
  v_b = d_b rho - (rho/c_s^2) d_b mu        1 mul + d fma
  per velocity pair, c = M_e S J^-1 C_alpha D2Q9: 0 (axis) or d adds (diagonal);
                                            cubic sets: (k-1) d adds; D3Q13: none
                                            (its d fma per pair are done once per
                                            mesh, k_pair_metric, and c is read)
  then, for D2Q9 and D3Q13 (one t v per moving weight):
  per node and moving weight, t v_b         d mul
  per moving velocity                       d chains t v_b - d_b g (n fma
                                            each), c.x: 1 mul + (d-1) fma
  and for the cubic sets (two or three weights, t c.v formed per pair):
  per velocity pair, t c.v                  1 mul + (d-1) fma, 1 mul
  per moving velocity                       d derivatives, d fma (t c.v - c.dg)
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
# sets whose pair coefficients M_e S J^-1 C are stored per node (k_rhs reads
# (Q-1)/2 x d of them instead of the d x d metric)
_STORED_PAIRS = ("D3Q13",)
# sets whose streaming derivative chains start from t v (one product per moving
# weight and node), and the number of distinct weights of the moving velocities
_TV_START = ("D2Q9", "D3Q13")
_MOVING_WEIGHTS = {"D2Q9": 2, "D3Q13": 1, "D3Q19": 2, "D3Q27": 3}


def _pair_coeff_work(lattice, d):
    """c_b = (J^-1 C)_b for every pair: adds for unit components.  D3Q13's
    coefficients (an fma with phi each) are stored per node at setup."""
    if lattice in _STORED_PAIRS:
        return 0, 0
    ops = flops = 0
    for k in _REP_NONZERO[lattice]:
        ops += (k - 1) * d
        flops += (k - 1) * d
    return ops, flops


def rhs_work_per_node(lattice, N):
    n, d = N + 1, _DIM[lattice]
    M = 2 * len(_REP_NONZERO[lattice])   # moving velocities
    dv = _deriv(n)
    ops = d * dv["ops"] + 1 + d
    flops = d * dv["flops"] + 1 + 2 * d
    po, pf = _pair_coeff_work(lattice, d)
    ops += po
    flops += pf
    if lattice in _TV_START:
        ops += _MOVING_WEIGHTS[lattice] * d
        flops += _MOVING_WEIGHTS[lattice] * d
        per_v_ops = d * n + d
        per_v_flops = d * 2 * n + 2 * d - 1
    else:
        P = M // 2
        ops += P * (d + 1)
        flops += P * (2 * d - 1 + 1)
        per_v_ops = d * dv["ops"] + d
        per_v_flops = d * dv["flops"] + 2 * d
    return {"ops": ops + M * per_v_ops, "flops": flops + M * per_v_flops}


def rhs_work(lattice, N, n_local, n_wall_nodes):
    """FP64 ops and flops of one k_rhs launch over the whole mesh."""
    Q = 2 * len(_REP_NONZERO[lattice]) + 1
    w = rhs_work_per_node(lattice, N)
    return {"ops": w["ops"] * n_local + 2 * (Q - 1) * n_wall_nodes,
            "flops": w["flops"] * n_local + 3 * (Q - 1) * n_wall_nodes}


def rhs_bytes_per_node(lattice, N):
    """Minimum DRAM bytes of k_rhs per node: read g (Q-1), rho, mu, grad rho (d),
    the metric M_e S J^-1 (d^2; or the stored pair coefficients, (Q-1)/2 x d),
    M_e, wall slot (4 B); write r (Q-1)."""
    d = _DIM[lattice]
    Q = 2 * len(_REP_NONZERO[lattice]) + 1
    metric = (Q - 1) // 2 * d if lattice in _STORED_PAIRS else d * d
    return 8 * ((Q - 1) + 2 + d + metric + 1 + (Q - 1)) + 4


# ---------------------------------------------------------------------------
# FP64 work of one whole time step (all 14 kernels), for the step roofline.
# Per element-local node (V of them), per node group (G; a group is one mesh
# node, summed over its copies), per extra copy (V - G) and per wall record R.
# A double division counts as one operation.
# ---------------------------------------------------------------------------
def _cdot_ops(lattice):
    """FP64 ops of C_a . v for each representative velocity."""
    if lattice == "D3Q13":
        return [1] * 6                       # one fma with phi
    return [k - 1 for k in _REP_NONZERO[lattice]]


def step_work(lattice, N, n_local, n_groups, n_wall_nodes):
    """(ops, flops) of the 14 kernels of one time step."""
    n, d = N + 1, _DIM[lattice]
    Q = 2 * len(_REP_NONZERO[lattice]) + 1
    M = Q - 1
    V, G, R = n_local, n_groups, n_wall_nodes
    X = V - G                                  # extra copies of shared nodes
    S1 = 0 if lattice in ("D2Q9", "D3Q19", "D3Q27") else 1   # |e| scale multiplies
    dv = _deriv(n)
    ops = flops = 0

    def add(o, f, count):
        nonlocal ops, flops
        ops += o * count
        flops += f * count

    # k_lap (x3): grad rho, metric products, D^T contraction; wall wetting term
    add(2 * d * dv["ops"] + d * d + (d - 1),
        2 * d * dv["flops"] + d * (2 * d - 1) + (d - 1), 3 * V)
    add(4, 5, 3 * R)
    # k_dss_mu (x3): sum of copies, 1/M, mu0 and -kappa lap
    add(10, 11, 3 * G)
    add(1, 1, 3 * X)
    # k_force (x1): grad mu, reference (c^2 d rho - rho d mu)/S (the first term
    # scaled by the force_split factor: 1 mul), metric M_e S J^-1
    add(d * dv["ops"] + 2 + 2 * d + d * d,
        d * dv["flops"] + 2 + 3 * d + d * (2 * d - 1), V)
    # k_dss_collide (x1): force average, momentum, equilibrium and F**
    cd = _cdot_ops(lattice)
    mom = sum(1 + k for k in _REP_NONZERO[lattice])            # difference + components
    per_group = d + mom + 1 + d + 2 * (2 * d - 1) + 1 + 4 + 4
    per_group += sum(2 * c + S1 + 1 + 1 + 2 + 1 + 8 for c in cd)
    add(per_group, per_group + 8 * len(cd) + 6, G)
    add(d, d, X)
    # k_rhs (x3)
    w = rhs_work_per_node(lattice, N)
    add(w["ops"], w["flops"], 3 * V)
    add(2 * M, 3 * M, 3 * R)
    # k_dss_rk (x3): sums of copies, dt/M, stage update, rho
    add(M, M, 3 * X)
    add(1 + M + Q, 1 + 2 * M + Q, G)                          # stage 1
    add(2 * (2 + 3 * M + 2 + Q), 2 * (2 + 5 * M + 3 + Q), G)  # stages 2 and 3
    return {"ops": ops, "flops": flops}
