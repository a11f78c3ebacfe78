"""The algorithmic FP64 counts behind bench.py's rooflines (flops.py), pinned by
hand counts of the formulations the kernels evaluate.  A fused multiply-add is
2 flops and 1 pipe operation; an add or a multiply 1 of each."""
from paper_2609_00535_b300 import flops


def test_streaming_kernel_d3q13_n5():
    """D3Q13 at N = 5 (n = 6, d = 3, 12 moving velocities, one moving weight):
    grad mu 3 x (1 mul + 5 fma) = 18 ops / 33 flops; v_b = d_b rho - 3 rho d_b mu:
    1 mul + 3 fma = 4 / 7; t v_b: 3 mul; per velocity three chains of 6 fma from
    t v_b (18 / 36) and c.x: 1 mul + 2 fma (3 / 5).  The pair coefficients are
    read, not computed."""
    w = flops.rhs_work_per_node("D3Q13", 5)
    assert w == {"ops": 18 + 4 + 3 + 12 * 21, "flops": 33 + 7 + 3 + 12 * 41}
    assert w == {"ops": 277, "flops": 535}


def test_streaming_kernel_d2q9_n4():
    """D2Q9 at N = 4 (n = 5, d = 2, 8 moving velocities, weights 1/9 and 1/36):
    grad mu 2 x 5 = 10 / 18; v 3 / 5; pair coefficients: 2 adds for each diagonal
    pair (4 / 4); t v_b per weight 2 x 2 mul; per velocity 2 chains of 5 fma
    (10 / 20) and c.x 1 mul + 1 fma (2 / 3)."""
    w = flops.rhs_work_per_node("D2Q9", 4)
    assert w == {"ops": 10 + 3 + 4 + 4 + 8 * 12, "flops": 18 + 5 + 4 + 4 + 8 * 23}


def test_streaming_kernel_cubic_sets_form_t_c_v_per_pair():
    """D3Q19 at N = 5: 9 pairs (3 axis, 6 face diagonals); pair coefficients
    3 adds per diagonal (18); t c.v per pair 1 mul + 2 fma + 1 mul (4 / 6); per
    velocity 3 derivatives (1 mul + 5 fma) and 3 fma (21 / 39)."""
    w = flops.rhs_work_per_node("D3Q19", 5)
    assert w == {"ops": 18 + 4 + 18 + 9 * 4 + 18 * 21, "flops": 33 + 7 + 18 + 9 * 6 + 18 * 39}


def test_launch_totals_add_the_wall_records():
    """A launch is the per-node count times the nodes, plus 2 ops / 3 flops per
    moving velocity of each wall record."""
    per = flops.rhs_work_per_node("D3Q13", 5)
    tot = flops.rhs_work("D3Q13", 5, 1000, 10)
    assert tot == {"ops": 1000 * per["ops"] + 10 * 2 * 12, "flops": 1000 * per["flops"] + 10 * 3 * 12}
    assert flops.rhs_bytes_per_node("D3Q13", 5) == 8 * (12 + 2 + 3 + 18 + 1 + 12) + 4
