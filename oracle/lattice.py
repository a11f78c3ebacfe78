"""Discrete velocity sets for the oracle (test infrastructure only).

* D2Q9, the 2D set of Sec. 2.1 (standard weights 4/9, 1/9, 1/36; c_s^2 = 1/3).
* D3Q19 and D3Q27, the standard cubic 3D sets (alternatives to D3Q13).
* D3Q13 for the 3D case of Sec. 3.2.  The paper cites Shan (2006) without a
  table.  Reading used here: the rest velocity plus the 12 vertices of an
  icosahedron, |e| = sqrt(5 c_s^2), weights 2/5 and 1/20, c_s^2 = 1/3.  That is
  the 13-point degree-5 quadrature of the Maxwellian; the spectral element
  streaming does not require lattice-conforming velocities.

Pinned by tests/test_oracle_tables.py (test_velocity_set_moments,
test_d3q13_speed): the weight moments sum(t) = 1,
sum(t e) = 0, sum(t e e) = c_s^2 I, odd moments zero to rank 5 and the rank-4
isotropic tensor c_s^4 (dd + dd + dd), plus closure of the set under e -> -e.
"""
import numpy as np

CS2 = 1.0 / 3.0


class Lattice:
    def __init__(self, name, e, t):
        self.name = name
        self.e = np.asarray(e, dtype=np.float64)      # [Q, d]
        self.t = np.asarray(t, dtype=np.float64)      # [Q]
        self.Q, self.dim = self.e.shape
        self.cs2 = CS2
        # opposite direction index (bounce-back partner)
        opp = []
        for a in range(self.Q):
            match = [b for b in range(self.Q) if np.allclose(self.e[b], -self.e[a], atol=1e-14)]
            if len(match) != 1:
                raise ValueError("velocity set is not closed under e -> -e")
            opp.append(match[0])
        self.opp = np.array(opp)


def d2q9():
    e = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    t = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
    return Lattice("D2Q9", e, t)


def d3q13():
    """Rest + 12 icosahedron vertices, ordered so that e_{a+6} = -e_a (a = 1..6)."""
    phi = (1 + np.sqrt(5.0)) / 2
    half = np.array([(0, 1, phi), (0, -1, phi), (1, phi, 0), (-1, phi, 0), (phi, 0, 1),
                     (phi, 0, -1)], dtype=np.float64)
    verts = np.vstack([half, -half])
    verts *= np.sqrt(5 * CS2) / np.linalg.norm(verts[0])
    e = np.vstack([np.zeros((1, 3)), verts])
    t = np.array([2 / 5] + [1 / 20] * 12)
    return Lattice("D3Q13", e, t)


_FACES = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
_EDGES = [(1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1), (0, 1, 1), (0, 1, -1)]
_CORNERS = [(1, 1, 1), (1, 1, -1), (1, -1, 1), (1, -1, -1)]


def _paired(half, weights, t0):
    half = np.array(half, dtype=np.float64)
    e = np.vstack([np.zeros((1, 3)), half, -half])
    t = np.array([t0] + list(weights) + list(weights))
    return e, t


def d3q19():
    """Rest, 6 face and 12 edge neighbours (weights 1/3, 1/18, 1/36); e_{a+9} = -e_a."""
    e, t = _paired(_FACES + _EDGES, [1 / 18] * 3 + [1 / 36] * 6, 1 / 3)
    return Lattice("D3Q19", e, t)


def d3q27():
    """Rest, faces, edges and corners (8/27, 2/27, 1/54, 1/216); e_{a+13} = -e_a."""
    e, t = _paired(_FACES + _EDGES + _CORNERS, [2 / 27] * 3 + [1 / 54] * 6 + [1 / 216] * 4, 8 / 27)
    return Lattice("D3Q27", e, t)


def by_name(name):
    return {"D2Q9": d2q9, "D3Q13": d3q13, "D3Q19": d3q19, "D3Q27": d3q27}[name]()
