"""Element geometry and gather-scatter for the oracle (test infrastructure only).

Everything is recomputed from the raw mesh arrays (GLL node coordinates per
element, global node ids, face kinds and tags):

* isoparametric Jacobian J_ab = dx_a/dxi_b by the GLL derivative matrix applied
  to the node coordinates; det J and J^-1 by numpy.linalg;
* local mass M_e = W det J (tensor GLL weights W) and the assembled diagonal
  mass M_g = sum of M_e over the copies of a global node (the mass matrix M of
  Eq. spetrum);
* wall faces: outward area vector from the face tangents (2D: the tangent
  rotated by -90 degrees; 3D: the cross product of the two tangent
  derivatives), times the GLL weights along the face.  It is kept per
  face-node, so a corner node on two wall faces carries two contributions:
  this is the per-face normal treatment that the flux bounce-back scheme
  relies on (Sec. 1, Sec. 2.2);
* direct-stiffness summation: copies with the same global id are summed with
  numpy's ``bincount`` (sequential accumulation) and the sum is scattered back.

Pinned by tests/test_oracle_operators.py: sum of M_e equals the area/volume of
affine meshes exactly and converges spectrally on curved meshes
(test_areas_and_volumes), the area vector equals det J times the matching row
of J^-1 (test_area_vector_is_cofactor_row), the discrete area vectors of a
closed wall sum to zero (test_closed_wall_area_vectors_sum_to_zero), wall nodes
lie on the curved walls, and the mass matrix and gather-scatter against the
independent dense assembly of tests/brute_dense.py (test_mass_matrix_dense,
test_dss_counts_shared_copies).
"""
import numpy as np

from . import gll


def deriv(u, D, b, dim, transpose=False):
    """Derivative along reference axis b of element-local nodal data.

    u has trailing shape (n,)*dim with the xi_1 index last (fastest).  With
    transpose=True the contraction uses D^T (sum_m D[m, i] u_m), the adjoint
    that the weak Laplacian needs.
    """
    lead = u.shape[:-dim]
    v = u.reshape((-1,) + u.shape[-dim:])
    axis = v.ndim - 1 - b
    out = np.tensordot(v, D, axes=([axis], [0 if transpose else 1]))
    out = np.moveaxis(out, -1, axis)
    return out.reshape(lead + u.shape[-dim:])


class Mesh:
    """Oracle view of a mesh: metrics, masses, wall face-nodes and DSS maps."""

    def __init__(self, dim, N, node_xyz, global_id, face_kind, face_tag):
        self.dim = dim
        self.N = N
        n = self.n = N + 1
        node_xyz = np.asarray(node_xyz, dtype=np.float64)
        E = self.E = node_xyz.shape[0]
        self.shape = (E,) + (n,) * dim
        self.xi, self.w, self.D = gll.tables(N)
        X = node_xyz.reshape(self.shape + (dim,))
        self.X = X

        J = np.empty(self.shape + (dim, dim))
        for a in range(dim):
            for b in range(dim):
                J[..., a, b] = deriv(X[..., a], self.D, b, dim)
        self.J = J
        self.detJ = np.linalg.det(J)
        if np.any(self.detJ <= 0):
            raise ValueError("mesh has an element with non-positive Jacobian")
        self.Jinv = np.linalg.inv(J)              # Jinv[..., b, a] = dxi_b / dx_a

        W = np.ones((n,) * dim)
        for b in range(dim):
            shp = [1] * dim
            shp[dim - 1 - b] = n
            W = W * self.w.reshape(shp)
        self.W = W
        self.Me = W[None] * self.detJ            # local mass, [E, n..]

        gid = np.asarray(global_id, dtype=np.int64).reshape(E, -1)
        uniq, inv = np.unique(gid.ravel(), return_inverse=True)
        self.G = len(uniq)
        self.inv = inv.reshape(self.shape)
        self.Mg = self.gather(self.assemble(self.Me))  # assembled mass at each copy

        self._build_walls(np.asarray(face_kind).reshape(E, 2 * dim),
                          np.asarray(face_tag).reshape(E, 2 * dim))

    # ---- direct-stiffness summation ------------------------------------
    def assemble(self, r):
        """Sum element-local copies per global node: returns [..., G]."""
        lead = r.shape[:-self.dim - 1]
        rr = r.reshape((-1, self.E) + r.shape[-self.dim:])
        out = np.zeros((rr.shape[0], self.G))
        idx = self.inv.ravel()
        for k in range(rr.shape[0]):
            # bincount accumulates in input order: a fixed, sequential summation
            out[k] = np.bincount(idx, weights=rr[k].ravel(), minlength=self.G)
        return out.reshape(lead + (self.G,))

    def gather(self, g):
        """Scatter a global-node field back to every element-local copy."""
        return g[..., self.inv]

    def dss_average(self, r):
        """DSS(r) / M_g at every element-local copy."""
        return self.gather(self.assemble(r)) / self.Mg

    # ---- walls -----------------------------------------------------------
    def _face_index(self, f):
        """Index tuple (over the element-local node axes) of face f = 2b + s."""
        b, s = divmod(f, 2)
        sl = [slice(None)] * self.dim
        sl[self.dim - 1 - b] = self.N if s == 1 else 0
        return tuple(sl)

    def _build_walls(self, face_kind, face_tag):
        dim, n = self.dim, self.n
        flat = np.arange(n ** dim).reshape((n,) * dim)
        elems, nodes, avec, tags = [], [], [], []
        for f in range(2 * dim):
            b, s = divmod(f, 2)
            sign = 1.0 if s == 1 else -1.0
            fi = self._face_index(f)
            wf = np.ones((n,) * dim)
            for c in range(dim):
                if c != b:
                    shp = [1] * dim
                    shp[dim - 1 - c] = n
                    wf = wf * self.w.reshape(shp)
            for e in np.nonzero(face_kind[:, f] == 1)[0]:
                Je = self.J[e][fi]                       # [face nodes.., a, b]
                if dim == 2:
                    if b == 0:
                        t = Je[..., :, 1]
                        a = np.stack([t[..., 1], -t[..., 0]], axis=-1)
                    else:
                        t = Je[..., :, 0]
                        a = np.stack([-t[..., 1], t[..., 0]], axis=-1)
                else:
                    c, d = (b + 1) % 3, (b + 2) % 3
                    a = np.cross(Je[..., :, c], Je[..., :, d])
                a = sign * a * wf[fi][..., None]
                elems.append(np.full(a.shape[:-1], e).ravel())
                nodes.append(flat[fi].ravel())
                avec.append(a.reshape(-1, dim))
                tags.append(np.full(elems[-1].shape, face_tag[e, f]))
        if elems:
            self.wall_elem = np.concatenate(elems)
            self.wall_node = np.concatenate(nodes)
            self.wall_area = np.concatenate(avec)    # w_face * outward area vector
            self.wall_tag = np.concatenate(tags)
        else:
            self.wall_elem = np.zeros(0, dtype=np.int64)
            self.wall_node = np.zeros(0, dtype=np.int64)
            self.wall_area = np.zeros((0, dim))
            self.wall_tag = np.zeros(0, dtype=np.int64)

    def add_wall_nodes(self, r, values):
        """r[..., e, node] + values for each wall face-node entry (r element-local)."""
        out = r.reshape(r.shape[:-self.dim] + (-1,)).copy()
        if out.ndim == 2:
            np.add.at(out, (self.wall_elem, self.wall_node), values)
        else:
            for k in range(out.shape[0]):
                np.add.at(out[k], (self.wall_elem, self.wall_node), values[k])
        return out.reshape(r.shape)

    def at_wall(self, u):
        """Values of an element-local field at the wall face-node entries."""
        uu = u.reshape(u.shape[:-self.dim] + (-1,))
        return uu[..., self.wall_elem, self.wall_node]

    # ---- collocated physical gradient -----------------------------------
    def grad(self, u):
        """Physical gradient of element-local nodal data: [..., d] (discontinuous)."""
        gxi = np.stack([deriv(u, self.D, b, self.dim) for b in range(self.dim)], axis=-1)
        # du/dx_a = sum_b (dxi_b/dx_a) du/dxi_b
        return np.einsum("...ba,...b->...a", self.Jinv, gxi)
