"""Dense brute-force assembly of the SEM operators on tiny meshes (test-only).

Independent of the oracle: GLL points from numpy's Legendre routines, the
Lagrange basis as numpy Polynomial objects (differentiated symbolically), the
isoparametric map and its Jacobian evaluated by summing over every basis
function, and the global matrices assembled densely by explicit quadrature of
products of global basis functions:

  M_IJ      = sum_e sum_q W_q detJ_q  Phi_I(q) Phi_J(q)
  K_IJ      = sum_e sum_q W_q detJ_q  grad Phi_I(q) . grad Phi_J(q)
  C[w]^a_IJ = sum_e sum_q W_q detJ_q  w_q Phi_I(q) e_a . grad Phi_J(q)
  wall      = sum over wall faces, face quadrature w_face |a| Phi_I(q) (...)

These are the matrices of Eq. (spetrum) and Eq. (weak).  Meant for 1-4
elements only (cost grows as (E n^d)^2).
"""
import numpy as np
from numpy.polynomial import Polynomial
from numpy.polynomial import legendre as L


def gll(N):
    inner = L.Legendre.basis(N).deriv().roots().real
    x = np.concatenate([[-1.0], np.sort(inner), [1.0]])
    PN = L.Legendre.basis(N)(x)
    w = 2.0 / (N * (N + 1) * PN ** 2)
    return x, w


class Dense:
    def __init__(self, mesh):
        self.dim, self.N = mesh.dim, mesh.N
        dim, N = self.dim, self.N
        n = self.n = N + 1
        self.x, self.w = gll(N)
        basis = []
        for j in range(n):
            others = np.delete(self.x, j)
            p = Polynomial.fromroots(others)
            basis.append(p / p(self.x[j]))
        self.ell = np.array([[b(xq) for xq in self.x] for b in basis])                 # [j, q]
        self.dell = np.array([[b.deriv()(xq) for xq in self.x] for b in basis])        # [j, q]
        self.mesh = mesh
        E = mesh.n_elem
        nl = n ** dim
        self.loc = np.indices((n,) * dim).reshape(dim, -1)[::-1].T                     # [nl, d]
        # global numbering
        uniq, inv = np.unique(mesh.global_id.ravel(), return_inverse=True)
        self.G = len(uniq)
        self.gmap = inv.reshape(E, nl)
        # basis values / reference gradients: phi[k, q], dphi[b, k, q]
        phi = np.ones((nl, nl))
        dphi = np.ones((dim, nl, nl))
        for c in range(dim):
            kc = self.loc[:, c][:, None]
            qc = self.loc[:, c][None, :]
            phi = phi * self.ell[kc, qc]
            for b in range(dim):
                dphi[b] = dphi[b] * (self.dell[kc, qc] if b == c else self.ell[kc, qc])
        self.phi, self.dphi = phi, dphi
        Wq = np.ones(nl)
        for c in range(dim):
            Wq = Wq * self.w[self.loc[:, c]]
        self.Wq = Wq
        # per element: Jacobian at quadrature points from the interpolated map
        self.detJ = np.zeros((E, nl))
        self.gradphi = np.zeros((E, dim, nl, nl))        # [e, a, k, q]: d Phi_k / dx_a at q
        self.Jq = np.zeros((E, nl, dim, dim))
        for e in range(E):
            X = mesh.node_xyz[e]                           # [k, a]
            J = np.einsum("ka,bkq->qab", X, dphi)          # J[q, a, b]
            self.Jq[e] = J
            self.detJ[e] = np.linalg.det(J)
            Ji = np.linalg.inv(J)                          # [q, b, a]
            self.gradphi[e] = np.einsum("qba,bkq->akq", Ji, dphi)
        self._walls()

    def _walls(self):
        m, dim, n = self.mesh, self.dim, self.n
        self.wall = []     # (e, face, q-indices, w*|a|, normal)
        for e in range(m.n_elem):
            for f in range(2 * dim):
                if m.face_kind[e, f] != 1:
                    continue
                b, s = divmod(f, 2)
                sel = np.nonzero(self.loc[:, b] == (self.N if s else 0))[0]
                tang = [c for c in range(dim) if c != b]
                J = self.Jq[e][sel]                          # [q, a, c]
                if dim == 2:
                    t = J[:, :, tang[0]]
                    a = np.stack([t[:, 1], -t[:, 0]], -1)     # t rotated by -90 deg
                    if b == 1:
                        a = -a
                else:
                    a = np.cross(J[:, :, tang[0]], J[:, :, tang[1]])
                    if b == 1:
                        a = -a
                # orient outward: compare with the reference normal mapped by J^-T
                ref = np.zeros(dim)
                ref[b] = 1.0 if s else -1.0
                outward = np.einsum("qba,b->qa", np.linalg.inv(J), ref)
                sgn = np.sign(np.einsum("qa,qa->q", a, outward))
                a = a * sgn[:, None]
                wf = np.ones(len(sel))
                for c in tang:
                    wf = wf * self.w[self.loc[sel, c]]
                area = np.linalg.norm(a, axis=1)
                self.wall.append((e, f, sel, wf * area, a / area[:, None], int(m.face_tag[e, f])))

    # ---- dense global matrices -------------------------------------------
    def mass(self):
        M = np.zeros((self.G, self.G))
        for e in range(self.mesh.n_elem):
            g = self.gmap[e]
            Me = np.einsum("q,kq,lq->kl", self.Wq * self.detJ[e], self.phi, self.phi)
            M[np.ix_(g, g)] += Me
        return M

    def stiffness(self):
        K = np.zeros((self.G, self.G))
        for e in range(self.mesh.n_elem):
            g = self.gmap[e]
            Ke = np.einsum("q,akq,alq->kl", self.Wq * self.detJ[e], self.gradphi[e], self.gradphi[e])
            K[np.ix_(g, g)] += Ke
        return K

    def convection(self, evec, weight=None):
        """C_IJ = int w Phi_I e.grad Phi_J (weight w given per global node)."""
        C = np.zeros((self.G, self.G))
        for e in range(self.mesh.n_elem):
            g = self.gmap[e]
            wq = np.ones(len(self.Wq)) if weight is None else weight[g]   # nodal = quadrature
            egrad = np.einsum("a,alq->lq", evec, self.gradphi[e])
            Ce = np.einsum("q,kq,lq->kl", self.Wq * self.detJ[e] * wq, self.phi, egrad)
            C[np.ix_(g, g)] += Ce
        return C

    def wall_vector(self, fn):
        """b_I = sum_wall faces sum_q w|a| Phi_I(q) fn(e, sel, normal, tag)."""
        b = np.zeros(self.G)
        for (e, f, sel, ws, nrm, tag) in self.wall:
            vals = fn(e, sel, nrm, tag)
            np.add.at(b, self.gmap[e], (self.phi[:, sel] * (ws * vals)[None, :]).sum(1))
        return b

    def to_global(self, u_local):
        """Element-local nodal field -> global vector (copies must agree)."""
        out = np.zeros(self.G)
        out[self.gmap.ravel()] = u_local.reshape(-1)
        return out

    def to_local(self, u_global):
        return u_global[self.gmap]
