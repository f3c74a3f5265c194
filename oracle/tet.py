"""SIPDG Poisson / screened-Poisson operator on affine tetrahedra (oracle).

TEST INFRASTRUCTURE ONLY.

Section 6 names three-dimensional tetrahedral meshes as the method's next
step; the bilinear form is the one of Eq. ellipticOp1 with volume integrals
over tetrahedra and surface integrals over their triangular faces:

  a_E(u, v) = (grad v, grad u)_E - (v, n.{grad u})_dE + 1/2 (n.grad v, [u])_dE
              - (v, tau [u])_dE + lambda (v, u)_E,

{w} = (w+ + w-)/2, [w] = w+ - w- (Eq. AverageJumpScalar), output the weak
coefficient vector (A u)_i = a_E(u, l_i). Readings for three dimensions (the
paper gives none):
  * penalty: Eq. PenaltyParameter with the three-dimensional trace-inverse
    constant, tau = (N+1)(N+3)/3 max(1/h+, 1/h-), h = |E| / |face| (the
    triangle's constant (N+1)(N+2)/2 is the d = 2 case of (N+1)(N+d)/d);
  * boundary faces as on triangles: Dirichlet ghost u+ = 2g - u-,
    grad u+ = grad u- (penalty 2 tau on the homogeneous operator); Neumann
    u+ = u-, grad u+ = -grad u- (no face terms); tau from the interior side;
  * nodes: the equispaced nodes of the reference tetrahedron
    (r, s, t) = (-1 + 2i/N, -1 + 2j/N, -1 + 2k/N), i + j + k <= N, ordered
    by k, then j, then i (the optimised three-dimensional node set is not in
    the paper; equispaced nodes are well conditioned at the degrees used
    here, N <= 4).
Reference tetrahedron: vertices v0 = (-1,-1,-1), v1 = (1,-1,-1),
v2 = (-1,1,-1), v3 = (-1,-1,1); local faces face 0 = (v0, v1, v2),
face 1 = (v0, v1, v3), face 2 = (v1, v2, v3), face 3 = (v0, v2, v3), opposite
vertices v3, v2, v0, v1.

The nodal basis is built from monomials r^a s^b t^c (a + b + c <= N) through
the nodal Vandermonde matrix, and every integral is taken by quadrature
exact for its integrand (collapsed Gauss-Jacobi on the tetrahedron, the
collapsed triangle rule on each face), the neighbour's basis evaluated at the
same physical face points through its own inverse map: no face-node
ordering is used.
"""
import numpy as np
import scipy.sparse as sp
from scipy.special import roots_jacobi

from .basis import triangle_quadrature

INTERIOR, DIRICHLET, NEUMANN = 0, 1, 2
TET_VERTS = np.array([[-1.0, -1.0, -1.0], [1.0, -1.0, -1.0], [-1.0, 1.0, -1.0], [-1.0, -1.0, 1.0]])
TET_FACES = np.array([[0, 1, 2], [0, 1, 3], [1, 2, 3], [0, 2, 3]])


def tet_nodes(N):
    """The equispaced nodes of the reference tetrahedron (the module's node reading)."""
    pts = [(-1.0 + 2.0 * i / N, -1.0 + 2.0 * j / N, -1.0 + 2.0 * k / N)
           for k in range(N + 1) for j in range(N + 1 - k) for i in range(N + 1 - k - j)]
    p = np.array(pts)
    return p[:, 0], p[:, 1], p[:, 2]


def monomial_exponents(N):
    return [(a, b, c) for c in range(N + 1) for b in range(N + 1 - c) for a in range(N + 1 - c - b)]


def monomials(N, r, s, t):
    """Values and r/s/t derivatives of the monomials r^a s^b t^c, a + b + c <= N."""
    r, s, t = (np.asarray(z, dtype=np.float64).ravel() for z in (r, s, t))
    ex = monomial_exponents(N)

    def pw(x, k):
        return x ** k if k >= 0 else np.zeros_like(x)
    V = np.stack([pw(r, a) * pw(s, b) * pw(t, c) for a, b, c in ex], axis=1)
    Vr = np.stack([a * pw(r, a - 1) * pw(s, b) * pw(t, c) for a, b, c in ex], axis=1)
    Vs = np.stack([b * pw(r, a) * pw(s, b - 1) * pw(t, c) for a, b, c in ex], axis=1)
    Vt = np.stack([c * pw(r, a) * pw(s, b) * pw(t, c - 1) for a, b, c in ex], axis=1)
    return V, Vr, Vs, Vt


def tet_quadrature(n):
    """Collapsed (Stroud) rule on the reference tetrahedron with n^3 points:
    a, b, c from n-point Gauss-Jacobi rules with weights 1, (1-b), (1-c)^2;
    r = (1+a)(1-b)(1-c)/4 - 1, s = (1+b)(1-c)/2 - 1, t = c, and
    dr ds dt = (1-b)(1-c)^2/32 da db dc. Exact to total degree 2n - 1."""
    xa, wa = roots_jacobi(n, 0.0, 0.0)
    xb, wb = roots_jacobi(n, 1.0, 0.0)
    xc, wc = roots_jacobi(n, 2.0, 0.0)
    A, B, C = np.meshgrid(xa, xb, xc, indexing="ij")
    W = np.einsum("i,j,k->ijk", wa, wb, wc) / 8.0
    r = 0.25 * (1.0 + A) * (1.0 - B) * (1.0 - C) - 1.0
    s = 0.5 * (1.0 + B) * (1.0 - C) - 1.0
    t = C
    return r.ravel(), s.ravel(), t.ravel(), W.ravel()


class TetGeometry:
    """Affine maps x = v0 + (r+1)/2 (v1-v0) + (s+1)/2 (v2-v0) + (t+1)/2 (v3-v0),
    their inverses, face normals and areas, and face neighbours."""

    def __init__(self, VX, VY, VZ, EToV):
        self.V = np.stack([np.asarray(VX, float), np.asarray(VY, float), np.asarray(VZ, float)], axis=1)
        self.EToV = np.asarray(EToV, dtype=np.int64)
        K = self.EToV.shape[0]
        self.K = K
        P = self.V[self.EToV]                                   # (K,4,3)
        self.P = P
        jac = np.stack([0.5 * (P[:, 1] - P[:, 0]), 0.5 * (P[:, 2] - P[:, 0]), 0.5 * (P[:, 3] - P[:, 0])],
                       axis=2)                                   # columns x_r, x_s, x_t
        self.jac = jac
        self.J = np.linalg.det(jac)
        if np.any(self.J <= 0):
            raise ValueError("tetrahedron with non-positive Jacobian")
        self.inv = np.linalg.inv(jac)                            # rows grad r, grad s, grad t
        self.vol = self.J * (4.0 / 3.0)
        self.normal = np.empty((K, 4, 3))
        self.area = np.empty((K, 4))
        cen = P.mean(axis=1)
        for f, (a, b, c) in enumerate(TET_FACES):
            nv = np.cross(P[:, b] - P[:, a], P[:, c] - P[:, a])
            ar = np.linalg.norm(nv, axis=1)
            nv = nv / ar[:, None]
            out = np.einsum("ki,ki->k", nv, P[:, a] - cen) > 0
            nv[~out] *= -1.0
            self.normal[:, f] = nv
            self.area[:, f] = 0.5 * ar
        keys = {}
        self.EToE = -np.ones((K, 4), dtype=np.int64)
        self.EToF = -np.ones((K, 4), dtype=np.int64)
        for e in range(K):
            for f in range(4):
                key = tuple(sorted(self.EToV[e, TET_FACES[f]]))
                if key in keys:
                    e2, f2 = keys.pop(key)
                    self.EToE[e, f], self.EToF[e, f] = e2, f2
                    self.EToE[e2, f2], self.EToF[e2, f2] = e, f
                else:
                    keys[key] = (e, f)

    def to_physical(self, e, r, s, t):
        """Physical points of elements e (E,) at reference points r, s, t
        broadcastable to (E, q): (E, q, 3)."""
        P = self.P[np.asarray(e)]
        r, s, t = (np.asarray(z, dtype=np.float64) for z in (r, s, t))
        return (P[:, None, 0, :] + 0.5 * (r + 1.0)[..., None] * (P[:, None, 1, :] - P[:, None, 0, :])
                + 0.5 * (s + 1.0)[..., None] * (P[:, None, 2, :] - P[:, None, 0, :])
                + 0.5 * (t + 1.0)[..., None] * (P[:, None, 3, :] - P[:, None, 0, :]))

    def to_reference(self, e, x):
        """x: (E, q, 3) physical points of elements e -> (r, s, t), each (E, q)."""
        d = x - self.P[e][:, None, 0, :]
        rst = np.einsum("eij,eqj->eqi", self.inv[e], d) - 1.0  # x - v0 = jac (rst + 1)
        return rst[..., 0], rst[..., 1], rst[..., 2]


class TetSipdg:
    """The SIPDG bilinear form on tetrahedra (module header) for degree N:
    element and face coupling blocks by exact quadrature, matrix-free apply,
    assembled matrix, right-hand side of the Dirichlet problem."""

    def __init__(self, VX, VY, VZ, EToV, bc, N):
        self.N = N
        self.Np = (N + 1) * (N + 2) * (N + 3) // 6
        self.geo = TetGeometry(VX, VY, VZ, EToV)
        self.K = self.geo.K
        self.bc = np.asarray(bc, dtype=np.int64)
        self.r, self.s, self.t = tet_nodes(N)
        V, _, _, _ = monomials(N, self.r, self.s, self.t)
        self.Vinv = np.linalg.inv(V)
        rq, sq, tq, self.wq = tet_quadrature(N + 1)
        self.Lq, self.Lrq, self.Lsq, self.Ltq = self._eval_basis(rq, sq, tq)
        # face quadrature: the collapsed triangle rule mapped onto each reference face
        ra, sa, wa = triangle_quadrature(N + 1)
        self.wf = wa                       # sums to 2 (the bi-unit triangle's area)
        self.face_ref = []
        for f in range(4):
            A, B, C = TET_VERTS[TET_FACES[f]]
            pts = A[None] + 0.5 * (ra + 1.0)[:, None] * (B - A)[None] + 0.5 * (sa + 1.0)[:, None] * (C - A)[None]
            self.face_ref.append((pts[:, 0], pts[:, 1], pts[:, 2]) + self._eval_basis(pts[:, 0], pts[:, 1], pts[:, 2]))
        g = self.geo
        inv_h = g.area / g.vol[:, None]    # 1/h = |face| / |E|
        inv_h_nb = np.where(g.EToE >= 0, inv_h[np.maximum(g.EToE, 0), np.maximum(g.EToF, 0)], 0.0)
        c = (N + 1) * (N + 3) / 3.0
        self.tau = c * np.where(g.EToE >= 0, np.maximum(inv_h, inv_h_nb), inv_h)
        X = g.to_physical(np.arange(self.K), self.r[None, :], self.s[None, :], self.t[None, :])
        self.x, self.y, self.z = X[..., 0], X[..., 1], X[..., 2]

    def _eval_basis(self, r, s, t):
        shp = np.asarray(r).shape
        V, Vr, Vs, Vt = monomials(self.N, r, s, t)
        out = [M @ self.Vinv for M in (V, Vr, Vs, Vt)]
        return tuple(o.reshape(shp + (self.Np,)) for o in out)

    def _grad(self, inv, Lr, Ls, Lt):
        """Physical gradient components of basis values given reference derivatives
        (inv: (E,3,3) rows grad r, grad s, grad t)."""
        return [inv[:, 0, d, None, None] * Lr + inv[:, 1, d, None, None] * Ls + inv[:, 2, d, None, None] * Lt
                for d in range(3)]

    def local_blocks(self, elems, lam=0.0):
        """Element matrix and face coupling matrices of the listed elements:
        Ke[e] = volume stiffness + lambda mass; faces[f] = (Fm, Fp, nbr, Fb, A1, A2, tau)."""
        g = self.geo
        elems = np.asarray(elems)
        inv = g.inv[elems]
        J = g.J[elems]
        E = len(elems)
        Lr = np.broadcast_to(self.Lrq, (E,) + self.Lrq.shape)
        Ls = np.broadcast_to(self.Lsq, (E,) + self.Lsq.shape)
        Lt = np.broadcast_to(self.Ltq, (E,) + self.Ltq.shape)
        gx, gy, gz = self._grad(inv, Lr, Ls, Lt)
        Ke = (np.einsum("q,eqi,eqj->eij", self.wq, gx, gx) + np.einsum("q,eqi,eqj->eij", self.wq, gy, gy)
              + np.einsum("q,eqi,eqj->eij", self.wq, gz, gz)) * J[:, None, None]
        if lam != 0.0:
            Mref = np.einsum("q,qi,qj->ij", self.wq, self.Lq, self.Lq)
            Ke = Ke + lam * J[:, None, None] * Mref[None]
        faces = []
        for f in range(4):
            rf, sf, tf, Lf, Lrf, Lsf, Ltf = self.face_ref[f]
            n = g.normal[elems, f]                                         # (E,3)
            W = self.wf[None, :] * 0.5 * g.area[elems, f][:, None]         # (E,nq)
            tau = self.tau[elems, f]
            E_ = (E,) + Lrf.shape
            fx, fy, fz = self._grad(inv, np.broadcast_to(Lrf, E_), np.broadcast_to(Lsf, E_), np.broadcast_to(Ltf, E_))
            dn_m = n[:, 0, None, None] * fx + n[:, 1, None, None] * fy + n[:, 2, None, None] * fz
            A1 = np.einsum("ek,ki,ekj->eij", W, Lf, dn_m)    # (l_i, n.grad l_j)
            A2 = np.einsum("ek,ki,kj->eij", W, Lf, Lf)       # (l_i, l_j)
            Fm = -0.5 * A1 - 0.5 * np.swapaxes(A1, 1, 2) + tau[:, None, None] * A2
            Fb = -A1 - np.swapaxes(A1, 1, 2) + 2.0 * tau[:, None, None] * A2
            nbr = g.EToE[elems, f]
            Fp = np.zeros_like(Fm)
            inter = nbr >= 0
            if np.any(inter):
                ei, en = elems[inter], nbr[inter]
                xq = g.to_physical(ei, rf[None, :], sf[None, :], tf[None, :])
                rp, spp, tp = g.to_reference(en, xq)
                Lp, Lrp, Lsp, Ltp = self._eval_basis(rp, spp, tp)
                px, py, pz = self._grad(g.inv[en], Lrp, Lsp, Ltp)
                ni = n[inter]
                dn_p = ni[:, 0, None, None] * px + ni[:, 1, None, None] * py + ni[:, 2, None, None] * pz
                Wi = W[inter]
                B1 = np.einsum("ek,ki,ekj->eij", Wi, Lf, dn_p)          # (l_i, n.grad l+_j)
                B2 = np.einsum("ek,eki,ekj->eij", Wi, dn_m[inter], Lp)  # (n.grad l_i, l+_j)
                B3 = np.einsum("ek,ki,ekj->eij", Wi, Lf, Lp)            # (l_i, l+_j)
                Fp[inter] = -0.5 * B1 + 0.5 * B2 - tau[inter, None, None] * B3
            faces.append((Fm, Fp, nbr, Fb, A1, A2, tau))
        return Ke, faces

    def _chunks(self, elems, size=1024):
        for i in range(0, len(elems), size):
            yield elems[i:i + size]

    def apply(self, u, lam=0.0):
        """(A u), u: (K, Np) or (B, K, Np)."""
        u = np.asarray(u, dtype=np.float64)
        U = u if u.ndim == 3 else u[None]
        out = np.zeros_like(U)
        for ch in self._chunks(np.arange(self.K)):
            Ke, faces = self.local_blocks(ch, lam)
            acc = np.einsum("eij,bej->bei", Ke, U[:, ch])
            for f in range(4):
                Fm, Fp, nbr, Fb, _, _, _ = faces[f]
                inter = nbr >= 0
                acc[:, inter] += np.einsum("eij,bej->bei", Fm[inter], U[:, ch[inter]])
                acc[:, inter] += np.einsum("eij,bej->bei", Fp[inter], U[:, nbr[inter]])
                d = self.bc[ch, f] == DIRICHLET
                acc[:, d] += np.einsum("eij,bej->bei", Fb[d], U[:, ch[d]])
            out[:, ch] = acc
        return out if u.ndim == 3 else out[0]

    def assemble(self, lam=0.0):
        """Sparse CSR matrix of the bilinear form, A[(e,i),(e',j)] = a(l_j^{e'}, l_i^e)."""
        rows, cols, vals = [], [], []
        Np = self.Np
        ii, jj = np.meshgrid(np.arange(Np), np.arange(Np), indexing="ij")
        for ch in self._chunks(np.arange(self.K)):
            Ke, faces = self.local_blocks(ch, lam)
            blocks = [(ch, ch, Ke)]
            for f in range(4):
                Fm, Fp, nbr, Fb, _, _, _ = faces[f]
                inter = nbr >= 0
                d = self.bc[ch, f] == DIRICHLET
                blocks += [(ch[inter], ch[inter], Fm[inter]), (ch[inter], nbr[inter], Fp[inter]), (ch[d], ch[d], Fb[d])]
            for er, ec, Bk in blocks:
                rows.append((er[:, None, None] * Np + ii[None]).ravel())
                cols.append((ec[:, None, None] * Np + jj[None]).ravel())
                vals.append(Bk.ravel())
        n = self.K * Np
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()
        A.sum_duplicates()
        return A

    def mass_apply(self, f):
        """J M f per element (f nodal, (K, Np) or (B, K, Np))."""
        Mref = np.einsum("q,qi,qj->ij", self.wq, self.Lq, self.Lq)
        return np.einsum("ij,...ej->...ei", Mref, np.asarray(f, dtype=np.float64)) * self.geo.J[:, None]

    def dirichlet_lift(self, g):
        """L(g)_i = sum over Dirichlet faces of (n.grad l_i, g) - 2 tau (l_i, g), g nodal."""
        g = np.asarray(g, dtype=np.float64)
        out = np.zeros((self.K, self.Np))
        for ch in self._chunks(np.arange(self.K)):
            _, faces = self.local_blocks(ch, 0.0)
            for f in range(4):
                _, _, _, _, A1, A2, tau = faces[f]
                d = self.bc[ch, f] == DIRICHLET
                Lg = np.swapaxes(A1[d], 1, 2) - 2.0 * tau[d, None, None] * A2[d]
                out[ch[d]] += np.einsum("eij,ej->ei", Lg, g[ch[d]])
        return out

    def rhs(self, f_nodal, g_nodal):
        """b = J M f - L(g): the weak right-hand side of -lap u = f, u = g on Dirichlet faces."""
        return self.mass_apply(f_nodal) - self.dirichlet_lift(g_nodal)
