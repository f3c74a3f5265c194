"""SIPDG Poisson / screened-Poisson operator from its bilinear form (oracle).

TEST INFRASTRUCTURE ONLY.

Eq. ellipticOp1 (equivalently Eq. INS_SD_5 with the lambda term) defines, for
each element E and every test function v in P_N(E),

  a_E(u, v) = (grad v, grad u)_E - (v, n.{grad u})_dE + 1/2 (n.grad v, [u])_dE
              - (v, tau [u])_dE + lambda (v, u)_E,

with {w} = (w+ + w-)/2 and [w] = w+ - w- (Eq. AverageJumpScalar; "-" is the
element's own trace, "+" the neighbour's) and the per-face penalty of
Eq. PenaltyParameter, tau = (N+1)(N+2)/2 max(1/h+, 1/h-), h = |E| / |face|.
The operator's output is the weak coefficient vector (A u)_i = a_E(u, l_i).

Every integral is taken by quadrature that is exact for the integrand: a
collapsed Gauss rule on the triangle and Gauss-Legendre on each face, with
the neighbour's basis evaluated at the same physical face points through the
neighbour's own inverse map. No face-node ordering or lift operator is used,
so agreement with a factored implementation (Eq. ellipticOp3) also checks the
factorisation.

Readings taken where the paper is silent (Section 2.1 only says boundary
conditions are imposed "analogously"):
  * Dirichlet face: ghost state u+ = 2 g - u-, grad u+ = grad u-. The
    homogeneous operator then carries the boundary penalty 2 tau, and the data
    enter the right-hand side as b = M f - L(g) with
    L(g)_i = (n.grad l_i, g)_dD - 2 tau (l_i, g)_dD, g the nodal trace.
  * Neumann face (zero flux): u+ = u-, grad u+ = -grad u-; no face terms.
  * Boundary penalty uses the interior element only: tau = (N+1)(N+2)/2 / h-.
"""
import numpy as np
import scipy.sparse as sp

from . import basis
from .geometry import Geometry, REF_VERTS

INTERIOR, DIRICHLET, NEUMANN = 0, 1, 2


class Sipdg:
    """Reference data plus per-element quadrature for degree N on a mesh: the
    SIPDG bilinear form of Eq. ellipticOp1 (Section 5.2; Eq. INS_SD_5 in Section 2.1)."""

    def __init__(self, VX, VY, EToV, bc, N):
        self.N = N
        self.Np = (N + 1) * (N + 2) // 2
        self.geo = Geometry(VX, VY, EToV)
        self.K = self.geo.K
        self.bc = np.asarray(bc, dtype=np.int64)
        bnd = self.geo.EToE < 0
        if np.any(bnd & (self.bc == INTERIOR)) or np.any(~bnd & (self.bc != INTERIOR)):
            raise ValueError("boundary tags disagree with the face connectivity")
        self.r, self.s = basis.warp_blend_nodes(N)
        self.V = basis.vandermonde(N, self.r, self.s)
        self.Vinv = np.linalg.inv(self.V)
        # volume rule, exact to degree 2N+1
        rq, sq, wq = basis.triangle_quadrature(N + 1)
        self.wq = wq
        self.Lq = basis.vandermonde(N, rq, sq) @ self.Vinv
        Vr, Vs = basis.vandermonde_grad(N, rq, sq)
        self.Lrq, self.Lsq = Vr @ self.Vinv, Vs @ self.Vinv
        # face rule, exact to degree 2N+1, on each reference face
        t, w = basis.gauss_legendre(N + 1)
        self.tf, self.wf = t, w
        self.face_ref = []
        for f in range(3):
            va, vb = REF_VERTS[f], REF_VERTS[(f + 1) % 3]
            rf = va[0] + 0.5 * (t + 1.0) * (vb[0] - va[0])
            sf = va[1] + 0.5 * (t + 1.0) * (vb[1] - va[1])
            Lf = basis.vandermonde(N, rf, sf) @ self.Vinv
            Vr, Vs = basis.vandermonde_grad(N, rf, sf)
            self.face_ref.append((rf, sf, Lf, Vr @ self.Vinv, Vs @ self.Vinv))
        # physical node coordinates (K, Np)
        self.x, self.y = self.geo.to_physical(np.arange(self.K), self.r[None, :], self.s[None, :])
        c = (N + 1) * (N + 2) / 2.0
        inv_h = self.geo.face_len / self.geo.area[:, None]              # 1/h- per face
        nb = np.where(self.geo.EToE >= 0, self.geo.EToE, 0)
        inv_h_nb = self.geo.face_len / self.geo.area[nb]
        self.tau = c * np.where(self.geo.EToE >= 0, np.maximum(inv_h, inv_h_nb), inv_h)

    # -- basis evaluation at arbitrary reference points --------------------
    def _eval_basis(self, r, s):
        shp = r.shape
        rr, ss = r.ravel(), s.ravel()
        L = basis.vandermonde(self.N, rr, ss) @ self.Vinv
        Vr, Vs = basis.vandermonde_grad(self.N, rr, ss)
        return (L.reshape(shp + (self.Np,)), (Vr @ self.Vinv).reshape(shp + (self.Np,)),
                (Vs @ self.Vinv).reshape(shp + (self.Np,)))

    def local_blocks(self, elems, lam=0.0):
        """Element matrix and face coupling matrices for the listed elements: the
        volume and face integrals of Eq. ellipticOp1, with the penalty of
        Eq. PenaltyParameter and the averages and jumps of Eq. AverageJumpScalar.

        Returns (Ke, faces) where Ke[e] = volume stiffness + lambda mass and
        faces[f] = (Fm, Fp, nbr, Fb_dir, A1, A2, tau) per face f.
        """
        g = self.geo
        elems = np.asarray(elems)
        inv = g.inv[elems]
        rx, ry = inv[:, 0, 0], inv[:, 0, 1]
        sx, sy = inv[:, 1, 0], inv[:, 1, 1]
        J = g.J[elems]
        lx = rx[:, None, None] * self.Lrq[None] + sx[:, None, None] * self.Lsq[None]
        ly = ry[:, None, None] * self.Lrq[None] + sy[:, None, None] * self.Lsq[None]
        Ke = (np.einsum("q,eqi,eqj->eij", self.wq, lx, lx)
              + np.einsum("q,eqi,eqj->eij", self.wq, ly, ly)) * J[:, None, None]
        if lam != 0.0:
            Mref = np.einsum("q,qi,qj->ij", self.wq, self.Lq, self.Lq)
            Ke = Ke + lam * J[:, None, None] * Mref[None]
        faces = []
        for f in range(3):
            rf, sf, Lf, Lrf, Lsf = self.face_ref[f]
            n = g.normal[elems, f]                                      # (E,2)
            W = self.wf[None, :] * 0.5 * g.face_len[elems, f][:, None]  # (E,nq)
            tau = self.tau[elems, f]
            gx = rx[:, None, None] * Lrf[None] + sx[:, None, None] * Lsf[None]
            gy = ry[:, None, None] * Lrf[None] + sy[:, None, None] * Lsf[None]
            dn_m = n[:, 0, None, None] * gx + n[:, 1, None, None] * gy   # (E,nq,Np)
            A1 = np.einsum("ek,ki,ekj->eij", W, Lf, dn_m)    # (l_i, n.grad l_j)
            A2 = np.einsum("ek,ki,kj->eij", W, Lf, Lf)       # (l_i, l_j)
            Fm = -0.5 * A1 - 0.5 * np.swapaxes(A1, 1, 2) + tau[:, None, None] * A2
            Fb = -A1 - np.swapaxes(A1, 1, 2) + 2.0 * tau[:, None, None] * A2
            nbr = g.EToE[elems, f]
            Fp = np.zeros_like(Fm)
            inter = nbr >= 0
            if np.any(inter):
                ei = elems[inter]
                en = nbr[inter]
                xq, yq = g.to_physical(ei, rf[None, :], sf[None, :])
                rp, spp = g.to_reference(en, xq, yq)
                Lp, Lrp, Lsp = self._eval_basis(rp, spp)
                invn = g.inv[en]
                gpx = invn[:, 0, 0, None, None] * Lrp + invn[:, 1, 0, None, None] * Lsp
                gpy = invn[:, 0, 1, None, None] * Lrp + invn[:, 1, 1, None, None] * Lsp
                ni = n[inter]
                dn_p = ni[:, 0, None, None] * gpx + ni[:, 1, None, None] * gpy
                Wi = W[inter]
                B1 = np.einsum("ek,ki,ekj->eij", Wi, Lf, dn_p)          # (l_i, n.grad l+_j)
                B2 = np.einsum("ek,eki,ekj->eij", Wi, dn_m[inter], Lp)  # (n.grad l_i, l+_j)
                B3 = np.einsum("ek,ki,ekj->eij", Wi, Lf, Lp)            # (l_i, l+_j)
                Fp[inter] = -0.5 * B1 + 0.5 * B2 - tau[inter, None, None] * B3
            faces.append((Fm, Fp, nbr, Fb, A1, A2, tau))
        return Ke, faces

    def _chunks(self, elems, size=2048):
        for i in range(0, len(elems), size):
            yield elems[i:i + size]

    def apply(self, u, lam=0.0, elems=None):
        """(A u) of Eq. ellipticOp1, matrix-free, on the listed elements (default all).
        u: (K, Np) or (B, K, Np)."""
        u = np.asarray(u, dtype=np.float64)
        batched = u.ndim == 3
        U = u if batched else u[None]
        elems = np.arange(self.K) if elems is None else np.asarray(elems)
        out = np.zeros((U.shape[0], len(elems), self.Np))
        pos = 0
        for ch in self._chunks(elems):
            Ke, faces = self.local_blocks(ch, lam)
            acc = np.einsum("eij,bej->bei", Ke, U[:, ch])
            for f in range(3):
                Fm, Fp, nbr, Fb, _, _, _ = faces[f]
                tag = self.bc[ch, f]
                inter = nbr >= 0
                acc[:, inter] += np.einsum("eij,bej->bei", Fm[inter], U[:, ch[inter]])
                acc[:, inter] += np.einsum("eij,bej->bei", Fp[inter], U[:, nbr[inter]])
                d = tag == DIRICHLET
                acc[:, d] += np.einsum("eij,bej->bei", Fb[d], U[:, ch[d]])
            out[:, pos:pos + len(ch)] = acc
            pos += len(ch)
        return out if batched else out[0]

    def assemble(self, lam=0.0):
        """Sparse CSR matrix A with A[(e,i),(e',j)] = a(l_j^{e'}, l_i^e), a the bilinear
        form of Eq. ellipticOp1."""
        rows, cols, vals = [], [], []
        Np = self.Np
        ii, jj = np.meshgrid(np.arange(Np), np.arange(Np), indexing="ij")
        for ch in self._chunks(np.arange(self.K)):
            Ke, faces = self.local_blocks(ch, lam)
            blocks = [(ch, ch, Ke)]
            for f in range(3):
                Fm, Fp, nbr, Fb, _, _, _ = faces[f]
                inter = nbr >= 0
                d = self.bc[ch, f] == DIRICHLET
                blocks.append((ch[inter], ch[inter], Fm[inter]))
                blocks.append((ch[inter], nbr[inter], Fp[inter]))
                blocks.append((ch[d], ch[d], Fb[d]))
            for er, ec, B in blocks:
                rows.append((er[:, None, None] * Np + ii[None]).ravel())
                cols.append((ec[:, None, None] * Np + jj[None]).ravel())
                vals.append(B.ravel())
        n = self.K * Np
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(n, n)).tocsr()
        A.sum_duplicates()
        return A

    def diagonal(self, lam=0.0):
        """diag(A) as a (K, Np) array (the Jacobi preconditioner of Section 3)."""
        out = np.zeros((self.K, self.Np))
        for ch in self._chunks(np.arange(self.K)):
            Ke, faces = self.local_blocks(ch, lam)
            dg = np.einsum("eii->ei", Ke).copy()
            for f in range(3):
                Fm, _, nbr, Fb, _, _, _ = faces[f]
                inter = nbr >= 0
                d = self.bc[ch, f] == DIRICHLET
                dg[inter] += np.einsum("eii->ei", Fm[inter])
                dg[d] += np.einsum("eii->ei", Fb[d])
            out[ch] = dg
        return out

    def mass_matrix_ref(self):
        """Reference mass matrix (l_i, l_j) on the bi-unit triangle, by quadrature
        (Eq. elMass)."""
        return np.einsum("q,qi,qj->ij", self.wq, self.Lq, self.Lq)

    def mass_apply(self, f):
        """(l_i, f_h)_E = J^e M f_e for a nodal field f (K, Np) or (B, K, Np) (the
        lambda term of Eq. ellipticOp1, and the load of the right-hand side)."""
        M = self.mass_matrix_ref()
        return np.einsum("ij,...ej->...ei", M, f) * self.geo.J[:, None]

    def dirichlet_lift(self, g):
        """L(g)_i = sum over Dirichlet faces of (n.grad l_i, g) - 2 tau (l_i, g),
        g the nodal trace of a field given at all nodes (K, Np): the data part of
        the Dirichlet faces of Eq. ellipticOp1 under the ghost state u+ = 2g - u-
        (a reading: Section 2.1 calls the boundary treatment analogous)."""
        g = np.asarray(g, dtype=np.float64)
        out = np.zeros((self.K, self.Np))
        for ch in self._chunks(np.arange(self.K)):
            _, faces = self.local_blocks(ch, 0.0)
            for f in range(3):
                _, _, _, _, A1, A2, tau = faces[f]
                d = self.bc[ch, f] == DIRICHLET
                Lg = np.swapaxes(A1[d], 1, 2) - 2.0 * tau[d, None, None] * A2[d]
                out[ch[d]] += np.einsum("eij,ej->ei", Lg, g[ch[d]])
        return out

    def rhs(self, f_nodal, g_nodal):
        """Weak right-hand side b = M f - L(g) of the Dirichlet problem (Eq. DirichletBC
        data; f interpolated at the nodes, a reading)."""
        return self.mass_apply(f_nodal) - self.dirichlet_lift(g_nodal)

    def l2_error(self, u_nodal, exact):
        """L2 norm of (u_h - exact) over the mesh, by the volume quadrature (the error
        norm of the convergence studies of Section 4)."""
        rq, sq, wq = basis.triangle_quadrature(self.N + 3)
        Lq = basis.vandermonde(self.N, rq, sq) @ self.Vinv
        xq, yq = self.geo.to_physical(np.arange(self.K), rq[None, :], sq[None, :])
        uh = np.einsum("qj,ej->eq", Lq, u_nodal)
        err = uh - exact(xq, yq)
        return float(np.sqrt(np.sum(wq[None, :] * err ** 2 * self.geo.J[:, None])))
