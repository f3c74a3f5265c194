"""Reference-element operators of Section 5.2 (oracle).

TEST INFRASTRUCTURE ONLY.

Eq. elMass, elStiff, elLift on the bi-unit triangle with the nodal basis:
  M_ij   = (l_i, l_j)                 = ((V V^T)^{-1})_ij  (V orthonormal-mode Vandermonde)
  Dr_ij  = dl_j/dr at node i          = (V_r V^{-1})_ij,   Ds likewise
  Mf     = 1-D face mass on the N+1 face nodes, in the face parameter t in [-1,1]
  LIFT   = M^{-1} E, E placing Mf of face f at that face's nodes (Np x 3(N+1))
and the p-multigrid interpolation P_{f<-c} = V_c(r_f, s_f) V_c^{-1} (the
coarse nodal polynomial evaluated at the fine nodes; restriction R = P^T).
"""
import numpy as np

from . import basis


def reference_operators(N):
    """Nodes, M, Dr, Ds, the face mass and LIFT of degree N on the reference
    triangle (Section 5.2, Eq. elMass, Eq. operators1, Eq. elLift)."""
    r, s = basis.warp_blend_nodes(N)
    V = basis.vandermonde(N, r, s)
    Vinv = np.linalg.inv(V)
    Vr, Vs = basis.vandermonde_grad(N, r, s)
    M = np.linalg.inv(V @ V.T)
    Dr = Vr @ Vinv
    Ds = Vs @ Vinv
    fl = basis.face_node_lists(N)
    Nfp = N + 1
    t = basis.gauss_lobatto(N)
    V1 = np.stack([basis.jacobi_normalized(t, 0, 0, k) for k in range(N + 1)], axis=1)
    Mf = np.linalg.inv(V1 @ V1.T)
    Np = len(r)
    E = np.zeros((Np, 3 * Nfp))
    for f in range(3):
        for a in range(Nfp):
            for b in range(Nfp):
                E[fl[f][a], f * Nfp + b] += Mf[a, b]
    LIFT = np.linalg.solve(M, E)
    return dict(r=r, s=s, V=V, M=M, Dr=Dr, Ds=Ds, Mf=Mf, LIFT=LIFT, E=E, faces=fl, t=t)


def interpolation(Nf, Nc):
    """P (Np_f x Np_c): values at the degree-Nf nodes of the degree-Nc nodal basis,
    the prolongation of the degree-coarsening multigrid of Section 3 (its form is
    a reading: the paper does not print the transfer operators)."""
    rf, sf = basis.warp_blend_nodes(Nf)
    rc, sc = basis.warp_blend_nodes(Nc)
    Vc = basis.vandermonde(Nc, rc, sc)
    return basis.vandermonde(Nc, rf, sf) @ np.linalg.inv(Vc)
