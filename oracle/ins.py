"""Semi-implicit INS time step with semi-Lagrangian subcycling (oracle).

TEST INFRASTRUCTURE ONLY. FP64 throughout; every integral by quadrature with
the neighbour's basis evaluated at the same physical face points.

Section 2.2 (Eq. INS_TD_2, INS_TD_3) with the second-order BDF/EXT
coefficients and a first-order pressure increment (Section 4 uses it), and
Section 2.3 (Eq. SS_2, SS_3, INS_CUB_N) for the advection stage:

  (i)   U^ = sum_i beta_i U~^{n-i}: each U^{n-i} is advected from t^{n-i} to
        t^{n+1} by dU~/dt = -N~(Ubar, U~) with LSERK(5,4) substeps of dt/Ns,
        Ubar(t) the linear extrapolant through U^n, U^{n-1};
  (ii)  (-L + gamma/(nu dt)) U^^ = U^/(nu dt) - (1/nu) G P^n;
  (iii) -L dP = -(gamma/dt) D.U^^;
  (iv)  U^{n+1} = U^^ - (dt/gamma) G dP,  P^{n+1} = P^n + dP.

G and D carry central fluxes (Eq. INS_SD_4_1, INS_SD_4_2). N~ is the weak
form of Eq. INS_CUB_N with the local Lax-Friedrichs flux
  n.F* = 1/2 (n.Ubar- u- + n.Ubar+ u+) + 1/2 Lambda (u- - u+),
  Lambda = max(|n.Ubar-|, |n.Ubar+|),
with the dissipative sign of the paper's surface-kernel algorithm (the printed
Eq. INS_SD_3 has the opposite, anti-dissipative sign).

Readings where the paper is silent or inconsistent:
  * BDF2 beta_1 = -1/2 (the printed +1/2 violates sum beta = gamma);
    start-up step: BDF1/EXT1 (gamma = 1, beta_0 = 1, Ubar = U^0);
  * boundary data: velocity-Dirichlet faces take u+ = g (advection), u* = g
    (divergence); pressure-Dirichlet faces take p* = g_p (gradient); on
    pressure-Neumann faces p* = p-; on velocity-Neumann faces u* = u-. Steady
    data (the Kovasznay flow) make the pressure increment zero on
    pressure-Dirichlet faces. Time-dependent data g(t), g_p(t) (the Taylor
    vortex of Section 4.1) enter at the times each stage needs them: the
    advection stage at time t uses g(t), the Helmholtz solve and the
    divergence use g(t^{n+1}), G P^n uses g_p(t^n), and the increment takes
    g_p(t^{n+1}) - g_p(t^n) on pressure-Dirichlet faces;
  * the cubature is the collapsed Gauss rule with ceil((3N+1)/2) points per
    direction on the triangle and Gauss-Legendre with as many points per face
    (exact for the degree-3N advection integrands);
  * LSERK(5,4) coefficients of Carpenter & Kennedy (1994), cited by the paper.
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import basis
from .geometry import REF_VERTS
from .sipdg import DIRICHLET, NEUMANN

# Carpenter & Kennedy (1994), five-stage fourth-order 2N-storage Runge-Kutta
LSERK_A = np.array([0.0,
                    -567301805773.0 / 1357537059087.0,
                    -2404267990393.0 / 2016746695238.0,
                    -3550918686646.0 / 2091501179385.0,
                    -1275806237668.0 / 842570457699.0])
LSERK_B = np.array([1432997174477.0 / 9575080441755.0,
                    5161836677717.0 / 13612068292357.0,
                    1720146321549.0 / 2090206949498.0,
                    3134564353537.0 / 4481467310338.0,
                    2277821191437.0 / 14882151754819.0])
LSERK_C = np.array([0.0,
                    1432997174477.0 / 9575080441755.0,
                    2526269341429.0 / 6820363962896.0,
                    2006345519317.0 / 3224310063776.0,
                    2802321613138.0 / 2924317926251.0])


def lserk_integrate(f, y, t, dt, nsteps):
    """Integrate y' = f(t, y) with LSERK(5,4) (2N-storage form): the substep
    integrator of the subcycling of Section 2.3 (Carpenter & Kennedy 1994, which
    the paper cites)."""
    res = np.zeros_like(y)
    for _ in range(nsteps):
        for s in range(5):
            res = LSERK_A[s] * res + dt * f(t + LSERK_C[s] * dt, y)
            y = y + LSERK_B[s] * res
        t = t + dt
    return y


class InsOracle:
    """Operators of the split scheme of Section 2.2 (G, D of Eq. INS_SD_4_1-2,
    the advection of Eq. INS_CUB_N) on a velocity-tagged and a pressure-tagged
    SIPDG discretisation of the same mesh and degree."""

    def __init__(self, Su, Sp):
        assert Su.N == Sp.N and Su.K == Sp.K
        self.Su, self.Sp = Su, Sp
        self.N, self.Np, self.K = Su.N, Su.Np, Su.K
        g = Su.geo
        self.geo = g
        nc = -(-(3 * self.N + 1) // 2)
        self.nc = nc
        rq, sq, wq = basis.triangle_quadrature(nc)
        self.wq = wq
        self.Lq = basis.vandermonde(self.N, rq, sq) @ Su.Vinv
        Vr, Vs = basis.vandermonde_grad(self.N, rq, sq)
        self.Lrq, self.Lsq = Vr @ Su.Vinv, Vs @ Su.Vinv
        t, w = basis.gauss_legendre(nc)
        self.tf, self.wf = t, w
        self.face = []
        for f in range(3):
            va, vb = REF_VERTS[f], REF_VERTS[(f + 1) % 3]
            rf = va[0] + 0.5 * (t + 1.0) * (vb[0] - va[0])
            sf = va[1] + 0.5 * (t + 1.0) * (vb[1] - va[1])
            self.face.append((rf, sf, basis.vandermonde(self.N, rf, sf) @ Su.Vinv))
        self.Mref = np.einsum("q,qi,qj->ij", wq, self.Lq, self.Lq)
        self.Minv = np.linalg.inv(self.Mref)
        inv = g.inv
        self.rx, self.ry, self.sx, self.sy = inv[:, 0, 0], inv[:, 0, 1], inv[:, 1, 0], inv[:, 1, 1]
        # neighbour basis at every face quadrature point (K, nq, Np) per face
        self.nbr_basis = []
        for f in range(3):
            rf, sf, _ = self.face[f]
            nbr = g.EToE[:, f]
            Lp = np.zeros((self.K, nc, self.Np))
            inter = nbr >= 0
            e_in = np.nonzero(inter)[0]
            if len(e_in):
                xq, yq = g.to_physical(e_in, rf[None, :], sf[None, :])
                rp, spp = g.to_reference(nbr[e_in], xq, yq)
                Lp[e_in] = Su._eval_basis(rp, spp)[0]
            self.nbr_basis.append(Lp)

    # -- helpers ------------------------------------------------------------
    def _face_vals(self, f, field, nodal_bc, tags):
        """Interior and exterior traces of `field` (K, Np) at face f's
        quadrature points; exterior = neighbour's value on interior faces,
        the Dirichlet datum (nodal trace of nodal_bc) on Dirichlet faces and
        the interior value on Neumann faces."""
        _, _, Lf = self.face[f]
        um = field @ Lf.T                                          # (K, nq)
        nbr = self.geo.EToE[:, f]
        up = um.copy()
        inter = nbr >= 0
        up[inter] = np.einsum("eqj,ej->eq", self.nbr_basis[f][inter], field[nbr[inter]])
        d = tags[:, f] == DIRICHLET
        if nodal_bc is not None:
            up[d] = nodal_bc[d] @ Lf.T
        return um, up, d, tags[:, f] == NEUMANN

    def _face_weight(self, f):
        return self.wf[None, :] * 0.5 * self.geo.face_len[:, f][:, None]   # (K, nq)

    def weak_grad(self, p, gp):
        """(l_i, G p) per Eq. INS_SD_4_1 with p* = {p} inside, p* = g_p on
        pressure-Dirichlet faces and p* = p- on pressure-Neumann faces."""
        J = self.geo.J
        pr = p @ self.Lrq.T
        ps = p @ self.Lsq.T
        px = self.rx[:, None] * pr + self.sx[:, None] * ps
        py = self.ry[:, None] * pr + self.sy[:, None] * ps
        out = np.stack([np.einsum("q,qi,eq->ei", self.wq, self.Lq, px),
                        np.einsum("q,qi,eq->ei", self.wq, self.Lq, py)]) * J[None, :, None]
        tags = self.Sp.bc
        for f in range(3):
            _, _, Lf = self.face[f]
            pm, pp, d, neu = self._face_vals(f, p, gp, tags)
            jump = pp - pm
            jump[d] = 2.0 * (pp[d] - pm[d])       # p* = g  ->  p+ = 2 g - p-
            jump[neu] = 0.0
            W = self._face_weight(f)
            n = self.geo.normal[:, f]
            for c in range(2):
                out[c] += 0.5 * np.einsum("eq,qi,eq->ei", W, Lf, n[:, c, None] * jump)
        return out

    def weak_div(self, U, gU):
        """(l_i, D.U) per Eq. INS_SD_4_2 with u* = {u} inside, u* = g on
        velocity-Dirichlet faces and u* = u- on velocity-Neumann faces."""
        J = self.geo.J
        u, v = U
        ux = self.rx[:, None] * (u @ self.Lrq.T) + self.sx[:, None] * (u @ self.Lsq.T)
        vy = self.ry[:, None] * (v @ self.Lrq.T) + self.sy[:, None] * (v @ self.Lsq.T)
        out = np.einsum("q,qi,eq->ei", self.wq, self.Lq, ux + vy) * J[:, None]
        tags = self.Su.bc
        for f in range(3):
            _, _, Lf = self.face[f]
            W = self._face_weight(f)
            n = self.geo.normal[:, f]
            nj = np.zeros((self.K, self.nc))
            for c in range(2):
                um, up, d, neu = self._face_vals(f, U[c], None if gU is None else gU[c], tags)
                jump = up - um
                jump[d] = 2.0 * (up[d] - um[d])
                jump[neu] = 0.0
                nj += n[:, c, None] * jump
            out += 0.5 * np.einsum("eq,qi,eq->ei", W, Lf, nj)
        return out

    def to_strong(self, weak):
        """(J M)^{-1} applied element-wise: weak to nodal values with the element
        mass matrix of Eq. elMass."""
        return np.einsum("ij,...ej->...ei", self.Minv, weak) / self.geo.J[:, None]

    def advection(self, Ubar, Ut, gU):
        """Strong -N~(Ubar, U~) (the right-hand side of Eq. SS_3) for both
        components, by cubature (Eq. INS_CUB_N)."""
        J = self.geo.J
        ub = Ubar @ self.Lq.T       # (2, K, nq)
        ut = Ut @ self.Lq.T
        weak = np.zeros_like(Ut)
        for c in range(2):
            Fx = ub[0] * ut[c]
            Fy = ub[1] * ut[c]
            # -(grad l_i, Ubar u~_c)_E
            gx = self.rx[:, None, None] * self.Lrq[None] + self.sx[:, None, None] * self.Lsq[None]
            gy = self.ry[:, None, None] * self.Lrq[None] + self.sy[:, None, None] * self.Lsq[None]
            weak[c] = -J[:, None] * (np.einsum("q,eqi,eq->ei", self.wq, gx, Fx)
                                     + np.einsum("q,eqi,eq->ei", self.wq, gy, Fy))
        tags = self.Su.bc
        for f in range(3):
            _, _, Lf = self.face[f]
            W = self._face_weight(f)
            n = self.geo.normal[:, f]
            bm, bp = [], []
            for c in range(2):
                m_, p_, d, neu = self._face_vals(f, Ubar[c], gU[c], tags)
                bm.append(m_)
                bp.append(p_)
            unm = n[:, 0, None] * bm[0] + n[:, 1, None] * bm[1]
            unp = n[:, 0, None] * bp[0] + n[:, 1, None] * bp[1]
            lam = np.maximum(np.abs(unm), np.abs(unp))
            for c in range(2):
                tm, tp, _, _ = self._face_vals(f, Ut[c], gU[c], tags)
                flux = 0.5 * (unm * tm + unp * tp) + 0.5 * lam * (tm - tp)
                weak[c] += np.einsum("eq,qi,eq->ei", W, Lf, flux)
        return -self.to_strong(weak)

    # -- the split step -------------------------------------------------------
    def step(self, st, dt, nu, Ns, gU, gP, solve=None):
        """One time step of Eq. INS_TD_3 (steps (i)-(iv) of the module header)
        with the subcycled advection of Section 2.3; st = dict(U, Uold, P, n).
        gU, gP: steady nodal data, or callables of t returning them
        (time-dependent data, t^n = n dt). Returns the new state and the
        intermediate fields (U^, U^^, dP) for inspection."""
        U, Uold, P, n = st["U"], st["Uold"], st["P"], st["n"]
        t = n * dt
        unsteady = callable(gU)
        gUt = gU if unsteady else (lambda tt: gU)
        gPt = gP if unsteady else (lambda tt: gP)
        dts = dt / Ns
        if n == 0:
            gamma, betas = 1.0, [1.0]
            ubar = lambda tt: U
            starts = [(U, t, Ns)]
        else:
            gamma, betas = 1.5, [2.0, -0.5]
            ubar = lambda tt: U + (tt - t) / dt * (U - Uold)
            starts = [(U, t, Ns), (Uold, t - dt, 2 * Ns)]
        Uhat = np.zeros_like(U)
        for beta, (U0, t0, nsub) in zip(betas, starts):
            rhs = lambda tt, y: self.advection(ubar(tt), y, gUt(tt))
            Uhat += beta * lserk_integrate(rhs, U0, t0, dts, nsub)
        lam = gamma / (nu * dt)
        Au = self.Su.assemble(lam).tocsc()
        G = self.weak_grad(P, gPt(t))
        g1 = gUt(t + dt)
        Uhh = np.zeros_like(U)
        for c in range(2):
            b = self.Su.mass_apply(Uhat[c]) / (nu * dt) - G[c] / nu - self.Su.dirichlet_lift(g1[c])
            Uhh[c] = (solve or _direct)(Au, b)
        Ap = self.Sp.assemble(0.0).tocsc()
        bp = -(gamma / dt) * self.weak_div(Uhh, g1)
        gdP = gPt(t + dt) - gPt(t) if unsteady else np.zeros_like(P)
        if unsteady:
            bp = bp - self.Sp.dirichlet_lift(gdP)
        dP = (solve or _direct)(Ap, bp)
        Gd = self.to_strong(self.weak_grad(dP, gdP))
        Unew = Uhh - (dt / gamma) * Gd
        new = dict(U=Unew, Uold=U, P=P + dP, n=n + 1)
        return new, dict(Uhat=Uhat, Uhh=Uhh, dP=dP)


def _direct(A, b):
    return spla.spsolve(A, b.ravel()).reshape(b.shape)
