"""Krylov solvers, Chebyshev smoothing and the p-multigrid V-cycle (oracle).

TEST INFRASTRUCTURE ONLY. All arithmetic in FP64.

Section 3: both elliptic systems are solved by preconditioned conjugate
gradients; the screened-Poisson (velocity) system with the scaled inverse
mass matrix of each element as preconditioner, the pressure system with a
multigrid preconditioner that coarsens the polynomial degree N -> ... -> 1
matrix-free and smooths with a degree-2 Chebyshev iteration. Readings taken
where the paper is silent (the AMG tail at degree 1 is replaced by CG to a
loose relative tolerance):
  * coarse operators are the SIPDG operator rediscretised at each degree
    (penalty recomputed with that degree), not Galerkin products;
  * prolongation P interpolates the coarse nodal polynomial at the fine nodes,
    restriction R = P^T;
  * smoothing = Chebyshev iteration of the given degree on D^{-1} A, D =
    diag(A), on the interval [rho/10, 1.1 rho], rho ~ largest eigenvalue of
    D^{-1} A from a fixed number of power steps;
  * with a preconditioner that is not a fixed SPD operator (single-precision
    levels, inner CG) the outer iteration is flexible CG with
    beta = r_{k+1}^T (z_{k+1} - z_k) / r_k^T z_k.
The residual norm is ||b - A x||_2 / ||b||_2 on the weak coefficient vector.

Parity unpinned: the iteration counts of the p-multigrid preconditioned solve
(Section 4 reports them as figures only). What is pinned: the V-cycle's
symmetry with an exact coarse solve, the Chebyshev error factor against its
closed form, CG's finite termination, and every solution through its
residual against the assembled operator.
"""
import numpy as np


def cg(apply, b, x0=None, tol=1e-10, maxit=10000, prec=None, flexible=False):
    """(Flexible) preconditioned CG (Section 3; flexible beta with a variable
    preconditioner, a reading). Returns (x, iters, relres)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply(x)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, 0.0
    z = prec(r) if prec is not None else r.copy()
    p = z.copy()
    rz = float(np.vdot(r, z))
    it = 0
    relres = np.linalg.norm(r) / nb
    while relres > tol and it < maxit:
        Ap = apply(p)
        pAp = float(np.vdot(p, Ap))
        if not pAp > 0.0:
            raise FloatingPointError("CG breakdown: p^T A p <= 0")
        alpha = rz / pAp
        x = x + alpha * p
        r = r - alpha * Ap
        it += 1
        relres = np.linalg.norm(r) / nb
        if relres <= tol:
            break
        z_new = prec(r) if prec is not None else r.copy()
        if flexible:
            beta = float(np.vdot(r, z_new - z)) / rz
        else:
            beta = float(np.vdot(r, z_new)) / rz
        rz = float(np.vdot(r, z_new))
        z = z_new
        p = z + beta * p
    return x, it, relres


def chebyshev(apply, dinv, b, x, lmin, lmax, degree):
    """`degree` steps of the Chebyshev iteration for A x = b preconditioned by
    D = diag(A), eigenvalues of D^{-1}A assumed in [lmin, lmax] (Saad,
    Iterative Methods for Sparse Linear Systems, Alg. 12.1)."""
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = b - apply(x)
    d = dinv * r / theta
    for k in range(degree):
        x = x + d
        if k == degree - 1:
            break
        r = r - apply(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + 2.0 * rho_new / delta * (dinv * r)
        rho = rho_new
    return x


def power_rho(apply, dinv, shape, steps=20, seed=12345):
    """Largest eigenvalue of D^{-1} A estimated by `steps` power iterations
    from a seeded random start: the bound of the Chebyshev smoother of Section 3
    (its estimate is a reading: the paper does not say how it is obtained)."""
    v = np.random.default_rng(seed).standard_normal(shape)
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(steps):
        w = dinv * apply(v)
        lam = float(np.linalg.norm(w))
        v = w / lam
    return lam


class PMultigrid:
    """V-cycle over degrees levels[0] > levels[1] > ... > levels[-1]: the
    degree-coarsening multigrid preconditioner of Section 3.

    ops[l] = (apply, dinv) of the SIPDG operator at degree levels[l] on
    (K, Np_l) arrays; P[l] interpolates level l+1 to level l (Np_l x Np_{l+1}).
    The coarsest level is solved by CG to relative tolerance coarse_tol, or
    exactly by `coarse_solve` if given.
    """

    def __init__(self, ops, P, shapes, cheb_degree=2, coarse_tol=1e-2, coarse_solve=None,
                 power_steps=20, seed=12345):
        self.ops, self.P, self.shapes = ops, P, shapes
        self.cheb_degree = cheb_degree
        self.coarse_tol = coarse_tol
        self.coarse_solve = coarse_solve
        self.bounds = []
        for l in range(len(ops) - 1):
            apply, dinv = ops[l]
            rho = power_rho(apply, dinv, shapes[l], power_steps, seed)
            self.bounds.append((rho / 10.0, 1.1 * rho))
        self.coarse_iters = []

    def vcycle(self, r, l=0):
        """One V-cycle from level l (Section 3): Chebyshev pre-smoothing, residual,
        restriction by P^T, recursion, prolongation by P, post-smoothing."""
        if l == len(self.ops) - 1:
            apply, _ = self.ops[l]
            if self.coarse_solve is not None:
                return self.coarse_solve(r)
            x, it, _ = cg(apply, r, tol=self.coarse_tol, maxit=10000)
            self.coarse_iters.append(it)
            return x
        apply, dinv = self.ops[l]
        lmin, lmax = self.bounds[l]
        x = chebyshev(apply, dinv, r, np.zeros_like(r), lmin, lmax, self.cheb_degree)
        res = r - apply(x)
        rc = np.einsum("ij,...ei->...ej", self.P[l], res)        # R = P^T
        ec = self.vcycle(rc, l + 1)
        x = x + np.einsum("ij,...ej->...ei", self.P[l], ec)     # prolong
        x = chebyshev(apply, dinv, r, x, lmin, lmax, self.cheb_degree)
        return x


def inverse_mass_prec(sip, lam):
    """Block preconditioner z_e = (lam J_e M)^{-1} r_e (Section 3, screened Poisson)."""
    Minv = np.linalg.inv(sip.mass_matrix_ref())
    J = sip.geo.J

    def prec(r):
        """z_e = (lam J_e M)^{-1} r_e (Section 3)."""
        return np.einsum("ij,...ej->...ei", Minv, r) / (lam * J[:, None])
    return prec
