"""FP64 CPU oracle for the SIPDG pressure-Poisson hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the library imports this package; only
the tests, the smoke check and the CPU-baseline leg of the benchmark use it.
It is a plain, slow, obviously-correct restatement of the discretisation of
Karakus, Chalmers, Swirydowicz & Warburton (arXiv:1801.00246):

  basis.py      nodal basis on the triangle (Section 2.1), Warp & Blend nodes,
                orthonormal simplex basis, Gauss rules
  geometry.py   affine element maps, normals, face lengths, connectivity
                (Section 5.2, Eq. operators1-2)
  sipdg.py      the SIPDG bilinear form of Eq. ellipticOp1 / Eq. INS_SD_5,
                integrated by quadrature, assembled or applied element by element
  solvers.py    CG, PCG, flexible CG, Chebyshev smoothing, the p-multigrid
                V-cycle (Section 3)
  refops.py     reference-element operators M, Dr, Ds, LIFT (Eq. elMass,
                elStiff, elLift) used by the pins and by the p-multigrid
                transfer operators

Readings where the paper is silent or inconsistent are listed in the module
that takes them. Every function cites the passage it follows.
"""
