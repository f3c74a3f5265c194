"""Jittered structured tetrahedral meshes of a box.

Recipe: an n-by-n-by-n grid of cubes on [x0,x1]x[y0,y1]x[z0,z1]; vertices
numbered v = (k*(n+1) + j)*(n+1) + i; every interior vertex is shifted by
independent U(-jitter*h, jitter*h) draws per coordinate from numpy's
default_rng(seed), vertices in numbering order, x, y, z each. Each cube is cut
into six tetrahedra around its diagonal from corner (0,0,0) to (1,1,1): for
each ordering (p, q, r) of the three axes, the tetrahedron (000, 000+e_p,
000+e_p+e_q, 111), in the orderings (x,y,z), (x,z,y), (y,x,z), (y,z,x),
(z,x,y), (z,y,x); every cube is cut the same way, so faces conform. Two local
vertices are swapped where needed so that every element has a positive
Jacobian. Cubes are visited with i fastest, then j, then k.

Local faces of a tetrahedron: face 0 = (v0, v1, v2), face 1 = (v0, v1, v3),
face 2 = (v1, v2, v3), face 3 = (v0, v2, v3), opposite local vertices 3, 2, 0, 1. Boundary faces carry the tag of their side
(x0, x1, y0, y1, z0, z1 -> bc_sides[0..5]): 0 = interior, 1 = Dirichlet,
2 = Neumann.
"""
from dataclasses import dataclass
from itertools import permutations

import numpy as np

INTERIOR, DIRICHLET, NEUMANN = 0, 1, 2
_FACES = ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3))


@dataclass
class TetMesh:
    VX: np.ndarray
    VY: np.ndarray
    VZ: np.ndarray
    EToV: np.ndarray     # (K, 4) int32
    bc: np.ndarray       # (K, 4) int8

    @property
    def K(self):
        return int(self.EToV.shape[0])


def jittered_tet_grid(n, box=(0.0, 1.0, 0.0, 1.0, 0.0, 1.0), jitter=0.1, seed=0,
                      bc_sides=(DIRICHLET,) * 6):
    x0, x1, y0, y1, z0, z1 = box
    h = np.array([(x1 - x0) / n, (y1 - y0) / n, (z1 - z0) / n])
    idx = np.arange(n + 1)
    K3, J3, I3 = np.meshgrid(idx, idx, idx, indexing="ij")
    X = np.stack([x0 + I3.ravel() * h[0], y0 + J3.ravel() * h[1], z0 + K3.ravel() * h[2]], axis=1)
    rng = np.random.default_rng(seed)
    interior = ((I3 > 0) & (I3 < n) & (J3 > 0) & (J3 < n) & (K3 > 0) & (K3 < n)).ravel()
    for v in range(X.shape[0]):
        if interior[v]:
            X[v] += rng.uniform(-jitter, jitter, 3) * h
    vid = lambda i, j, k: (k * (n + 1) + j) * (n + 1) + i
    tets = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                for order in permutations(range(3)):
                    c = [0, 0, 0]
                    corners = [tuple(c)]
                    for ax in order[:2]:
                        c[ax] = 1
                        corners.append(tuple(c))
                    corners.append((1, 1, 1))
                    t = [vid(i + a, j + b, k + d) for a, b, d in corners]
                    P = X[t]
                    if np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]], axis=1)) < 0:
                        t[1], t[2] = t[2], t[1]
                    tets.append(t)
    EToV = np.array(tets, dtype=np.int32)
    # boundary tags: a face on a side plane of the box
    bc = np.zeros((len(tets), 4), dtype=np.int8)
    seen = {}
    for e, t in enumerate(tets):
        for f, loc in enumerate(_FACES):
            key = tuple(sorted(t[q] for q in loc))
            seen.setdefault(key, []).append((e, f))
    lo, hi = np.array([x0, y0, z0]), np.array([x1, y1, z1])
    for key, owners in seen.items():
        if len(owners) != 1:
            continue
        P = X[list(key)]
        tag = None
        for ax in range(3):
            if np.all(np.abs(P[:, ax] - lo[ax]) < 1e-12):
                tag = bc_sides[2 * ax]
            elif np.all(np.abs(P[:, ax] - hi[ax]) < 1e-12):
                tag = bc_sides[2 * ax + 1]
        if tag is None:
            raise RuntimeError("boundary face off the box sides")
        e, f = owners[0]
        bc[e, f] = tag
    return TetMesh(X[:, 0].copy(), X[:, 1].copy(), X[:, 2].copy(), EToV, bc)


def permute_local_vertices(mesh, seed):
    """The same mesh with each element's local vertices renumbered by an even
    permutation p drawn from default_rng(seed) (even permutations keep the
    orientation; new local vertex i is old local vertex p[i]), and the face tags
    moved with them: new face f is opposite new vertex OPP[f], which was old
    vertex p[OPP[f]], whose opposite face was old face FACE_OPP[p[OPP[f]]]."""
    from itertools import permutations as _perms
    OPP = (3, 2, 0, 1)        # the local vertex opposite face f
    FACE_OPP = (2, 3, 1, 0)   # the local face opposite vertex v
    even = [p for p in _perms(range(4))
            if sum(1 for i in range(4) for j in range(i + 1, 4) if p[i] > p[j]) % 2 == 0]
    rng = np.random.default_rng(seed)
    pick = rng.integers(0, len(even), size=mesh.K)
    EToV = np.empty_like(mesh.EToV)
    bc = np.empty_like(mesh.bc)
    for e in range(mesh.K):
        p = even[pick[e]]
        EToV[e] = mesh.EToV[e, list(p)]
        for f in range(4):
            bc[e, f] = mesh.bc[e, FACE_OPP[p[OPP[f]]]]
    return TetMesh(mesh.VX.copy(), mesh.VY.copy(), mesh.VZ.copy(), EToV, bc)
