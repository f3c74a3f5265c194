"""Affine element maps, face data and face connectivity (oracle).

TEST INFRASTRUCTURE ONLY.

Section 5.2 (Eq. operators1, operators2): each triangle is the affine image
x = Phi^e(r, s) of the bi-unit triangle with vertices (-1,-1), (1,-1), (-1,1);
G^e = [[r_x, s_x], [r_y, s_y]] and J^e = det of the map's Jacobian. Here the
map and its inverse are written out directly from the vertex coordinates,
face normals from the edge vectors, so nothing depends on node orderings.
"""
import numpy as np

REF_VERTS = np.array([[-1.0, -1.0], [1.0, -1.0], [-1.0, 1.0]])


class Geometry:
    """Per-element affine map, its inverse metric G^e and Jacobian J^e, edge
    normals and lengths, and face neighbours (Section 5.2, Eq. operators2)."""

    def __init__(self, VX, VY, EToV):
        self.VX = np.asarray(VX, dtype=np.float64)
        self.VY = np.asarray(VY, dtype=np.float64)
        self.EToV = np.asarray(EToV, dtype=np.int64)
        K = self.EToV.shape[0]
        self.K = K
        P = np.stack([self.VX[self.EToV], self.VY[self.EToV]], axis=-1)  # (K,3,2)
        self.P = P
        # x = P0 + 0.5*(P1-P0)*(r+1) + 0.5*(P2-P0)*(s+1)
        jac = np.empty((K, 2, 2))
        jac[:, :, 0] = 0.5 * (P[:, 1] - P[:, 0])   # (x_r, y_r)
        jac[:, :, 1] = 0.5 * (P[:, 2] - P[:, 0])   # (x_s, y_s)
        self.jac = jac                               # [[x_r, x_s], [y_r, y_s]]
        self.J = np.linalg.det(jac)
        if np.any(self.J <= 0):
            raise ValueError("element with non-positive Jacobian (vertices not counter-clockwise)")
        self.inv = np.linalg.inv(jac)                # [[r_x, r_y], [s_x, s_y]]
        self.area = 2.0 * self.J
        # faces: f joins local vertices f and f+1
        self.face_len = np.empty((K, 3))
        self.normal = np.empty((K, 3, 2))
        for f in range(3):
            d = P[:, (f + 1) % 3] - P[:, f]
            L = np.hypot(d[:, 0], d[:, 1])
            self.face_len[:, f] = L
            self.normal[:, f, 0] = d[:, 1] / L
            self.normal[:, f, 1] = -d[:, 0] / L
        self.EToE, self.EToF = self._connect()

    def _connect(self):
        """Neighbour element and face across each face (-1 on the boundary)."""
        K = self.K
        EToE = -np.ones((K, 3), dtype=np.int64)
        EToF = -np.ones((K, 3), dtype=np.int64)
        seen = {}
        for e in range(K):
            for f in range(3):
                a = int(self.EToV[e, f])
                b = int(self.EToV[e, (f + 1) % 3])
                key = (min(a, b), max(a, b))
                if key in seen:
                    e2, f2 = seen.pop(key)
                    EToE[e, f], EToF[e, f] = e2, f2
                    EToE[e2, f2], EToF[e2, f2] = e, f
                else:
                    seen[key] = (e, f)
        return EToE, EToF

    def to_physical(self, elems, r, s):
        """Physical coordinates of reference points (r, s) in elements `elems`
        (the affine map of Eq. operators2). r, s broadcast against elems[:, None]."""
        P0 = self.P[elems, 0]
        jac = self.jac[elems]
        rr = np.asarray(r) + 1.0
        ss = np.asarray(s) + 1.0
        x = P0[:, 0, None] + jac[:, 0, 0, None] * rr + jac[:, 0, 1, None] * ss
        y = P0[:, 1, None] + jac[:, 1, 0, None] * rr + jac[:, 1, 1, None] * ss
        return x, y

    def to_reference(self, elems, x, y):
        """Reference coordinates in elements `elems` of physical points (x, y),
        arrays of shape (len(elems), n): the inverse of the map of Eq. operators2,
        used to evaluate a neighbour's basis at shared face points."""
        P0 = self.P[elems, 0]
        inv = self.inv[elems]
        dx = x - P0[:, 0, None]
        dy = y - P0[:, 1, None]
        r = inv[:, 0, 0, None] * dx + inv[:, 0, 1, None] * dy - 1.0
        s = inv[:, 1, 0, None] * dx + inv[:, 1, 1, None] * dy - 1.0
        return r, s
