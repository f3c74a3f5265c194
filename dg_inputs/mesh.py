"""Jittered structured triangulations of a rectangle.

Recipe (the paper's unstructured meshes are not available, so these stand in
for them): an nx-by-ny grid of squares on [x0,x1]x[y0,y1]; square (i, j) with
corners a=(i,j), b=(i+1,j), c=(i+1,j+1), d=(i,j+1) is split along the diagonal
a-c into the lower triangle (a, b, c) and then the upper triangle (a, c, d),
both counter-clockwise; squares are visited row by row (j outer, i inner).
Vertices are numbered row-major, v = j*(nx+1) + i. Every interior vertex is
shifted by independent U(-jitter*hx, jitter*hx) and U(-jitter*hy, jitter*hy)
draws taken from numpy's default_rng(seed) (PCG64), vertices in row-major
order, x before y. Boundary vertices stay on the boundary.

Local face f of an element joins its local vertices f and (f+1) mod 3.
Boundary faces carry a tag per side (x0, x1, y0, y1 -> bc_sides[0..3]):
0 = interior face, 1 = Dirichlet, 2 = Neumann.
"""
from dataclasses import dataclass, field

import numpy as np

INTERIOR, DIRICHLET, NEUMANN = 0, 1, 2


@dataclass
class Mesh:
    VX: np.ndarray          # (Nv,) float64
    VY: np.ndarray          # (Nv,) float64
    EToV: np.ndarray        # (K, 3) int32, counter-clockwise
    bc: np.ndarray          # (K, 3) int8, tag of face f = (v_f, v_{f+1})
    nx: int = 0
    ny: int = 0
    box: tuple = (0.0, 1.0, 0.0, 1.0)
    meta: dict = field(default_factory=dict)

    @property
    def K(self):
        return int(self.EToV.shape[0])

    @property
    def Nv(self):
        return int(self.VX.shape[0])


def jittered_grid(nx, ny, box=(0.0, 1.0, 0.0, 1.0), jitter=0.1, seed=0,
                  bc_sides=(DIRICHLET, DIRICHLET, DIRICHLET, DIRICHLET)):
    x0, x1, y0, y1 = box
    hx = (x1 - x0) / nx
    hy = (y1 - y0) / ny
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    VX = (x0 + ii * hx).astype(np.float64).ravel()
    VY = (y0 + jj * hy).astype(np.float64).ravel()
    interior = ((ii > 0) & (ii < nx) & (jj > 0) & (jj < ny)).ravel()
    if jitter != 0.0:
        rng = np.random.default_rng(seed)
        n_int = int(interior.sum())
        d = rng.uniform(-1.0, 1.0, size=(n_int, 2))
        VX[interior] += jitter * hx * d[:, 0]
        VY[interior] += jitter * hy * d[:, 1]
    # exact boundary coordinates (no rounding drift from x0 + i*hx)
    VX[(ii == nx).ravel()] = x1
    VY[(jj == ny).ravel()] = y1

    i = np.tile(np.arange(nx), ny)
    j = np.repeat(np.arange(ny), nx)
    a = j * (nx + 1) + i
    b = a + 1
    c = a + (nx + 1) + 1
    d = a + (nx + 1)
    lower = np.stack([a, b, c], axis=1)
    upper = np.stack([a, c, d], axis=1)
    EToV = np.empty((2 * nx * ny, 3), dtype=np.int32)
    EToV[0::2] = lower
    EToV[1::2] = upper

    # boundary tags from the grid structure (face f joins local vertices f, f+1)
    gi = np.tile(np.arange(nx + 1), ny + 1)
    gj = np.repeat(np.arange(ny + 1), nx + 1)
    bc = np.zeros((EToV.shape[0], 3), dtype=np.int8)
    for f in range(3):
        va = EToV[:, f]
        vb = EToV[:, (f + 1) % 3]
        for side, (arr, val) in enumerate(((gi, 0), (gi, nx), (gj, 0), (gj, ny))):
            on = (arr[va] == val) & (arr[vb] == val)
            bc[on, f] = bc_sides[side]
    return Mesh(VX=VX, VY=VY, EToV=EToV, bc=bc, nx=nx, ny=ny, box=tuple(box),
                meta=dict(jitter=jitter, seed=seed, bc_sides=tuple(bc_sides)))


# The five workloads: name -> (nx, ny, box, jitter, seed, bc_sides, N)
CONFIG_MESHES = {
    # 16x16 on the unit square, N=3, Dirichlet everywhere
    "c1_poisson_512tri_N3": (16, 16, (0.0, 1.0, 0.0, 1.0), 0.1, 0, (1, 1, 1, 1), 3),
    # 128x128 on the unit square, N=6, Dirichlet everywhere
    "c2_pmg_32768tri_N6": (128, 128, (0.0, 1.0, 0.0, 1.0), 0.1, 0, (1, 1, 1, 1), 6),
    # 64x64 on [-0.5,1]x[-0.5,1.5], N=8; velocity Dirichlet on every side (the
    # pressure-increment tags come from ins_pressure_tags)
    "c3_ins_8192tri_N8": (64, 64, (-0.5, 1.0, -0.5, 1.5), 0.0, 0, (1, 1, 1, 1), 8),
    # c2 mesh, batch of 64 right-hand sides
    "c4_adjoint_32768tri_N6": (128, 128, (0.0, 1.0, 0.0, 1.0), 0.1, 0, (1, 1, 1, 1), 6),
    # 512x512 on the unit square, N=8 headline (N=1..8 swept)
    "c5_sweep_524288tri_N8": (512, 512, (0.0, 1.0, 0.0, 1.0), 0.1, 0, (1, 1, 1, 1), 8),
}


def config_mesh(name):
    nx, ny, box, jit, seed, sides, N = CONFIG_MESHES[name]
    return jittered_grid(nx, ny, box=box, jitter=jit, seed=seed, bc_sides=sides), N


def rotate_local_vertices(mesh, seed):
    """Same triangulation with each element's local vertex list cyclically
    rotated by a seeded random shift (orientation stays counter-clockwise), so
    that every pairing of local face indices across a shared face occurs."""
    rng = np.random.default_rng(seed)
    k = rng.integers(0, 3, size=mesh.K)
    idx = (np.arange(3)[None, :] + k[:, None]) % 3
    EToV = np.take_along_axis(mesh.EToV, idx, axis=1).astype(np.int32)
    bc = np.take_along_axis(mesh.bc, idx, axis=1).astype(np.int8)
    return Mesh(VX=mesh.VX.copy(), VY=mesh.VY.copy(), EToV=EToV, bc=bc, nx=mesh.nx, ny=mesh.ny,
                box=mesh.box, meta=dict(mesh.meta, rotated_seed=seed))


def with_all_neumann(mesh):
    bc = np.where(mesh.bc != INTERIOR, NEUMANN, INTERIOR).astype(np.int8)
    return Mesh(VX=mesh.VX, VY=mesh.VY, EToV=mesh.EToV, bc=bc, nx=mesh.nx, ny=mesh.ny,
                box=mesh.box, meta=dict(mesh.meta, all_neumann=True))


def ins_pressure_tags(mesh, dirichlet_sides=(1,)):
    """Copy of a velocity mesh whose boundary tags are those of the pressure
    increment: Dirichlet on the listed sides (0: x0, 1: x1, 2: y0, 3: y1),
    Neumann on the others."""
    x0, x1, y0, y1 = mesh.box
    bc = mesh.bc.copy()
    for f in range(3):
        va = mesh.EToV[:, f]
        vb = mesh.EToV[:, (f + 1) % 3]
        bnd = mesh.bc[:, f] != INTERIOR
        bc[bnd, f] = NEUMANN
        for side, (arr, val) in enumerate(((mesh.VX, x0), (mesh.VX, x1), (mesh.VY, y0), (mesh.VY, y1))):
            if side in dirichlet_sides:
                on = bnd & np.isclose(arr[va], val) & np.isclose(arr[vb], val)
                bc[on, f] = DIRICHLET
    return Mesh(VX=mesh.VX, VY=mesh.VY, EToV=mesh.EToV, bc=bc, nx=mesh.nx, ny=mesh.ny, box=mesh.box,
                meta=dict(mesh.meta, pressure_tags=tuple(dirichlet_sides)))
