"""The seeded input generators shared by the oracle and the library
(dg_inputs): every workload mesh is counter-clockwise with positive areas,
its faces are conforming, its boundary tags sit exactly on the boundary, and
the draws are reproducible from the seed."""
import numpy as np
import pytest

from dg_inputs import config_mesh, jittered_grid, uniform_field
from dg_inputs.mesh import CONFIG_MESHES, DIRICHLET, INTERIOR, NEUMANN, ins_pressure_tags, rotate_local_vertices


def _areas(m):
    x, y = m.VX[m.EToV], m.VY[m.EToV]
    return 0.5 * ((x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0]))


def _face_counts(m):
    a = m.EToV
    b = np.roll(m.EToV, -1, axis=1)
    key = np.minimum(a, b).astype(np.int64) * m.Nv + np.maximum(a, b)
    _, inv, cnt = np.unique(key.ravel(), return_inverse=True, return_counts=True)
    return cnt[inv].reshape(m.K, 3)


@pytest.mark.parametrize("name", sorted(CONFIG_MESHES))
def test_workload_meshes_are_valid(name):
    m, N = config_mesh(name)
    nx, ny, box, jit, seed, sides, N0 = CONFIG_MESHES[name]
    assert m.K == 2 * nx * ny and N == N0
    A = _areas(m)
    h2 = (box[1] - box[0]) * (box[3] - box[2]) / (nx * ny)
    assert A.min() > 0.0                                   # counter-clockwise, J > 0
    assert abs(A.sum() - (box[1] - box[0]) * (box[3] - box[2])) < 1e-9 * A.sum()
    assert A.min() > 0.25 * h2 and A.max() < 0.75 * h2     # jitter 0.1 h keeps them well shaped
    cnt = _face_counts(m)
    assert cnt.max() == 2                                  # conforming: no face shared by three
    assert np.all((cnt == 1) == (m.bc != INTERIOR))        # boundary faces, and only they, carry a tag
    # each tagged face lies on the side whose tag it carries
    x0, x1, y0, y1 = box
    for f in range(3):
        va, vb = m.EToV[:, f], m.EToV[:, (f + 1) % 3]
        on = m.bc[:, f] != INTERIOR
        xa, xb, ya, yb = m.VX[va[on]], m.VX[vb[on]], m.VY[va[on]], m.VY[vb[on]]
        side = np.where((xa == x0) & (xb == x0), 0, np.where((xa == x1) & (xb == x1), 1,
                        np.where((ya == y0) & (yb == y0), 2, np.where((ya == y1) & (yb == y1), 3, -1))))
        assert np.all(side >= 0)
        assert np.all(m.bc[on, f] == np.asarray(sides)[side])


def test_draws_are_reproducible_from_the_seed():
    a, b, c = jittered_grid(6, 5, seed=3), jittered_grid(6, 5, seed=3), jittered_grid(6, 5, seed=4)
    assert np.array_equal(a.VX, b.VX) and np.array_equal(a.VY, b.VY) and np.array_equal(a.EToV, b.EToV)
    assert not np.array_equal(a.VX, c.VX)
    assert np.array_equal(uniform_field((4, 7), seed=1), uniform_field((4, 7), seed=1))
    u = uniform_field((1000,), seed=2)
    assert u.min() >= -1.0 and u.max() < 1.0


def test_rotation_and_pressure_tags_keep_the_mesh():
    m = jittered_grid(5, 4, seed=1, bc_sides=(DIRICHLET, NEUMANN, DIRICHLET, DIRICHLET))
    r = rotate_local_vertices(m, seed=2)
    assert np.allclose(np.sort(_areas(r)), np.sort(_areas(m))) and _areas(r).min() > 0
    assert np.array_equal(np.sort(np.sort(r.EToV, axis=1), axis=0), np.sort(np.sort(m.EToV, axis=1), axis=0))
    assert np.all((_face_counts(r) == 1) == (r.bc != INTERIOR))
    p = ins_pressure_tags(m, dirichlet_sides=(1,))
    on_x1 = np.zeros_like(p.bc, dtype=bool)
    for f in range(3):
        va, vb = m.EToV[:, f], m.EToV[:, (f + 1) % 3]
        on_x1[:, f] = (m.bc[:, f] != INTERIOR) & (m.VX[va] == m.box[1]) & (m.VX[vb] == m.box[1])
    assert np.all(p.bc[on_x1] == DIRICHLET)
    assert np.all(p.bc[(m.bc != INTERIOR) & ~on_x1] == NEUMANN)
    assert np.all(p.bc[m.bc == INTERIOR] == INTERIOR)
