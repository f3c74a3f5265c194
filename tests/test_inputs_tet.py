"""The seeded tetrahedral mesh generators: conforming, positively oriented,
boundary faces tagged by their side of the box, and local renumbering that moves
the face tags with the faces."""
import numpy as np
import pytest

from dg_inputs.tetmesh import jittered_tet_grid, permute_local_vertices

FACES = ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3))


def _faces(m):
    owners = {}
    for e, t in enumerate(m.EToV):
        for f, loc in enumerate(FACES):
            owners.setdefault(tuple(sorted(int(t[q]) for q in loc)), []).append((e, f))
    return owners


@pytest.mark.parametrize("n", [1, 2, 3])
def test_grid_counts_orientation_and_conformity(n):
    m = jittered_tet_grid(n, jitter=0.15, seed=n)
    assert m.K == 6 * n ** 3 and m.VX.size == (n + 1) ** 3
    P = np.stack([m.VX, m.VY, m.VZ], 1)[m.EToV]
    det = np.linalg.det(np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], 2))
    assert det.min() > 0
    assert abs(det.sum() / 6.0 - 1.0) < 1e-12          # the volumes fill the unit cube
    owners = _faces(m)
    assert all(len(o) in (1, 2) for o in owners.values())
    nb = sum(1 for o in owners.values() if len(o) == 1)
    assert nb == 12 * n * n                             # two triangles per boundary square


def test_boundary_tags_follow_the_sides():
    sides = (1, 2, 1, 2, 2, 1)
    m = jittered_tet_grid(2, jitter=0.1, seed=3, bc_sides=sides)
    X = np.stack([m.VX, m.VY, m.VZ], 1)
    for key, o in _faces(m).items():
        e, f = o[0]
        if len(o) == 2:
            assert m.bc[e, f] == 0 and m.bc[o[1]] == 0
            continue
        pts = X[list(key)]
        side = [s for ax in range(3) for s, v in ((2 * ax, 0.0), (2 * ax + 1, 1.0))
                if np.all(np.abs(pts[:, ax] - v) < 1e-12)]
        assert len(side) == 1 and m.bc[e, f] == sides[side[0]]


def test_renumbering_keeps_orientation_and_moves_tags_with_faces():
    m = jittered_tet_grid(2, jitter=0.1, seed=5, bc_sides=(1, 2, 2, 1, 1, 2))
    pm = permute_local_vertices(m, 11)
    P = np.stack([pm.VX, pm.VY, pm.VZ], 1)[pm.EToV]
    det = np.linalg.det(np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], 2))
    assert det.min() > 0
    tag = {}
    for e in range(m.K):
        for f, loc in enumerate(FACES):
            tag[(e, tuple(sorted(int(m.EToV[e, q]) for q in loc)))] = m.bc[e, f]
    for e in range(pm.K):
        assert sorted(pm.EToV[e]) == sorted(m.EToV[e])
        for f, loc in enumerate(FACES):
            assert pm.bc[e, f] == tag[(e, tuple(sorted(int(pm.EToV[e, q]) for q in loc)))]
    assert np.any(pm.EToV != m.EToV)
