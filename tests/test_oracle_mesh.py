"""Pins of the mesh-extraction oracle (marching tetrahedra): a linear field
gives triangles exactly on its zero plane with normals along the field's
descent; a sphere gives a closed, consistently oriented surface whose area
and enclosed volume match 4 pi r^2 and 4/3 pi r^3."""
import numpy as np

from oracle import mesh


def _field(fn, center, half, res):
    return fn(mesh.lattice(center, half, res))


def test_plane_is_exact_and_oriented():
    n = np.array([0.3, -0.5, 0.8])
    n /= np.linalg.norm(n)
    center, half, res = np.zeros(3), np.full(3, 1.0), 6
    occ = _field(lambda p: 0.5 + 0.2 * (p @ n - 0.1), center, half, res)
    tris = mesh.marching_tetrahedra(occ, center, half, res, 0.5)
    assert tris.shape[0] > 20
    assert np.max(np.abs(tris.reshape(-1, 3) @ n - 0.1)) < 1e-12
    normals = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    ok = np.linalg.norm(normals, axis=1) > 1e-12
    assert np.all(normals[ok] @ n < 0)          # inside (occ > level) is the +n side: normals point to -n


def test_sphere_is_closed_with_the_right_area_and_volume():
    r = 0.6
    center, half, res = np.array([0.1, -0.2, 0.3]), np.full(3, 0.8), 24
    occ = _field(lambda p: 1.0 / (1.0 + np.exp(-(r - np.linalg.norm(p - center, axis=1)) * 20)), center, half, res)
    tris = mesh.marching_tetrahedra(occ, center, half, res, 0.5)
    area = 0.5 * np.linalg.norm(np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0]), axis=1)
    keep = area > 1e-14
    t = tris[keep] - center
    assert abs(area.sum() - 4 * np.pi * r ** 2) / (4 * np.pi * r ** 2) < 0.02
    vol = np.einsum("ij,ij->i", t[:, 0], np.cross(t[:, 1], t[:, 2])).sum() / 6.0
    assert abs(vol - 4 / 3 * np.pi * r ** 3) / (4 / 3 * np.pi * r ** 3) < 0.02   # outward normals: positive
    # closed and consistently oriented: every directed edge is matched by its reverse exactly once
    key = lambda p: tuple(np.round(p, 9))
    edges = {}
    for tri in tris[keep]:
        for a, b in ((0, 1), (1, 2), (2, 0)):
            e = (key(tri[a]), key(tri[b]))
            edges[e] = edges.get(e, 0) + 1
    for (a, b), c in edges.items():
        assert c == 1 and edges.get((b, a), 0) == 1
