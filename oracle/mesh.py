"""Mesh extraction of one object (the reconstruction the paper evaluates,
section 4: object meshes from querying each object within its 3D bound).

TEST INFRASTRUCTURE (see oracle/__init__.py).

The object's occupancy is sampled on a (res+1)^3 lattice over its box
c +- half, and the level set occupancy = level is extracted by marching
tetrahedra (each cube split into the six Kuhn tetrahedra that share the
diagonal from corner 0 to corner 7, so neighbouring cubes split shared
faces the same way). Reading (PROPOSAL; the paper names no iso-surface
method): a lattice vertex is inside when its occupancy exceeds `level`.

Order of the output (the GPU kernels follow it): cubes by index
q = i + res (j + res k) (x fastest), in each cube the tetrahedra
[0, e_a, e_a + e_b, 7] for (a, b) = (0,1), (0,2), (1,0), (1,2), (2,0), (2,1)
(corner id = x + 2 y + 4 z), in each tetrahedron:
  one vertex on its own side (inside or outside) at tetrahedron position a,
    the others b < c < d:  triangle (E(a,b), E(a,c), E(a,d));
  two inside i < j, two outside k < l:
    triangles (E(i,k), E(i,l), E(j,l)) and (E(i,k), E(j,l), E(j,k));
where E(x, y) is the level crossing on the edge, interpolated from the lower
tetrahedron position to the higher one. Every triangle is then oriented so
its normal (B - A) x (C - A) points from the inside vertices' centroid to the
outside vertices' centroid (B and C swapped otherwise).
"""
import numpy as np

from . import vmap_step as vs

KUHN = [(0, 1), (0, 2), (1, 0), (1, 2), (2, 0), (2, 1)]


def tets():
    return [[0, 1 << a, (1 << a) | (1 << b), 7] for a, b in KUHN]


def lattice(center, half, res):
    """World points of the (res+1)^3 lattice, vertex v = i + (res+1)(j + (res+1) k)."""
    center = np.asarray(center, np.float64)
    half = np.asarray(half, np.float64)
    origin = center - half
    step = 2.0 * half / res
    k, j, i = np.meshgrid(np.arange(res + 1), np.arange(res + 1), np.arange(res + 1), indexing="ij")
    return origin + np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1) * step


def grid_occupancy(cfg, params, H, center, scale, half, res):
    occ, _ = vs.query(cfg, params, H, center, scale, lattice(center, half, res))
    return occ


def marching_tetrahedra(occ, center, half, res, level):
    """Triangles [n, 3, 3] (world coordinates) of the level set, in the order above."""
    center = np.asarray(center, np.float64)
    half = np.asarray(half, np.float64)
    origin = center - half
    step = 2.0 * half / res
    n1 = res + 1
    out = []
    T = tets()
    for k in range(res):
        for j in range(res):
            for i in range(res):
                cv = [(i + (c & 1)) + n1 * ((j + ((c >> 1) & 1)) + n1 * (k + ((c >> 2) & 1))) for c in range(8)]
                cp = [origin + np.array([i + (c & 1), j + ((c >> 1) & 1), k + ((c >> 2) & 1)]) * step
                      for c in range(8)]
                cf = [occ[v] for v in cv]
                if all(f > level for f in cf) or all(not (f > level) for f in cf):
                    continue
                for t in T:
                    P = [cp[c] for c in t]
                    F = [cf[c] for c in t]
                    inside = [f > level for f in F]
                    out.extend(_tet_triangles(P, F, inside, level))
    return np.array(out).reshape(-1, 3, 3)


def _edge(P, F, x, y, level):
    lo, hi = min(x, y), max(x, y)
    t = (level - F[lo]) / (F[hi] - F[lo])
    return P[lo] + t * (P[hi] - P[lo])


def _orient(tri, P, inside):
    A, B, C = tri
    pin = np.mean([P[q] for q in range(4) if inside[q]], axis=0)
    pout = np.mean([P[q] for q in range(4) if not inside[q]], axis=0)
    if np.dot(np.cross(B - A, C - A), pout - pin) < 0:
        return [A, C, B]
    return [A, B, C]


def _tet_triangles(P, F, inside, level):
    cnt = sum(inside)
    if cnt == 0 or cnt == 4:
        return []
    if cnt in (1, 3):
        lone = [q for q in range(4) if inside[q] == (cnt == 1)][0]
        rest = [q for q in range(4) if q != lone]
        tri = [_edge(P, F, lone, r, level) for r in rest]
        return [_orient(tri, P, inside)]
    i, j = [q for q in range(4) if inside[q]]
    k, l = [q for q in range(4) if not inside[q]]
    eik, eil, ejl, ejk = (_edge(P, F, i, k, level), _edge(P, F, i, l, level), _edge(P, F, j, l, level),
                          _edge(P, F, j, k, level))
    return [_orient([eik, eil, ejl], P, inside), _orient([eik, ejl, ejk], P, inside)]
