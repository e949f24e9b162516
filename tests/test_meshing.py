"""Host-side checks of the mesh metrics: exact point-triangle distances and
area-uniform sampling."""
import numpy as np
import torch

from paper_2302_01838_b300 import meshing


def test_point_triangle_distance_regions():
    tri = torch.tensor([[[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]]], dtype=torch.float64)
    p = torch.tensor([[0.2, 0.2, 0.5],      # above the face
                      [-1.0, -1.0, 0.0],    # beyond vertex a
                      [0.5, -2.0, 0.0],     # beyond edge ab
                      [1.0, 1.0, 0.0],      # beyond edge bc
                      [2.0, 0.0, 1.0]], dtype=torch.float64)
    d = meshing.point_triangle_distance(p, tri).numpy()
    want = [0.5, np.sqrt(2.0), 2.0, np.sqrt(0.5), np.sqrt(2.0)]
    assert np.allclose(d, want)
    # brute force against dense samples of the triangle
    rng = np.random.default_rng(0)
    q = torch.from_numpy(rng.uniform(-1, 2, (50, 3)))
    s = meshing.sample_triangles(tri, 200000, torch.Generator().manual_seed(1))
    brute = torch.cdist(q, s).min(1).values
    assert torch.all(meshing.point_triangle_distance(q, tri) <= brute + 1e-12)
    assert torch.max(brute - meshing.point_triangle_distance(q, tri)) < 1e-2


def test_sampling_is_area_uniform():
    tris = torch.tensor([[[0.0, 0, 0], [1, 0, 0], [0, 1, 0]], [[0, 0, 1], [2, 0, 1], [0, 2, 1]]], dtype=torch.float64)
    s = meshing.sample_triangles(tris, 40000, torch.Generator().manual_seed(2))
    frac_top = float((s[:, 2] > 0.5).double().mean())
    assert abs(frac_top - 0.8) < 0.01          # areas 0.5 and 2.0
