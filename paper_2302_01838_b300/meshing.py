"""Reconstruction metrics of extracted object meshes (the accuracy and
completion the paper reports for object meshes, section 4): distances
between points sampled on the mesh and the ground-truth surface, in both
directions. Evaluation only (torch on the GPU); meshes come from
VMap.extract_mesh."""
import torch


def sample_triangles(tris, n, generator=None):
    """n points uniformly (by area) on triangles [m, 3, 3]."""
    a, b, c = tris[:, 0], tris[:, 1], tris[:, 2]
    area = 0.5 * torch.linalg.norm(torch.cross(b - a, c - a, dim=1), dim=1)
    idx = torch.multinomial(area, n, replacement=True, generator=generator)
    u = torch.rand(n, 2, device=tris.device, generator=generator)
    flip = u.sum(1) > 1
    u[flip] = 1 - u[flip]
    return a[idx] + u[:, :1] * (b[idx] - a[idx]) + u[:, 1:] * (c[idx] - a[idx])


def point_triangle_distance(p, tris, chunk=4096):
    """Distance from each point p [n, 3] to the nearest triangle of tris [m, 3, 3]
    (exact point-triangle distance, brute force in chunks)."""
    out = []
    a, b, c = tris[:, 0], tris[:, 1], tris[:, 2]
    ab, ac = b - a, c - a
    for s in range(0, p.shape[0], chunk):
        q = p[s:s + chunk, None, :]                      # [k, 1, 3]
        ap = q - a                                       # [k, m, 3]
        d1, d2 = (ab * ap).sum(-1), (ac * ap).sum(-1)
        bp = q - b
        d3, d4 = (ab * bp).sum(-1), (ac * bp).sum(-1)
        cp = q - c
        d5, d6 = (ab * cp).sum(-1), (ac * cp).sum(-1)
        vc = d1 * d4 - d3 * d2
        vb = d5 * d2 - d1 * d6
        va = d3 * d6 - d5 * d4
        denom = (va + vb + vc).clamp_min(1e-30)
        v = vb / denom
        w = vc / denom
        closest = a + v[..., None] * ab + w[..., None] * ac          # inside the face
        # regions outside the face: clamp to the nearest edge
        def seg(x, y):
            e = y - x
            t = (((q - x) * e).sum(-1) / (e * e).sum(-1).clamp_min(1e-30)).clamp(0, 1)
            return x + t[..., None] * e
        inside = (va >= 0) & (vb >= 0) & (vc >= 0)
        cand = torch.stack([seg(a, b), seg(b, c), seg(c, a)], 0)      # [3, k, m, 3]
        dist_edges = torch.linalg.norm(cand - q, dim=-1).min(0).values
        dist_face = torch.linalg.norm(closest - q, dim=-1)
        d = torch.where(inside, dist_face, dist_edges)
        out.append(d.min(1).values)
    return torch.cat(out)


def accuracy_completion(tris, sdf, gt_points, n=20000, generator=None):
    """Accuracy: mean |sdf| at points sampled on the mesh; completion: mean
    distance from ground-truth surface points to the mesh."""
    pts = sample_triangles(tris, n, generator)
    acc = sdf(pts).abs().mean()
    comp = point_triangle_distance(gt_points, tris).mean()
    return float(acc), float(comp)
