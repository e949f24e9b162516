"""Held-out rendering of objects and of the composed scene.

TEST INFRASTRUCTURE (see oracle/__init__.py).

Section 3.4 ("Compositional Scene Rendering") bounds each object's rays by
intersecting them with the object's 3D box (the ray-box intersection of
Majercik et al.); between the entry and exit depths we place n evenly spaced
midpoints (no depth guidance: a held-out view has no depth input) and render
with Eq. 3. A ray that misses the box renders 0. The scene render then ranks
the objects' rendered depths along each ray for occlusion. Reading
(PROPOSAL): the objects a ray meets are ordered by their expected hit depth
D^_k / O^_k (ties: lower object index first; objects with O^_k = 0 are
skipped) and composed front to back as Eq. 3 composes samples:
D = sum_k A_k D^_k, C = sum_k A_k C^_k, O = sum_k A_k O^_k with
A_k = prod over the objects j before k of (1 - O^_j).
"""
import numpy as np

from . import vmap_step as vs


def ray_box(o, d, lo, hi):
    """Slab-method entry/exit depths (entry clamped at 0) of rays o + t d."""
    t_in = np.zeros(o.shape[0])
    t_out = np.full(o.shape[0], np.inf)
    for ax in range(3):
        with np.errstate(divide="ignore", invalid="ignore"):
            t1 = (lo[ax] - o[:, ax]) / d[:, ax]
            t2 = (hi[ax] - o[:, ax]) / d[:, ax]
        par = d[:, ax] == 0
        inside = (o[:, ax] >= lo[ax]) & (o[:, ax] <= hi[ax])
        # a ray parallel to the slab: no constraint inside it, a miss outside
        t1 = np.where(par, -np.inf, t1)
        t2 = np.where(par, np.where(inside, np.inf, -np.inf), t2)
        t_in = np.maximum(t_in, np.minimum(t1, t2))
        t_out = np.minimum(t_out, np.maximum(t1, t2))
    return t_in, t_out


def render_depth(cfg, params, H, center, scale, rays, box_half, n_samples):
    """Rendered depth of each ray with n_samples midpoints inside the box."""
    rays = np.asarray(rays, np.float64)
    c = np.asarray(center, np.float64)
    half = np.asarray(box_half, np.float64)
    t_in, t_out = ray_box(rays[:, 0:3], rays[:, 3:6], c - half, c + half)
    hit = (t_out > t_in) & (t_out > 0)
    span = np.where(hit, t_out - t_in, 0.0)
    t = t_in[:, None] + (np.arange(n_samples) + 0.5)[None, :] / n_samples * span[:, None]
    Ws, bs = vs.unpack(params, H)
    xt = vs.points(rays, t, c, scale)
    _, y = vs.mlp_forward(Ws, bs, vs.encode(xt.reshape(-1, 3), cfg.B))
    s = vs.sigmoid(y).reshape(rays.shape[0], n_samples, 4)
    rend = vs.render(s[:, :, 0], s[:, :, 1:], t)
    return np.where(hit, rend["D"], 0.0)


def render_object(cfg, params, H, center, scale, rays, box_half, n_samples):
    """(O^, D^, C^ [n, 3]) of each ray with n_samples midpoints inside the box;
    zeros for rays that miss it."""
    rays = np.asarray(rays, np.float64)
    c = np.asarray(center, np.float64)
    half = np.asarray(box_half, np.float64)
    t_in, t_out = ray_box(rays[:, 0:3], rays[:, 3:6], c - half, c + half)
    hit = (t_out > t_in) & (t_out > 0)
    span = np.where(hit, t_out - t_in, 0.0)
    t = t_in[:, None] + (np.arange(n_samples) + 0.5)[None, :] / n_samples * span[:, None]
    Ws, bs = vs.unpack(params, H)
    xt = vs.points(rays, t, c, scale)
    _, y = vs.mlp_forward(Ws, bs, vs.encode(xt.reshape(-1, 3), cfg.B))
    s = vs.sigmoid(y).reshape(rays.shape[0], n_samples, 4)
    rend = vs.render(s[:, :, 0], s[:, :, 1:], t)
    return (np.where(hit, rend["O"], 0.0), np.where(hit, rend["D"], 0.0),
            np.where(hit[:, None], rend["C"], 0.0))


def compose(records):
    """Scene render from per-object records [(O^ [n], D^ [n], C^ [n, 3]), ...]
    in object order: returns (D [n], C [n, 3], O [n])."""
    n = records[0][0].shape[0]
    D, C, O = np.zeros(n), np.zeros((n, 3)), np.zeros(n)
    for r in range(n):
        order = sorted((rec[1][r] / rec[0][r], k) for k, rec in enumerate(records) if rec[0][r] > 0)
        A = 1.0
        for _, k in order:
            Ok, Dk, Ck = records[k][0][r], records[k][1][r], records[k][2][r]
            D[r] += A * Dk
            C[r] += A * Ck
            O[r] += A * Ok
            A *= 1.0 - Ok
    return D, C, O
