"""Seeded synthetic inputs: object shapes, camera poses, ray pools, the PE matrix.

This module only generates inputs. It holds none of the training step's
arithmetic (no sampling of depths, encoding, MLP, rendering, loss or
optimiser); tests, the benchmark and the smoke check feed what it produces to
both the CUDA library and the CPU oracle.

Scene recipe (stands in for the Replica / ScanNet / TUM sequences the paper
trains on, none of which are available here):
  * an object is a union of 1-3 primitives (sphere or axis-aligned box) with
    radius / half-extents U[rmin, rmax] and a uniform random RGB each;
  * it is seen from 5 cameras at 2 m, viewing directions uniform on the
    sphere, looking at the object centre, up = +z;
  * pinhole 640 x 480, f = 500, principal point (320, 240);
  * a ray's direction is R_wc ((u + 0.5 - cx) / f, (v + 0.5 - cy) / f, 1),
    unnormalised, so the ray parameter t equals the camera z-depth;
  * the depth is the analytic first hit, the colour the hit primitive's RGB;
  * the pool keeps up to ``per_view`` hit pixels per view.
Ray record (12 float32): origin(3), direction(3), depth, rgb(3), mask, 0.
"""
import numpy as np

REC = 12
W_IMG, H_IMG, FOCAL, CX, CY = 640, 480, 500.0, 320.0, 240.0


def make_B(seed, n_freq=45, std=5.0):
    """Gaussian encoding matrix, entries N(0, std^2) (std 5 -> variance 25)."""
    return (np.random.default_rng(seed).standard_normal((n_freq, 3)) * std).astype(np.float32)


def random_shape(rng, n_prims, rmin=0.1, rmax=0.4, spread=0.0):
    prims = []
    for _ in range(n_prims):
        kind = "sphere" if rng.random() < 0.5 else "box"
        off = rng.uniform(-spread, spread, 3) if spread > 0 else np.zeros(3)
        if kind == "sphere":
            size = np.full(3, rng.uniform(rmin, rmax))
        else:
            size = rng.uniform(rmin, rmax, 3)
        prims.append(dict(kind=kind, offset=off, size=size, rgb=rng.uniform(0, 1, 3)))
    return prims


def bound_radius(prims):
    r = 0.0
    for p in prims:
        ext = p["size"][0] if p["kind"] == "sphere" else np.linalg.norm(p["size"])
        r = max(r, np.linalg.norm(p["offset"]) + ext)
    return r


def cast(prims, center, o, d):
    """First hit of rays o + t d (t > 0) with a union of primitives.

    Returns (t_hit [n] with inf for a miss, rgb [n, 3])."""
    n = o.shape[0]
    best = np.full(n, np.inf)
    rgb = np.zeros((n, 3))
    for p in prims:
        c = center + p["offset"]
        if p["kind"] == "sphere":
            r = p["size"][0]
            oc = o - c
            a = np.einsum("ij,ij->i", d, d)
            b = 2.0 * np.einsum("ij,ij->i", d, oc)
            cc = np.einsum("ij,ij->i", oc, oc) - r * r
            disc = b * b - 4 * a * cc
            sq = np.sqrt(np.maximum(disc, 0.0))
            t0 = (-b - sq) / (2 * a)
            t1 = (-b + sq) / (2 * a)
            t = np.where(t0 > 1e-6, t0, t1)
            t = np.where((disc >= 0) & (t > 1e-6), t, np.inf)
        else:
            h = p["size"]
            with np.errstate(divide="ignore", invalid="ignore"):
                inv = 1.0 / d
                ta = (c - h - o) * inv
                tb = (c + h - o) * inv
            tmin = np.nanmax(np.minimum(ta, tb), axis=1)
            tmax = np.nanmin(np.maximum(ta, tb), axis=1)
            t = np.where(tmin > 1e-6, tmin, tmax)
            t = np.where((tmax >= np.maximum(tmin, 0.0)) & (t > 1e-6), t, np.inf)
        closer = t < best
        best = np.where(closer, t, best)
        rgb[closer] = p["rgb"]
    return best, rgb


def union_sdf(prims, center, x):
    """Signed distance of points x [n, 3] to a union of primitives (negative
    inside): spheres |x - c| - r, boxes the exact box distance."""
    x = np.asarray(x, np.float64)
    best = np.full(x.shape[0], np.inf)
    for p in prims:
        q = x - (np.asarray(center, np.float64) + p["offset"])
        if p["kind"] == "sphere":
            d = np.linalg.norm(q, axis=1) - p["size"][0]
        else:
            a = np.abs(q) - p["size"]
            d = np.linalg.norm(np.maximum(a, 0.0), axis=1) + np.minimum(np.max(a, axis=1), 0.0)
        best = np.minimum(best, d)
    return best


def surface_points(rng, prims, center, n):
    """About n points on the surface of a union of primitives: points on each
    primitive's surface (area-proportional) that lie on the union's boundary."""
    pts, areas = [], []
    for p in prims:
        areas.append(4 * np.pi * p["size"][0] ** 2 if p["kind"] == "sphere"
                     else 8 * (p["size"][0] * p["size"][1] + p["size"][1] * p["size"][2] + p["size"][0] * p["size"][2]))
    areas = np.array(areas) / np.sum(areas)
    for p, w in zip(prims, areas):
        m = max(1, int(round(3 * n * w)))
        c = np.asarray(center, np.float64) + p["offset"]
        if p["kind"] == "sphere":
            v = rng.standard_normal((m, 3))
            q = c + p["size"][0] * v / np.linalg.norm(v, axis=1, keepdims=True)
        else:
            h = p["size"]
            face_area = np.array([h[1] * h[2], h[1] * h[2], h[0] * h[2], h[0] * h[2], h[0] * h[1], h[0] * h[1]])
            f = rng.choice(6, m, p=face_area / face_area.sum())
            u = rng.uniform(-1, 1, (m, 3)) * h
            ax, sgn = f // 2, np.where(f % 2 == 0, 1.0, -1.0)
            u[np.arange(m), ax] = sgn * h[ax]
            q = c + u
        pts.append(q)
    q = np.concatenate(pts)
    q = q[np.abs(union_sdf(prims, center, q)) < 1e-6]
    return q[rng.permutation(q.shape[0])[:n]]


def look_at(eye, target, up=np.array([0.0, 0.0, 1.0])):
    """Camera-to-world rotation for a camera with +z forward, +x right, +y down."""
    f = target - eye
    f = f / np.linalg.norm(f)
    r = np.cross(f, up)
    r = r / np.linalg.norm(r)
    dn = np.cross(f, r)
    return np.stack([r, dn, f], axis=1)


def camera_rays(R_wc, eye, u, v):
    dc = np.stack([(u + 0.5 - CX) / FOCAL, (v + 0.5 - CY) / FOCAL, np.ones_like(u)], axis=1)
    d = dc @ R_wc.T
    o = np.broadcast_to(eye, d.shape).copy()
    return o, d


def random_view(rng, center, dist=2.0):
    while True:
        w = rng.standard_normal(3)
        w /= np.linalg.norm(w)
        if abs(w[2]) <= 0.99:
            break
    eye = center + dist * w
    return eye, look_at(eye, center)


def object_pool(rng, prims, center, n_views=5, per_view=1024, dist=2.0, extra_views=0, offmask=0.0):
    """Ray pool of one object: hit pixels from ``n_views`` random views.

    Returns float32 [n, 12] records (mask = 1). With offmask > 0, up to
    offmask * per_view further pixels of the object's 2D box that miss it are
    added per training view with mask 0 (the paper's rays inside the box but
    outside the mask), their depth that of a background wall 1 m behind the
    object centre and their colour 0."""
    radius = bound_radius(prims)
    recs = []
    for vi in range(n_views + extra_views):
        eye, Rwc = random_view(rng, center, dist)
        half = FOCAL * radius / max(dist - radius, 1e-3) + 2.0
        n_cand = per_view * 3
        u = np.floor(rng.uniform(max(CX - half, 0), min(CX + half, W_IMG), n_cand))
        v = np.floor(rng.uniform(max(CY - half, 0), min(CY + half, H_IMG), n_cand))
        o, d = camera_rays(Rwc, eye, u, v)
        t, rgb = cast(prims, center, o, d)
        hit = np.isfinite(t)
        oh, dh, th, rgbh = o[hit][:per_view], d[hit][:per_view], t[hit][:per_view], rgb[hit][:per_view]
        rec = np.zeros((oh.shape[0], REC), np.float32)
        rec[:, 0:3], rec[:, 3:6], rec[:, 6], rec[:, 7:10], rec[:, 10] = oh, dh, th, rgbh, 1.0
        if offmask > 0 and vi < n_views:
            nm = int(offmask * per_view)
            om, dm = o[~hit][:nm], d[~hit][:nm]
            miss = np.zeros((om.shape[0], REC), np.float32)
            miss[:, 0:3], miss[:, 3:6], miss[:, 6] = om, dm, dist + 1.0
            rec = np.concatenate([rec, miss])
        recs.append(rec)
    return recs


def make_object(rng, n_prims=(1, 1), rmin=0.1, rmax=0.4, spread=0.0, H=32,
                n_views=5, per_view=1024, room=(2.0, 2.0, 0.6), heldout_views=0, offmask=0.0):
    """One object: shape, world centre, PE scale, ray pool (first n_views views)
    and, with heldout_views > 0, the rays of further views kept apart ("eval")."""
    k = int(rng.integers(n_prims[0], n_prims[1] + 1))
    prims = random_shape(rng, k, rmin, rmax, spread)
    center = np.array([rng.uniform(-room[0], room[0]), rng.uniform(-room[1], room[1]),
                       1.0 + rng.uniform(-room[2], room[2])])
    views = object_pool(rng, prims, center, n_views=n_views, per_view=per_view,
                        extra_views=heldout_views, offmask=offmask)
    pool = np.concatenate(views[:n_views], axis=0)
    scale = 1.1 * bound_radius(prims)
    out = dict(prims=prims, center=center.astype(np.float32), scale=np.float32(scale),
               pool=pool, H=H)
    if heldout_views:
        out["eval"] = np.concatenate(views[n_views:], axis=0)
    return out


def first_keyframe_samples(rng, obj, n=256, view=0, per_view=1024):
    """Set-encoder input of an object: n (x~, occupancy, rgb) samples from the
    rays of its first keyframe (the first view of the pool): n/2 surface hits
    (occupancy 1, the hit colour) and n/2 free-space points before the hit
    (occupancy 0, colour 0), x~ = (x - c) / s. Returns float32 [n, 7]."""
    pool = obj["pool"]
    rays = pool[view * per_view:(view + 1) * per_view] if pool.shape[0] >= per_view else pool
    rays = rays[rays[:, 10] > 0]          # in-mask pixels of the keyframe
    h = n // 2
    i = rng.integers(0, rays.shape[0], h)
    j = rng.integers(0, rays.shape[0], n - h)
    hit = rays[i, 0:3] + rays[i, 6:7] * rays[i, 3:6]
    frac = rng.uniform(0.2, 0.9, (n - h, 1))
    free = rays[j, 0:3] + frac * rays[j, 6:7] * rays[j, 3:6]
    x = (np.concatenate([hit, free]) - obj["center"]) / obj["scale"]
    occ = np.concatenate([np.ones(h), np.zeros(n - h)])[:, None]
    rgb = np.concatenate([rays[i, 7:10], np.zeros((n - h, 3))])
    return np.concatenate([x, occ, rgb], axis=1).astype(np.float32)


def scene_shapes(seed, n_objects, heldout_views=1, per_view=512, offmask=0.0):
    """Shapes for the warm-start experiments: unions of 1-3 primitives,
    hidden 32, 120 rays per step, one held-out view per object; every object
    starts from the same seeded initial weights (so converged weights share
    one basin)."""
    rng = np.random.default_rng(seed)
    init = init_weights(np.random.default_rng(12345), 32)
    objs = []
    for _ in range(n_objects):
        o = make_object(rng, (1, 3), 0.1, 0.3, 0.25, H=32, per_view=per_view, heldout_views=heldout_views,
                        offmask=offmask)
        o["init"] = init
        o["rays"] = 120
        o["n_surface"], o["n_strat"] = 10, 12
        o["set_input"] = first_keyframe_samples(rng, o, per_view=per_view)
        objs.append(o)
    return dict(objects=objs, B=make_B(1000 + 5), seed=seed)


def background_object(rng, half=(3.0, 3.0, 1.5), n_views=5, per_view=2048, H=128, scale=2.5):
    """A room box seen from inside: the background model's training rays.

    Each of the six walls has its own colour; a ray's depth is where it
    leaves the box."""
    half = np.asarray(half)
    center = np.array([0.0, 0.0, half[2]])
    wall_rgb = rng.uniform(0, 1, (6, 3))
    recs = []
    for _ in range(n_views):
        eye = center + rng.uniform(-0.6, 0.6, 3) * half
        yaw = rng.uniform(0, 2 * np.pi)
        target = eye + np.array([np.cos(yaw), np.sin(yaw), rng.uniform(-0.3, 0.3)])
        Rwc = look_at(eye, target)
        u = np.floor(rng.uniform(0, W_IMG, per_view))
        v = np.floor(rng.uniform(0, H_IMG, per_view))
        o, d = camera_rays(Rwc, eye, u, v)
        with np.errstate(divide="ignore"):
            inv = 1.0 / d
        ta = (center - half - o) * inv
        tb = (center + half - o) * inv
        tmax_axis = np.maximum(ta, tb)
        axis = np.argmin(tmax_axis, axis=1)
        t = tmax_axis[np.arange(len(axis)), axis]
        side = (d[np.arange(len(axis)), axis] > 0).astype(int)
        rgb = wall_rgb[2 * axis + side]
        rec = np.zeros((o.shape[0], REC), np.float32)
        rec[:, 0:3], rec[:, 3:6], rec[:, 6], rec[:, 7:10], rec[:, 10] = o, d, t, rgb, 1.0
        recs.append(rec)
    return dict(prims=None, center=center.astype(np.float32), scale=np.float32(scale),
                pool=np.concatenate(recs, axis=0), H=H)


def init_weights(rng, H):
    """Explicit U(-1/sqrt(fan_in), 1/sqrt(fan_in)) initial weights, canonical packed layout
    (W1, b1, ..., W5, b5; W row-major [out, in])."""
    parts = []
    for (o, i) in [(H, 93), (H, H), (H, H), (H, H), (4, H)]:
        bound = 1.0 / np.sqrt(i)
        parts.append(rng.uniform(-bound, bound, o * i))
        parts.append(rng.uniform(-bound, bound, o))
    return np.concatenate(parts).astype(np.float32)


def loguniform_int(rng, lo, hi, n):
    return np.round(np.exp(rng.uniform(np.log(lo), np.log(hi), n))).astype(np.int64)


# ----------------------------------------------------------------------------
# the benchmark / parity workloads
# ----------------------------------------------------------------------------
def scene_small(seed=1, n_objects=4, rays=120):
    """4 objects, each one sphere or box (radius/half-extent U[0.1, 0.4] m), 120 rays/step."""
    rng = np.random.default_rng(seed)
    objs = [make_object(rng, (1, 1), 0.1, 0.4, 0.0, H=32) for _ in range(n_objects)]
    for o in objs:
        o["init"] = init_weights(rng, o["H"])
        o["rays"] = rays
        o["n_surface"], o["n_strat"] = 10, 12
    return dict(objects=objs, B=make_B(seed + 1000), seed=seed)


def scene_room(seed=2, n_objects=50, with_background=True, per_view=512):
    """50 objects (unions of 1-3 primitives, hidden 32, rays log-uniform in 32-600)
    plus a background room model (hidden 128, 1,200 rays)."""
    rng = np.random.default_rng(seed)
    objs = []
    rays = loguniform_int(rng, 32, 600, n_objects)
    for k in range(n_objects):
        o = make_object(rng, (1, 3), 0.1, 0.3, 0.25, H=32, per_view=per_view)
        o["rays"] = int(rays[k])
        objs.append(o)
    if with_background:
        bg = background_object(rng)
        bg["rays"] = 1200
        objs.append(bg)
    for o in objs:
        o["init"] = init_weights(rng, o["H"])
        o["n_surface"], o["n_strat"] = 10, 12
    return dict(objects=objs, B=make_B(seed + 1000), seed=seed)


def scene_many(seed=4, n_objects=1000, per_view=256):
    """1,000 objects, hidden in {16, 32, 64}, rays log-uniform 16-1,024,
    samples per ray in {16, 22, 32}."""
    rng = np.random.default_rng(seed)
    objs = []
    rays = loguniform_int(rng, 16, 1024, n_objects)
    split = {16: (7, 9), 22: (10, 12), 32: (15, 17)}
    for k in range(n_objects):
        H = int(rng.choice([16, 32, 64]))
        S = int(rng.choice([16, 22, 32]))
        o = make_object(rng, (1, 3), 0.1, 0.3, 0.25, H=H, per_view=per_view)
        o["rays"] = int(rays[k])
        o["n_surface"], o["n_strat"] = split[S]
        o["init"] = init_weights(rng, H)
        objs.append(o)
    return dict(objects=objs, B=make_B(seed + 1000), seed=seed)
