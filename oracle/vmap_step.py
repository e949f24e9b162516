"""FP64 CPU oracle of the vMAP vectorised training step.

TEST INFRASTRUCTURE. This is the plain, slow, obviously-correct restatement of
the method that the CUDA library is checked against. Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline leg and its
``--impl reference`` arm) may import or run it. It shares no code with the
CUDA path; the two meet only in the seeded input generators.

What one step computes for every object k (vMAP, Kong et al., CVPR 2023):

  1. pick R_k rays uniformly, with replacement, from the object's own ray pool
     (each object samples pixels from its own keyframes, section 3.2
     "Object Supervision");
  2. depth-guided samples per ray: N_c stratified in [t_n, t_s + pad] (Eq. 1)
     and N_s ~ N(t_s, d_sigma^2) (Eq. 2), t_s = depth, or t_far when the depth
     is invalid; sorted ascending;
  3. x = o + t d, x~ = (x - c_k) / s_k (object-level scale, supplementary B),
     Gaussian encoding gamma = [x~, sin(B x~), cos(B x~)] (93 values);
  4. MLP 93 -> H -> H -> H -> H -> 4 with ReLU hidden units, sigmoid on the
     occupancy and the three colour outputs (section 4.1 "Implementation
     Details" gives hidden 32 / 128);
  5. occupancy rendering, Eq. 3: T_i = o_i prod_{j<i}(1 - o_j),
     O^ = sum T_i, D^ = sum T_i t_i, C^ = sum T_i c_i;
  6. losses, Eq. 4-5, read as means over the batch (see ``object_loss``);
  7. the exact gradient of that loss (hand-derived, pinned against finite
     differences and autograd in the tests);
  8. Adam (Kingma & Ba 2015, Algorithm 1) with the object's own step count.

Every function is FP64 numpy; matrix products use ``@`` as a library
primitive and nothing is blocked, fused or reordered beyond the definitions.
"""
from dataclasses import dataclass, field

import numpy as np

from .philox import ray_words, word_to_unit, word_to_index, philox4x32_10, seed_key

N_FREQ = 45
D_IN = 3 + 2 * N_FREQ   # 93 encoded features per point
N_OUT = 4               # occupancy + rgb

# ray record: 12 floats per ray
REC = 12
R_O, R_D, R_DEPTH, R_RGB, R_MASK = slice(0, 3), slice(3, 6), 6, slice(7, 10), 10


@dataclass
class Config:
    """Hyper-parameters of the step (defaults: section 3.3 and section 4.1)."""
    t_near: float = 0.05        # near bound t_n
    depth_pad: float = 0.10     # stratified samples reach depth + pad
    d_sigma: float = 0.03       # 3 cm, section 3.3
    t_far: float = 8.0          # far bound t_f used when the depth is invalid
    lambda_colour: float = 5.0  # lambda_1, Eq. 5
    lambda_occ: float = 0.0     # lambda_2, Eq. 5 (10 in the paper's full objective)
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    seed: int = 0
    B: np.ndarray = field(default_factory=lambda: np.zeros((N_FREQ, 3)))


def param_count(H):
    """Parameters of the 93 -> H -> H -> H -> H -> 4 MLP (weights + biases)."""
    return D_IN * H + H + 3 * (H * H + H) + N_OUT * H + N_OUT


def layer_shapes(H):
    """(out, in) of the five linear maps, in order."""
    return [(H, D_IN), (H, H), (H, H), (H, H), (N_OUT, H)]


def unpack(flat, H):
    """Canonical packed layout: W1, b1, W2, b2, ..., W5, b5; W row-major (out, in)."""
    flat = np.asarray(flat, dtype=np.float64)
    Ws, bs, off = [], [], 0
    for (o, i) in layer_shapes(H):
        Ws.append(flat[off:off + o * i].reshape(o, i)); off += o * i
        bs.append(flat[off:off + o]); off += o
    assert off == flat.size == param_count(H)
    return Ws, bs


def pack(Ws, bs):
    parts = []
    for W, b in zip(Ws, bs):
        parts.append(np.asarray(W, np.float64).ravel())
        parts.append(np.asarray(b, np.float64).ravel())
    return np.concatenate(parts)


def init_params(seed, stream, H):
    """Seeded default initialisation (PyTorch nn.Linear's U(-1/sqrt(fan_in), +1/sqrt(fan_in))
    for weights and biases; the paper does not state its init).

    Parameter p draws Philox word p % 4 of block p // 4 with counter
    (block, 0, 0xFFFFFFFF, stream): the step word 0xFFFFFFFF is reserved for
    initialisation so it never collides with a training step's draws.
    """
    P = param_count(H)
    n_blocks = (P + 3) // 4
    ctr = np.zeros((n_blocks, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(n_blocks)
    ctr[:, 2] = 0xFFFFFFFF
    ctr[:, 3] = int(stream) & 0xFFFFFFFF
    u = word_to_unit(philox4x32_10(ctr, seed_key(seed)).reshape(-1)[:P])
    fan_in = np.empty(P)
    off = 0
    for (o, i) in layer_shapes(H):
        fan_in[off:off + o * i + o] = i
        off += o * i + o
    return (2.0 * u - 1.0) / np.sqrt(fan_in)


# ----------------------------------------------------------------------------
# 1-2. ray picking and depth-guided sampling (section 3.3, Eq. 1 and Eq. 2)
# ----------------------------------------------------------------------------
def words_per_ray(n_surface, n_strat):
    """One pick word, one word per stratified sample, two per Box-Muller pair."""
    return 1 + n_strat + 2 * ((n_surface + 1) // 2)


def sample_object(cfg, pool, n_rays, n_surface, n_strat, stream, step):
    """Pick rays and draw their sorted sample depths.

    Returns (pick [R] int64, t [R, n_surface + n_strat] float64).
    Word 0 picks the ray; words 1..N_c give the stratified uniforms u_j,
    t_j = t_n + (j + u_j) / N_c * (t_s + pad - t_n)            (Eq. 1);
    the next words, in pairs (u1, u2), give Box-Muller normals
    z = sqrt(-2 ln u1) * (cos 2 pi u2, sin 2 pi u2), t = t_s + d_sigma z (Eq. 2),
    clamped below at t_n. Surface samples come first, then the stratified
    ones, and a stable ascending sort orders them. Rays off the object's mask
    (M = 0) end where they hit a surface (supplementary "depth guided
    sampling": rays through the box that do not belong to the object are
    terminated at the surface they hit): their stratified range stops at t_s
    and their Gaussian samples are clamped above at t_s.
    """
    n_words = words_per_ray(n_surface, n_strat)
    w = ray_words(cfg.seed, stream, step, np.arange(n_rays), n_words)
    pick = word_to_index(w[:, 0], pool.shape[0])
    depth = pool[pick, R_DEPTH].astype(np.float64)
    return pick, sample_depths(cfg, depth, w, n_surface, n_strat, pool[pick, R_MASK])


def sample_given(cfg, rays, n_surface, n_strat, stream, step):
    """Sorted sample depths for rays the caller chose: the same draws as
    ``sample_object`` with word 0 (the pick) unused."""
    n_words = words_per_ray(n_surface, n_strat)
    w = ray_words(cfg.seed, stream, step, np.arange(rays.shape[0]), n_words)
    return sample_depths(cfg, rays[:, R_DEPTH].astype(np.float64), w, n_surface, n_strat, rays[:, R_MASK])


def sample_depths(cfg, depth, w, n_surface, n_strat, mask=None):
    """Eq. 1 and Eq. 2 for rays of the given depths from their Philox words w;
    rays with mask 0 are terminated at t_s (see ``sample_object``)."""
    n_rays = depth.shape[0]
    on = np.ones(n_rays, bool) if mask is None else np.asarray(mask) > 0
    ts = np.where(depth > 0.0, depth, cfg.t_far)
    lo = cfg.t_near
    hi = ts + np.where(on, cfg.depth_pad, 0.0)
    strat = np.empty((n_rays, n_strat))
    for j in range(n_strat):
        u = word_to_unit(w[:, 1 + j])
        strat[:, j] = lo + (j + u) / n_strat * (hi - lo)
    z = np.empty((n_rays, 2 * ((n_surface + 1) // 2)))
    for p in range((n_surface + 1) // 2):
        u1 = word_to_unit(w[:, 1 + n_strat + 2 * p])
        u2 = word_to_unit(w[:, 2 + n_strat + 2 * p])
        rho = np.sqrt(-2.0 * np.log(u1))
        z[:, 2 * p] = rho * np.cos(2.0 * np.pi * u2)
        z[:, 2 * p + 1] = rho * np.sin(2.0 * np.pi * u2)
    surf = np.maximum(ts[:, None] + cfg.d_sigma * z[:, :n_surface], cfg.t_near)
    surf = np.where(on[:, None], surf, np.minimum(surf, ts[:, None]))
    t = np.concatenate([surf, strat], axis=1)
    return np.sort(t, axis=1, kind="stable")


# ----------------------------------------------------------------------------
# 3. points and Gaussian positional encoding (supplementary B: object scale s)
# ----------------------------------------------------------------------------
def points(rays, t, center, scale):
    """x~ = (o + t d - c) / s for every sample: [R, S, 3]."""
    o = rays[:, R_O].astype(np.float64)
    d = rays[:, R_D].astype(np.float64)
    x = o[:, None, :] + t[:, :, None] * d[:, None, :]
    return (x - np.asarray(center, np.float64)) / float(scale)


def encode(xt, B):
    """gamma(x~) = [x~, sin(B x~), cos(B x~)]  -> [n, 93]."""
    proj = xt @ np.asarray(B, np.float64).T
    return np.concatenate([xt, np.sin(proj), np.cos(proj)], axis=1)


# ----------------------------------------------------------------------------
# 4. the object MLP
# ----------------------------------------------------------------------------
def sigmoid(y):
    return 1.0 / (1.0 + np.exp(-y))


def mlp_forward(Ws, bs, gamma):
    """Returns (activations [a0=gamma, a1..a4], y [n, 4] pre-sigmoid)."""
    acts = [gamma]
    a = gamma
    for l in range(4):
        a = np.maximum(a @ Ws[l].T + bs[l], 0.0)
        acts.append(a)
    y = a @ Ws[4].T + bs[4]
    return acts, y


# ----------------------------------------------------------------------------
# 5. occupancy rendering (Eq. 3)
# ----------------------------------------------------------------------------
def render(o, c, t):
    """o [R,S], c [R,S,3], t [R,S] -> dict with P (prod_{j<i}(1-o_j)), T, O^, D^, C^."""
    R, S = o.shape
    P = np.ones((R, S))
    for i in range(1, S):
        P[:, i] = P[:, i - 1] * (1.0 - o[:, i - 1])
    T = o * P
    return dict(P=P, T=T, O=T.sum(1), D=(T * t).sum(1), C=(T[:, :, None] * c).sum(1))


# ----------------------------------------------------------------------------
# 6. losses (Eq. 4-5)
# ----------------------------------------------------------------------------
def object_loss(cfg, rays, rend):
    """L_k = mean_r M|D^-D| + lambda_1 mean_{r,ch} M|C^-C| + lambda_2 mean_r |O^-M|.

    Eq. 4 writes sums over the rays of the object's box; we read them as
    means over the R_k drawn rays (depth over R_k, colour over 3 R_k) so the
    loss scale does not depend on R_k. The depth term is also dropped for
    rays whose depth is invalid (depth <= 0).
    Returns (L_k, L_depth, L_colour, L_occupancy).
    """
    R = rays.shape[0]
    D = rays[:, R_DEPTH].astype(np.float64)
    C = rays[:, R_RGB].astype(np.float64)
    M = rays[:, R_MASK].astype(np.float64)
    valid = (D > 0.0).astype(np.float64)
    Ld = np.sum(M * valid * np.abs(rend["D"] - D)) / R
    Lc = np.sum(M[:, None] * np.abs(rend["C"] - C)) / (3 * R)
    Lo = np.sum(np.abs(rend["O"] - M)) / R
    return Ld + cfg.lambda_colour * Lc + cfg.lambda_occ * Lo, Ld, Lc, Lo


# ----------------------------------------------------------------------------
# 7. backward
# ----------------------------------------------------------------------------
def render_backward(cfg, rays, t, o, c, rend):
    """dL/do [R,S] and dL/dc [R,S,3] through Eq. 3 and the losses.

    With g_i = dL/dT_i = a t_i + b . c_i + e (a = dL/dD^, b = dL/dC^,
    e = dL/dO^), the reverse recursion S_{N+1} = 0,
    S_i = o_i g_i + (1 - o_i) S_{i+1} gives dL/do_i = P_i (g_i - S_{i+1}),
    and dL/dc_i = T_i b. Nothing divides by (1 - o_i).
    sign(0) = 0 for the L1 terms.
    """
    R, S = o.shape
    D = rays[:, R_DEPTH].astype(np.float64)
    C = rays[:, R_RGB].astype(np.float64)
    M = rays[:, R_MASK].astype(np.float64)
    valid = (D > 0.0).astype(np.float64)
    a = M * valid * np.sign(rend["D"] - D) / R
    b = cfg.lambda_colour * M[:, None] * np.sign(rend["C"] - C) / (3 * R)
    e = cfg.lambda_occ * np.sign(rend["O"] - M) / R
    g = a[:, None] * t + np.einsum("rsc,rc->rs", c, b) + e[:, None]
    Snext = np.zeros(R)
    dLdo = np.empty((R, S))
    for i in range(S - 1, -1, -1):
        dLdo[:, i] = rend["P"][:, i] * (g[:, i] - Snext)
        Snext = o[:, i] * g[:, i] + (1.0 - o[:, i]) * Snext
    dLdc = rend["T"][:, :, None] * b[:, None, :]
    return dLdo, dLdc


def mlp_backward(Ws, acts, dy):
    """Gradients of the five linear maps given dL/dy [n,4] (y pre-sigmoid).

    ReLU'(0) = 0. Returns (dWs, dbs, dgamma).
    """
    dWs, dbs = [None] * 5, [None] * 5
    dz = dy
    for l in range(4, -1, -1):
        dWs[l] = dz.T @ acts[l]
        dbs[l] = dz.sum(0)
        da = dz @ Ws[l]
        if l > 0:
            dz = da * (acts[l] > 0.0)
    return dWs, dbs, da


def encode_backward(xt, B, dgamma):
    """dL/dx~ from dL/dgamma: d sin(b.x~)/dx~ = cos(b.x~) b, d cos(b.x~)/dx~ = -sin(b.x~) b."""
    B = np.asarray(B, np.float64)
    proj = xt @ B.T
    return (dgamma[:, 0:3]
            + (dgamma[:, 3:3 + N_FREQ] * np.cos(proj)) @ B
            - (dgamma[:, 3 + N_FREQ:] * np.sin(proj)) @ B)


def object_forward_backward(cfg, params, H, rays, t, center, scale, want_center_grad=False):
    """Loss and gradients of one object on one batch of rays with given t.

    Returns dict(loss, Ld, Lc, Lo, grad (flat), render) and, with
    want_center_grad, dcenter (3,) and the per-ray gradients dray_o, dray_d [R, 3]."""
    Ws, bs = unpack(params, H)
    R, S = t.shape
    xt = points(rays, t, center, scale)
    gamma = encode(xt.reshape(-1, 3), cfg.B)
    acts, y = mlp_forward(Ws, bs, gamma)
    oc = sigmoid(y).reshape(R, S, N_OUT)
    o, c = oc[:, :, 0], oc[:, :, 1:]
    rend = render(o, c, t)
    L, Ld, Lc, Lo = object_loss(cfg, rays, rend)
    dLdo, dLdc = render_backward(cfg, rays, t, o, c, rend)
    dy = np.concatenate([(dLdo * o * (1 - o))[:, :, None], dLdc * c * (1 - c)], axis=2)
    dWs, dbs, dgamma = mlp_backward(Ws, acts, dy.reshape(-1, N_OUT))
    out = dict(loss=L, Ld=Ld, Lc=Lc, Lo=Lo, grad=pack(dWs, dbs), render=rend)
    if want_center_grad:
        dxt = encode_backward(xt.reshape(-1, 3), cfg.B, dgamma)
        out["dcenter"] = -dxt.sum(0) / float(scale)
        # per ray, through x = o + t d with the sample depths t held fixed:
        # dL/do = sum_i dL/dx_i, dL/dd = sum_i t_i dL/dx_i, dL/dx = dL/dx~ / s
        dx = dxt.reshape(R, S, 3) / float(scale)
        out["dray_o"] = dx.sum(1)
        out["dray_d"] = (dx * t[:, :, None]).sum(1)
    return out


# ----------------------------------------------------------------------------
# 8. Adam
# ----------------------------------------------------------------------------
def adam_update(cfg, theta, grad, m, v, step):
    """One Adam step (Kingma & Ba 2015, Algorithm 1; epsilon added to sqrt(v^)
    as PyTorch places it; no weight decay). Returns (theta, m, v, step)."""
    step = step + 1
    m = cfg.beta1 * m + (1.0 - cfg.beta1) * grad
    v = cfg.beta2 * v + (1.0 - cfg.beta2) * grad * grad
    mhat = m / (1.0 - cfg.beta1 ** step)
    vhat = v / (1.0 - cfg.beta2 ** step)
    return theta - cfg.lr * mhat / (np.sqrt(vhat) + cfg.eps), m, v, step


# ----------------------------------------------------------------------------
# the vectorised step over many independent objects
# ----------------------------------------------------------------------------
@dataclass
class ObjectState:
    H: int
    pool: np.ndarray            # [n_pool, 12] ray records (float32 values)
    center: np.ndarray          # (3,)
    scale: float
    n_surface: int = 10
    n_strat: int = 12
    stream: int = 0
    params: np.ndarray = None   # flat FP64
    m: np.ndarray = None
    v: np.ndarray = None
    step: int = 0
    active: bool = True
    faulted: bool = False

    def __post_init__(self):
        P = param_count(self.H)
        if self.params is None:
            raise ValueError("params required")
        self.params = np.asarray(self.params, np.float64).copy()
        assert self.params.size == P
        if self.m is None:
            self.m = np.zeros(P)
        if self.v is None:
            self.v = np.zeros(P)


def train_step(cfg, objects, rays_per_object, given=None):
    """One vectorised step: every active object trains on its own batch.

    given: optional list of per-object ray arrays chosen by the caller (the
    pick is then skipped, see ``sample_given``).

    Objects are independent: nothing of object j enters object k's loss or
    update (the objective of Eq. 5 is a plain sum over objects). Returns the
    per-object losses computed before the update (NaN for inactive ones).
    An object whose loss or gradient is not finite is frozen (state kept)
    and flagged.
    """
    losses = np.full(len(objects), np.nan)
    for k, (ob, R) in enumerate(zip(objects, rays_per_object)):
        if not ob.active or R <= 0:
            continue
        if given is None:
            pick, t = sample_object(cfg, ob.pool, R, ob.n_surface, ob.n_strat, ob.stream, ob.step)
            rays = ob.pool[pick].astype(np.float64)
        else:
            rays = np.asarray(given[k], np.float64)
            t = sample_given(cfg, rays, ob.n_surface, ob.n_strat, ob.stream, ob.step)
        res = object_forward_backward(cfg, ob.params, ob.H, rays, t, ob.center, ob.scale)
        losses[k] = res["loss"]
        if not (np.isfinite(res["loss"]) and np.all(np.isfinite(res["grad"]))):
            ob.faulted = True
            ob.active = False
            continue
        ob.params, ob.m, ob.v, ob.step = adam_update(cfg, ob.params, res["grad"], ob.m, ob.v, ob.step)
    return losses


def query(cfg, params, H, center, scale, pts):
    """Occupancy and colour of arbitrary world points for one object."""
    Ws, bs = unpack(params, H)
    xt = (np.asarray(pts, np.float64) - np.asarray(center, np.float64)) / float(scale)
    _, y = mlp_forward(Ws, bs, encode(xt, cfg.B))
    s = sigmoid(y)
    return s[:, 0], s[:, 1:]
