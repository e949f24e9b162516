"""Rounding model of the library's BF16 tensor-core step, on the CPU.

TEST INFRASTRUCTURE (see oracle/__init__.py).

The paper trains in full precision; the BF16 path is this library's
extension (tensor-core GEMMs with BF16 operands, FP32 accumulation, FP32
master weights, moments, rendering and losses). This module states exactly
which values that path rounds, so the GPU path can be checked to much tighter
bounds than its distance from the FP64 oracle allows:

  forward   gamma (the encoding), W1..W5 and h1..h4 (after the ReLU) are
            rounded to BF16; every product is then exact-accumulated (FP64
            here), biases are added unrounded;
  backward  dL/dy and dZ_l = (dZ_{l+1} W_{l+1}) * [h_l > 0] are rounded to
            BF16 before they enter a product; the masks come from the
            unrounded pre-activations; bias gradients are sums of the rounded
            dZ_l (and of the rounded dL/dy for b5).

Everything else (points, rendering, losses, sigmoid derivatives) is the FP64
oracle's own arithmetic. ``round_bf16`` is round-to-nearest-even of the FP32
value to 8 significant bits, written with integer operations on the FP32 bit
pattern; ``rounding=False`` turns every rounding off, which must give back
the FP64 oracle exactly.
"""
import numpy as np

from . import vmap_step as vs


def round_bf16(x):
    """Round to the nearest BF16 (ties to even) via FP32; returns FP64.
    NaN and infinities pass through."""
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    special = ~np.isfinite(f)
    return np.where(special, f.astype(np.float64), out)


def object_forward_backward(cfg, params, H, rays, t, center, scale, rounding=True):
    """Loss and gradient of one object with the BF16 path's roundings
    (same inputs and outputs as the FP64 oracle's function of that name)."""
    rb = round_bf16 if rounding else (lambda a: np.asarray(a, np.float64))
    Ws, bs = vs.unpack(params, H)
    Wr = [rb(W) for W in Ws]
    R, S = t.shape
    xt = vs.points(rays, t, center, scale)
    a = rb(vs.encode(xt.reshape(-1, 3), cfg.B))
    acts, masks = [a], []
    for l in range(4):
        z = a @ Wr[l].T + bs[l]
        masks.append(z > 0.0)
        a = rb(np.maximum(z, 0.0))
        acts.append(a)
    y = a @ Wr[4].T + bs[4]
    oc = vs.sigmoid(y).reshape(R, S, vs.N_OUT)
    o, c = oc[:, :, 0], oc[:, :, 1:]
    rend = vs.render(o, c, t)
    L, Ld, Lc, Lo = vs.object_loss(cfg, rays, rend)
    dLdo, dLdc = vs.render_backward(cfg, rays, t, o, c, rend)
    dy = np.concatenate([(dLdo * o * (1 - o))[:, :, None], dLdc * c * (1 - c)], axis=2)
    dz = rb(dy.reshape(-1, vs.N_OUT))
    dWs, dbs = [None] * 5, [None] * 5
    for l in range(4, -1, -1):
        dWs[l] = dz.T @ acts[l]
        dbs[l] = dz.sum(0)
        if l > 0:
            dz = rb((dz @ Wr[l]) * masks[l - 1])
    return dict(loss=L, Ld=Ld, Lc=Lc, Lo=Lo, grad=vs.pack(dWs, dbs), render=rend)
