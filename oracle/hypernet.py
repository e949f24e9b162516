"""FP64 oracle of the warm-start set-encoder hypernetwork.

TEST INFRASTRUCTURE (see oracle/__init__.py).

The paper has no such network; it is a learned extension of the method: from a
set of N points (x~, occupancy, rgb) taken from a newly seen object's first
keyframe, predict initial weights for the object's MLP.

  per point:  h1 = ReLU(W1 x + b1), h2 = ReLU(W2 h1 + b2), h3 = ReLU(W3 h2 + b3)
  set:        z = max over points of h3 (per channel; ties -> lowest point index)
  head:       u = Wa z + ba (rank r), theta = Wb u + bb (P outputs)
  loss:       L = sum_{b,p} (theta_bp - target_bp)^2 / (B P)

Parameters (flat, in this order): W1 [w][7], b1, W2 [w][w], b2, W3 [w][w], b3,
Wa [r][w], ba [r], Wb [P][r], bb [P].

With bf16=True the functions follow the library's BF16 mode: the operands
of the GEMMs of the 128-wide layers (h1 W2^T, h2 W3^T in the forward; dZ3 W3,
dZ2 W2 and the weight gradients dZ3^T h2, dZ2^T h1 in the backward) are
rounded to BF16 (round to nearest even, oracle.bf16_model.round_bf16);
everything else stays FP64.
"""
import numpy as np

from .bf16_model import round_bf16


def _rb(on):
    return round_bf16 if on else (lambda a: a)


def shapes(width=128, rank=16, P=6308, d_in=7):
    return [(width, d_in), (width,), (width, width), (width,), (width, width), (width,),
            (rank, width), (rank,), (P, rank), (P,)]


def count(width=128, rank=16, P=6308, d_in=7):
    return int(sum(np.prod(s) for s in shapes(width, rank, P, d_in)))


def unpack(flat, width=128, rank=16, P=6308, d_in=7):
    flat = np.asarray(flat, np.float64)
    out, off = [], 0
    for s in shapes(width, rank, P, d_in):
        n = int(np.prod(s))
        out.append(flat[off:off + n].reshape(s))
        off += n
    assert off == flat.size
    return out


def pack(parts):
    return np.concatenate([np.asarray(p, np.float64).ravel() for p in parts])


def forward(params, X, width=128, rank=16, P=6308, bf16=False):
    """X [B, N, 7] -> (theta [B, P], cache)."""
    rb = _rb(bf16)
    W1, b1, W2, b2, W3, b3, Wa, ba, Wb, bb = unpack(params, width, rank, P, X.shape[-1])
    X = np.asarray(X, np.float64)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(rb(h1) @ rb(W2).T + b2, 0.0)
    h3 = np.maximum(rb(h2) @ rb(W3).T + b3, 0.0)
    arg = h3.argmax(axis=1)                      # first occurrence of the maximum
    z = np.take_along_axis(h3, arg[:, None, :], axis=1)[:, 0, :]
    u = z @ Wa.T + ba
    theta = u @ Wb.T + bb
    return theta, dict(X=X, h1=h1, h2=h2, h3=h3, arg=arg, z=z, u=u)


def loss(theta, target):
    d = theta - np.asarray(target, np.float64)
    return float(np.sum(d * d) / d.size)


def backward(params, cache, theta, target, width=128, rank=16, P=6308, bf16=False):
    """Gradient of ``loss`` with respect to the flat parameters."""
    rb = _rb(bf16)
    W1, b1, W2, b2, W3, b3, Wa, ba, Wb, bb = unpack(params, width, rank, P, cache["X"].shape[-1])
    B, N, _ = cache["X"].shape
    dth = 2.0 * (theta - np.asarray(target, np.float64)) / theta.size
    dWb = dth.T @ cache["u"]
    dbb = dth.sum(0)
    du = dth @ Wb
    dWa = du.T @ cache["z"]
    dba = du.sum(0)
    dz = du @ Wa
    dh3 = np.zeros_like(cache["h3"])
    b_idx = np.arange(B)[:, None]
    c_idx = np.arange(width)[None, :]
    dh3[b_idx, cache["arg"], c_idx] = dz            # max-pool routes to the arg-max point
    dz3 = dh3 * (cache["h3"] > 0)
    dW3 = np.einsum("bnc,bnk->ck", rb(dz3), rb(cache["h2"]))
    db3 = dz3.sum((0, 1))
    dz2 = (rb(dz3) @ rb(W3)) * (cache["h2"] > 0)
    dW2 = np.einsum("bnc,bnk->ck", rb(dz2), rb(cache["h1"]))
    db2 = dz2.sum((0, 1))
    dz1 = (rb(dz2) @ rb(W2)) * (cache["h1"] > 0)
    dW1 = np.einsum("bnc,bnk->ck", dz1, cache["X"])
    db1 = dz1.sum((0, 1))
    return pack([dW1, db1, dW2, db2, dW3, db3, dWa, dba, dWb, dbb])
