"""Pins of the warm-start hypernetwork oracle: finite differences and torch
autograd for the gradient, the max-pool routing, and a closed-form case."""
import numpy as np
import torch

from oracle import hypernet as hn


def _case(seed=0, B=3, N=9, w=8, r=3, P=11):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((B, N, 7))
    p = rng.standard_normal(hn.count(w, r, P)) * 0.4
    T = rng.standard_normal((B, P))
    return X, p, T, dict(width=w, rank=r, P=P)


def test_gradient_matches_finite_differences():
    X, p, T, kw = _case()
    th, cache = hn.forward(p, X, **kw)
    g = hn.backward(p, cache, th, T, **kw)
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p); e[i] = h
        fd[i] = (hn.loss(hn.forward(p + e, X, **kw)[0], T) - hn.loss(hn.forward(p - e, X, **kw)[0], T)) / (2 * h)
    assert np.max(np.abs(fd - g)) < 1e-7 * max(1.0, np.abs(fd).max())


def test_gradient_matches_torch_autograd():
    X, p, T, kw = _case(seed=1, B=4, N=16, w=12, r=4, P=20)
    th, cache = hn.forward(p, X, **kw)
    g = hn.backward(p, cache, th, T, **kw)
    P = torch.tensor(p, requires_grad=True)
    parts, off = [], 0
    for s in hn.shapes(kw["width"], kw["rank"], kw["P"]):
        n = int(np.prod(s)); parts.append(P[off:off + n].view(*s)); off += n
    W1, b1, W2, b2, W3, b3, Wa, ba, Wb, bb = parts
    x = torch.tensor(X)
    h = torch.relu(x @ W1.T + b1); h = torch.relu(h @ W2.T + b2); h = torch.relu(h @ W3.T + b3)
    z = h.max(dim=1).values
    out = (z @ Wa.T + ba) @ Wb.T + bb
    L = ((out - torch.tensor(T)) ** 2).mean()
    L.backward()
    assert abs(L.item() - hn.loss(th, T)) < 1e-12
    assert np.allclose(P.grad.numpy(), g, rtol=1e-9, atol=1e-12)


def test_max_pool_picks_the_largest_point_and_lowest_index_on_ties():
    w, r, P = 2, 1, 2
    # W1 = I on the first two inputs, everything else identity-like so h3 = relu(x[:, :2])
    parts = [np.zeros((w, 7)), np.zeros(w), np.eye(w), np.zeros(w), np.eye(w), np.zeros(w),
             np.ones((r, w)), np.zeros(r), np.ones((P, r)), np.zeros(P)]
    parts[0][0, 0] = parts[0][1, 1] = 1.0
    p = hn.pack(parts)
    X = np.zeros((1, 4, 7))
    X[0, :, 0] = [0.5, 2.0, 2.0, 1.0]
    X[0, :, 1] = [3.0, -1.0, 0.0, 3.0]
    th, cache = hn.forward(p, X, width=w, rank=r, P=P)
    assert list(cache["arg"][0]) == [1, 0]
    assert np.allclose(cache["z"][0], [2.0, 3.0])
    assert np.allclose(th[0], [5.0, 5.0])          # u = 2 + 3, theta = u


def test_bf16_hypernet_model_reduces_to_fp64_and_stays_close():
    """The hypernetwork's BF16 rounding model: bf16=False is the FP64 model
    bitwise; bf16=True stays within BF16-level relative error of it."""
    import numpy as np
    from oracle import hypernet as hn
    rng = np.random.default_rng(7)
    B, N, P = 3, 24, 100
    p = rng.standard_normal(hn.count(P=P)) * 0.1
    X = rng.standard_normal((B, N, 7))
    T = rng.standard_normal((B, P)) * 0.1
    th0, c0 = hn.forward(p, X, P=P)
    th1, c1 = hn.forward(p, X, P=P, bf16=False)
    assert np.array_equal(th0, th1)
    g0 = hn.backward(p, c0, th0, T, P=P)
    assert np.array_equal(g0, hn.backward(p, c1, th1, T, P=P, bf16=False))
    thb, cb = hn.forward(p, X, P=P, bf16=True)
    gb = hn.backward(p, cb, thb, T, P=P, bf16=True)
    assert 0 < np.linalg.norm(thb - th0) <= 2e-2 * np.linalg.norm(th0)
    assert 0 < np.linalg.norm(gb - g0) <= 5e-2 * np.linalg.norm(g0)
