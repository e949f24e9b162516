"""Pins of the oracle's hand-written backward and of its Adam.

Backward: central finite differences in FP64 for every parameter and for the
object centre (the encoding backward), plus PyTorch autograd on an
independent torch formulation of the forward. Adam: the closed-form first
step and torch.optim.Adam over several steps."""
import numpy as np
import pytest
import torch

from oracle import vmap_step as vs


def _tiny_case(H=4, R=3, S=5, seed=0, lam_occ=0.0, mask=None):
    rng = np.random.default_rng(seed)
    cfg = vs.Config(B=rng.standard_normal((45, 3)) * 2.0, lambda_occ=lam_occ)
    rays = np.zeros((R, 12))
    rays[:, 0:3] = rng.uniform(-1, 1, (R, 3))
    rays[:, 3:6] = rng.uniform(-0.5, 0.5, (R, 3))
    rays[:, 6] = rng.uniform(0.5, 1.5, R)
    rays[:, 7:10] = rng.uniform(0, 1, (R, 3))
    rays[:, 10] = 1.0 if mask is None else mask
    t = np.sort(rng.uniform(0.1, 2.0, (R, S)), axis=1)
    p = rng.standard_normal(vs.param_count(H)) * 0.7
    center = rng.uniform(-0.3, 0.3, 3)
    return cfg, rays, t, p, center, 0.8


def _loss(cfg, p, H, rays, t, center, scale):
    return vs.object_forward_backward(cfg, p, H, rays, t, center, scale)["loss"]


@pytest.mark.parametrize("lam_occ,mask", [(0.0, None), (10.0, [1.0, 0.0, 1.0])])
def test_backward_matches_finite_differences(lam_occ, mask):
    H = 4
    cfg, rays, t, p, center, scale = _tiny_case(H=H, lam_occ=lam_occ, mask=mask)
    res = vs.object_forward_backward(cfg, p, H, rays, t, center, scale, want_center_grad=True)
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p); e[i] = h
        fd[i] = (_loss(cfg, p + e, H, rays, t, center, scale)
                 - _loss(cfg, p - e, H, rays, t, center, scale)) / (2 * h)
    err = np.abs(fd - res["grad"])
    assert np.max(err) < 1e-7 * max(1.0, np.max(np.abs(fd))), np.argmax(err)
    fdc = np.empty(3)
    for i in range(3):
        e = np.zeros(3); e[i] = h
        fdc[i] = (_loss(cfg, p, H, rays, t, center + e, scale)
                  - _loss(cfg, p, H, rays, t, center - e, scale)) / (2 * h)
    assert np.allclose(res["dcenter"], fdc, rtol=1e-6, atol=1e-8)


def test_backward_matches_torch_autograd():
    """An independent torch formulation of the forward, differentiated by autograd."""
    H, R, S = 6, 4, 7
    cfg, rays, t, p, center, scale = _tiny_case(H=H, R=R, S=S, seed=3, lam_occ=10.0)
    res = vs.object_forward_backward(cfg, p, H, rays, t, center, scale, want_center_grad=True)

    P = torch.tensor(p, requires_grad=True)
    c = torch.tensor(center, requires_grad=True)
    rt = torch.tensor(rays)
    tt = torch.tensor(t)
    B = torch.tensor(cfg.B)
    x = (rt[:, None, 0:3] + tt[..., None] * rt[:, None, 3:6] - c) / scale
    proj = x @ B.T
    h = torch.cat([x, torch.sin(proj), torch.cos(proj)], -1)
    off = 0
    for li, (o, i) in enumerate(vs.layer_shapes(H)):
        W = P[off:off + o * i].view(o, i); off += o * i
        b = P[off:off + o]; off += o
        h = torch.nn.functional.linear(h, W, b)
        if li < 4:
            h = torch.relu(h)
    s = torch.sigmoid(h)
    occ, col = s[..., 0], s[..., 1:]
    trans = torch.cumprod(torch.cat([torch.ones(R, 1, dtype=occ.dtype), 1 - occ[:, :-1]], 1), 1)
    w = occ * trans
    Dh = (w * tt).sum(1)
    Ch = (w[..., None] * col).sum(1)
    Oh = w.sum(1)
    Dg, Cg, Mg = rt[:, 6], rt[:, 7:10], rt[:, 10]
    L = ((Mg * (Dh - Dg).abs()).sum() / R + 5 * (Mg[:, None] * (Ch - Cg).abs()).sum() / (3 * R)
         + 10 * (Oh - Mg).abs().sum() / R)
    L.backward()
    assert abs(L.item() - res["loss"]) < 1e-13
    assert np.allclose(P.grad.numpy(), res["grad"], rtol=1e-10, atol=1e-13)
    assert np.allclose(c.grad.numpy(), res["dcenter"], rtol=1e-10, atol=1e-13)


def test_render_gradient_saturated_occupancy():
    """o = 1 exactly (FP32 sigmoid saturation): the recursion must not divide by 1 - o."""
    cfg = vs.Config()
    rays = np.zeros((1, 12)); rays[0, 6] = 1.0; rays[0, 7:10] = 0.5; rays[0, 10] = 1
    t = np.array([[0.5, 1.0, 1.5, 2.0]])
    o = np.array([[0.2, 1.0, 0.3, 0.9]])
    c = np.full((1, 4, 3), 0.25)
    rend = vs.render(o, c, t)
    dLdo, dLdc = vs.render_backward(cfg, rays, t, o, c, rend)
    assert np.all(np.isfinite(dLdo))
    # behind a fully occupied sample nothing matters
    assert dLdo[0, 2] == 0 and dLdo[0, 3] == 0 and np.all(dLdc[0, 2:] == 0)
    # FD on o_0 and o_1 (only from the left, o <= 1)
    def L(o_):
        return vs.object_loss(cfg, rays, vs.render(o_, c, t))[0]
    h = 1e-7
    for i in (0,):
        e = np.zeros_like(o); e[0, i] = h
        assert abs((L(o + e) - L(o - e)) / (2 * h) - dLdo[0, i]) < 1e-6
    e = np.zeros_like(o); e[0, 1] = h
    assert abs((L(o) - L(o - e)) / h - dLdo[0, 1]) < 1e-5


def test_adam_first_step_closed_form():
    cfg = vs.Config(lr=1e-3)
    g = np.array([3.0, -2e-4, 0.0, 1e-12])
    th, m, v, st = vs.adam_update(cfg, np.zeros(4), g, np.zeros(4), np.zeros(4), 0)
    assert st == 1
    assert np.allclose(th, -cfg.lr * g / (np.abs(g) + cfg.eps), rtol=1e-12, atol=0)


def test_adam_matches_torch_optim():
    rng = np.random.default_rng(4)
    cfg = vs.Config(lr=3e-3, beta1=0.85, beta2=0.99, eps=1e-7)
    theta = rng.standard_normal(50)
    m = np.zeros(50); v = np.zeros(50); st = 0
    tp = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=cfg.lr, betas=(cfg.beta1, cfg.beta2), eps=cfg.eps)
    for k in range(12):
        g = rng.standard_normal(50) * 10.0 ** rng.uniform(-6, 1)
        theta, m, v, st = vs.adam_update(cfg, theta, g, m, v, st)
        tp.grad = torch.tensor(g)
        opt.step()
    assert np.allclose(theta, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_per_ray_origin_and_direction_gradients_by_finite_differences():
    """dL/do and dL/dd of single rays (sample depths held fixed), the
    primitive of camera-pose refinement, against central differences."""
    import numpy as np
    from oracle import vmap_step as vs
    from paper_2302_01838_b300 import scenes
    rng = np.random.default_rng(31)
    o = scenes.make_object(rng, (1, 2), 0.1, 0.3, 0.2, H=16, per_view=64)
    cfg = vs.Config(seed=2, B=scenes.make_B(8))
    p = scenes.init_weights(rng, 16).astype(np.float64)
    pick, t = vs.sample_object(cfg, o["pool"], 12, 10, 12, 0, 0)
    rays = o["pool"][pick].astype(np.float64)
    c = np.asarray(o["center"], np.float64)
    res = vs.object_forward_backward(cfg, p, 16, rays, t, c, float(o["scale"]), want_center_grad=True)
    h = 1e-6
    for r in (0, 5, 11):
        for a in range(3):
            for col, key in ((a, "dray_o"), (3 + a, "dray_d")):
                rp, rm = rays.copy(), rays.copy()
                rp[r, col] += h
                rm[r, col] -= h
                Lp = vs.object_forward_backward(cfg, p, 16, rp, t, c, float(o["scale"]))["loss"]
                Lm = vs.object_forward_backward(cfg, p, 16, rm, t, c, float(o["scale"]))["loss"]
                fd = (Lp - Lm) / (2 * h)
                assert abs(fd - res[key][r, a]) <= 1e-5 * max(1.0, abs(fd)), (r, a, key, fd, res[key][r, a])
    # the centre gradient is minus the sum of the origin gradients
    assert np.allclose(res["dcenter"], -res["dray_o"].sum(0))
