"""The warm-start hypernetwork's GPU forward/backward against the FP64 oracle,
its training, and the warm start through the C ABI.

Tolerances: loss 1e-5 relative; gradient relative L2 per parameter tensor
1e-4 (FP32 sums over 256-point sets and batches)."""
import numpy as np
import pytest
import torch

from oracle import hypernet as hn
from paper_2302_01838_b300 import scenes

import vmap_harness as vh

pytestmark = pytest.mark.gpu


def _inputs(B, seed=0):
    sc = scenes.scene_shapes(seed, B)
    X = np.stack([o["set_input"] for o in sc["objects"]])
    return sc, X


def test_hypernet_gradient_matches_oracle():
    from paper_2302_01838_b300.api import HyperNet
    B = 6
    sc, X = _inputs(B, seed=3)
    rng = np.random.default_rng(1)
    hyp = HyperNet(max_batch=8, seed=5)
    p = rng.standard_normal(hyp.n_params).astype(np.float32) * 0.1
    T = rng.standard_normal((B, hyp.P)).astype(np.float32) * 0.2
    hyp.set_params(torch.from_numpy(p).cuda())
    g, loss = hyp.grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    th, cache = hn.forward(p.astype(np.float64), X.astype(np.float64))
    gref = hn.backward(p.astype(np.float64), cache, th, T)
    assert abs(loss.item() - hn.loss(th, T)) <= 1e-5 * hn.loss(th, T)
    g = g.cpu().numpy()
    parts_g = hn.unpack(g)
    parts_r = hn.unpack(gref)
    for i, (a, b) in enumerate(zip(parts_g, parts_r)):
        assert vh.rel_l2(a, b) <= 1e-4, (i, vh.rel_l2(a, b))
    pred = hyp.predict(torch.from_numpy(X).cuda()).cpu().numpy()
    assert np.max(np.abs(pred - th)) <= 1e-4 * max(1.0, np.abs(th).max())


def test_hypernet_training_and_warmstart():
    from paper_2302_01838_b300.api import HyperNet
    B = 16
    sc, X = _inputs(B, seed=4)
    rng = np.random.default_rng(2)
    T = (rng.standard_normal((B, 6308)) * 0.1).astype(np.float32)
    hyp = HyperNet(max_batch=B, seed=6)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    loss = torch.empty(1, device="cuda")
    hyp.train_step(Xd, Td, 1e-3, loss)
    first = loss.item()
    for _ in range(200):
        hyp.train_step(Xd, Td, 1e-3, loss)
    assert loss.item() < 0.5 * first
    # warm start installs exactly the prediction, with fresh optimiser state
    vm = vh.library_context(dict(objects=sc["objects"][:2], B=sc["B"], seed=sc["seed"]))
    vm.sample_rays([120, 120]); vm.train_step()
    vm.warmstart(1, hyp, Xd[1])
    p, m, v, st = vm.get_object_state(1)
    pred = hyp.predict(Xd[1:2])[0]
    assert torch.equal(p, pred) and st == 0
    assert float(m.abs().max()) == 0.0 and float(v.abs().max()) == 0.0
    vm.sample_rays([120, 120]); vm.train_step()
    assert vm.get_object_state(1)[3] == 1 and vm.get_object_state(0)[3] == 2


def test_bf16_hypernet_gradient_matches_rounding_model():
    """BF16 mode (tensor-core GEMMs for the 128-wide layers) against the
    oracle's BF16 rounding model (tight) and the FP64 model (BF16-level)."""
    from paper_2302_01838_b300.api import HyperNet
    from paper_2302_01838_b300.native import VMAP_BF16
    B = 6
    sc, X = _inputs(B, seed=3)
    rng = np.random.default_rng(1)
    hyp = HyperNet(max_batch=8, seed=5)
    hyp.set_precision(VMAP_BF16)
    p = rng.standard_normal(hyp.n_params).astype(np.float32) * 0.1
    T = rng.standard_normal((B, hyp.P)).astype(np.float32) * 0.2
    hyp.set_params(torch.from_numpy(p).cuda())
    g, loss = hyp.grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    g = g.cpu().numpy()
    for bf16, tol in ((True, 1e-2), (False, 1e-1)):
        th, cache = hn.forward(p.astype(np.float64), X.astype(np.float64), bf16=bf16)
        gref = hn.backward(p.astype(np.float64), cache, th, T, bf16=bf16)
        assert abs(loss.item() - hn.loss(th, T)) <= (1e-4 if bf16 else 1e-2) * hn.loss(th, T)
        errs = [vh.rel_l2(a, b) for a, b in zip(hn.unpack(g), hn.unpack(gref))]
        assert max(errs) <= tol, (bf16, errs)
    # training in BF16 mode lowers the loss
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    out = torch.empty(1, device="cuda")
    hyp.train_step(Xd, Td, 1e-3, out)
    first = out.item()
    for _ in range(100):
        hyp.train_step(Xd, Td, 1e-3, out)
    assert out.item() < 0.7 * first
