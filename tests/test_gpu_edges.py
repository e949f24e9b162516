"""Degenerate and boundary cases of the step, FP32 and BF16, against the
oracle: an empty batch, rays with invalid depth (sampled up to t_far), one
sample per ray, the maximum of 32 samples per ray, a single-ray batch, and
capacity limits reached exactly."""
import numpy as np
import pytest
import torch

from oracle import bf16_model as bm
from oracle import vmap_step as vs
from paper_2302_01838_b300 import scenes
from paper_2302_01838_b300.native import VMAP_BF16, VmapError

import vmap_harness as vh

pytestmark = pytest.mark.gpu


def _scene(seed, specs):
    """specs: (H, n_surface, n_strat, rays, invalid_depth_fraction)."""
    rng = np.random.default_rng(seed)
    objs = []
    for H, ns, nc, R, bad in specs:
        o = scenes.make_object(rng, (1, 2), 0.1, 0.3, 0.2, H=H, per_view=128)
        if bad:
            pool = o["pool"].copy()
            pool[rng.random(pool.shape[0]) < bad, 6] = 0.0     # no depth measured
            o["pool"] = pool
        o["init"] = scenes.init_weights(rng, H)
        o["n_surface"], o["n_strat"], o["rays"] = ns, nc, R
        objs.append(o)
    return dict(objects=objs, B=scenes.make_B(seed + 1), seed=seed)


SPECS = [(32, 1, 0, 40, 0.0),      # one Gaussian sample per ray
         (16, 0, 1, 33, 0.0),      # one stratified sample per ray
         (64, 15, 17, 17, 0.3),    # 32 samples per ray, some rays without depth
         (32, 10, 12, 1, 0.0),     # a single ray
         (128, 10, 12, 9, 0.5)]    # hidden 128, half the rays without depth


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_degenerate_batches_match_the_oracle(precision):
    sc = _scene(91, SPECS)
    cfg = vh.oracle_config(sc)
    R = [o["rays"] for o in sc["objects"]]
    kw = dict(precision=VMAP_BF16) if precision == "bf16" else {}
    vm = vh.library_context(sc, **kw)
    vm.sample_rays(R)
    L = torch.empty(len(R), device="cuda")
    vm.forward(L)
    gp = torch.zeros(vm.arena_size(), device="cuda")
    vm.backward(gp)
    assert vm.sync_status() == []
    L, gp = L.cpu().numpy(), gp.cpu().numpy()
    for k, o in enumerate(sc["objects"]):
        pk, tk = vs.sample_object(cfg, o["pool"], R[k], o["n_surface"], o["n_strat"], k, 0)
        if o["n_surface"] + o["n_strat"] == 32 or k == 4:
            # rays without depth sample up to t_far (an 8 m ray through the box)
            bad = o["pool"][pk, 6] <= 0
            if bad.any():
                assert np.max(tk[bad]) > 1.0
        rays = o["pool"][pk].astype(np.float64)
        args = (cfg, np.asarray(o["init"], np.float64), o["H"], rays, tk, np.asarray(o["center"], np.float64),
                float(o["scale"]))
        ref = bm.object_forward_backward(*args) if precision == "bf16" else vs.object_forward_backward(*args)
        info = vm.object_info(k)
        g = gp[info["param_offset"]:info["param_offset"] + info["param_count"]]
        ltol, gtol = (1e-5, 1e-2) if precision == "bf16" else (1e-5, 1e-4)
        assert abs(L[k] - ref["loss"]) <= ltol * abs(ref["loss"]) + 1e-7, (k, L[k], ref["loss"])
        errs = vh.layer_errors(g, ref["grad"], o["H"])
        assert max(errs) <= gtol, (k, errs)


def test_empty_batch_and_exact_capacity():
    sc = _scene(93, [(32, 10, 12, 8, 0.0), (16, 7, 9, 8, 0.0)])
    vm = vh.library_context(sc, max_rays=24)
    # nothing requested: the step trains nothing and reports NaN losses
    vm.sample_rays([0, 0])
    L = torch.zeros(2, device="cuda")
    vm.train_step(L)
    assert torch.isnan(L).all() and vm.get_object_state(0)[3] == 0 and vm.get_object_state(1)[3] == 0
    # exactly max_rays_total rays is allowed, one more is refused
    vm.sample_rays([12, 12])
    vm.train_step(L)
    assert torch.isfinite(L).all() and vm.get_object_state(1)[3] == 1
    with pytest.raises(VmapError, match="ERR_CAPACITY"):
        vm.sample_rays([13, 12])
    # the context is intact: the next step trains object 0 only
    vm.sample_rays([5, 0])
    vm.train_step(L)
    assert torch.isfinite(L[0]) and torch.isnan(L[1])
    assert vm.get_object_state(0)[3] == 2 and vm.get_object_state(1)[3] == 1


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_combined_step_on_degenerate_batches_and_capacity(precision):
    """vmap_step, replayed, on the degenerate batches above (one sample per ray,
    32 samples, rays without depth, a single ray, hidden 128), an empty batch
    and a half-empty one equals the separate calls bitwise; a request past the
    capacity is refused before anything is launched and the context trains on."""
    sc = _scene(95, SPECS)
    R = [o["rays"] for o in sc["objects"]]
    K = len(R)
    kw = dict(precision=VMAP_BF16) if precision == "bf16" else {}
    a = vh.library_context(sc, **kw)
    b = vh.library_context(sc, **kw)
    b.set_graph(True)
    half = [r if k % 2 else 0 for k, r in enumerate(R)]
    for plan in (R, [0] * K, R, half, half, R):
        la, lb = torch.empty(K, device="cuda"), torch.empty(K, device="cuda")
        a.sample_rays(plan); a.train_step(la)
        b.step(plan, lb)
        assert torch.allclose(la, lb, rtol=0, atol=0, equal_nan=True), (plan, la, lb)
        assert all(bool(torch.isnan(lb[k])) == (plan[k] == 0) for k in range(K))
    with pytest.raises(VmapError, match="ERR_CAPACITY"):
        b.step([10 ** 6] + R[1:], lb)
    a.sample_rays(R); a.train_step(la)
    b.step(R, lb)
    assert torch.equal(la, lb)
    assert torch.equal(a.get_params(), b.get_params())
    assert a.sync_status() == [] and b.sync_status() == []
