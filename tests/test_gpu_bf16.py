"""The BF16 tensor-core path (tcgen05 MMAs, FP32 accumulation, FP32 master
weights, moments, rendering and losses).

Implementation parity: against the BF16 rounding model (oracle/bf16_model.py:
the FP64 oracle with the path's GEMM operands rounded to BF16), loss within
MODEL_LOSS_RTOL and every weight / bias gradient tensor within MODEL_G_RTOL
(relative L2); what remains is FP32 accumulation order, FP32 sin/cos before
rounding and the rare rounding or ReLU decision that these flip.

Precision (BF16 operands carry 8 significant bits), against the FP64 oracle:
  * per-step loss: 1e-3 relative on the first step, and within 2e-2 of the
    oracle over 60 steps (30 for hidden 128);
  * gradients: relative L2 error per tensor <= 1e-1 for any batch, <= 5e-2
    on batches of 100 rays or more (the error of a sum over few samples is
    larger; the rounding model shows the same numbers there).
Hidden width 128 runs as two kernels (forward / input gradients, then
split-K weight gradients) under the same bounds."""
import numpy as np
import pytest
import torch

from oracle import bf16_model as bm
from oracle import vmap_step as vs
from paper_2302_01838_b300 import scenes
from paper_2302_01838_b300.native import VMAP_BF16

import vmap_harness as vh

pytestmark = pytest.mark.gpu

MODEL_LOSS_RTOL = 1e-5
MODEL_G_RTOL = 1e-2


def _check_against_oracles(cfg, o, k, R, step, L, g):
    args = (cfg, np.asarray(o["init"], np.float64), o["H"])
    pk, tk = vs.sample_object(cfg, o["pool"], R, o["n_surface"], o["n_strat"], k, step)
    rays = o["pool"][pk].astype(np.float64)
    geo = (rays, tk, np.asarray(o["center"], np.float64), float(o["scale"]))
    m = bm.object_forward_backward(*args, *geo)
    assert abs(L - m["loss"]) <= MODEL_LOSS_RTOL * m["loss"], (k, L, m["loss"])
    em = vh.layer_errors(g, m["grad"], o["H"])
    assert max(em) <= MODEL_G_RTOL, (k, o["H"], em)
    f = vs.object_forward_backward(*args, *geo)
    assert abs(L - f["loss"]) <= 1e-3 * f["loss"], (k, L, f["loss"])
    ef = vh.layer_errors(g, f["grad"], o["H"])
    assert max(ef) <= (5e-2 if R >= 100 else 1e-1), (k, o["H"], R, ef)
    return max(em), max(ef)


def test_bf16_gradients_and_loss_vs_oracle():
    sc = vh.mixed_scene(seed=41)
    cfg = vh.oracle_config(sc)
    K = len(sc["objects"])
    R = [o["rays"] for o in sc["objects"]]
    vm = vh.library_context(sc, precision=VMAP_BF16)
    vm.sample_rays(R)
    L = torch.empty(K, device="cuda")
    vm.forward(L)
    gp = torch.zeros(vm.arena_size(), device="cuda")
    vm.backward(gp)
    assert vm.sync_status() == []
    L, gp = L.cpu().numpy(), gp.cpu().numpy()
    for k, o in enumerate(sc["objects"]):
        info = vm.object_info(k)
        g = gp[info["param_offset"]:info["param_offset"] + info["param_count"]]
        _check_against_oracles(cfg, o, k, R[k], 0, L[k], g)


def _wide_scene(seed, n_small=2, bg_rays=1200):
    """A room background (hidden 128, bg_rays rays: hundreds of tiles spread
    over every CTA range) and n_small hidden-32 objects."""
    rng = np.random.default_rng(seed)
    bg = scenes.background_object(rng)
    bg["rays"] = bg_rays
    objs = [bg]
    for _ in range(n_small):
        o = scenes.make_object(rng, (1, 2), 0.1, 0.3, 0.2, H=32, per_view=200)
        o["rays"] = 100
        objs.append(o)
    for o in objs:
        o["init"] = scenes.init_weights(rng, o["H"])
        o["n_surface"], o["n_strat"] = 10, 12
    return dict(objects=objs, B=scenes.make_B(seed + 1000), seed=seed)


def test_bf16_width_128_background_gradients_vs_oracle():
    sc = _wide_scene(45)
    cfg = vh.oracle_config(sc)
    K = len(sc["objects"])
    R = [o["rays"] for o in sc["objects"]]
    vm = vh.library_context(sc, precision=VMAP_BF16)
    vm.sample_rays(R)
    L = torch.empty(K, device="cuda")
    vm.forward(L)
    gp = torch.zeros(vm.arena_size(), device="cuda")
    vm.backward(gp)
    assert vm.sync_status() == []
    L, gp = L.cpu().numpy(), gp.cpu().numpy()
    for k, o in enumerate(sc["objects"]):
        info = vm.object_info(k)
        g = gp[info["param_offset"]:info["param_offset"] + info["param_count"]]
        _check_against_oracles(cfg, o, k, R[k], 0, L[k], g)
    # the training step's loss equals the forward's (same batch, before the update)
    lt = torch.empty(K, device="cuda")
    vm.train_step(lt)
    assert np.array_equal(lt.cpu().numpy(), L)


def test_bf16_width_128_training_follows_the_oracle():
    sc = _wide_scene(46, n_small=1, bg_rays=150)
    cfg = vh.oracle_config(sc)
    ost = vh.oracle_states(sc)
    vm = vh.library_context(sc, precision=VMAP_BF16)
    K = len(ost)
    R = [o["rays"] for o in sc["objects"]]
    loss = torch.empty(K, device="cuda")
    for step in range(30):
        vm.sample_rays(R)
        vm.train_step(loss)
        Lo = vs.train_step(cfg, ost, R)
        rel = np.abs(loss.cpu().numpy() - Lo) / np.abs(Lo)
        assert np.all(rel <= 2e-2), (step, rel)
    assert vm.sync_status() == []
    for k in range(K):
        p = vm.get_object_state(k)[0].cpu().numpy()
        errs = vh.layer_errors(p, ost[k].params, ost[k].H)
        assert max(errs) <= 5e-2, (k, errs)


def test_bf16_training_follows_the_oracle():
    sc = scenes.scene_small(seed=42, n_objects=6, rays=120)
    cfg = vh.oracle_config(sc)
    ost = vh.oracle_states(sc)
    vm = vh.library_context(sc, precision=VMAP_BF16)
    K = len(ost)
    loss = torch.empty(K, device="cuda")
    worst = 0.0
    for step in range(60):
        vm.sample_rays([120] * K)
        vm.train_step(loss)
        Lo = vs.train_step(cfg, ost, [120] * K)
        rel = np.abs(loss.cpu().numpy() - Lo) / np.abs(Lo)
        worst = max(worst, float(rel.max()))
        assert np.all(rel <= 2e-2), (step, rel)
    assert vm.sync_status() == []
    for k in range(K):
        p = vm.get_object_state(k)[0].cpu().numpy()
        errs = vh.layer_errors(p, ost[k].params, 32)
        assert max(errs) <= 5e-2, (k, errs)


def test_bf16_graph_replay_matches_eager_bitwise():
    sc = vh.mixed_scene(seed=43)
    R = [o["rays"] for o in sc["objects"]]
    a = vh.library_context(sc, precision=VMAP_BF16)
    b = vh.library_context(sc, precision=VMAP_BF16)
    b.set_graph(True)
    K = len(R)
    la, lb = torch.empty(K, device="cuda"), torch.empty(K, device="cuda")
    for _ in range(3):
        a.sample_rays(R); a.train_step(la)
        b.sample_rays(R); b.train_step(lb)
        assert torch.equal(la, lb)
    assert torch.equal(a.get_params(), b.get_params())
    # more width-128 rays than the activation buffer holds: it grows, and the
    # captured graph (which reads the buffer's address from device memory) stays valid
    R2 = [r * 6 if o["H"] == 128 else r for r, o in zip(R, sc["objects"])]
    for _ in range(2):
        a.sample_rays(R2); a.train_step(la)
        b.sample_rays(R2); b.train_step(lb)
        assert torch.equal(la, lb)
    assert torch.equal(a.get_params(), b.get_params())


def test_bf16_checkpoint_resume_refreshes_the_operand_images():
    sc = scenes.scene_small(seed=44, n_objects=2, rays=64)
    a = vh.library_context(sc, precision=VMAP_BF16)
    for _ in range(3):
        a.sample_rays([64, 64]); a.train_step()
    saved = [a.get_object_state(k) for k in range(2)]
    b = vh.library_context(sc, precision=VMAP_BF16)
    for k, (p, m, v, st) in enumerate(saved):
        b.set_object_state(k, p, m, v, st)
    la, lb = torch.empty(2, device="cuda"), torch.empty(2, device="cuda")
    for _ in range(2):
        a.sample_rays([64, 64]); a.train_step(la)
        b.sample_rays([64, 64]); b.train_step(lb)
        assert torch.equal(la, lb)


def test_bf16_training_then_queries_see_the_current_weights():
    """BF16 steps update the master weights; the FP32 query and depth-render
    kernels must evaluate exactly those weights afterwards."""
    sc = _wide_scene(47, n_small=2, bg_rays=64)
    cfg = vh.oracle_config(sc)
    R = [o["rays"] for o in sc["objects"]]
    vm = vh.library_context(sc, precision=VMAP_BF16)
    vm.set_graph(True)                       # replayed steps too
    rng = np.random.default_rng(0)
    for rep in range(2):
        for _ in range(5):
            vm.sample_rays(R)
            vm.train_step()
        _check_queries(vm, sc, cfg, rng)


def _check_queries(vm, sc, cfg, rng):
    for k, o in enumerate(sc["objects"]):
        p = vm.get_object_state(k)[0].cpu().numpy().astype(np.float64)
        pts = (np.asarray(o["center"], np.float64) + rng.uniform(-0.3, 0.3, (200, 3))).astype(np.float32)
        occ = torch.empty(200, device="cuda")
        vm.query_occupancy(k, torch.from_numpy(pts).cuda(), occ)
        ref, _ = vs.query(cfg, p, o["H"], np.asarray(o["center"], np.float64), float(o["scale"]), pts)
        assert np.max(np.abs(occ.cpu().numpy() - ref)) <= 1e-5, k


def test_bf16_overlapped_launches_match_serial_launches_bitwise():
    """With profiling off the width-128 kernels start behind the tile kernel on
    the SMs it frees (programmatic dependent launch); with profiling on every
    kernel runs alone between its timing events. Same results, bitwise."""
    sc = vh.mixed_scene(seed=47)
    R = [o["rays"] for o in sc["objects"]]
    a = vh.library_context(sc, precision=VMAP_BF16)
    b = vh.library_context(sc, precision=VMAP_BF16)
    b.profile_enable(True)
    K = len(R)
    la, lb = torch.empty(K, device="cuda"), torch.empty(K, device="cuda")
    for _ in range(4):
        a.sample_rays(R); a.train_step(la)
        b.sample_rays(R); b.train_step(lb)
        assert torch.equal(la, lb)
    assert torch.equal(a.get_params(), b.get_params())
    assert a.sync_status() == [] and b.sync_status() == []


def test_changing_ray_counts_rebuild_the_layout_in_graph_mode():
    """The batch layout is rebuilt only when its inputs change; alternating ray
    counts (and a paused object) in graph mode give the eager results bitwise and
    follow the FP64 oracle."""
    sc = scenes.scene_small(seed=48, n_objects=3, rays=60)
    cfg = vh.oracle_config(sc)
    ost = vh.oracle_states(sc)
    a = vh.library_context(sc, max_rays=400)
    b = vh.library_context(sc, max_rays=400)
    b.set_graph(True)
    plans = [[60, 60, 60], [60, 60, 60], [30, 90, 10], [30, 90, 10], [60, 60, 60], [0, 45, 60], [0, 45, 60]]
    la, lb = torch.empty(3, device="cuda"), torch.empty(3, device="cuda")
    for R in plans:
        a.sample_rays(R); a.train_step(la)
        b.sample_rays(R); b.train_step(lb)
        live = [k for k in range(3) if R[k] > 0]
        Lo = vs.train_step(cfg, [ost[k] for k in live], [R[k] for k in live])
        assert torch.equal(la[live], lb[live])
        rel = np.abs(la[live].cpu().numpy() - Lo) / np.abs(Lo)
        assert np.all(rel <= 1e-5), (R, rel)
    assert torch.equal(a.get_params(), b.get_params())
    assert [a.get_object_state(k)[3] for k in range(3)] == [5, 7, 7]


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_train_step_writes_losses_to_the_callers_buffer_in_graph_mode(precision):
    """The step's reduce writes the losses straight to the caller's buffer, whose
    address the replayed graph reads from device memory: switching buffers (or
    passing none) between replays gives the eager losses bitwise, NaN for an
    object outside the batch, and leaves the other buffers untouched."""
    from paper_2302_01838_b300.native import VMAP_FP32
    prec = VMAP_BF16 if precision == "bf16" else VMAP_FP32
    sc = scenes.scene_small(seed=49, n_objects=3, rays=60)
    a = vh.library_context(sc, max_rays=400, precision=prec)
    b = vh.library_context(sc, max_rays=400, precision=prec)
    b.set_graph(True)
    x = torch.full((3,), 7.0, device="cuda")
    y = torch.full((3,), 7.0, device="cuda")
    plans = [([60, 60, 60], x), ([60, 60, 60], y), ([0, 45, 60], x), ([60, 60, 60], None), ([30, 0, 60], y),
             ([60, 60, 60], x)]
    for R, dest in plans:
        ref = torch.empty(3, device="cuda")
        a.sample_rays(R); a.train_step(ref)
        before = {id(t): t.clone() for t in (x, y)}
        b.sample_rays(R); b.train_step(dest)
        torch.cuda.synchronize()
        for t in (x, y):
            if t is not dest:
                assert torch.allclose(t, before[id(t)], rtol=0, atol=0, equal_nan=True)
        if dest is None:
            continue
        gone = [k for k in range(3) if R[k] == 0]
        assert torch.isnan(ref[gone]).all() and torch.isnan(dest[gone]).all()
        live = [k for k in range(3) if R[k] > 0]
        assert torch.isfinite(ref[live]).all()
        assert torch.equal(ref[live], dest[live])
    assert torch.equal(a.get_params(), b.get_params())


def test_combined_step_matches_separate_calls_bitwise():
    """vmap_step (the sampler, then the tile kernel launched behind it with a
    programmatic dependency, then the width-128 kernels behind that) gives the
    results of vmap_sample_rays + vmap_train_step bitwise: eager, replayed, and
    with profiling events between every launch; across layout rebuilds, with a
    paused object, with no hidden-32 rays at all (the tile kernel's CTAs have no
    tiles and the width-128 kernels still read the sampler's output) and with
    no background rays."""
    sc = _wide_scene(50, n_small=3, bg_rays=600)
    R0 = [o["rays"] for o in sc["objects"]]
    K = len(R0)
    ctxs = [vh.library_context(sc, precision=VMAP_BF16, max_rays=4000) for _ in range(4)]
    sep, eager, graph, prof = ctxs
    graph.set_graph(True)
    prof.profile_enable(True)
    plans = [R0, R0, [1500] + R0[1:], [1500] + R0[1:], [600, 0, 100, 100], [600, 0, 0, 0], [600, 0, 0, 0],
             [0, 100, 100, 100], R0, R0]
    for R in plans:
        ref = torch.empty(K, device="cuda")
        sep.sample_rays(R); sep.train_step(ref)
        live = [k for k in range(K) if R[k] > 0]
        gone = [k for k in range(K) if R[k] == 0]
        for vm in (eager, graph, prof):
            out = torch.empty(K, device="cuda")
            vm.step(R, out)
            assert torch.equal(out[live], ref[live]), (R, out, ref)
            assert torch.isnan(out[gone]).all() and torch.isnan(ref[gone]).all()
    p = sep.get_params()
    for vm in (eager, graph, prof):
        assert torch.equal(vm.get_params(), p)
        assert vm.sync_status() == []


def test_host_buffer_step_in_graph_mode_matches_separate_calls_bitwise():
    """vmap_train_step_host (pinned host rays, one replayed launch sequence with
    the sampler, host losses) equals vmap_sample_rays_given + vmap_train_step on
    the same rays, including the width-128 background, a changed ray count (a
    layout rebuild) and an object outside the batch."""
    sc = _wide_scene(51, n_small=2, bg_rays=300)
    K = len(sc["objects"])
    dev = vh.library_context(sc, precision=VMAP_BF16, max_rays=2000)
    host = vh.library_context(sc, precision=VMAP_BF16, max_rays=2000)
    host.set_graph(True)
    rng = np.random.default_rng(9)
    loss_d = torch.empty(K, device="cuda")
    loss_h = torch.empty(K).pin_memory()
    for R in ([300, 100, 100], [300, 100, 100], [500, 0, 60], [500, 0, 60], [300, 100, 100]):
        given = [o["pool"][rng.integers(0, o["pool"].shape[0], max(R[k], 1))][:R[k]]
                 for k, o in enumerate(sc["objects"])]
        flat = np.concatenate([g for g in given if g.shape[0]]).astype(np.float32)
        dev.sample_rays_given(torch.from_numpy(flat).cuda(), R)
        dev.train_step(loss_d)
        host.train_step_host(torch.from_numpy(flat).pin_memory(), R, loss_h)
        assert np.array_equal(loss_d.cpu().numpy(), loss_h.numpy(), equal_nan=True)
        assert all(np.isnan(loss_h.numpy()[k]) == (R[k] == 0) for k in range(K))
    assert torch.equal(dev.get_params(), host.get_params())
    assert dev.sync_status() == [] and host.sync_status() == []


def test_mixed_pool_and_host_steps_in_graph_mode():
    """Alternating vmap_step (pool rays), vmap_train_step_host (caller rays) and the
    separate calls on one replayed context (each switch of ray source rebuilds
    the layout) trains exactly like a context doing the same with separate calls."""
    sc = _wide_scene(53, n_small=2, bg_rays=300)
    K = len(sc["objects"])
    R = [o["rays"] for o in sc["objects"]]
    ref = vh.library_context(sc, precision=VMAP_BF16, max_rays=2000)
    mix = vh.library_context(sc, precision=VMAP_BF16, max_rays=2000)
    mix.set_graph(True)
    rng = np.random.default_rng(4)
    lr, lm = torch.empty(K, device="cuda"), torch.empty(K, device="cuda")
    lh = torch.empty(K).pin_memory()
    for kind in ("step", "host", "step", "sep", "host", "host", "step"):
        if kind == "host":
            flat = np.concatenate([o["pool"][rng.integers(0, o["pool"].shape[0], R[k])]
                                   for k, o in enumerate(sc["objects"])]).astype(np.float32)
            ref.sample_rays_given(torch.from_numpy(flat).cuda(), R); ref.train_step(lr)
            mix.train_step_host(torch.from_numpy(flat).pin_memory(), R, lh)
            assert np.array_equal(lr.cpu().numpy(), lh.numpy())
        else:
            ref.sample_rays(R); ref.train_step(lr)
            if kind == "step":
                mix.step(R, lm)
            else:
                mix.sample_rays(R); mix.train_step(lm)
            assert torch.equal(lr, lm)
    assert torch.equal(ref.get_params(), mix.get_params())
    assert mix.sync_status() == []
