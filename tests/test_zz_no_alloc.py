"""The allocation-free entry point (vmap_object_grad_static) against the
context-based path, through the C ABI.

Callers such as custom allocators, real-time loops or hosts that plan every
device allocation cannot call cudaMalloc; this entry point serves them from a
static device array. Its gradient and loss must match what a context computes
for the same object, the same rays and the same step count (vmap_sample_rays_given
+ vmap_forward + vmap_backward), within the tolerances of the other parity
tests, on two calls in a row (the second call must not see stale scratch)."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2302_01838_b300 import native, scenes

import vmap_harness as vh

pytestmark = pytest.mark.gpu


def _static_grad(lib, cfg, o, rays, params, step, stream_id):
    d = native.VmapObjectDesc()
    d.hidden = o["H"]
    d.n_surface, d.n_strat = o["n_surface"], o["n_strat"]
    for a in range(3):
        d.center[a] = float(o["center"][a])
    d.scale = float(o["scale"])
    d.rays = rays.data_ptr()
    d.n_rays = rays.shape[0]
    d.stream = stream_id
    P = params.numel()
    grad = torch.full((P,), float("nan"), device="cuda")
    loss = torch.full((1,), float("nan"), device="cuda")
    st = lib.vmap_object_grad_static(ctypes.byref(cfg), ctypes.byref(d), ctypes.c_void_p(params.data_ptr()),
                                     step, ctypes.c_void_p(grad.data_ptr()), ctypes.c_void_p(loss.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, native.STATUS_NAMES.get(st, st)
    torch.cuda.synchronize()
    return grad, loss


def test_static_entry_point_matches_context_path_twice():
    lib = native.load()
    sc = vh.mixed_scene(seed=31)
    rng = np.random.default_rng(5)
    cfg = native.VmapConfig()
    lib.vmap_default_config(ctypes.byref(cfg))
    B = np.ascontiguousarray(np.asarray(sc["B"], np.float32))
    cfg.B = B.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    cfg.seed = sc["seed"]
    for k in (1, 3, 0, 2):                    # hidden 32, 128, 16, 64
        o = sc["objects"][k]
        one = dict(objects=[o], B=sc["B"], seed=sc["seed"])
        vm = vh.library_context(one, max_rays=2048)
        params = torch.from_numpy(np.asarray(o["init"], np.float32)).cuda()
        for call in range(2):                 # two calls in a row, different rays
            n = [300, 1024][call]
            rays = torch.from_numpy(o["pool"][rng.integers(0, o["pool"].shape[0], n)]).cuda().contiguous()
            # the object sits at index 0 with stream id 0 in the one-object context
            g_static, l_static = _static_grad(lib, cfg, o, rays, params, 0, 0)
            vm.sample_rays_given(rays, [n])
            l_ctx = torch.empty(1, device="cuda")
            vm.forward(l_ctx)
            g_ctx = torch.zeros(vm.arena_size(), device="cuda")
            vm.backward(g_ctx)
            P = params.numel()
            assert abs(l_static.item() - l_ctx.item()) <= 1e-5 * abs(l_ctx.item())
            errs = vh.layer_errors(g_static.cpu().numpy(), g_ctx[:P].cpu().numpy().astype(np.float64), o["H"])
            assert max(errs) <= 1e-4, (k, call, errs)


def test_static_entry_point_rejects_oversized_batches():
    lib = native.load()
    sc = scenes.scene_small(seed=32, n_objects=1, rays=8)
    o = sc["objects"][0]
    cfg = native.VmapConfig()
    lib.vmap_default_config(ctypes.byref(cfg))
    B = np.ascontiguousarray(np.asarray(sc["B"], np.float32))
    cfg.B = B.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    rays = torch.from_numpy(np.repeat(o["pool"][:1], 1025, axis=0)).cuda().contiguous()
    d = native.VmapObjectDesc()
    d.hidden, d.n_surface, d.n_strat, d.scale = 32, 10, 12, float(o["scale"])
    d.rays, d.n_rays = rays.data_ptr(), 1025
    params = torch.zeros(6308, device="cuda")
    out = torch.zeros(6309, device="cuda")
    st = lib.vmap_object_grad_static(ctypes.byref(cfg), ctypes.byref(d), ctypes.c_void_p(params.data_ptr()), 0,
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(out.data_ptr() + 4 * 6308),
                                     None)
    assert native.STATUS_NAMES[st] == "VMAP_ERR_CAPACITY"
