"""Thin Python wrapper over the C ABI (argument marshalling only).

torch is used for device memory and streams: tensors are passed to the
library as raw pointers, the context runs on torch's current CUDA stream.
"""
import ctypes

import numpy as np
import torch

from . import native
from .native import VmapConfig, VmapError, VmapObjectDesc


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


class VMap:
    """One training context: a stack of per-object MLPs trained together."""

    def __init__(self, max_objects, max_rays_total, max_pool_rays, B, seed=0,
                 max_param_floats=0, stream=None, **hyper):
        self.lib = native.load()
        if not torch.cuda.is_available():
            raise RuntimeError("the vMAP library needs a CUDA device")
        cfg = VmapConfig()
        self.lib.vmap_default_config(ctypes.byref(cfg))
        cfg.max_objects = int(max_objects)
        cfg.max_rays_total = int(max_rays_total)
        cfg.max_pool_rays = int(max_pool_rays)
        cfg.max_param_floats = int(max_param_floats)
        cfg.seed = int(seed)
        for k, v in hyper.items():
            if not hasattr(cfg, k):
                raise TypeError(f"unknown hyper-parameter {k}")
            setattr(cfg, k, v)
        self._B = np.ascontiguousarray(np.asarray(B, np.float32).reshape(native.N_FREQ, 3))
        cfg.B = self._B.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = self.lib.vmap_init_objects(ctypes.byref(h), ctypes.byref(cfg),
                                        ctypes.c_void_p(self.stream.cuda_stream))
        if st != 0:
            raise VmapError(st, "vmap_init_objects failed")
        self.h = h
        self.cfg = cfg

    # ------------------------------------------------------------------
    def _counts(self, rays_per_object):
        """Host int array of the rays per object (the last one is reused while unchanged)."""
        key = tuple(rays_per_object)
        if key != getattr(self, "_counts_key", None):
            self._counts_arr = (ctypes.c_int * len(key))(*[int(r) for r in key])
            self._counts_key = key
        return self._counts_arr

    def _check(self, st):
        if st != 0:
            raise VmapError(st, self.lib.vmap_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.vmap_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------
    def add_object(self, rays, hidden=32, center=(0, 0, 0), scale=1.0, n_surface=10, n_strat=12,
                   init_params=None, stream_id=None):
        rays = torch.as_tensor(rays, dtype=torch.float32).reshape(-1, native.REC_FLOATS)
        rays = rays.to("cuda").contiguous()
        d = VmapObjectDesc()
        d.hidden = int(hidden)
        d.n_surface = int(n_surface)
        d.n_strat = int(n_strat)
        for a in range(3):
            d.center[a] = float(center[a])
        d.scale = float(scale)
        d.rays = _ptr(rays).value
        d.n_rays = rays.shape[0]
        d.stream = self.num_objects() if stream_id is None else int(stream_id)
        ip = None
        if init_params is not None:
            init_params = torch.as_tensor(init_params, dtype=torch.float32).to("cuda").contiguous()
            ip = _ptr(init_params)
        oid = ctypes.c_int()
        self._check(self.lib.vmap_add_object(self.h, ctypes.byref(d), ip, ctypes.byref(oid)))
        return oid.value

    def num_objects(self):
        n = ctypes.c_int()
        self._check(self.lib.vmap_num_objects(self.h, ctypes.byref(n)))
        return n.value

    def sample_rays(self, rays_per_object):
        arr = self._counts(rays_per_object)
        self._check(self.lib.vmap_sample_rays(self.h, arr))

    def sample_rays_given(self, rays, rays_per_object):
        arr = self._counts(rays_per_object)
        self._check(self.lib.vmap_sample_rays_given(self.h, _ptr(rays), arr))

    def train_step_host(self, rays, rays_per_object, loss_out):
        """rays, loss_out: CPU tensors (pinned for an asynchronous copy)."""
        if rays.is_cuda or loss_out.is_cuda:
            raise ValueError("train_step_host takes host tensors")
        arr = self._counts(rays_per_object)
        self._check(self.lib.vmap_train_step_host(self.h, ctypes.c_void_p(rays.data_ptr()), arr,
                                                  ctypes.c_void_p(loss_out.data_ptr())))
        return loss_out

    def profile_enable(self, on=True):
        self._check(self.lib.vmap_profile_enable(self.h, int(bool(on))))

    def profile_reset(self):
        self._check(self.lib.vmap_profile_reset(self.h))

    def profile(self):
        """{kernel name: (launches, total device ms)} since the last reset."""
        out = {}
        slot = 0
        while True:
            name = ctypes.c_char_p()
            n = ctypes.c_longlong()
            ms = ctypes.c_double()
            st = self.lib.vmap_profile_read(self.h, slot, ctypes.byref(name), ctypes.byref(n),
                                            ctypes.byref(ms))
            if st != 0:
                break
            if n.value:
                out[name.value.decode()] = (n.value, ms.value)
            slot += 1
        return out

    def warmstart(self, obj, hyper, X):
        """Install hypernetwork-predicted weights for object obj (X: [n_points, 7] CUDA)."""
        self._check(self.lib.vmap_warmstart(self.h, int(obj), hyper.h, _ptr(X.contiguous())))

    def set_graph(self, on=True):
        self._check(self.lib.vmap_set_graph(self.h, int(bool(on))))

    def set_wait_limit(self, polls):
        """Polls before a tensor-core wait gives up (default 2**26; 0: at once)."""
        self._check(self.lib.vmap_set_wait_limit(self.h, int(polls)))

    def get_launch(self):
        rt, gm = (ctypes.c_int * 4)(), (ctypes.c_int * 4)()
        self._check(self.lib.vmap_get_launch(self.h, rt, gm))
        return list(rt), list(gm)

    def set_launch(self, rays_per_tile=None, grid_mult=None):
        rt = (ctypes.c_int * 4)(*rays_per_tile) if rays_per_tile is not None else None
        gm = (ctypes.c_int * 4)(*grid_mult) if grid_mult is not None else None
        self._check(self.lib.vmap_set_launch(self.h, rt, gm))

    def autotune(self, rays_per_object, reps=3):
        arr = self._counts(rays_per_object)
        best = (ctypes.c_float * 4)()
        self._check(self.lib.vmap_autotune(self.h, arr, int(reps), best))
        return list(best)

    def train_step(self, out_loss=None):
        self._check(self.lib.vmap_train_step(self.h, _ptr(out_loss)))
        return out_loss

    def step(self, rays_per_object, out_loss=None):
        """sample_rays(rays_per_object) then train_step(out_loss), as one launch sequence."""
        arr = self._counts(rays_per_object)
        self._check(self.lib.vmap_step(self.h, arr, _ptr(out_loss)))
        return out_loss

    def forward(self, out_loss):
        self._check(self.lib.vmap_forward(self.h, _ptr(out_loss)))
        return out_loss

    def backward(self, grad_params, grad_loss=None, grad_center=None):
        self._check(self.lib.vmap_backward(self.h, _ptr(grad_loss), _ptr(grad_params),
                                           _ptr(grad_center)))

    def query_occupancy(self, obj, pts, occ, rgb=None):
        self._check(self.lib.vmap_query_occupancy(self.h, int(obj), _ptr(pts), pts.shape[0],
                                                  _ptr(occ), _ptr(rgb)))

    def pose_step(self, obj, dc, meas, pose, adam, lr_t, lr_r, rays_work, grad_work, loss):
        """One device iteration of camera-pose refinement (vmap_pose_step); every
        argument tensor is CUDA float32: dc [n, 3], meas [n, 5], pose [12], adam [13],
        rays_work [n, 12], grad_work [n, 6], loss [n_objects]."""
        self._check(self.lib.vmap_pose_step(self.h, int(obj), _ptr(dc), _ptr(meas), int(dc.shape[0]), _ptr(pose),
                                            _ptr(adam), float(lr_t), float(lr_r), _ptr(rays_work), _ptr(grad_work),
                                            _ptr(loss)))

    def ray_gradients(self, out):
        """(dL/do, dL/dd) of every ray of the current batch into out [n_rays, 6] (CUDA)."""
        self._check(self.lib.vmap_ray_gradients(self.h, _ptr(out)))

    def extract_mesh(self, obj, box_half, res, level=0.5):
        """Triangles [n, 3, 3] (CUDA, world space) of the object's occupancy level set."""
        hb = np.ascontiguousarray(np.asarray(box_half, np.float32).reshape(3))
        hp = hb.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        n = ctypes.c_longlong()
        self._check(self.lib.vmap_extract_mesh(self.h, int(obj), hp, int(res), float(level), None, 0, ctypes.byref(n)))
        tris = torch.empty(max(n.value, 1), 3, 3, device="cuda")
        self._check(self.lib.vmap_extract_mesh(self.h, int(obj), hp, int(res), float(level), _ptr(tris), n.value,
                                               ctypes.byref(n)))
        return tris[:n.value]

    def render_scene(self, rays, objs, box_half, n_samples, depth, rgb=None, occ=None):
        """Occlusion-aware render of the listed objects (vmap_render_scene)."""
        objs = list(objs)
        oa = (ctypes.c_int * len(objs))(*objs)
        hb = np.ascontiguousarray(np.asarray(box_half, np.float32).reshape(len(objs), 3))
        self._check(self.lib.vmap_render_scene(self.h, _ptr(rays), rays.shape[0], oa, len(objs),
                                               hb.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), int(n_samples),
                                               _ptr(depth), _ptr(rgb), _ptr(occ)))

    def render_depth(self, obj, rays, box_half, n_samples, depth):
        hb = (ctypes.c_float * 3)(*[float(x) for x in box_half])
        self._check(self.lib.vmap_render_depth(self.h, int(obj), _ptr(rays), rays.shape[0], hb,
                                               int(n_samples), _ptr(depth)))

    def object_info(self, obj):
        H, P, S = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        off = ctypes.c_longlong()
        self._check(self.lib.vmap_object_info(self.h, int(obj), ctypes.byref(H), ctypes.byref(P),
                                              ctypes.byref(off), ctypes.byref(S)))
        return dict(hidden=H.value, param_count=P.value, param_offset=off.value,
                    samples_per_ray=S.value)

    def get_object_state(self, obj):
        P = self.object_info(obj)["param_count"]
        p = torch.empty(P, device="cuda")
        m = torch.empty(P, device="cuda")
        v = torch.empty(P, device="cuda")
        st = ctypes.c_int()
        self._check(self.lib.vmap_get_object_state(self.h, int(obj), _ptr(p), _ptr(m), _ptr(v),
                                                   ctypes.byref(st)))
        return p, m, v, st.value

    def set_object_state(self, obj, params=None, m=None, v=None, step=0):
        self._check(self.lib.vmap_set_object_state(self.h, int(obj), _ptr(params), _ptr(m),
                                                   _ptr(v), int(step)))

    def arena_size(self):
        n = ctypes.c_longlong()
        self._check(self.lib.vmap_param_arena_size(self.h, ctypes.byref(n)))
        return n.value

    def get_params(self):
        out = torch.empty(self.arena_size(), device="cuda")
        self._check(self.lib.vmap_get_params(self.h, _ptr(out)))
        return out

    def set_params(self, arena):
        self._check(self.lib.vmap_set_params(self.h, _ptr(arena)))

    def set_object_active(self, obj, active):
        self._check(self.lib.vmap_set_object_active(self.h, int(obj), int(bool(active))))

    def set_object_center(self, obj, center):
        c = (ctypes.c_float * 3)(*[float(x) for x in center])
        self._check(self.lib.vmap_set_object_center(self.h, int(obj), c))

    def batch_info(self):
        r, s = ctypes.c_int(), ctypes.c_longlong()
        self._check(self.lib.vmap_batch_info(self.h, ctypes.byref(r), ctypes.byref(s)))
        return r.value, s.value

    def get_samples(self):
        r, s = self.batch_info()
        pick = torch.empty(r, dtype=torch.int32, device="cuda")
        t = torch.empty(s, dtype=torch.float32, device="cuda")
        self._check(self.lib.vmap_get_samples(self.h, _ptr(pick), _ptr(t)))
        return pick, t

    def sync_status(self, max_ids=1024):
        n = ctypes.c_int()
        ids = (ctypes.c_int * max_ids)()
        st = self.lib.vmap_sync_status(self.h, ctypes.byref(n), ids, max_ids)
        if st not in (0, -4):
            self._check(st)
        return [ids[i] for i in range(min(n.value, max_ids))]


class VMapLoss(torch.autograd.Function):
    """Per-object losses of the current batch as a differentiable function of the
    whole parameter arena and of the object centres; forward and backward run
    in the library (vmap_forward / vmap_backward)."""

    @staticmethod
    def forward(ctx, vm, params, centers):
        vm.set_params(params.detach().contiguous())
        for k in range(vm.num_objects()):
            vm.set_object_center(k, centers[k].tolist())
        loss = torch.empty(vm.num_objects(), device="cuda")
        vm.forward(loss)
        ctx.vm = vm
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        vm = ctx.vm
        gp = torch.zeros(vm.arena_size(), device="cuda")
        gc = torch.zeros(vm.num_objects(), 3, device="cuda")
        vm.backward(gp, grad_loss=grad_loss.contiguous(), grad_center=gc)
        return None, gp, gc


class HyperNet:
    """Warm-start set-encoder hypernetwork (C ABI vmap_hyper_*)."""

    def __init__(self, n_points=256, width=128, rank=16, hidden=32, max_batch=256, seed=0, stream=None):
        self.lib = native.load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = self.lib.vmap_hyper_create(ctypes.byref(h), n_points, width, rank, hidden, max_batch, seed,
                                        ctypes.c_void_p(self.stream.cuda_stream))
        if st != 0:
            raise VmapError(st, "vmap_hyper_create failed")
        self.h = h
        n, P = ctypes.c_longlong(), ctypes.c_int()
        self.lib.vmap_hyper_param_count(h, ctypes.byref(n), ctypes.byref(P))
        self.n_params, self.P = n.value, P.value
        self.n_points = n_points

    def _check(self, st):
        if st != 0:
            raise VmapError(st, self.lib.vmap_hyper_last_error(self.h).decode())

    def set_precision(self, precision):
        """native.VMAP_FP32 or native.VMAP_BF16 (tensor-core GEMMs of the 128-wide layers)."""
        self._check(self.lib.vmap_hyper_set_precision(self.h, int(precision)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.vmap_hyper_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        out = torch.empty(self.n_params, device="cuda")
        self._check(self.lib.vmap_hyper_get_params(self.h, _ptr(out)))
        return out

    def set_params(self, flat):
        self._check(self.lib.vmap_hyper_set_params(self.h, _ptr(flat.contiguous())))

    def predict(self, X):
        out = torch.empty(X.shape[0], self.P, device="cuda")
        self._check(self.lib.vmap_hyper_predict(self.h, X.shape[0], _ptr(X.contiguous()), _ptr(out)))
        return out

    def grad(self, X, T):
        g = torch.empty(self.n_params, device="cuda")
        loss = torch.empty(1, device="cuda")
        self._check(self.lib.vmap_hyper_grad(self.h, X.shape[0], _ptr(X.contiguous()), _ptr(T.contiguous()),
                                             _ptr(g), _ptr(loss)))
        return g, loss

    def train_step(self, X, T, lr, loss=None):
        self._check(self.lib.vmap_hyper_train_step(self.h, X.shape[0], _ptr(X.contiguous()), _ptr(T.contiguous()),
                                                   ctypes.c_float(lr), _ptr(loss)))
