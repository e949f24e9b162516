"""ctypes binding of libvmap.so (the C ABI declared in include/vmap.h).

Argument marshalling only: every step of the training path runs in the CUDA
library. Loading fails loudly if the library is missing; there is no CPU
fallback.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvmap.so")

VMAP_OK = 0
STATUS_NAMES = {0: "VMAP_OK", -1: "VMAP_ERR_ARG", -2: "VMAP_ERR_CAPACITY", -3: "VMAP_ERR_CUDA",
                -4: "VMAP_ERR_NAN", -5: "VMAP_ERR_TIMEOUT", -6: "VMAP_ERR_STATE"}
VMAP_FP32, VMAP_BF16 = 0, 1
REC_FLOATS = 12
N_FREQ = 45


class VmapConfig(ctypes.Structure):
    _fields_ = [
        ("max_objects", ctypes.c_int),
        ("max_rays_total", ctypes.c_int),
        ("max_pool_rays", ctypes.c_longlong),
        ("max_param_floats", ctypes.c_longlong),
        ("t_near", ctypes.c_float),
        ("depth_pad", ctypes.c_float),
        ("d_sigma", ctypes.c_float),
        ("t_far", ctypes.c_float),
        ("lambda_colour", ctypes.c_float),
        ("lambda_occ", ctypes.c_float),
        ("lr", ctypes.c_float),
        ("beta1", ctypes.c_float),
        ("beta2", ctypes.c_float),
        ("eps", ctypes.c_float),
        ("precision", ctypes.c_int),
        ("seed", ctypes.c_ulonglong),
        ("B", ctypes.POINTER(ctypes.c_float)),
    ]


class VmapObjectDesc(ctypes.Structure):
    _fields_ = [
        ("hidden", ctypes.c_int),
        ("n_surface", ctypes.c_int),
        ("n_strat", ctypes.c_int),
        ("center", ctypes.c_float * 3),
        ("scale", ctypes.c_float),
        ("rays", ctypes.c_void_p),
        ("n_rays", ctypes.c_longlong),
        ("stream", ctypes.c_uint),
    ]


_P = ctypes.c_void_p
_I = ctypes.c_int
_LL = ctypes.c_longlong
_IP = ctypes.POINTER(ctypes.c_int)
_LLP = ctypes.POINTER(ctypes.c_longlong)

# name -> (restype, argtypes)
SIGNATURES = {
    "vmap_default_config": (None, [ctypes.POINTER(VmapConfig)]),
    "vmap_init_objects": (_I, [ctypes.POINTER(_P), ctypes.POINTER(VmapConfig), _P]),
    "vmap_destroy": (_I, [_P]),
    "vmap_last_error": (ctypes.c_char_p, [_P]),
    "vmap_add_object": (_I, [_P, ctypes.POINTER(VmapObjectDesc), _P, _IP]),
    "vmap_sample_rays": (_I, [_P, _IP]),
    "vmap_sample_rays_given": (_I, [_P, _P, _IP]),
    "vmap_train_step_host": (_I, [_P, _P, _IP, _P]),
    "vmap_profile_enable": (_I, [_P, _I]),
    "vmap_profile_reset": (_I, [_P]),
    "vmap_profile_read": (_I, [_P, _I, ctypes.POINTER(ctypes.c_char_p), _LLP,
                                ctypes.POINTER(ctypes.c_double)]),
    "vmap_train_step": (_I, [_P, _P]),
    "vmap_step": (_I, [_P, _IP, _P]),
    "vmap_set_graph": (_I, [_P, _I]),
    "vmap_set_wait_limit": (_I, [_P, _LL]),
    "vmap_pose_step": (_I, [_P, _I, _P, _P, _I, _P, _P, ctypes.c_float, ctypes.c_float, _P, _P, _P]),
    "vmap_get_launch": (_I, [_P, _IP, _IP]),
    "vmap_set_launch": (_I, [_P, _IP, _IP]),
    "vmap_autotune": (_I, [_P, _IP, _I, ctypes.POINTER(ctypes.c_float)]),
    "vmap_forward": (_I, [_P, _P]),
    "vmap_backward": (_I, [_P, _P, _P, _P]),
    "vmap_query_occupancy": (_I, [_P, _I, _P, _LL, _P, _P]),
    "vmap_render_depth": (_I, [_P, _I, _P, _LL, ctypes.POINTER(ctypes.c_float), _I, _P]),
    "vmap_extract_mesh": (_I, [_P, _I, ctypes.POINTER(ctypes.c_float), _I, ctypes.c_float, _P, _LL,
                               ctypes.POINTER(ctypes.c_longlong)]),
    "vmap_ray_gradients": (_I, [_P, _P]),
    "vmap_hyper_set_precision": (_I, [_P, _I]),
    "vmap_render_scene": (_I, [_P, _P, _LL, ctypes.POINTER(ctypes.c_int), _I, ctypes.POINTER(ctypes.c_float), _I,
                               _P, _P, _P]),
    "vmap_get_object_state": (_I, [_P, _I, _P, _P, _P, _IP]),
    "vmap_set_object_state": (_I, [_P, _I, _P, _P, _P, _I]),
    "vmap_get_params": (_I, [_P, _P]),
    "vmap_set_params": (_I, [_P, _P]),
    "vmap_param_arena_size": (_I, [_P, _LLP]),
    "vmap_set_object_active": (_I, [_P, _I, _I]),
    "vmap_set_object_center": (_I, [_P, _I, ctypes.POINTER(ctypes.c_float)]),
    "vmap_object_info": (_I, [_P, _I, _IP, _IP, _LLP, _IP]),
    "vmap_num_objects": (_I, [_P, _IP]),
    "vmap_batch_info": (_I, [_P, _IP, _LLP]),
    "vmap_get_samples": (_I, [_P, _P, _P]),
    "vmap_sync_status": (_I, [_P, _IP, _IP, _I]),
    "vmap_hyper_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I, _I, ctypes.c_ulonglong, _P]),
    "vmap_hyper_destroy": (_I, [_P]),
    "vmap_hyper_last_error": (ctypes.c_char_p, [_P]),
    "vmap_hyper_param_count": (_I, [_P, _LLP, _IP]),
    "vmap_hyper_get_params": (_I, [_P, _P]),
    "vmap_hyper_set_params": (_I, [_P, _P]),
    "vmap_hyper_predict": (_I, [_P, _I, _P, _P]),
    "vmap_hyper_grad": (_I, [_P, _I, _P, _P, _P, _P]),
    "vmap_hyper_train_step": (_I, [_P, _I, _P, _P, ctypes.c_float, _P]),
    "vmap_warmstart": (_I, [_P, _I, _P, _P]),
    "vmap_object_grad_static": (_I, [ctypes.POINTER(VmapConfig), ctypes.POINTER(VmapObjectDesc), _P, _I,
                                     _P, _P, _P]),
}

_lib = None


def load(path=LIB_PATH):
    """Load libvmap.so and declare every exported signature (no GPU needed)."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libvmap.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == LIB_PATH:
        _lib = lib
    return lib


class VmapError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status
