"""The C-ABI library loads on a machine without a GPU and exports every
function include/vmap.h declares (no compute call is made here)."""
import ctypes
import os
import re

from paper_2302_01838_b300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:vmap_status|void|const char\s*\*)\s*(vmap_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("vmap_init_objects", "vmap_add_object", "vmap_sample_rays", "vmap_train_step",
                     "vmap_query_occupancy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = native.load()
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in native.SIGNATURES, f"{name} has no binding signature"


def test_binding_struct_sizes_match_the_header_layout():
    # vmap_config: 2 ints, 2 long longs, 10 floats, 1 int (+pad), 1 ull, 1 pointer
    assert ctypes.sizeof(native.VmapConfig) == 4 * 2 + 8 * 2 + 4 * 10 + 8 + 8 + 8
    # vmap_object_desc: 3 ints, 4 floats (+pad), pointer, long long, uint (+pad)
    assert ctypes.sizeof(native.VmapObjectDesc) == 3 * 4 + 4 * 4 + 4 + 8 + 8 + 8


def test_default_config_without_a_gpu():
    lib = native.load()
    cfg = native.VmapConfig()
    lib.vmap_default_config(ctypes.byref(cfg))
    assert abs(cfg.d_sigma - 0.03) < 1e-9 and cfg.lambda_colour == 5.0 and abs(cfg.lr - 1e-3) < 1e-9
    assert cfg.precision == native.VMAP_FP32


def test_binding_reuses_the_ray_count_array_only_while_the_counts_are_unchanged():
    """The binding's host array of rays per object is rebuilt whenever the
    counts change, also when the caller mutates the same list in place."""
    import types
    from paper_2302_01838_b300.api import VMap
    holder = types.SimpleNamespace()
    counts = [3, 0, 7]
    a = VMap._counts(holder, counts)
    assert list(a) == [3, 0, 7]
    assert VMap._counts(holder, [3, 0, 7]) is a
    counts[1] = 5
    b = VMap._counts(holder, counts)
    assert list(b) == [3, 5, 7]
    assert list(VMap._counts(holder, (1, 2))) == [1, 2]
    import numpy as np
    assert list(VMap._counts(holder, np.array([4, 4, 4]))) == [4, 4, 4]
