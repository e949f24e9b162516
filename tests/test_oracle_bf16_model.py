"""Pins of the BF16 rounding model (oracle/bf16_model.py): its rounding is
round-to-nearest-even at 8 significant bits (checked on hand-worked values,
against the error bound, and against an independent library conversion), and
with rounding switched off the model is exactly the FP64 oracle."""
import numpy as np
import torch

from oracle import bf16_model as bm
from oracle import vmap_step as vs
from paper_2302_01838_b300 import scenes


def test_round_bf16_hand_worked_values():
    u = 2.0 ** -7                       # BF16 spacing on [1, 2)
    cases = [(1.0, 1.0), (1 + u / 2, 1.0),                 # tie -> even mantissa (0)
             (1 + 3 * u / 2, 1 + 2 * u),                    # tie -> even mantissa (2)
             (1 + u / 2 + 2.0 ** -20, 1 + u),               # just above the tie
             (-2.5, -2.5), (np.float32(np.pi), 3.140625), (0.0, 0.0),
             (65280.0, 65280.0), (1e-30, np.float32(1e-30).astype(np.float64))]
    got = bm.round_bf16(np.array([c[0] for c in cases]))
    for (x, want), g in zip(cases[:-1], got[:-1]):
        assert g == want, (x, g, want)
    # 1e-30 is normal in FP32 and BF16: within half a BF16 ulp of the FP32 value
    assert abs(got[-1] - cases[-1][1]) <= 2.0 ** -9 * abs(cases[-1][1])
    assert np.isnan(bm.round_bf16(np.nan)) and bm.round_bf16(np.inf) == np.inf


def test_round_bf16_error_bound_and_library_conversion():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-20, 20, 20000),
                        (1 + (2 * rng.integers(0, 128, 2000) + 1) * 2.0 ** -8) * 2.0 ** rng.integers(-5, 5, 2000)])
    r = bm.round_bf16(x)
    f32 = x.astype(np.float32).astype(np.float64)
    assert np.all(np.abs(r - f32) <= 2.0 ** -8 * np.abs(f32))        # half an ulp at 8 bits
    assert np.array_equal(bm.round_bf16(r), r)                         # idempotent
    lib = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(r, lib)


def _object(seed=3, H=32):
    rng = np.random.default_rng(seed)
    o = scenes.make_object(rng, (1, 2), 0.1, 0.3, 0.2, H=H, per_view=128)
    cfg = vs.Config(seed=seed, B=scenes.make_B(seed))
    pk, t = vs.sample_object(cfg, o["pool"], 40, 10, 12, 0, 0)
    return cfg, scenes.init_weights(rng, H).astype(np.float64), o["pool"][pk].astype(np.float64), t, o


def test_model_without_rounding_is_the_fp64_oracle():
    for H in (16, 128):
        cfg, p, rays, t, o = _object(H=H)
        a = bm.object_forward_backward(cfg, p, H, rays, t, np.asarray(o["center"], np.float64),
                                       float(o["scale"]), rounding=False)
        b = vs.object_forward_backward(cfg, p, H, rays, t, np.asarray(o["center"], np.float64), float(o["scale"]))
        assert a["loss"] == b["loss"]
        assert np.array_equal(a["grad"], b["grad"])


def test_model_with_rounding_stays_near_the_fp64_oracle():
    cfg, p, rays, t, o = _object(H=32)
    a = bm.object_forward_backward(cfg, p, 32, rays, t, np.asarray(o["center"], np.float64), float(o["scale"]))
    b = vs.object_forward_backward(cfg, p, 32, rays, t, np.asarray(o["center"], np.float64), float(o["scale"]))
    assert 0 < abs(a["loss"] - b["loss"]) <= 1e-2 * b["loss"]
    err = np.linalg.norm(a["grad"] - b["grad"]) / np.linalg.norm(b["grad"])
    assert 0 < err <= 5e-2
