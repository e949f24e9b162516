"""Whole-step pins of the oracle: objects are independent (N objects trained
together equal N separate trainings, bitwise), a non-finite object is frozen
without touching the others, and training lowers the loss."""
import numpy as np

from oracle import vmap_step as vs
from paper_2302_01838_b300 import scenes


def _states(scene, streams=None):
    out = []
    for k, o in enumerate(scene["objects"]):
        out.append(vs.ObjectState(H=o["H"], pool=o["pool"], center=o["center"], scale=o["scale"],
                                  n_surface=o["n_surface"], n_strat=o["n_strat"],
                                  stream=k if streams is None else streams[k], params=o["init"]))
    return out


def test_together_equals_separate():
    sc = scenes.scene_small(seed=21, n_objects=3, rays=40)
    cfg = vs.Config(seed=sc["seed"], B=sc["B"].astype(np.float64))
    together = _states(sc)
    L_tog = [vs.train_step(cfg, together, [40, 17, 33]) for _ in range(4)]
    for k in range(3):
        alone = _states(sc)[k:k + 1]
        alone[0].stream = k
        L_alone = [vs.train_step(cfg, alone, [[40, 17, 33][k]])[0] for _ in range(4)]
        assert [L[k] for L in L_tog] == L_alone
        assert np.array_equal(alone[0].params, together[k].params)
        assert np.array_equal(alone[0].v, together[k].v)


def test_nonfinite_object_frozen_others_unaffected():
    sc = scenes.scene_small(seed=22, n_objects=3, rays=30)
    cfg = vs.Config(seed=sc["seed"], B=sc["B"].astype(np.float64))
    ref = _states(sc)
    bad = _states(sc)
    bad[1].pool = bad[1].pool.copy()
    bad[1].pool[:, 7] = np.nan
    before = bad[1].params.copy()
    for _ in range(3):
        Lr = vs.train_step(cfg, ref, [30, 30, 30])
        Lb = vs.train_step(cfg, bad, [30, 30, 30])
    assert bad[1].faulted and not bad[1].active and bad[1].step == 0
    assert np.array_equal(bad[1].params, before)
    for k in (0, 2):
        assert Lr[k] == Lb[k] and np.array_equal(ref[k].params, bad[k].params)


def test_training_lowers_the_loss():
    sc = scenes.scene_small(seed=23, n_objects=2, rays=120)
    cfg = vs.Config(seed=sc["seed"], B=sc["B"].astype(np.float64), lr=5e-3)
    st = _states(sc)
    first = vs.train_step(cfg, st, [120, 120])
    for _ in range(150):
        last = vs.train_step(cfg, st, [120, 120])
    assert np.all(last < 0.5 * first)


def test_inactive_and_empty_objects_are_skipped():
    sc = scenes.scene_small(seed=24, n_objects=2, rays=10)
    cfg = vs.Config(seed=sc["seed"], B=sc["B"].astype(np.float64))
    st = _states(sc)
    st[0].active = False
    p0 = st[0].params.copy()
    L = vs.train_step(cfg, st, [10, 0])
    assert np.isnan(L[0]) and np.isnan(L[1])
    assert np.array_equal(st[0].params, p0) and st[1].step == 0
