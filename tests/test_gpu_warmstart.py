"""The learned warm start pays: a hypernetwork trained on MLPs that the
library itself converged predicts initial weights for unseen objects that
(a) start at a lower training loss than the seeded random initialisation and
(b) reach a held-out depth-L1 target in fewer steps.

Reduced sizes (1,536 training shapes x 1,000 steps, 48 held-out objects) so
the whole test takes well under a minute; the full-size experiment is
``python -m paper_2302_01838_b300.warmstart``."""
import pytest

from paper_2302_01838_b300 import scenes, warmstart as ws

pytestmark = pytest.mark.gpu


def test_warmstart_gain():
    X, T = ws.produce_dataset(1536, seed=7, steps=1000, chunk=768)
    assert X.shape == (1536, 256, 7) and T.shape == (1536, 6308)
    hyp = ws.train_hypernet(X, T, epochs=150, batch=128)
    held = scenes.scene_shapes(7 + 10 ** 6, 48, offmask=ws.OFFMASK)
    objs, B = held["objects"], held["B"]
    l_rand = ws.initial_loss(objs, B, 7)
    l_warm = ws.initial_loss(objs, B, 7, hyp)
    assert l_warm < 0.9 * l_rand, (l_warm, l_rand)
    cold = ws.time_to_target(objs, B, 7, "batched", target=0.05, max_steps=1500)
    warm = ws.time_to_target(objs, B, 7, "warm", hyper=hyp, target=0.05, max_steps=1500)
    assert warm["reached"], warm
    assert warm["steps"] < cold["steps"], (warm["steps"], cold["steps"])
