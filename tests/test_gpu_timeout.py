"""Failure detection of the tensor-core kernels without a GPU fault.

Every wait of the BF16 kernels (hidden 16/32/64 tile kernel, the width-128
forward and weight-gradient kernels) polls its mbarrier a bounded number of
times. With the limit set to 0 every such wait gives up at once, although the
MMAs and copies it waits for complete normally: the CTA drains the work it
has issued, frees its tensor memory and exits, and the context's error flag is
set. Nothing here makes an MMA fail, hang or fault.

Checked: the step is reported as VMAP_ERR_TIMEOUT by vmap_sync_status (once),
its losses are NaN, no object's weights, moments or step count change, and
once the default limit is back the context trains on exactly (bitwise) like a
context that never timed out, with losses equal to the oracle's BF16 rounding
model."""
import numpy as np
import pytest
import torch

from oracle import bf16_model as bm
from oracle import vmap_step as vs
from paper_2302_01838_b300.native import VMAP_BF16, VmapError

import vmap_harness as vh

pytestmark = pytest.mark.gpu

DEFAULT_POLLS = 1 << 26


def _states(vm, K):
    return [tuple(x.cpu().numpy().copy() if torch.is_tensor(x) else x for x in vm.get_object_state(k))
            for k in range(K)]


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("graph", [False, True])
def test_wait_limit_zero_reports_timeout_and_the_context_trains_on(graph):
    sc = vh.mixed_scene(seed=41)
    K = len(sc["objects"])
    R = [o["rays"] for o in sc["objects"]]
    vm = vh.library_context(sc, precision=VMAP_BF16)
    ref = vh.library_context(sc, precision=VMAP_BF16)
    for c in (vm, ref):
        c.set_graph(graph)
    loss, lref = torch.empty(K, device="cuda"), torch.empty(K, device="cuda")
    for c, l in ((vm, loss), (ref, lref)):
        c.sample_rays(R)
        c.train_step(l)
    before = _states(vm, K)
    assert all(_same(a, b) for a, b in zip(before, _states(ref, K)))

    # every tensor-core wait gives up at once: the step is void
    vm.set_wait_limit(0)
    vm.sample_rays(R)
    vm.train_step(loss)
    with pytest.raises(VmapError) as e:
        vm.sync_status()
    assert e.value.status == -5                       # VMAP_ERR_TIMEOUT
    assert torch.isnan(loss).all()
    after = _states(vm, K)
    assert all(_same(a, b) for a, b in zip(before, after)), "a void step changed an object"
    assert vm.sync_status() == []                     # reported once

    # default limit: trains on exactly as a context that never timed out
    vm.set_wait_limit(DEFAULT_POLLS)
    cfg = vh.oracle_config(sc)
    for step in range(3):
        pre = _states(vm, K)
        for c, l in ((vm, loss), (ref, lref)):
            c.sample_rays(R)
            c.train_step(l)
        assert torch.equal(loss, lref), step
        assert all(_same(a, b) for a, b in zip(_states(vm, K), _states(ref, K))), step
        # the step's losses against the BF16 rounding model of the oracle (objects of every width)
        for k in (0, 1, 2, 3):
            o = sc["objects"][k]
            pk, tk = vs.sample_object(cfg, o["pool"], R[k], o["n_surface"], o["n_strat"], k, pre[k][3])
            m = bm.object_forward_backward(cfg, np.asarray(pre[k][0], np.float64), o["H"],
                                           o["pool"][pk].astype(np.float64), tk,
                                           np.asarray(o["center"], np.float64), float(o["scale"]))
            assert abs(float(loss[k]) - m["loss"]) <= 1e-5 * m["loss"], (step, k, float(loss[k]), m["loss"])
    assert vm.sync_status() == []
    vm.close()
    ref.close()


def test_wait_limit_rejects_negative():
    sc = vh.mixed_scene(seed=42)
    vm = vh.library_context(sc, precision=VMAP_BF16)
    with pytest.raises(VmapError) as e:
        vm.set_wait_limit(-1)
    assert e.value.status == -1
    vm.close()
