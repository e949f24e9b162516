"""Camera-pose refinement through the encoding backward: per-ray origin and
direction gradients against the oracle, and a perturbed camera pulled back
to its true pose by a trained object."""
import numpy as np
import pytest
import torch

from oracle import vmap_step as vs
from paper_2302_01838_b300 import scenes, tracking

import vmap_harness as vh

pytestmark = pytest.mark.gpu


def test_ray_gradients_match_oracle():
    sc = vh.mixed_scene(seed=81)
    sc["objects"] = [o for o in sc["objects"] if o["rays"] > 1]
    cfg = vh.oracle_config(sc)
    R = [o["rays"] for o in sc["objects"]]
    vm = vh.library_context(sc)
    vm.sample_rays(R)
    g = torch.empty(sum(R), 6, device="cuda")
    vm.ray_gradients(g)
    g = g.cpu().numpy().astype(np.float64)
    r0 = 0
    for k, o in enumerate(sc["objects"]):
        pk, tk = vs.sample_object(cfg, o["pool"], R[k], o["n_surface"], o["n_strat"], k, 0)
        res = vs.object_forward_backward(cfg, np.asarray(o["init"], np.float64), o["H"], o["pool"][pk].astype(np.float64),
                                         tk, np.asarray(o["center"], np.float64), float(o["scale"]), want_center_grad=True)
        for key, sl in (("dray_o", slice(0, 3)), ("dray_d", slice(3, 6))):
            assert vh.rel_l2(g[r0:r0 + R[k], sl], res[key]) <= 1e-4, (k, key)
        r0 += R[k]


def _trained_view(seed=83):
    rng = np.random.default_rng(seed)
    # an asymmetric union of primitives with distinct colours: a single sphere would
    # leave orbiting the camera about it unobservable
    o = scenes.make_object(rng, (3, 3), 0.1, 0.25, 0.25, H=32, per_view=1024, offmask=0.5)
    o["init"] = scenes.init_weights(rng, 32)
    o["n_surface"], o["n_strat"], o["rays"] = 10, 12, 512
    sc = dict(objects=[o], B=scenes.make_B(seed + 1), seed=seed)
    vm = vh.library_context(sc, lambda_occ=1.0, max_rays=4096)
    for _ in range(3000):
        vm.sample_rays([512])
        vm.train_step()
    # a new view of the object: measured depth and colour from the true pose
    center = np.asarray(o["center"], np.float64)
    eye, Rwc = scenes.random_view(rng, center, 2.0)
    u, v = np.meshgrid(np.arange(0, scenes.W_IMG, 4), np.arange(0, scenes.H_IMG, 4))
    u, v = u.ravel().astype(np.float64), v.ravel().astype(np.float64)
    dc = np.stack([(u + 0.5 - scenes.CX) / scenes.FOCAL, (v + 0.5 - scenes.CY) / scenes.FOCAL, np.ones_like(u)], 1)
    orig, d = scenes.camera_rays(Rwc, eye, u, v)
    t_hit, rgb = scenes.cast(o["prims"], center, orig, d)
    sel = np.nonzero(np.isfinite(t_hit))[0][:600]
    meas = np.zeros((sel.size, 5))
    meas[:, 0], meas[:, 1:4], meas[:, 4] = t_hit[sel], rgb[sel], 1.0
    return vm, rng, eye, Rwc, dc[sel], meas


def test_pose_gradient_and_refinement():
    """The pose gradient assembled from the per-ray gradients equals central
    differences of the loss; refinement from a perturbed camera (2 cm, 1
    degree) reaches a pose the trained map explains at least as well as the
    true pose (the map's own centimetre-level errors bound the pose accuracy)."""
    vm, rng, eye, Rwc, dc, meas = _trained_view()
    loss_at = lambda p, R: tracking.refine_pose(vm, 0, 1, dc, meas, p, R, iters=1)[2][0]
    dp = rng.normal(size=3)
    dp *= 0.02 / np.linalg.norm(dp)
    ax = rng.normal(size=3)
    ax *= np.deg2rad(1.0) / np.linalg.norm(ax)
    p0, R0 = eye + dp, tracking.rodrigues(ax) @ Rwc
    # pose gradient against central differences at the perturbed pose
    rec, d = tracking._records(p0, R0, dc, meas)
    vm.sample_rays_given(rec, [dc.shape[0]])
    g = torch.empty(dc.shape[0], 6, device="cuda")
    vm.ray_gradients(g)
    gg = g.double().cpu().numpy()
    gp, gw = gg[:, :3].sum(0), np.cross(d, gg[:, 3:]).sum(0)
    h = 1e-4
    fdp = np.array([(loss_at(p0 + h * e, R0) - loss_at(p0 - h * e, R0)) / (2 * h) for e in np.eye(3)])
    fdw = np.array([(loss_at(p0, tracking.rodrigues(h * e) @ R0) - loss_at(p0, tracking.rodrigues(-h * e) @ R0)) / (2 * h)
                    for e in np.eye(3)])
    assert np.linalg.norm(gp - fdp) <= 5e-2 * np.linalg.norm(fdp), (gp, fdp)
    assert np.linalg.norm(gw - fdw) <= 5e-2 * np.linalg.norm(fdw), (gw, fdw)
    # refinement
    p, Rf, losses = tracking.refine_pose(vm, 0, 1, dc, meas, p0, R0, iters=300, lr_t=5e-4, lr_r=1e-3)
    true_loss = loss_at(eye, Rwc)
    rot_err = lambda Ra: np.degrees(np.arccos(np.clip((np.trace(Ra.T @ Rwc) - 1) / 2, -1, 1)))
    print(f"pose: translation {np.linalg.norm(p0 - eye) * 100:.2f} -> {np.linalg.norm(p - eye) * 100:.2f} cm, "
          f"rotation {rot_err(R0):.2f} -> {rot_err(Rf):.2f} deg, loss {losses[0]:.4f} -> {losses[-1]:.4f} "
          f"(true pose {true_loss:.4f})")
    assert losses[-1] <= true_loss and losses[-1] < 0.8 * losses[0]
    assert np.linalg.norm(p - eye) < 0.03 and rot_err(Rf) < 1.0


def test_device_pose_step_matches_its_definition():
    """vmap_pose_step against the same iteration spelled out from library
    outputs: rays from the pose, the per-ray gradients of the same batch
    (vmap_ray_gradients), dL/dp = sum dL/do, dL/dw = sum d x dL/dd, one Adam
    step (float64 here), R <- exp([w]x) R; and the loss it reports equals
    vmap_forward on the same batch."""
    rng = np.random.default_rng(91)
    o = scenes.make_object(rng, (2, 2), 0.1, 0.25, 0.25, H=32, per_view=256)
    o["init"] = scenes.init_weights(rng, 32)
    o["n_surface"], o["n_strat"], o["rays"] = 10, 12, 64
    sc = dict(objects=[o], B=scenes.make_B(92), seed=91)
    vm = vh.library_context(sc, max_rays=1024)
    center = np.asarray(o["center"], np.float64)
    eye, Rwc = scenes.random_view(rng, center, 2.0)
    u, v = np.meshgrid(np.arange(0, scenes.W_IMG, 8), np.arange(0, scenes.H_IMG, 8))
    u, v = u.ravel().astype(np.float64), v.ravel().astype(np.float64)
    dc = np.stack([(u + 0.5 - scenes.CX) / scenes.FOCAL, (v + 0.5 - scenes.CY) / scenes.FOCAL, np.ones_like(u)], 1)
    orig, d = scenes.camera_rays(Rwc, eye, u, v)
    t_hit, rgb = scenes.cast(o["prims"], center, orig, d)
    sel = np.nonzero(np.isfinite(t_hit))[0][:300]
    meas = np.zeros((sel.size, 5))
    meas[:, 0], meas[:, 1:4], meas[:, 4] = t_hit[sel], rgb[sel], 1.0
    dc = dc[sel]
    n = sel.size
    p0 = eye + np.array([0.01, -0.02, 0.015])
    R0 = tracking.rodrigues(np.array([0.01, 0.02, -0.015])) @ Rwc
    dcd = torch.from_numpy(dc.astype(np.float32)).cuda()
    measd = torch.from_numpy(meas.astype(np.float32)).cuda()
    pose = torch.from_numpy(np.concatenate([p0, R0.ravel()]).astype(np.float32)).cuda()
    pose_before = pose.double().cpu().numpy()
    adam = torch.zeros(13, device="cuda")
    rays = torch.empty(n, 12, device="cuda")
    gw = torch.empty(n, 6, device="cuda")
    loss = torch.empty(1, device="cuda")
    lr_t, lr_r = 2e-3, 4e-3
    vm.pose_step(0, dcd, measd, pose, adam, lr_t, lr_r, rays, gw, loss)
    # the same batch (same rays, same draws: the step count is unchanged)
    g = torch.empty(n, 6, device="cuda")
    vm.ray_gradients(g)
    lf = torch.empty(1, device="cuda")
    vm.forward(lf)
    assert float(loss[0]) == float(lf[0])
    g = g.double().cpu().numpy()
    rec = rays.double().cpu().numpy()
    assert np.allclose(rec[:, 0:3], pose_before[:3]) and np.allclose(rec[:, 6:11], meas.astype(np.float32))
    assert np.allclose(rec[:, 3:6], dc.astype(np.float32) @ pose_before[3:].reshape(3, 3).T, atol=1e-6)
    grad = np.concatenate([g[:, :3].sum(0), np.cross(rec[:, 3:6], g[:, 3:]).sum(0)])
    a = adam.double().cpu().numpy()
    # the pose gradient (FP32 sums on the device, FP64 here) through Adam's first moments
    assert np.linalg.norm(a[:6] - 0.1 * grad) <= 1e-4 * np.linalg.norm(0.1 * grad), (a[:6], 0.1 * grad)
    assert np.linalg.norm(a[6:12] - 0.001 * grad * grad) <= 1e-4 * np.linalg.norm(0.001 * grad * grad)
    assert a[12] == 1.0
    # the update from the device's moments (the first Adam step is about lr * sign(g) per
    # component, so a component near zero must not decide the comparison)
    step = (a[:6] / 0.1) / (np.sqrt(a[6:12] / 0.001) + 1e-12)
    p_exp = pose_before[:3] - lr_t * step[:3]
    R_exp = tracking.rodrigues(-lr_r * step[3:]) @ pose_before[3:].reshape(3, 3)
    got = pose.double().cpu().numpy()
    assert np.allclose(got[:3], p_exp, atol=1e-6), (got[:3], p_exp)
    assert np.allclose(got[3:].reshape(3, 3), R_exp, atol=1e-6), (got[3:], R_exp)
