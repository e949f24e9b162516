"""Camera-pose refinement against a trained object (the map held fixed):
the per-ray gradients of the object's loss with respect to ray origin and
direction (vmap_ray_gradients, the encoding backward) give the pose
gradient, which Adam follows. A camera at position p with rotation R maps
camera-frame directions d_c to d = R d_c, so dL/dp = sum_rays dL/do and,
for a rotation update exp([w]x) R, dL/dw = sum_rays d x dL/dd.

Library calls only (vmap_sample_rays_given, vmap_ray_gradients,
vmap_forward); FP32 contexts."""
import numpy as np
import torch


def rodrigues(w):
    """Rotation matrix exp([w]x)."""
    th = float(np.linalg.norm(w))
    if th < 1e-12:
        return np.eye(3)
    k = w / th
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * (K @ K)


def _records(p, R, dc, meas):
    d = dc @ R.T
    rec = np.zeros((dc.shape[0], 12), np.float32)
    rec[:, 0:3] = p
    rec[:, 3:6] = d
    rec[:, 6:11] = meas          # depth, rgb, mask
    return torch.from_numpy(rec).cuda(), d


def refine_pose(vm, obj, n_objects, dc, meas, p0, R0, iters=150, lr_t=2e-3, lr_r=4e-3):
    """Refine a camera pose (p0, R0) so the object's rendering of the camera's
    rays matches their measurements.
      dc:   camera-frame ray directions [n, 3] ((u + 1/2 - cx)/f, (v + 1/2 - cy)/f, 1)
      meas: [n, 5] measured depth, rgb and mask per ray
    Returns (p, R, losses)."""
    p, R = np.asarray(p0, np.float64).copy(), np.asarray(R0, np.float64).copy()
    n = dc.shape[0]
    R_req = [0] * n_objects
    R_req[obj] = n
    g = torch.empty(n, 6, device="cuda")
    loss = torch.empty(n_objects, device="cuda")
    m = np.zeros(6)
    v = np.zeros(6)
    losses = []
    for it in range(1, iters + 1):
        rec, d = _records(p, R, dc, meas)
        vm.sample_rays_given(rec, R_req)
        vm.forward(loss)
        losses.append(float(loss[obj]))
        vm.ray_gradients(g)
        gg = g.double().cpu().numpy()
        grad = np.concatenate([gg[:, :3].sum(0), np.cross(d, gg[:, 3:]).sum(0)])
        m = 0.9 * m + 0.1 * grad
        v = 0.999 * v + 0.001 * grad * grad
        step = (m / (1 - 0.9 ** it)) / (np.sqrt(v / (1 - 0.999 ** it)) + 1e-12)
        p = p - lr_t * step[:3]
        R = rodrigues(-lr_r * step[3:]) @ R
    return p, R, losses
