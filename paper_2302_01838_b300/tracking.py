"""Camera-pose refinement against a trained object (the map held fixed):
the per-ray gradients of the object's loss with respect to ray origin and
direction (the encoding backward) give the pose gradient, which Adam
follows. A camera at position p with rotation R maps camera-frame directions
d_c to d = R d_c, so dL/dp = sum_rays dL/do and, for a rotation update
exp([w]x) R, dL/dw = sum_rays d x dL/dd.

Each iteration is one library call (vmap_pose_step: rays from the pose,
samples, loss and per-ray gradients in one pass, pose gradient and Adam on
the device); the host reads the pose and the loss curve once at the end.
FP32 contexts."""
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
    Returns (p, R, losses): the loss of each iteration is taken before its update."""
    n = dc.shape[0]
    dcd = torch.from_numpy(np.ascontiguousarray(dc, np.float32)).cuda()
    measd = torch.from_numpy(np.ascontiguousarray(meas, np.float32)).cuda()
    pose = torch.from_numpy(np.concatenate([np.asarray(p0, np.float64).ravel(),
                                            np.asarray(R0, np.float64).ravel()]).astype(np.float32)).cuda()
    adam = torch.zeros(13, device="cuda")
    rays_work = torch.empty(n, 12, device="cuda")
    grad_work = torch.empty(n, 6, device="cuda")
    losses = torch.empty(iters, n_objects, device="cuda")
    for it in range(iters):
        vm.pose_step(obj, dcd, measd, pose, adam, lr_t, lr_r, rays_work, grad_work, losses[it])
    pose = pose.double().cpu().numpy()
    return pose[:3], pose[3:].reshape(3, 3), losses[:, obj].double().cpu().numpy().tolist()
