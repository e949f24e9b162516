"""Mesh extraction on the GPU: the same triangles, in the same order, as the
oracle's marching tetrahedra on the oracle's occupancy lattice; and the mesh
of a trained object lies on the ground-truth surface (accuracy and
completion against the shape's exact distance field)."""
import numpy as np
import pytest
import torch

from oracle import mesh as om
from oracle import vmap_step as vs
from paper_2302_01838_b300 import meshing, scenes

import vmap_harness as vh

pytestmark = pytest.mark.gpu


def _level_with_margin(occ):
    """A level between two lattice values near the median, as far from both as possible."""
    s = np.sort(occ)
    lo, hi = int(0.4 * s.size), int(0.6 * s.size)
    g = np.argmax(np.diff(s[lo:hi])) + lo
    return 0.5 * (s[g] + s[g + 1]), 0.5 * (s[g + 1] - s[g])


def test_mesh_matches_oracle_marching_tetrahedra():
    rng = np.random.default_rng(71)
    o = scenes.make_object(rng, (1, 2), 0.15, 0.3, 0.2, H=32, per_view=64)
    # a random MLP with its output layer scaled up: a field that varies across a
    # lattice cell, so the interpolated crossings are well conditioned
    Ws, bs = vs.unpack(scenes.init_weights(rng, 32).astype(np.float64), 32)
    Ws[4] *= 20.0
    o["init"] = vs.pack(Ws, bs).astype(np.float32)
    o["n_surface"], o["n_strat"], o["rays"] = 10, 12, 32
    sc = dict(objects=[o], B=scenes.make_B(72), seed=71)
    vm = vh.library_context(sc)
    half = np.full(3, float(o["scale"]))
    res = 20
    cfg = vh.oracle_config(sc)
    occ = om.grid_occupancy(cfg, o["init"].astype(np.float64), 32, o["center"], o["scale"], half, res)
    level, margin = _level_with_margin(occ)
    assert margin > 1e-6
    ref = om.marching_tetrahedra(occ, o["center"], half, res, level)
    tris = vm.extract_mesh(0, half, res, level).cpu().numpy().astype(np.float64)
    assert ref.shape[0] > 100 and tris.shape == ref.shape
    step = 2 * half[0] / res
    assert np.max(np.abs(tris - ref)) <= 1e-3 * step
    # orientation agrees wherever the triangle is not degenerate
    n_ref = np.cross(ref[:, 1] - ref[:, 0], ref[:, 2] - ref[:, 0])
    n_gpu = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    big = np.linalg.norm(n_ref, axis=1) > 1e-6 * step * step
    assert np.all(np.einsum("ij,ij->i", n_ref[big], n_gpu[big]) > 0)


def test_trained_object_mesh_lies_on_the_surface():
    rng = np.random.default_rng(73)
    o = scenes.make_object(rng, (1, 2), 0.15, 0.3, 0.15, H=32, per_view=1024, offmask=0.5)
    o["init"] = scenes.init_weights(rng, 32)
    o["n_surface"], o["n_strat"], o["rays"] = 10, 12, 512
    sc = dict(objects=[o], B=scenes.make_B(74), seed=73)
    vm = vh.library_context(sc, lambda_occ=1.0)
    for _ in range(3000):
        vm.sample_rays([512])
        vm.train_step()
    half = np.full(3, 1.2 * float(o["scale"]))
    tris = vm.extract_mesh(0, half, 64, 0.5)
    assert tris.shape[0] > 500
    center = np.asarray(o["center"], np.float64)
    sdf = lambda p: torch.from_numpy(scenes.union_sdf(o["prims"], center, p.cpu().numpy().astype(np.float64))).to(p)
    gt = torch.from_numpy(scenes.surface_points(rng, o["prims"], center, 4000)).float().cuda()
    acc, comp = meshing.accuracy_completion(tris, sdf, gt, n=20000, generator=torch.Generator(device="cuda").manual_seed(0))
    print(f"mesh accuracy {acc * 100:.2f} cm, completion {comp * 100:.2f} cm, {tris.shape[0]} triangles")
    assert acc < 0.02 and comp < 0.02, (acc, comp)
