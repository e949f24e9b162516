"""Pins of the oracle's generator and depth-guided sampler (section 3.3, Eq. 1-2).

The generator is pinned to the published Philox4x32-10 known-answer vectors;
the sampler to the distributions Eq. 1 and Eq. 2 define (one stratified
sample per stratum, uniform inside it; Gaussian samples around the depth)."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox
from oracle import vmap_step as vs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat_rows())
def test_philox_known_answers(ctr, key, out):
    got = philox.philox4x32_10(np.array(ctr), np.array(key))
    assert [int(x) for x in got] == out


def test_unit_map_open_interval_and_float32_exact():
    w = np.array([0, 1, 511, 512, 2**31, 2**32 - 1], dtype=np.uint64)
    u = philox.word_to_unit(w)
    assert np.all(u > 0) and np.all(u < 1)
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)
    assert u[0] == 2.0 ** -24 and u[-1] == 1.0 - 2.0 ** -24


def test_index_map_range_and_uniformity():
    w = philox.ray_words(7, 3, 0, np.arange(200000), 1)[:, 0]
    idx = philox.word_to_index(w, 37)
    assert idx.min() == 0 and idx.max() == 36
    counts = np.bincount(idx, minlength=37)
    assert stats.chisquare(counts).pvalue > 1e-3


def _pool_single(depth, n=1):
    pool = np.zeros((n, 12), np.float32)
    pool[:, 6] = depth
    pool[:, 10] = 1.0
    return pool


def test_stratified_one_per_stratum_and_uniform():
    cfg = vs.Config(seed=11)
    D = 1.7
    R, Nc = 4000, 12
    _, t = vs.sample_object(cfg, _pool_single(D), R, 0, Nc, stream=5, step=3)
    lo, hi = cfg.t_near, D + cfg.depth_pad
    pos = (t - lo) / (hi - lo) * Nc
    j = np.floor(pos)
    # sorted output has exactly the j-th sample in the j-th stratum (Eq. 1)
    assert np.array_equal(j, np.broadcast_to(np.arange(Nc), t.shape))
    frac = (pos - j).ravel()
    assert stats.kstest(frac, "uniform").pvalue > 1e-3
    assert np.all(np.diff(t, axis=1) >= 0)


def test_surface_samples_gaussian_around_depth():
    cfg = vs.Config(seed=12)
    D = 2.3
    _, t = vs.sample_object(cfg, _pool_single(D), 3000, 10, 0, stream=1, step=0)
    z = (t.ravel() - D) / cfg.d_sigma
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 0.05 and abs(z.std() - 1) < 0.05
    # odd Gaussian count uses a cos without its sin partner: still N(0, 1)
    _, t = vs.sample_object(cfg, _pool_single(D), 3000, 7, 0, stream=1, step=0)
    assert t.shape == (3000, 7)
    assert stats.kstest(((t.ravel() - D) / cfg.d_sigma), "norm").pvalue > 1e-3


def test_invalid_depth_uses_far_bound_and_clamps_near():
    cfg = vs.Config(seed=13)
    _, t = vs.sample_object(cfg, _pool_single(0.0), 500, 10, 12, stream=0, step=0)
    assert np.all(t >= cfg.t_near)
    assert np.all(t <= cfg.t_far + 0.5)
    # 10 surface samples sit near t_far
    assert np.mean(np.abs(t - cfg.t_far) < 0.2) > 10 / 22 - 0.05
    # a depth right at the near bound: surface samples below t_n are clamped to t_n
    _, t = vs.sample_object(cfg, _pool_single(cfg.t_near), 500, 10, 0, stream=0, step=0)
    assert np.all(t >= cfg.t_near)
    assert np.mean(t == np.float64(cfg.t_near)) > 0.4


def test_pick_uniform_and_stream_independence():
    cfg = vs.Config(seed=14)
    pool = _pool_single(1.0, n=50)
    pick, _ = vs.sample_object(cfg, pool, 50000, 10, 12, stream=2, step=9)
    assert stats.chisquare(np.bincount(pick, minlength=50)).pvalue > 1e-3
    p2, t2 = vs.sample_object(cfg, pool, 100, 10, 12, stream=2, step=9)
    p3, t3 = vs.sample_object(cfg, pool, 100, 10, 12, stream=2, step=9)
    assert np.array_equal(p2, p3) and np.array_equal(t2, t3)
    p4, _ = vs.sample_object(cfg, pool, 100, 10, 12, stream=3, step=9)
    p5, _ = vs.sample_object(cfg, pool, 100, 10, 12, stream=2, step=10)
    assert not np.array_equal(p2, p4) and not np.array_equal(p2, p5)
    # a longer batch extends a shorter one (the counter is the ray index)
    p6, t6 = vs.sample_object(cfg, pool, 160, 10, 12, stream=2, step=9)
    assert np.array_equal(p6[:100], p2) and np.array_equal(t6[:100], t2)


def test_init_params_bounds_and_uniformity():
    H = 32
    p = vs.init_params(5, 7, H)
    assert p.size == vs.param_count(H) == 6308
    Ws, bs = vs.unpack(p, H)
    for W, b, (o, i) in zip(Ws, bs, vs.layer_shapes(H)):
        bound = 1 / np.sqrt(i)
        assert np.all(np.abs(W) < bound) and np.all(np.abs(b) < bound)
    assert stats.kstest(Ws[0].ravel() * np.sqrt(93) * 0.5 + 0.5, "uniform").pvalue > 1e-3
    assert not np.array_equal(p, vs.init_params(5, 8, H))


def test_given_rays_reuse_the_pick_stream_layout():
    """Depths drawn for caller-given rays equal the depths drawn for the same
    rays when the generator picked them (word 0 is skipped, not shifted)."""
    cfg = vs.Config(seed=15)
    pool = np.zeros((40, 12), np.float32)
    pool[:, 6] = np.linspace(0.5, 3.0, 40)
    pick, t = vs.sample_object(cfg, pool, 64, 10, 12, stream=4, step=2)
    t2 = vs.sample_given(cfg, pool[pick], 10, 12, stream=4, step=2)
    assert np.array_equal(t, t2)


def test_off_mask_rays_end_at_their_surface():
    """Rays off the object's mask stop at the surface they hit: every sample
    <= t_s, one stratified sample per stratum of [t_n, t_s]; rays on the mask
    draw exactly what they draw without a mask column."""
    from oracle import vmap_step as vs
    from oracle.philox import ray_words
    cfg = vs.Config(seed=9)
    rng = np.random.default_rng(3)
    depth = rng.uniform(0.5, 3.0, 400)
    mask = (np.arange(400) % 3 != 0).astype(np.float64)
    ns, nc = 10, 12
    w = ray_words(cfg.seed, 4, 7, np.arange(400), vs.words_per_ray(ns, nc))
    t = vs.sample_depths(cfg, depth, w, ns, nc, mask)
    t_plain = vs.sample_depths(cfg, depth, w, ns, nc)
    on = mask > 0
    assert np.array_equal(t[on], t_plain[on])
    off = ~on
    assert np.all(t[off] <= depth[off, None]) and np.all(t[off] >= cfg.t_near)
    # stratified samples of off-mask rays: u_j from words 1..N_c, t_j in stratum j of [t_n, t_s]
    u = vs.word_to_unit(w[off, 1:1 + nc])
    strat = cfg.t_near + (np.arange(nc) + u) / nc * (depth[off, None] - cfg.t_near)
    for r in range(strat.shape[0]):
        for j in range(nc):
            assert np.any(np.isclose(t[off][r], strat[r, j], rtol=0, atol=1e-12))
    # some Gaussian samples would have passed t_s: they sit exactly at t_s
    assert np.sum(t[off] == depth[off, None]) > 0
