"""Pins of the oracle's encoding, MLP, rendering (Eq. 3) and losses (Eq. 4-5)
against closed forms, hand-worked cases and brute force."""
import itertools
import math

import numpy as np

from oracle import vmap_step as vs


def _brute_render(o, c, t):
    """Eq. 3 with every product written out term by term (pure Python)."""
    S = len(o)
    O = D = 0.0
    C = [0.0, 0.0, 0.0]
    for i in range(S):
        Ti = o[i]
        for j in range(i):
            Ti *= (1.0 - o[j])
        O += Ti
        D += Ti * t[i]
        for ch in range(3):
            C[ch] += Ti * c[i][ch]
    return O, D, C


def test_render_matches_brute_force_products():
    rng = np.random.default_rng(0)
    o = rng.uniform(0, 1, (6, 7))
    c = rng.uniform(0, 1, (6, 7, 3))
    t = np.sort(rng.uniform(0.1, 3, (6, 7)), axis=1)
    r = vs.render(o, c, t)
    for k in range(6):
        O, D, C = _brute_render(o[k], c[k], t[k])
        assert abs(r["O"][k] - O) < 1e-14 and abs(r["D"][k] - D) < 1e-14
        assert np.allclose(r["C"][k], C, atol=1e-14, rtol=0)


def test_render_closed_forms():
    rng = np.random.default_rng(1)
    t = np.sort(rng.uniform(0.1, 3, (1, 9)), axis=1)
    c = rng.uniform(0, 1, (1, 9, 3))
    # a single fully occupied sample renders exactly its depth and colour
    for i in range(9):
        o = np.zeros((1, 9)); o[0, i] = 1.0
        r = vs.render(o, c, t)
        assert r["D"][0] == t[0, i] and np.array_equal(r["C"][0], c[0, i]) and r["O"][0] == 1.0
    # the first occupied sample hides everything behind it
    o = rng.uniform(0, 1, (1, 9)); o[0, 3] = 1.0
    r1 = vs.render(o, c, t)
    o2 = o.copy(); o2[0, 4:] = rng.uniform(0, 1, 5)
    r2 = vs.render(o2, c, t)
    assert r1["D"][0] == r2["D"][0] and np.array_equal(r1["C"], r2["C"])
    # o = 1/2 everywhere: T_i = 2^-i (1-based), D^ = sum 2^-i t_i
    o = np.full((1, 9), 0.5)
    r = vs.render(o, c, t)
    assert abs(r["D"][0] - sum(2.0 ** -(i + 1) * t[0, i] for i in range(9))) < 1e-15
    assert abs(r["O"][0] - (1 - 2.0 ** -9)) < 1e-15
    # telescoping: sum T = 1 - prod(1 - o) <= 1
    o = rng.uniform(0, 1, (50, 22))
    r = vs.render(o, rng.uniform(0, 1, (50, 22, 3)), np.sort(rng.uniform(0, 3, (50, 22)), 1))
    assert np.allclose(r["O"], 1 - np.prod(1 - o, axis=1), atol=1e-15, rtol=0)
    assert np.all(r["O"] <= 1.0)
    # empty space renders nothing
    r = vs.render(np.zeros((1, 5)), np.ones((1, 5, 3)), np.ones((1, 5)))
    assert r["O"][0] == 0 and r["D"][0] == 0 and np.all(r["C"] == 0)


def test_encoding_special_cases():
    B = np.random.default_rng(2).standard_normal((45, 3)) * 5
    g = vs.encode(np.zeros((1, 3)), B)
    assert g.shape == (1, 93)
    assert np.all(g[0, :48] == 0) and np.all(g[0, 48:] == 1)
    # B rows (pi/2) e_axis: sin = 1, cos = 0 at x~ = e_axis; cos = -1 at 2 e_axis
    Bq = np.zeros((45, 3))
    for j in range(45):
        Bq[j, j % 3] = math.pi / 2
    g = vs.encode(np.array([[1.0, 0.0, 0.0], [2.0, 0.0, 0.0]]), Bq)
    on_x = np.arange(45) % 3 == 0
    assert np.allclose(g[0, 3:48][on_x], 1) and np.allclose(g[0, 48:][on_x], 0, atol=1e-15)
    assert np.allclose(g[1, 48:][on_x], -1) and np.allclose(g[0, 3:48][~on_x], 0)
    assert np.array_equal(g[0, :3], [1, 0, 0])


def test_mlp_zero_weights_give_one_half():
    H = 8
    Ws, bs = vs.unpack(np.zeros(vs.param_count(H)), H)
    _, y = vs.mlp_forward(Ws, bs, np.random.default_rng(3).standard_normal((5, 93)))
    assert np.all(vs.sigmoid(y) == 0.5)


def test_mlp_hand_worked_h2():
    """H = 2, inputs x~ = (0.5, -1, 0) with B = 0 (sin = 0, cos = 1).

    W1 picks (x~0, -x~1):  z1 = (0.5, 1) + b1 (0, -0.25) = (0.5, 0.75)
    W2 = [[1, 1], [1, -1]]: z2 = (1.25, -0.25) -> a2 = (1.25, 0)
    W3 = [[2, 0], [0, 1]], b3 = (-3, 0.5): z3 = (-0.5, 0.5) -> a3 = (0, 0.5)
    W4 = I, b4 = 0: a4 = (0, 0.5)
    W5 = [[0, 2], [1, 1], [0, -4], [0, 0]], b5 = (0, 0, 0, 0.3): y = (1, 0.5, -2, 0.3)
    """
    H = 2
    Ws = [np.zeros((2, 93)), np.array([[1.0, 1], [1, -1]]), np.array([[2.0, 0], [0, 1]]),
          np.eye(2), np.array([[0.0, 2], [1, 1], [0, -4], [0, 0]])]
    Ws[0][0, 0] = 1.0
    Ws[0][1, 1] = -1.0
    bs = [np.array([0.0, -0.25]), np.zeros(2), np.array([-3.0, 0.5]), np.zeros(2),
          np.array([0.0, 0, 0, 0.3])]
    g = vs.encode(np.array([[0.5, -1.0, 0.0]]), np.zeros((45, 3)))
    acts, y = vs.mlp_forward(Ws, bs, g)
    assert np.allclose(acts[1], [[0.5, 0.75]]) and np.allclose(acts[2], [[1.25, 0]])
    assert np.allclose(acts[3], [[0, 0.5]])
    assert np.allclose(y, [[1.0, 0.5, -2.0, 0.3]])
    p = vs.pack(Ws, bs)
    o, c = vs.query(vs.Config(B=np.zeros((45, 3))), p, H, np.zeros(3), 1.0, [[0.5, -1.0, 0.0]])
    assert abs(o[0] - 1 / (1 + math.exp(-1))) < 1e-15
    assert np.allclose(c[0], [1 / (1 + math.exp(-0.5)), 1 / (1 + math.exp(2)), 1 / (1 + math.exp(-0.3))])


def test_points_and_scale():
    rays = np.zeros((1, 12)); rays[0, 0:3] = [1, 2, 3]; rays[0, 3:6] = [0.5, 0, -1]
    xt = vs.points(rays, np.array([[2.0]]), center=[1, 1, 1], scale=2.0)
    assert np.allclose(xt[0, 0], [(1 + 1 - 1) / 2, (2 - 1) / 2, (3 - 2 - 1) / 2])


def test_loss_closed_form():
    cfg = vs.Config(lambda_colour=5.0, lambda_occ=10.0)
    rays = np.zeros((2, 12))
    rays[:, 6] = [1.0, 2.0]
    rays[:, 7:10] = [[0.2, 0.4, 0.6], [1, 1, 1]]
    rays[:, 10] = [1.0, 0.0]
    rend = dict(D=np.array([1.5, 0.0]), C=np.array([[0.2, 0.5, 0.5], [0, 0, 0]]),
                O=np.array([0.75, 0.25]))
    L, Ld, Lc, Lo = vs.object_loss(cfg, rays, rend)
    assert abs(Ld - 0.5 / 2) < 1e-15            # only the in-mask ray counts
    assert abs(Lc - 0.2 / 6) < 1e-15
    assert abs(Lo - (0.25 + 0.25) / 2) < 1e-15
    assert abs(L - (Ld + 5 * Lc + 10 * Lo)) < 1e-15
    rays[0, 6] = 0.0                             # invalid depth: no depth term
    assert vs.object_loss(cfg, rays, rend)[1] == 0.0


def test_param_counts():
    assert [vs.param_count(h) for h in (16, 32, 64, 128)] == [2388, 6308, 18756, 62084]
    for H in (2, 32):
        p = np.arange(vs.param_count(H), dtype=np.float64)
        Ws, bs = vs.unpack(p, H)
        assert np.array_equal(vs.pack(Ws, bs), p)
        assert Ws[0][0, 1] == 1 and bs[0][0] == 93 * H and Ws[1][0, 0] == 94 * H
    assert list(itertools.chain(*vs.layer_shapes(4))) == [4, 93, 4, 4, 4, 4, 4, 4, 4, 4]


def test_eval_ray_box_and_render_closed_forms():
    from oracle import evaluate as ev
    o = np.array([[-5.0, 0.2, 0.1], [0.0, 3.0, 0.0], [0.0, 0.0, 0.0], [2.0, 2.0, 5.0]])
    d = np.array([[2.0, 0.0, 0.0], [0.0, -1.0, 0.0], [0.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
    t_in, t_out = ev.ray_box(o, d, np.array([-1.0, -1, -1]), np.array([1.0, 1, 1]))
    assert np.allclose([t_in[0], t_out[0]], [2.0, 3.0])      # enters at x=-1, leaves at x=1
    assert np.allclose([t_in[1], t_out[1]], [2.0, 4.0])
    assert t_in[2] == 0.0 and t_out[2] == 1.0                # starts inside
    assert t_out[3] < t_in[3]                                # parallel and outside: miss
    # an MLP that is fully occupied everywhere renders its first midpoint
    H = 4
    p = np.zeros(vs.param_count(H))
    Ws, bs = vs.unpack(p, H)
    bs[4][0] = 40.0                                          # sigmoid(40) == 1 in FP64
    p = vs.pack(Ws, bs)
    cfg = vs.Config(B=np.zeros((45, 3)))
    rays = np.zeros((2, 12)); rays[:, 0:3] = o[:2]; rays[:, 3:6] = d[:2]
    D = ev.render_depth(cfg, p, H, np.zeros(3), 1.0, rays, [1, 1, 1], 10)
    assert np.allclose(D, [2.0 + 0.05 * 1.0, 2.0 + 0.05 * 2.0], rtol=1e-15)
    # a miss renders 0
    rays[1, 0:3] = [5, 5, 5]
    assert ev.render_depth(cfg, p, H, np.zeros(3), 1.0, rays, [1, 1, 1], 10)[1] == 0.0


def test_scene_compose_closed_forms():
    """Scene composition (occlusion by rendered depth): one object is its own
    render; an opaque nearer object hides the farther; two semi-transparent
    layers compose as D1 + (1 - O1) D2; listing order does not matter."""
    from oracle import evaluate as ev
    rng = np.random.default_rng(0)
    n = 50
    def rec(O, z):
        O = np.asarray(O, np.float64)
        return O, O * z, O[:, None] * rng.uniform(0, 1, (n, 3))
    a = rec(rng.uniform(0.1, 0.9, n), 1.0)
    b = rec(rng.uniform(0.1, 0.9, n), 2.0)
    D, C, O = ev.compose([a])
    assert np.allclose(D, a[1]) and np.allclose(C, a[2]) and np.allclose(O, a[0])
    opaque = rec(np.ones(n), 0.5)
    D, C, O = ev.compose([b, opaque])
    assert np.allclose(D, opaque[1]) and np.allclose(C, opaque[2]) and np.allclose(O, 1.0)
    D, C, O = ev.compose([b, a])
    assert np.allclose(D, a[1] + (1 - a[0]) * b[1])
    assert np.allclose(C, a[2] + (1 - a[0])[:, None] * b[2])
    assert np.allclose(O, 1 - (1 - a[0]) * (1 - b[0]))
    D2, C2, O2 = ev.compose([a, b])
    assert np.array_equal(D, D2) and np.array_equal(C, C2)
    # a ray no object meets renders nothing
    empty = (np.zeros(n), np.zeros(n), np.zeros((n, 3)))
    D, C, O = ev.compose([empty, empty])
    assert not D.any() and not C.any() and not O.any()


def test_render_object_matches_depth_render():
    from oracle import evaluate as ev
    from oracle import vmap_step as vs
    from paper_2302_01838_b300 import scenes
    rng = np.random.default_rng(4)
    o = scenes.make_object(rng, (1, 2), 0.1, 0.3, 0.2, H=16, per_view=64)
    cfg = vs.Config(seed=1, B=scenes.make_B(5))
    p = scenes.init_weights(rng, 16).astype(np.float64)
    rays = o["pool"][:40].astype(np.float64)
    half = [0.4, 0.4, 0.4]
    O, D, C = ev.render_object(cfg, p, 16, o["center"], o["scale"], rays, half, 24)
    assert np.allclose(D, ev.render_depth(cfg, p, 16, o["center"], o["scale"], rays, half, 24))
    assert np.all((O >= 0) & (O <= 1)) and np.all(C >= 0) and np.all(C <= O[:, None] + 1e-12)
