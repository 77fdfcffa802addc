"""Pins of the oracle's depth fusion of several objects (the frame composer of
Sec. 5.1; reading: (t, object index) order, the K nearest hits, straight-alpha
"over" front to back, pixel (C / A, A)).

- one object: the fused pixel is that object's own render;
- opaque hits (alpha = 1): the fusion is a z-buffer, the nearest hit's colour;
- the same pixels by the back-to-front "over" recursion on premultiplied
  colour (a different algorithm for the same operator);
- equal opacities: coverage 1 - (1 - a)^k in closed form;
- a hand-worked two-object pixel (tests/golden/composite_two_objects.txt);
- the K cut drops the farthest hits, not the highest object indices.
"""
import os
from fractions import Fraction

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "composite_two_objects.txt")


def _random_layers(rng, n_obj, n, alpha=None, p_hit=0.6):
    hit = rng.random((n_obj, n)) < p_hit
    # coarse t values so that ties between objects occur
    t = (rng.integers(1, 40, size=(n_obj, n)) * 0.25).astype(np.float32)
    rgba = rng.random((n_obj, n, 4))
    if alpha is not None:
        rgba[..., 3] = alpha
    else:
        rgba[..., 3] = 0.05 + 0.9 * rgba[..., 3]
    return hit, t, rgba


def test_one_object_reproduces_its_render(tiny, tiny_oracle):
    rng = np.random.default_rng(3)
    n = 3000
    eye = rng.normal(size=(n, 3))
    eye = (2.7 * eye / np.linalg.norm(eye, axis=1, keepdims=True)).astype(np.float32)
    d = rng.uniform(-1.0, 1.0, size=(n, 3)) - eye
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    ref = tiny_oracle.render_rays(eye, d)
    got = oracle.render_scene([tiny_oracle], [(0.0, 0.0, 0.0)], eye, d, K=4)
    hit = ref["tri"] >= 0
    assert 0.2 < hit.mean() < 0.9
    assert np.array_equal(got["used"], hit.astype(np.int32))
    assert np.allclose(got["rgba"], ref["rgba"], rtol=1e-13, atol=1e-15)
    assert (got["rgba"][~hit] == 0).all()


def test_translation_moves_the_object(tiny, tiny_oracle):
    # an object placed at T seen by world rays o is the object at the origin
    # seen from o - T
    rng = np.random.default_rng(4)
    n = 500
    T = np.array([2.5, -1.0, 0.75], np.float32)
    eye = rng.normal(size=(n, 3))
    eye = (2.7 * eye / np.linalg.norm(eye, axis=1, keepdims=True)).astype(np.float32)
    d = rng.uniform(-1.0, 1.0, size=(n, 3)) - eye
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    world = (eye + T).astype(np.float32)
    got = oracle.render_scene([tiny_oracle], [T], world, d, K=1)
    ref = tiny_oracle.render_rays((world - T).astype(np.float32), d)
    assert np.array_equal(got["per"][0]["tri"], ref["tri"])
    assert (ref["tri"] >= 0).mean() > 0.2


def test_opaque_hits_give_a_z_buffer():
    rng = np.random.default_rng(5)
    n_obj, n = 7, 4000
    hit, t, rgba = _random_layers(rng, n_obj, n, alpha=1.0)
    out, used = oracle.composite(hit, t, rgba, K=4)
    for r in range(n):
        ks = [k for k in range(n_obj) if hit[k, r]]
        if not ks:
            assert (out[r] == 0).all() and used[r] == 0
            continue
        front = min(ks, key=lambda k: (t[k, r], k))
        assert np.array_equal(out[r, :3], rgba[front, r, :3])
        assert out[r, 3] == 1.0
        assert used[r] == min(len(ks), 4)


def test_back_to_front_over_gives_the_same_pixels():
    rng = np.random.default_rng(6)
    n_obj, n = 6, 3000
    hit, t, rgba = _random_layers(rng, n_obj, n)
    out, _ = oracle.composite(hit, t, rgba, K=n_obj)
    for r in range(n):
        ks = sorted((k for k in range(n_obj) if hit[k, r]), key=lambda k: (t[k, r], k))
        P, A = np.zeros(3), 0.0  # premultiplied colour and coverage, farthest first
        for k in reversed(ks):
            a = rgba[k, r, 3]
            P = a * rgba[k, r, :3] + (1 - a) * P
            A = a + (1 - a) * A
        want = np.concatenate([P / A, [A]]) if A > 0 else np.zeros(4)
        assert np.allclose(out[r], want, rtol=1e-12, atol=1e-14)


def test_equal_opacities_cover_in_closed_form():
    rng = np.random.default_rng(7)
    for k in range(1, 6):
        hit = np.ones((k, 1), bool)
        t = rng.permutation(np.arange(1, k + 1, dtype=np.float32)).reshape(k, 1)
        rgba = rng.random((k, 1, 4))
        rgba[..., 3] = 0.3
        out, used = oracle.composite(hit, t, rgba, K=8)
        assert used[0] == k
        assert abs(out[0, 3] - (1 - 0.7 ** k)) < 1e-15


def _golden():
    cases = {}
    for ln in open(GOLDEN):
        ln = ln.strip()
        if not ln or ln.startswith("#"):
            continue
        f = ln.split()
        c = cases.setdefault(int(f[1]), {"in": {}, "out": None})
        if f[0] == "in":
            c["in"][int(f[2])] = (int(f[3]), float(f[4]), [float(Fraction(x)) for x in f[5:9]])
        else:
            c["out"] = [float(Fraction(x)) for x in f[2:6]]
    return cases


def test_hand_worked_two_object_pixels():
    cases = _golden()
    assert len(cases) == 5
    for cid, c in sorted(cases.items()):
        ks = sorted(c["in"])
        hit = np.array([[c["in"][k][0]] for k in ks])
        t = np.array([[c["in"][k][1]] for k in ks], np.float32)
        rgba = np.array([[c["in"][k][2]] for k in ks])
        out, _ = oracle.composite(hit, t, rgba, K=4)
        assert np.allclose(out[0], c["out"], rtol=0, atol=1e-15), (cid, out[0], c["out"])


def test_k_cut_drops_the_farthest_hits():
    # five overlapping objects, object 0 farthest: K = 4 keeps objects 4..1
    rng = np.random.default_rng(8)
    rgba = rng.random((5, 1, 4))
    rgba[..., 3] = 0.5
    t = np.array([[5.0], [4.0], [3.0], [2.0], [1.0]], np.float32)
    hit = np.ones((5, 1), bool)
    out4, used4 = oracle.composite(hit, t, rgba, K=4)
    near4, _ = oracle.composite(hit[1:], t[1:], rgba[1:], K=4)
    by_index, _ = oracle.composite(hit[:4], t[:4], rgba[:4], K=4)
    out5, used5 = oracle.composite(hit, t, rgba, K=5)
    assert used4[0] == 4 and used5[0] == 5
    assert np.allclose(out4, near4, rtol=0, atol=1e-15)
    assert abs(out4[0, 3] - (1 - 0.5 ** 4)) < 1e-15
    assert np.abs(out4 - by_index).max() > 1e-3
    assert np.abs(out4 - out5).max() > 1e-3
