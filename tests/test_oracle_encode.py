"""Pins of the oracle's encoding step (Sec. 4.1: p = floor(N x), features of
the 8 voxel corners, trilinear interpolation) and of Eq. 1 as the oracle
evaluates it for checking hashes."""
import os

import numpy as np
import pytest

import oracle
from paper_2303_04086_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hits(scene, cam, W=128, H=128):
    o, d = oracle.raygen(cam, W, H)
    tri, t, _ = oracle.BVH(scene.vertices, scene.triangles).hit(o, d)
    m = tri >= 0
    return o[m], d[m], t[m]


def test_cell_contains_hit_point(tiny, tiny_cam):
    o, d, t = _hits(tiny, tiny_cam)
    for N in tiny.resolutions:
        c, f = oracle.cells(N, o, d, t)
        P = o.astype(np.float64) + t.astype(np.float64)[:, None] * d.astype(np.float64)
        h = 3.0 / N
        lo = -1.5 + c * h
        assert np.all(c >= 0) and np.all(c < N)
        assert np.all(P >= lo - 1e-5) and np.all(P <= lo + h + 1e-5)
        assert np.all(f >= 0) and np.all(f <= 1)
        # f is the position inside the cell in units of the cell size
        assert np.abs((lo + f * h) - P).max() < 1e-5


def test_no_corner_lookup_leaves_the_occupied_set(tiny_oracle, tiny_cam):
    r = tiny_oracle.render_pixels(tiny_cam, 128, 128)
    assert r["missing"] == 0
    hit = r["tri"] >= 0
    assert 0.5 < hit.mean() < 0.65
    assert np.all(r["rgba"][~hit] == 0)
    assert np.all((r["rgba"][hit] > 0) & (r["rgba"][hit] < 1))


def _affine_scene(tiny, A, B):
    s = synth.Scene(tiny.vertices, tiny.triangles, tiny.resolutions, tiny.keys,
                    [None] * len(tiny.keys), tiny.w1, tiny.w2, tiny.w3)
    feats = []
    for l, k in enumerate(tiny.keys):
        p = synth.unpack_keys(k).astype(np.float64)
        feats.append((p @ A[l].T + B[l]).astype(np.float32))
    s.features = feats
    return s


def test_trilinear_reproduces_affine_fields(tiny, tiny_cam):
    # features f(p) = A p + b (small integers: exact in FP32) -> the trilinear
    # interpolant of an affine field is the field itself: E = A u + b, u = c + f
    rng = np.random.default_rng(3)
    L = tiny.n_levels
    A = rng.integers(-3, 4, size=(L, 2, 3)).astype(np.float64)
    B = rng.integers(-5, 6, size=(L, 2)).astype(np.float64)
    s = _affine_scene(tiny, A, B)
    orc = oracle.Oracle(s)
    o, d, t = _hits(tiny, tiny_cam, 64, 64)
    out = orc.render_rays(o, d, with_E=True)
    assert out["missing"] == 0
    for l, N in enumerate(tiny.resolutions):
        c, f = oracle.cells(N, o, d, t)
        u = c.astype(np.float64) + f.astype(np.float64)
        ref = u @ A[l].T + B[l]
        got = out["E"][:, 2 * l:2 * l + 2]
        assert np.abs(got - ref).max() < 1e-9


def test_interpolation_at_corner_is_corner_value(tiny):
    # a ray that ends exactly on a grid vertex (f = 0): E = that vertex's feature
    orc = oracle.Oracle(tiny)
    N = tiny.resolutions[0]
    # vertex (8, 8, 13) of level 0 is the point (0, 0, 0.9375), next to the
    # +z pole of the unit sphere; (0.9375 + 1.5) * (float)(1/3) rounds to
    # 0.8125 in FP32, so u = 13 and f = 0 on every axis
    k = synth.unpack_keys(tiny.keys[0])
    z = 13
    assert any(v[0] == 8 and v[1] == 8 and v[2] == z for v in k)
    P = np.array([(8 / N) * 3 - 1.5, (8 / N) * 3 - 1.5, (z / N) * 3 - 1.5], np.float32)
    idx, w = orc.corners(P[None] - np.float32([0, 0, 1]), np.float32([[0, 0, 1]]), np.float32([1.0]))
    assert idx[0, 0, 0] >= 0
    assert w[0, 0, 0] == 1.0 and np.all(w[0, 0, 1:] == 0.0)
    row = np.searchsorted(tiny.keys[0], synth.pack_keys(np.array([[8, 8, z]]))[0])
    assert idx[0, 0, 0] == row


def test_psh_formula_hand_worked():
    rows = np.loadtxt(os.path.join(GOLDEN, "psh_tiny.txt"), dtype=np.int64)
    m, r = 3, 2
    offs = [(0, 0, 0), (1, 0, 0), (0, 2, 0), (2, 1, 1)] + [(0, 0, 1)] * 4
    phi = np.array([a | (b << 10) | (c << 20) for a, b, c in offs], np.uint32)
    got = oracle.psh_slots(phi, m, r, rows[:, :3].astype(np.int32))
    assert np.array_equal(got, rows[:, 3])


def test_features_are_keyed_by_coordinate(tiny):
    # the generator's value of a vertex does not depend on the list it sits in
    k = tiny.keys[2]
    sub = k[::7].copy()
    f_all = synth.features(0, 2, k)
    f_sub = synth.features(0, 2, sub)
    assert np.array_equal(f_all[::7], f_sub)
    assert abs(f_all.std() - 0.1) < 0.01 and abs(f_all.mean()) < 0.01
