"""inolf_build_hash (host-only part of the library) against Eq. 1 as the
oracle evaluates it: injective on the point set, in range, Phi entries in
range, deterministic, and the CRT conditions on (m, r)."""
import math

import numpy as np
import pytest

import oracle
from paper_2303_04086_gb300 import build, inolf, synth


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def _check(h, coords, extent):
    s = oracle.psh_slots(h.phi, h.m, h.r, coords)
    assert np.array_equal(s, h.slot_of.astype(np.int64))
    assert len(np.unique(s)) == len(s)
    assert s.min() >= 0 and s.max() < h.m ** 3
    assert math.gcd(h.m, h.r) == 1 and h.m * h.r >= extent + 1
    assert h.m ** 3 >= len(coords)
    e = h.phi
    for sh in (0, 10, 20):
        assert ((e >> sh) & 1023).max() < h.m
    assert (e >> 30).max() == 0


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_hash_tiny_scene_levels(tiny, level):
    c = synth.unpack_keys(tiny.keys[level])
    h = inolf.build_hash(c, tiny.resolutions[level])
    _check(h, c, tiny.resolutions[level])
    # equal to the dense map: feature row i of the slot table is feature i
    table = np.zeros((h.m ** 3, 2), np.float32)
    table[h.slot_of] = tiny.features[level]
    assert np.array_equal(table[oracle.psh_slots(h.phi, h.m, h.r, c)], tiny.features[level])


def test_hash_carries_its_points(tiny):
    # object creation lays out the corner bundles from the points the hash
    # keeps: they must be the input points, in input order
    c = synth.unpack_keys(tiny.keys[1])
    h = inolf.build_hash(c, tiny.resolutions[1])
    got = np.ctypeslib.as_array(h._h.contents.coords, shape=(h.n * 3,)).reshape(-1, 3)
    assert np.array_equal(got, c.astype(np.int32))


def test_hash_is_deterministic(tiny):
    c = synth.unpack_keys(tiny.keys[2])
    a = inolf.build_hash(c, tiny.resolutions[2])
    b = inolf.build_hash(c, tiny.resolutions[2])
    assert np.array_equal(a.phi, b.phi) and np.array_equal(a.slot_of, b.slot_of)


def test_hash_edge_cases():
    # single point, dense full grid, random sparse sets, all corners of a box
    h = inolf.build_hash(np.array([[3, 4, 5]]), 7)
    _check(h, np.array([[3, 4, 5]], np.int32), 7)
    g = np.stack(np.meshgrid(*[np.arange(9)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(np.int32)
    h = inolf.build_hash(g, 8)
    _check(h, g, 8)
    rng = np.random.default_rng(0)
    for n, ext in [(10, 1000), (5000, 300), (20000, 64)]:
        keys = np.unique(rng.integers(0, ext + 1, size=(n, 3)), axis=0).astype(np.int32)
        h = inolf.build_hash(keys, ext)
        _check(h, keys, ext)
    h = inolf.build_hash(np.zeros((0, 3), np.int32), 4)
    assert h.n == 0


def test_hash_rejects_bad_input():
    with pytest.raises(inolf.InolfError) as e:
        inolf.build_hash(np.array([[1, 2, 3], [1, 2, 3]]), 5)
    assert e.value.status == inolf.E_INVALID
    with pytest.raises(inolf.InolfError):
        inolf.build_hash(np.array([[1, 2, 9]]), 5)
    with pytest.raises(inolf.InolfError):
        inolf.build_hash(np.array([[1, -2, 3]]), 5)


def test_neighbouring_points_share_offsets(tiny):
    # the coherence heuristic: a good share of x-neighbour pairs sit in
    # consecutive slots (Fig. 3 of the paper: adjacent points -> adjacent slots)
    k = tiny.keys[3]
    c = synth.unpack_keys(k)
    h = inolf.build_hash(c, tiny.resolutions[3])
    kx = k + np.uint64(1)
    idx = np.searchsorted(k, kx)
    idx[idx >= len(k)] = 0
    has = k[idx] == kx
    s = h.slot_of.astype(np.int64)
    assert (s[idx[has]] == s[has] + 1).mean() > 0.2
