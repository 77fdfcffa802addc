"""Pins of the oracle's decoupled variant (Sec. 4.2): the density texture
cubes, the hit-point march of Eq. 4 (hit = first sample of largest blending
weight, alpha_c = accumulated weight), the alpha_c input of Eq. 5 and the
diffuse/specular combination of Eq. 7.  Every expected value here comes from a
closed form, an invariant or a special case, not from the oracle itself."""
import math

import numpy as np
import pytest

import oracle
from paper_2303_04086_gb300 import synth

LO, SIDE = -1.5, 3.0


def _cubes(b, r, cells, vertex_value, diffuse_value=None, step=None, t_min=1e-4, alpha_miss=1e-4):
    """A synth.Cubes record whose vertex values come from a function of the
    global fine vertex coordinate (so cubes sharing a face agree)."""
    cells = np.asarray(cells, np.int32).reshape(-1, 3)
    g = np.stack(np.meshgrid(np.arange(r + 1), np.arange(r + 1), np.arange(r + 1), indexing="ij"), -1)
    local = g.transpose(2, 1, 0, 3).reshape(-1, 3)  # x fastest
    dens = np.empty((len(cells), (r + 1) ** 3), np.float32)
    diff = None if diffuse_value is None else np.empty((len(cells), (r + 1) ** 3, 4), np.float32)
    for i, c in enumerate(cells):
        v = c[None, :] * r + local
        dens[i] = vertex_value(v)
        if diff is not None:
            diff[i] = diffuse_value(v)
    K = b * r
    step = float(np.float32(SIDE / K)) if step is None else step
    return synth.Cubes(b, r, cells, dens, diff, step, t_min, alpha_miss)


def _all_cells(b):
    return [(x, y, z) for z in range(b) for y in range(b) for x in range(b)]


def _rays(o, d):
    o = np.asarray(o, np.float32).reshape(-1, 3)
    d = np.asarray(d, np.float64).reshape(-1, 3)
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    return o, d


def test_homogeneous_medium_closed_forms():
    # sigma = S everywhere: every sample has sigma = S exactly, so
    # w_k = e^k (1 - e) with e = exp(-S delta): the entry sample is the hit,
    # w_0 = 1 - e, w_1 = e (1 - e) (a missing transmittance update would tie
    # them), and T after n samples is e^n, so the march stops at the first n
    # with e^n < t_min and alpha_c = 1 - e^n.
    b, r, S = 4, 4, 10.0
    cub = _cubes(b, r, _all_cells(b), lambda v: np.full(len(v), S))
    oc = oracle.Cubes(cub)
    o, d = _rays([[0.1, 0.2, 3.0], [0.3, -0.4, 0.2]], [[0.0, 0.0, -1.0], [0.2, 0.3, -1.0]])
    m = oc.march(o, d)
    e = math.exp(-S * cub.step)
    n = math.ceil(math.log(cub.t_min) / math.log(e))
    assert abs(e ** n - cub.t_min) > 1e-3 * cub.t_min  # not a near-threshold case
    # ray 0 enters the cube at z = 1.5 (t0 = 1.5); ray 1 starts inside (t0 = 0)
    assert m["k"].tolist() == [0, 0]
    assert m["t"][0] == np.float32(1.5) and m["t"][1] == 0.0
    np.testing.assert_allclose(m["wmax"], 1 - e, rtol=1e-5)
    np.testing.assert_allclose(m["w2"], e * (1 - e), rtol=1e-5)
    assert m["k2"].tolist() == [1, 1]
    assert m["n"].tolist() == [n, n]
    np.testing.assert_allclose(m["alpha"], 1 - e ** n, atol=1e-6)


def test_sample_spacing_and_cube_span():
    # a ray that never stops early takes the samples t0 + k delta inside the
    # cube: floor((t1 - t0) / delta) + 1 of them (t1 - t0 = 3 on an axis ray)
    b, r = 4, 4
    cub = _cubes(b, r, _all_cells(b), lambda v: np.full(len(v), 1e-3))
    oc = oracle.Cubes(cub)
    o, d = _rays([[0.05, 0.05, 3.0], [-3.0, 0.1, 0.2]], [[0, 0, -1.0], [1.0, 0, 0]])
    m = oc.march(o, d)
    K = b * r
    assert m["n"].tolist() == [K + 1, K + 1]  # delta = side / K exactly
    # each sample contributes sigma delta of optical depth (Eq. 4's sum):
    # alpha_c = 1 - exp(-sigma delta (K + 1)), up to the FP32 rounding of the
    # K + 1 transmittance products (about (K + 1) half-ulps of 1)
    np.testing.assert_allclose(m["alpha"], 1 - math.exp(-1e-3 * cub.step * (K + 1)), rtol=0, atol=2e-6)
    # rays that miss the cube take no sample
    o2, d2 = _rays([[5.0, 5.0, 5.0], [0.0, 2.0, 0.0]], [[1.0, 0, 0], [1.0, 0, 0]])
    m2 = oc.march(o2, d2)
    assert m2["n"].tolist() == [0, 0] and m2["k"].tolist() == [-1, -1]


def test_zero_density_misses():
    b, r = 4, 4
    cub = _cubes(b, r, _all_cells(b), lambda v: np.zeros(len(v)))
    m = oracle.Cubes(cub).march(*_rays([[0.0, 0.0, 3.0]] * 3, [[0, 0, -1.0], [0.1, 0.2, -1], [0.3, 0, -1]]))
    assert np.all(m["k"] == -1) and np.all(m["alpha"] == 0) and np.all(m["wmax"] == 0)


def test_unlisted_cubes_are_empty_space():
    # a medium that fills only the lower half (base cells z = 0, 1 of 4): the
    # density is S for z <= 0, falls linearly to 0 across the fine cell above
    # z = 0 (its upper vertices belong to unlisted cubes), and is 0 above.  A
    # vertical ray from above hits within one sample of that ramp.
    b, r, S = 4, 8, 400.0
    cells = [c for c in _all_cells(b) if c[2] < 2]
    cub = _cubes(b, r, cells, lambda v: np.full(len(v), S))
    oc = oracle.Cubes(cub)
    o, d = _rays([[0.11, -0.23, 3.0], [0.7, 0.6, 3.0]], [[0, 0, -1.0], [0, 0, -1.0]])
    m = oc.march(o, d)
    h = SIDE / (b * r)
    zhit = o[:, 2] + m["t"] * d[:, 2]
    assert np.all(m["k"] >= 0)
    assert np.all(zhit <= h + 1e-6) and np.all(zhit >= -cub.step - 1e-6)
    # density probes: S below, the ramp value at a quarter of the cell above z = 0, 0 above
    t = np.array([3.0 + 0.5, 3.0 - 0.25 * h, 3.0 - 2 * h], np.float32)
    sig = oc.density(np.repeat(o[:1], 3, 0), np.repeat(d[:1], 3, 0), t)
    np.testing.assert_allclose(sig, [S, 0.75 * S, 0.0], rtol=1e-5, atol=1e-4)


def test_density_reproduces_affine_fields():
    # sigma(v) = a . v + c on the vertices -> the trilinear interpolant is the
    # affine function a . u + c of the FP32 fine coordinate u = K x; distinct
    # per-axis slopes catch a transposed or mis-ordered corner
    b, r = 4, 4
    K = b * r
    a = np.array([1.0, 4.0, 16.0])
    cub = _cubes(b, r, _all_cells(b), lambda v: v @ a + 2.0)
    oc = oracle.Cubes(cub)
    rng = np.random.default_rng(0)
    n = 200
    o = rng.uniform(-1.4, 1.4, (n, 3)).astype(np.float32)
    d = np.tile(np.float32([0, 0, 1.0]), (n, 1))
    t = np.zeros(n, np.float32)
    sig = oc.density(o, d, t)
    x = (o.astype(np.float32) - np.float32(LO)) * np.float32(1.0 / 3.0)
    u = x.astype(np.float64) * K
    np.testing.assert_allclose(sig, u @ a + 2.0, rtol=2e-6)


def test_sphere_shell_hits_lie_in_the_shell():
    # tiny_density_scene: shell of half-width w around the unit sphere with
    # optical depth 12 across it.  Hit points lie within w plus one fine-cell
    # diagonal of the sphere; rays passing well inside the sphere's silhouette
    # are opaque hits, rays passing well outside it miss.
    s = synth.tiny_density_scene()
    oc = oracle.Cubes(s.cubes)
    cam = synth.camera((0.0, 0.0, 3.0))
    o, d = oracle.raygen(cam, 96, 96)
    m = oc.march(o, d)
    w = s.cubes.meta["w"]
    h = SIDE / (s.cubes.b * s.cubes.r)
    hit = m["k"] >= 0
    P = o.astype(np.float64) + m["t"].astype(np.float64)[:, None] * d
    rad = np.linalg.norm(P[hit], axis=1)
    assert rad.min() >= 1 - w - math.sqrt(3) * h and rad.max() <= 1 + w + math.sqrt(3) * h
    # impact parameter: distance of the ray's line from the origin
    oo = o.astype(np.float64)
    dd = d.astype(np.float64)
    imp = np.linalg.norm(oo - (oo * dd).sum(1, keepdims=True) * dd, axis=1)
    inside = imp < 0.9
    outside = imp > 1 + w + math.sqrt(3) * h
    assert inside.sum() > 1000 and outside.sum() > 1000
    assert np.all(hit[inside]) and np.all(m["alpha"][inside] > 0.999)
    assert not np.any(hit[outside])
    # the hit is the sample where the ray enters the dense part of the shell:
    # on the outer side of the sphere
    assert np.all(rad >= 1.0 - 1e-6)


def _variant_scene(diffuse_value, zero_alpha_column=False):
    s = synth.tiny_density_scene()
    c = s.cubes
    g = np.stack(np.meshgrid(np.arange(c.r + 1), np.arange(c.r + 1), np.arange(c.r + 1), indexing="ij"), -1)
    local = g.transpose(2, 1, 0, 3).reshape(-1, 3)
    diff = np.empty_like(c.diffuse)
    for i, cell in enumerate(c.cells):
        diff[i] = diffuse_value(cell[None, :] * c.r + local)
    s.cubes = synth.Cubes(c.b, c.r, c.cells, c.density, diff, c.step, c.t_min, c.alpha_miss, meta=c.meta)
    if zero_alpha_column:
        s.w1 = s.w1.copy()
        s.w1[:, -1] = 0.0
    return s


def _hit_rays(orc, n=400):
    cam = synth.camera((0.3, 0.2, 3.0))
    o, d = oracle.raygen(cam, 64, 64)
    m = orc.cubes.march(o, d)
    hit = np.nonzero(m["k"] >= 0)[0][:n]
    return o[hit], d[hit], m["t"][hit], m["alpha"][hit]


def test_eq7_diffuse_plus_tinted_specular():
    # c = c_d + t c_s (Eq. 7) checked through special cases of the diffuse
    # texture:  (c_d = 0, t = 1) gives c_s alone; (c_d, t = 0) gives the
    # interpolated c_d alone; the general case is their tint-weighted sum,
    # with the tint read back as the interpolated c_d of a texture holding it.
    rng = np.random.default_rng(1)
    A = rng.uniform(0.01, 0.03, (4, 3))

    def field(v):  # affine per channel, positive
        return (v @ A.T + 0.05).astype(np.float32)

    base = _variant_scene(field)
    orc = oracle.Oracle(base)
    o, d, t, a = _hit_rays(orc)
    full = orc.shade_variant_at(o, d, t, a)

    def only(mod):
        return oracle.Oracle(_variant_scene(mod)).shade_variant_at(o, d, t, a)

    cs = only(lambda v: np.tile(np.float32([0, 0, 0, 1.0]), (len(v), 1)))
    cd = only(lambda v: np.concatenate([field(v)[:, :3], np.zeros((len(v), 1), np.float32)], 1))
    tint = only(lambda v: np.concatenate([np.repeat(field(v)[:, 3:], 3, 1), np.zeros((len(v), 1), np.float32)],
                                         1))[:, 0]
    assert np.all((cs[:, :3] > 0) & (cs[:, :3] < 1))
    np.testing.assert_allclose(full[:, :3], cd[:, :3] + tint[:, None] * cs[:, :3], rtol=1e-12, atol=1e-12)
    # the opacity channel is F_s's alone: independent of the diffuse texture
    np.testing.assert_array_equal(full[:, 3], cs[:, 3])
    np.testing.assert_array_equal(full[:, 3], cd[:, 3])
    # an affine diffuse field is reproduced at the hit point
    x = (o.astype(np.float32) + t[:, None] * d.astype(np.float32) - np.float32(LO)) * np.float32(1.0 / 3.0)
    u = x.astype(np.float64) * (base.cubes.b * base.cubes.r)
    np.testing.assert_allclose(cd[:, :3], u @ A[:3].T + 0.05, rtol=1e-5)


def test_eq5_alpha_c_is_an_mlp_input():
    # with W1's alpha_c column zeroed the output cannot depend on alpha_c; with
    # the generated column it does
    diff_const = lambda v: np.tile(np.float32([0.1, 0.2, 0.3, 0.5]), (len(v), 1))
    z = oracle.Oracle(_variant_scene(diff_const, zero_alpha_column=True))
    nz = oracle.Oracle(_variant_scene(diff_const))
    o, d, t, _ = _hit_rays(z, 100)
    lo = np.full(len(o), 0.05, np.float32)
    hi = np.full(len(o), 0.95, np.float32)
    np.testing.assert_array_equal(z.shade_variant_at(o, d, t, lo), z.shade_variant_at(o, d, t, hi))
    assert np.abs(nz.shade_variant_at(o, d, t, lo) - nz.shade_variant_at(o, d, t, hi)).max() > 1e-3


def test_variant_render_end_to_end_is_consistent():
    s = synth.tiny_density_scene()
    orc = oracle.Oracle(s)
    cam = synth.camera((0.0, 0.0, 3.0))
    r = orc.render_variant_pixels(cam, 64, 64)
    assert r["missing"] == 0
    hit = r["k"] >= 0
    assert 0.5 < hit.mean() < 0.8
    assert np.all(r["rgba"][~hit] == 0)
    assert np.all(r["alpha"][hit] > s.cubes.alpha_miss)
    o, d = oracle.raygen(cam, 64, 64)
    again = orc.shade_variant_at(o[hit], d[hit], r["t"][hit], r["alpha"][hit])
    np.testing.assert_array_equal(again, r["rgba"][hit])
