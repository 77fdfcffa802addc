"""Pin of the oracle's analytic FP64 gradient (the L2 objective of Eq. 8,
back-propagated through F_s and the trilinear corner weights) by central
finite differences in FP64."""
import numpy as np
import pytest

import oracle


def _rays(tiny_oracle, cam, n=64, seed=0):
    o, d = oracle.raygen(cam, 128, 128)
    r = tiny_oracle.render_rays(o, d)
    hit = np.nonzero(r["tri"] >= 0)[0]
    sel = np.random.default_rng(seed).choice(hit, n, replace=False)
    return o[sel], d[sel]


def _loss(orc, o, d, target):
    y = orc.render_rays(o, d)["rgba"]
    return ((y - target) ** 2).sum() / len(o)


def test_gradient_matches_central_differences(tiny, tiny_cam):
    orc = oracle.Oracle(tiny)
    o, d = _rays(orc, tiny_cam)
    rng = np.random.default_rng(1)
    target = rng.uniform(0, 1, size=(len(o), 4))
    y = orc.render_rays(o, d)["rgba"]
    g_out = 2.0 * (y - target) / len(o)
    g1, g2, g3, gf = orc.backward(o, d, g_out)
    z1_0, z2_0 = orc.preacts(o, d)

    checked = kinks = 0
    params = [(0, 0, g1.ravel()), (1, 0, g2.ravel()), (2, 0, g3.ravel())]
    for l in range(tiny.n_levels):
        params.append((3, l, gf[l].ravel()))
    for which, level, g in params:
        theta = orc.param(which, level)
        if which == 3:
            idx = np.nonzero(g)[0]
            idx = rng.choice(idx, min(60, len(idx)), replace=False)
        else:
            idx = rng.choice(len(theta), min(120, len(theta)), replace=False)
        for i in idx:
            t0 = theta[i]
            eps = 1e-6 * max(1.0, abs(t0))
            theta[i] = t0 + eps
            lp = _loss(orc, o, d, target)
            zp1, zp2 = orc.preacts(o, d)
            theta[i] = t0 - eps
            lm = _loss(orc, o, d, target)
            zm1, zm2 = orc.preacts(o, d)
            theta[i] = t0
            flips = (np.any(np.sign(zp1) != np.sign(z1_0)) or np.any(np.sign(zm1) != np.sign(z1_0)) or
                     np.any(np.sign(zp2) != np.sign(z2_0)) or np.any(np.sign(zm2) != np.sign(z2_0)))
            if flips:
                kinks += 1
                continue
            fd = (lp - lm) / (2 * eps)
            if abs(g[i]) > 1e-7:
                assert abs(fd - g[i]) <= 1e-3 * abs(g[i]) + 1e-9, (which, level, i, fd, g[i])
            else:
                assert abs(fd) < 1e-6
            checked += 1
    assert checked > 400
    assert kinks < checked // 10


def test_gradient_is_linear_in_upstream(tiny, tiny_cam):
    orc = oracle.Oracle(tiny)
    o, d = _rays(orc, tiny_cam, n=16, seed=3)
    a = np.random.default_rng(5).normal(size=(len(o), 4))
    b = np.random.default_rng(6).normal(size=(len(o), 4))
    ga = orc.backward(o, d, a)
    gb = orc.backward(o, d, b)
    gab = orc.backward(o, d, 2 * a - b)
    for x, y, z in zip(ga[:3], gb[:3], gab[:3]):
        assert np.abs(2 * x - y - z).max() < 1e-12
