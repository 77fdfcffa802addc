"""Pins of the oracle's view encoding (real SH of degree <= 3 of the view
direction v that enters F_s, Sec. 4.2 Eq. 3) and of the MLP F_s itself."""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_sh_band0_closed_form():
    y = oracle.sh16(_unit(np.random.default_rng(0), 10))
    assert np.abs(y[:, 0] - 1.0 / (2.0 * math.sqrt(math.pi))).max() < 1e-15


def test_sh_band1_convention():
    # index l*l + l + m: (1,-1) ~ y, (1,0) ~ z, (1,1) ~ x, constant sqrt(3 / (4 pi))
    c = math.sqrt(3.0 / (4.0 * math.pi))
    d = _unit(np.random.default_rng(1), 20)
    y = oracle.sh16(d)
    assert np.abs(y[:, 1] - c * d[:, 1]).max() < 1e-14
    assert np.abs(y[:, 2] - c * d[:, 2]).max() < 1e-14
    assert np.abs(y[:, 3] - c * d[:, 0]).max() < 1e-14


def test_sh_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform phi: exact for the degree-6 products
    zs, wz = np.polynomial.legendre.leggauss(8)
    nphi = 16
    phis = 2 * math.pi * np.arange(nphi) / nphi
    dirs, w = [], []
    for z, wzz in zip(zs, wz):
        s = math.sqrt(1 - z * z)
        for ph in phis:
            dirs.append((s * math.cos(ph), s * math.sin(ph), z))
            w.append(wzz * 2 * math.pi / nphi)
    Y = oracle.sh16(np.array(dirs))
    G = (Y * np.array(w)[:, None]).T @ Y
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_sh_addition_theorem():
    # sum_m Y_lm(a) Y_lm(b) = (2l+1)/(4 pi) P_l(a . b)
    rng = np.random.default_rng(2)
    a, b = _unit(rng, 50), _unit(rng, 50)
    Ya, Yb = oracle.sh16(a), oracle.sh16(b)
    cosg = np.einsum("ij,ij->i", a, b)
    for l in range(4):
        sl = slice(l * l, (l + 1) * (l + 1))
        lhs = (Ya[:, sl] * Yb[:, sl]).sum(1)
        Pl = np.polynomial.legendre.legval(cosg, [0] * l + [1])
        assert np.abs(lhs - (2 * l + 1) / (4 * math.pi) * Pl).max() < 1e-13


def test_sh_matches_scipy_complex_harmonics():
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    d = _unit(np.random.default_rng(3), 40)
    th = np.arccos(np.clip(d[:, 2], -1, 1))
    ph = np.arctan2(d[:, 1], d[:, 0])
    Y = oracle.sh16(d)
    for l in range(4):
        for m in range(-l, l + 1):
            c = sp.sph_harm_y(l, abs(m), th, ph)  # includes the Condon-Shortley phase
            if m > 0:
                ref = math.sqrt(2) * (-1) ** m * c.real
            elif m < 0:
                ref = math.sqrt(2) * (-1) ** m * c.imag
            else:
                ref = c.real
            assert np.abs(Y[:, l * l + l + m] - ref).max() < 1e-12, (l, m)


def test_mlp_two_rays_hand_worked():
    rows = np.loadtxt(os.path.join(GOLDEN, "mlp_two_rays.txt"))
    W1 = np.array([[1, -1], [2, 1]], np.float64)
    W2 = np.array([[1, 1], [-1, 2]], np.float64)
    W3 = np.array([[1, -2]], np.float64)
    out = oracle.mlp(W1, W2, W3, rows[:, :2])
    ref = 1.0 / (1.0 + np.exp(-rows[:, 2]))
    assert np.abs(out[:, 0] - ref).max() < 1e-15


def test_mlp_zero_weights_give_one_half(tiny):
    w1 = np.zeros_like(tiny.w1); w2 = np.zeros_like(tiny.w2); w3 = np.zeros_like(tiny.w3)
    x = np.random.default_rng(4).normal(size=(5, tiny.d_in))
    assert np.all(oracle.mlp(w1, w2, w3, x) == 0.5)


def test_render_is_mlp_of_encoding(tiny, tiny_oracle, tiny_cam):
    # the renderer's output is F_s applied to [E(p), SH(v)] of the same ray
    o, d = oracle.raygen(tiny_cam, 32, 32)
    r = tiny_oracle.render_rays(o, d, with_E=True)
    hit = r["tri"] >= 0
    x = r["E"][hit]
    sh = oracle.sh16(d[hit].astype(np.float64))
    assert np.abs(x[:, tiny.n_levels * 2:] - sh).max() < 1e-15
    ref = oracle.mlp(tiny.w1, tiny.w2, tiny.w3, x)
    assert np.abs(ref - r["rgba"][hit]).max() < 1e-15
