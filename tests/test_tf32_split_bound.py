"""The error bound behind the FP32 path's split-TF32 products, checked in
exact (float64) arithmetic on the FP32 values.

Each FP32 operand x is held as hi = tf32(x) and lo = tf32(x - hi), both
rounded to nearest with ties away from zero by adding bit 12 and clearing the
low 13 bits.  A product a * w then runs as lo_a hi_w + hi_a lo_w + hi_a hi_w
with the lo * lo term dropped.  The claims: x - hi is exact in FP32, hi + lo
matches x to 2^-22 relative, and the three products match a * w to 2^-21
relative, far below the FP32 path's 1e-4 bar."""
import numpy as np


def _tf32_rna(x32: np.ndarray) -> np.ndarray:
    u = x32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return r.view(np.float32)


def _split(x32):
    hi = _tf32_rna(x32)
    d = (x32 - hi).astype(np.float32)  # FP32 subtraction
    lo = _tf32_rna(d)
    return hi, d, lo


def test_split_parts_are_tf32_and_close():
    rng = np.random.default_rng(0)
    # magnitudes of the MLP's weights and activations, and a wide range around them
    x = (rng.standard_normal(200_000) * np.exp(rng.uniform(-12, 4, 200_000))).astype(np.float32)
    hi, d, lo = _split(x)
    assert np.all(hi.view(np.uint32) & 0x1FFF == 0)
    assert np.all(lo.view(np.uint32) & 0x1FFF == 0)
    # x - hi is exact in FP32
    assert np.array_equal(d.astype(np.float64), x.astype(np.float64) - hi.astype(np.float64))
    # hi is within half a TF32 unit of x, lo within half a unit of x - hi
    rel_hi = np.abs(x.astype(np.float64) - hi) / np.abs(x.astype(np.float64))
    assert rel_hi.max() <= 2.0 ** -11
    rel = np.abs(x.astype(np.float64) - hi - lo) / np.abs(x.astype(np.float64))
    assert rel.max() <= 2.0 ** -22


def test_three_products_match_the_fp32_product():
    rng = np.random.default_rng(1)
    a = rng.uniform(-3, 3, 200_000).astype(np.float32)
    w = rng.uniform(-0.3, 0.3, 200_000).astype(np.float32)
    ah, _, al = _split(a)
    wh, _, wl = _split(w)
    exact = a.astype(np.float64) * w.astype(np.float64)
    three = (al.astype(np.float64) * wh + ah.astype(np.float64) * wl + ah.astype(np.float64) * wh)
    rel = np.abs(three - exact) / np.abs(exact)
    assert rel.max() <= 2.0 ** -21
    # one TF32 product alone is far coarser: the split is what keeps FP32 accuracy
    one = ah.astype(np.float64) * wh
    assert (np.abs(one - exact) / np.abs(exact)).max() > 2.0 ** -13


def test_rounding_is_to_nearest_ties_away():
    # 1 + 2^-11 is exactly half a TF32 unit above 1: rounds away from zero to
    # 1 + 2^-10; just below the half rounds down; signs are symmetric
    vals = np.array([1 + 2.0 ** -11, 1 + 2.0 ** -11 - 2.0 ** -23, -(1 + 2.0 ** -11), 3.0], np.float32)
    got = _tf32_rna(vals)
    assert got[0] == np.float32(1 + 2.0 ** -10)
    assert got[1] == np.float32(1.0)
    assert got[2] == np.float32(-(1 + 2.0 ** -10))
    assert got[3] == np.float32(3.0)
