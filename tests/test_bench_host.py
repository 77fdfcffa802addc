"""Host arithmetic of the bench line (no GPU): the per-kernel roofline entries
of the FP32 split shade and the per-hit work figures they use."""
from types import SimpleNamespace

import pytest

import bench


@pytest.fixture
def full_scene():
    # the benchmark scene's shape: 16 levels, F = 2 FP32 features, d_in = 48
    return SimpleNamespace(n_levels=16, d_in=48, feature_fp16=False)


def test_per_hit_work_figures(full_scene):
    s = full_scene
    assert bench.algorithmic_bytes_per_hit(s) == 16 * 8 * (2 * 4 + 4) == 1536
    assert bench.mlp_flops_per_hit(s) == 2 * (64 * 48 + 64 * 64 + 4 * 64) == 14848
    assert bench.tf32_k1(s) == 48 and bench.tf32_k1(SimpleNamespace(d_in=49)) == 56
    assert bench.tf32_row_bytes(s) == 192
    # three products per layer, layer 1 at K1 columns, layer 3 at 16 outputs
    assert bench.tf32x3_flops_per_hit(s) == 3 * 2 * (64 * 48 + 64 * 64 + 16 * 64) == 49152
    assert bench.encode_bytes_per_hit(s) == 1536 + 8 + 192
    fp16 = SimpleNamespace(n_levels=4, d_in=24, feature_fp16=True)
    assert bench.algorithmic_bytes_per_hit(fp16) == 4 * 8 * (2 * 2 + 4) == 256


def test_fp32_split_shade_rooflines(full_scene):
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
    steps, n_hit, n_rays = 5, 256_000_000, 530_000_000
    kernels = {"k_encode_tc_f32": {"launches": 190 * steps, "ms": 30.0 * steps},
               "k_mlp_tc_f32": {"launches": 190 * steps, "ms": 45.0 * steps},
               "k_trace": {"launches": steps, "ms": 31.0 * steps}}
    r = bench.kernel_rooflines(kernels, full_scene, n_rays, n_hit, steps, peaks)
    mlp = r["k_mlp_tc_f32"]
    want_tf = 49152 * n_hit / 0.045 / 1e12
    assert mlp["tensor_tflops"] == pytest.approx(want_tf)
    assert mlp["tf32_peak_tflops"] == pytest.approx(1900.0 * 1.1 / 2.25)
    assert mlp["frac_tf32_peak"] == pytest.approx(want_tf / (1900.0 * 1.1 / 2.25))
    assert mlp["mlp_tflops"] == pytest.approx(14848 * n_hit / 0.045 / 1e12)
    assert mlp["launches_per_step"] == 190
    enc = r["k_encode_tc_f32"]
    assert enc["gbs"] == pytest.approx((1536 + 8 + 192) * n_hit / 0.030 / 1e9)
    assert enc["frac_hbm"] == pytest.approx(enc["gbs"] / 6800.0)
    tr = r["k_trace"]
    assert tr["bound"] == "alu (issue)"
    assert tr["grays_per_s"] == pytest.approx(n_rays / 0.031 / 1e9)
