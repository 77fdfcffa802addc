"""FP32 shading on the tensor cores as split TF32 (k_encode_tc<FP32> +
k_mlp_tf32): every FP32 input and weight is carried as a TF32 hi part and a
TF32 lo part and each layer's product as lo*hi + hi*lo + hi*hi (kind::tf32,
FP32 accumulation), which keeps FP32-level accuracy.  This path runs
whenever the render workspace holds operand tiles; the FP32 SIMT kernel
(k_shade_f32_ws) runs otherwise.  Both are held to the FP32 bar against the
FP64 oracle (1e-4 max-abs), and to each other within 2e-5, five times
tighter than that bar and far below the BF16 path's error (about 1e-3)."""
import os

import numpy as np
import pytest

import oracle
from paper_2303_04086_gb300 import synth

pytestmark = pytest.mark.gpu

RGBA_TOL = 1e-4    # FP32 path vs FP64 oracle, max-abs
PATHS_TOL = 2e-5   # split-TF32 tensor-core shade vs FP32 SIMT shade, max-abs


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04086_gb300 import build
    build.build()
    return torch


class _no_tiles:
    """INOLF_TC_CHUNK_ROWS=0 for a block: no operand tiles, so FP32 shades
    on the CUDA cores."""

    def __enter__(self):
        self.old = os.environ.get("INOLF_TC_CHUNK_ROWS")
        os.environ["INOLF_TC_CHUNK_ROWS"] = "0"

    def __exit__(self, *exc):
        if self.old is None:
            os.environ.pop("INOLF_TC_CHUNK_ROWS", None)
        else:
            os.environ["INOLF_TC_CHUNK_ROWS"] = self.old


def _both(torch, inolf, obj, cams, W, H):
    inolf.stats_enable(True)
    inolf.stats_reset()
    tc = inolf.render(obj, cams, W, H, "fp32").cpu().numpy()
    st = inolf.stats_read()
    with _no_tiles():
        simt = inolf.render(obj, cams, W, H, "fp32").cpu().numpy()
    inolf.stats_enable(False)
    torch.cuda.synchronize()
    # the tensor-core path really ran for the first render
    assert st.get("k_mlp_tc_f32", {}).get("launches", 0) > 0
    assert st.get("k_shade_f32", {}).get("launches", 0) == 0
    return tc, simt


@pytest.mark.parametrize("fp16,seed", [(False, 0), (True, 1)])
def test_fp32_tensor_cores_against_oracle_and_simt(torch_cuda, fp16, seed, record_property):
    from paper_2303_04086_gb300 import inolf
    torch = torch_cuda
    scene = synth.tiny_scene(seed=seed, fp16=fp16)
    obj = inolf.object_create(scene)
    orc = oracle.Oracle(scene)
    cams = synth.ring_cameras(3, 2.9)
    W, H = 160, 112  # 3 x 17 920 rays: many 128-row tiles and a ragged last pair
    tc, simt = _both(torch, inolf, obj, cams, W, H)
    worst = 0.0
    for v in range(len(cams)):
        ref = orc.render_pixels(cams[v], W, H)
        assert ref["missing"] == 0
        want = ref["rgba"].reshape(H, W, 4)
        hit = ref["tri"].reshape(H, W) >= 0
        assert hit.sum() > 3000
        assert np.all(tc[v][~hit] == 0)
        worst = max(worst, float(np.abs(tc[v] - want).max()))
        assert np.abs(simt[v] - want).max() <= RGBA_TOL
    d = float(np.abs(tc - simt).max())
    record_property("max_abs_vs_oracle", worst)
    record_property("max_abs_vs_simt", d)
    assert worst <= RGBA_TOL
    assert d <= PATHS_TOL


def test_fp32_tensor_cores_density_cube_object(torch_cuda):
    # the decoupled variant: alpha_c as the last input (d_in = L F + 17, so
    # K1 = 56 after padding) and c = c_d + tint c_s in the MLP kernel's store
    from paper_2303_04086_gb300 import inolf
    torch = torch_cuda
    obj = inolf.object_create(synth.tiny_density_scene(seed=0))
    cams = synth.ring_cameras(2, 2.7)
    tc, simt = _both(torch, inolf, obj, cams, 144, 96)
    assert (tc[..., 3] > 0).sum() > 1000
    assert np.isfinite(tc).all()
    assert float(np.abs(tc - simt).max()) <= PATHS_TOL


def test_fp32_tensor_cores_explicit_rays_and_tile_ranges(torch_cuda):
    # explicit rays: one sub-range, many sub-ranges (a tile region of 700
    # rows of 128 B holds 768-row ranges of the 96-byte FP32 rows of this
    # scene), and the FP32 SIMT kernel, all against the oracle
    from paper_2303_04086_gb300 import inolf
    torch = torch_cuda
    scene = synth.tiny_scene(seed=2)
    obj = inolf.object_create(scene)
    orc = oracle.Oracle(scene)
    o, d = oracle.raygen(synth.camera((0.4, 0.3, 2.9)), 128, 96)
    rng = np.random.default_rng(5)
    idx = rng.permutation(len(o))[:7001]
    o, d = np.ascontiguousarray(o[idx]), np.ascontiguousarray(d[idx])
    ref = orc.render_rays(o, d)
    assert ref["missing"] == 0
    ot = torch.tensor(o, dtype=torch.float32, device="cuda")
    dt = torch.tensor(d, dtype=torch.float32, device="cuda")
    out = {}
    out["tc"] = inolf.render_rays(obj, ot, dt, "fp32").cpu().numpy()
    old = os.environ.get("INOLF_TC_CHUNK_ROWS")
    try:
        os.environ["INOLF_TC_CHUNK_ROWS"] = "700"
        out["tc_ranges"] = inolf.render_rays(obj, ot, dt, "fp32").cpu().numpy()
    finally:
        if old is None:
            os.environ.pop("INOLF_TC_CHUNK_ROWS", None)
        else:
            os.environ["INOLF_TC_CHUNK_ROWS"] = old
    with _no_tiles():
        out["simt"] = inolf.render_rays(obj, ot, dt, "fp32").cpu().numpy()
    torch.cuda.synchronize()
    assert np.array_equal(out["tc"], out["tc_ranges"])  # the same rows through the same MMAs
    for k, v in out.items():
        assert np.abs(v - ref["rgba"]).max() <= RGBA_TOL, k
    assert np.abs(out["tc"] - out["simt"]).max() <= PATHS_TOL
