"""The BF16 / FP8 shade runs either as one fused kernel or, when the render
workspace holds operand tiles, as an encode kernel and an MLP kernel over
sub-ranges of the hit list.  Both encode each hit with the same code and run
the same MMAs and epilogues, so their frames must agree bit for bit:
  - split with the default workspace (one sub-range per launch chunk);
  - split with sub-ranges of a few hundred rows (many ranges, a ragged last
    range, launches past the last hit);
  - a small workspace (room for the hit records of the whole call only):
    renders take one view per chunk with the operand tiles that one view's
    hit records leave room for, explicit rays run fused (no room for 256
    rows of tiles);
  - fused, with the operand tiles switched off (INOLF_TC_CHUNK_ROWS=0).
Mesh objects and density-cube objects (alpha_c input, c = c_d + tint c_s)
are both covered; the accuracy of these paths against the oracle is checked
by the precision tests."""
import os

import numpy as np
import pytest

from paper_2303_04086_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04086_gb300 import build
    build.build()
    return torch


class _env:
    """Sets INOLF_TC_CHUNK_ROWS for the duration of a block."""

    def __init__(self, value):
        self.value = value

    def __enter__(self):
        self.old = os.environ.get("INOLF_TC_CHUNK_ROWS")
        if self.value is None:
            os.environ.pop("INOLF_TC_CHUNK_ROWS", None)
        else:
            os.environ["INOLF_TC_CHUNK_ROWS"] = str(self.value)

    def __exit__(self, *exc):
        if self.old is None:
            os.environ.pop("INOLF_TC_CHUNK_ROWS", None)
        else:
            os.environ["INOLF_TC_CHUNK_ROWS"] = self.old


def _frames(torch, inolf, obj, cams, W, H, prec):
    n = len(cams) * W * H
    hit_bytes = 12 * n + 256
    out = {}
    with _env(None):
        out["split"] = inolf.render(obj, cams, W, H, prec).cpu().numpy()
        small = torch.empty((hit_bytes + 15) // 16 * 4, dtype=torch.int32, device="cuda")
        out["small_ws"] = inolf.render(obj, cams, W, H, prec, workspace=small).cpu().numpy()
    with _env(300):  # tiles for 300 rows of 128 B: ranges of 512 (BF16) or 1024 (FP8) hits
        out["split_many"] = inolf.render(obj, cams, W, H, prec).cpu().numpy()
    with _env(0):
        out["fused_off"] = inolf.render(obj, cams, W, H, prec).cpu().numpy()
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_split_equals_fused_mesh(torch_cuda, prec):
    from paper_2303_04086_gb300 import inolf
    torch = torch_cuda
    scene = synth.tiny_scene(seed=0, fp16=True)
    obj = inolf.object_create(scene)
    cams = synth.ring_cameras(3, 3.0)
    W, H = 200, 120
    if prec == "fp8":
        inolf.calibrate_fp8(obj, cams[:1], W, H)
    out = _frames(torch, inolf, obj, cams, W, H, prec)
    ref = out["split"]
    hit = ref[..., 3] > 0
    assert hit.sum() > 10000  # enough hits for many 256-row ranges
    assert np.isfinite(ref).all()
    for k, v in out.items():
        assert np.array_equal(v, ref), k


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_split_equals_fused_density_cubes(torch_cuda, prec):
    from paper_2303_04086_gb300 import inolf
    torch = torch_cuda
    scene = synth.tiny_density_scene(seed=0)
    obj = inolf.object_create(scene)
    cams = synth.ring_cameras(2, 2.7)
    W, H = 160, 96
    if prec == "fp8":
        inolf.calibrate_fp8(obj, cams[:1], W, H)
    out = _frames(torch, inolf, obj, cams, W, H, prec)
    ref = out["split"]
    assert (ref[..., 3] > 0).sum() > 1000
    for k, v in out.items():
        assert np.array_equal(v, ref), k


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_split_equals_fused_explicit_rays(torch_cuda, prec):
    """Explicit rays (inolf_render_rays): the split path over one and over many
    sub-ranges, the fused kernel, and the allocation-free entry point (its
    fixed scratch) give the same colours."""
    from paper_2303_04086_gb300 import inolf
    import oracle
    torch = torch_cuda
    scene = synth.tiny_scene(seed=1, fp16=False)
    obj = inolf.object_create(scene)
    cams = synth.ring_cameras(2, 2.8)
    W, H = 96, 80
    if prec == "fp8":
        inolf.calibrate_fp8(obj, cams[:1], W, H)
    o, d = oracle.raygen(cams[1], W, H)
    rng = np.random.default_rng(3)
    idx = rng.permutation(len(o))[:5000]  # scattered rays, ragged count
    o = torch.tensor(np.ascontiguousarray(o[idx]), dtype=torch.float32, device="cuda")
    d = torch.tensor(np.ascontiguousarray(d[idx]), dtype=torch.float32, device="cuda")
    n = o.shape[0]
    out = {}
    with _env(None):
        out["default"] = inolf.render_rays(obj, o, d, prec).cpu().numpy()
        small = torch.empty((12 * n + 256 + 15) // 16 * 4, dtype=torch.int32, device="cuda")
        out["small_ws"] = inolf.render_rays(obj, o, d, prec, workspace=small).cpu().numpy()
        out["noalloc"] = inolf.render_rays_noalloc(obj, o, d, prec).cpu().numpy()
    with _env(300):
        out["split_many"] = inolf.render_rays(obj, o, d, prec).cpu().numpy()
    torch.cuda.synchronize()
    ref = out["default"]
    assert (ref[:, 3] > 0).sum() > 1000
    for k, v in out.items():
        assert np.array_equal(v, ref), k


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_split_with_no_hits_and_a_ragged_hit_count(torch_cuda, prec):
    """A view with no hit at all (every encode / MLP launch returns at once)
    beside a view with a few hits: misses are exact zeros, the failure flags
    stay clear, and the hit view matches the fused kernel."""
    from paper_2303_04086_gb300 import inolf
    torch = torch_cuda
    scene = synth.tiny_scene(seed=2, fp16=True)
    obj = inolf.object_create(scene)
    W, H = 120, 72
    away = synth.camera((0.0, 0.0, 3.0), target=(0.0, 0.0, 6.0))  # looks away from the object
    far = synth.camera((0.0, 0.0, 12.0))                          # the object covers a few pixels
    cams = np.stack([away, far])
    if prec == "fp8":
        inolf.calibrate_fp8(obj, cams[1:], W, H)
    with _env(None):
        split = inolf.render(obj, cams, W, H, prec).cpu().numpy()
        small = torch.empty((12 * 2 * W * H + 256 + 15) // 16 * 4, dtype=torch.int32, device="cuda")
        fused = inolf.render(obj, cams, W, H, prec, workspace=small).cpu().numpy()
    torch.cuda.synchronize()
    assert np.all(split[0] == 0)
    n_hit = int((split[1][..., 3] > 0).sum())
    assert 0 < n_hit < 2000
    assert np.array_equal(split, fused)
