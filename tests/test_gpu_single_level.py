"""L = 1, the paper's single-resolution PSH encoding (Sec. 4.1), as a special
case of the multi-level path: forward FP32 / BF16 / FP8 and backward against
the FP64 oracle for PSH-128 and PSH-512 single-level scenes."""
import numpy as np
import pytest

import oracle
from paper_2303_04086_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[128, 512])
def single(request):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04086_gb300 import build, inolf
    build.build()
    sc = synth.tiny_scene(seed=3, resolutions=(request.param,), band=0.02)
    return torch, inolf, sc, inolf.object_create(sc), oracle.Oracle(sc)


def test_single_level_forward(single):
    torch, inolf, sc, obj, orc = single
    assert sc.n_levels == 1 and sc.d_in == 18
    cam = synth.camera((0.4, 0.3, 2.8))
    ref = orc.render_pixels(cam, 96, 80)
    assert ref["missing"] == 0
    hit = ref["tri"] >= 0
    tri = torch.empty((1, 80, 96), dtype=torch.int32, device="cuda")
    got = inolf.render(obj, cam[None], 96, 80, "fp32", tri_out=tri).cpu().numpy().reshape(-1, 4)
    assert np.array_equal(tri.cpu().numpy().ravel(), ref["tri"])
    assert np.abs(got - ref["rgba"]).max() <= 1e-4
    bf = inolf.render(obj, cam[None], 96, 80, "bf16").cpu().numpy().reshape(-1, 4)
    assert np.abs(bf - ref["rgba"]).max() <= 1e-2
    inolf.calibrate_fp8(obj, cam[None], 96, 80)
    f8 = inolf.render(obj, cam[None], 96, 80, "fp8").cpu().numpy().reshape(-1, 4)
    mse = np.mean((f8[hit] - ref["rgba"][hit]) ** 2)
    assert 10 * np.log10(1 / mse) >= 38.0


def test_single_level_backward(single):
    torch, inolf, sc, obj, orc = single
    cam = synth.camera((0.0, 0.0, 3.0))
    o, d = oracle.raygen(cam, 64, 64)
    r = orc.render_rays(o, d)
    sel = np.nonzero(r["tri"] >= 0)[0][:500]
    o, d = o[sel], d[sel]
    g = np.random.default_rng(0).normal(size=(len(o), 4))
    gt = [torch.zeros((obj.table_rows(0), 2), device="cuda")]
    gw = [torch.zeros((64, obj.d_in), device="cuda"), torch.zeros((64, 64), device="cuda"),
          torch.zeros((4, 64), device="cuda")]
    inolf.backward(obj, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(),
                   torch.from_numpy(g.astype(np.float32)).cuda(), gt, *gw)
    r1, r2, r3, rf = orc.backward(o, d, g)
    for a, b in zip([x.cpu().numpy() for x in gw], (r1, r2, r3)):
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 1e-4
    got = gt[0].cpu().numpy()[obj.hashes[0].slot_of]
    assert np.linalg.norm(got - rf[0]) / np.linalg.norm(rf[0]) <= 1e-4
