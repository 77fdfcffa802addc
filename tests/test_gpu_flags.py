"""Device-side failure flags reach the caller (no GPU fault involved).

With the test-only injection INOLF_INJECT_RING_STALL the gather warps of the
warp-specialised FP32 shade kernel never hand their tiles to the MLP warps, so
every hand-over wait runs out after the (shortened) limit and the kernel sets
INOLF_FLAG_WAIT_TIMEOUT and returns.  The flag must be visible through
inolf_workspace_flags for the asynchronous calls, turned into INOLF_E_TIMEOUT
by the calls that synchronise (inolf_render_host, the allocation-free entry
point), and the context must stay usable: the next call, without injection,
matches the oracle with its flags clear.  The FP32 shade runs on the CUDA
cores (k_shade_f32_ws) only when the workspace carries no operand tiles, so
the injected calls switch the tiles off (INOLF_TC_CHUNK_ROWS=0)."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(tiny):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04086_gb300 import build, inolf
    build.build()
    return torch, inolf, inolf.object_create(tiny)


def test_wait_timeout_is_reported_and_the_context_survives(env, tiny_oracle, tiny_cam):
    torch, inolf, obj = env
    W = H = 128
    ws = torch.empty((inolf.render_workspace_bytes(W * H) + 15) // 16 * 4, dtype=torch.int32, device="cuda")
    rgba = torch.empty((1, H, W, 4), device="cuda")
    checking = inolf._check_flags
    inolf.check_device_flags(False)
    old_rows = os.environ.get("INOLF_TC_CHUNK_ROWS")
    os.environ["INOLF_TC_CHUNK_ROWS"] = "0"
    try:
        inolf.set_wait_limit_ns(1_000_000)  # 1 ms
        inolf.set_fault_injection(inolf.INJECT_RING_STALL)
        inolf.render(obj, tiny_cam[None], W, H, "fp32", rgba_out=rgba, workspace=ws)
        assert inolf.workspace_flags(ws) == inolf.FLAG_WAIT_TIMEOUT
        with pytest.raises(inolf.InolfError) as e:
            inolf._check(inolf.lib().inolf_workspace_flags(ws.data_ptr(), None, None))
        assert e.value.status == inolf.E_INVALID  # NULL flags pointer
        with pytest.raises(inolf.InolfError) as e:
            inolf.render_host(obj, tiny_cam[None], W, H, "fp32")
        assert e.value.status == inolf.E_TIMEOUT
        o, d = (torch.from_numpy(a).cuda() for a in __import__("oracle").raygen(tiny_cam, W, H))
        with pytest.raises(inolf.InolfError) as e:
            inolf.render_rays_noalloc(obj, o, d, "fp32")
        assert e.value.status == inolf.E_TIMEOUT
        assert "bounded wait" in inolf.last_error()
    finally:
        inolf.set_fault_injection(0)
        inolf.set_wait_limit_ns(0)
        inolf.check_device_flags(checking)
        if old_rows is None:
            os.environ.pop("INOLF_TC_CHUNK_ROWS", None)
        else:
            os.environ["INOLF_TC_CHUNK_ROWS"] = old_rows
    # the context is intact: the same render, without injection, is right
    tri = torch.empty((1, H, W), dtype=torch.int32, device="cuda")
    inolf.render(obj, tiny_cam[None], W, H, "fp32", rgba_out=rgba, tri_out=tri, workspace=ws)
    assert inolf.workspace_flags(ws) == 0
    ref = tiny_oracle.render_pixels(tiny_cam, W, H)
    assert np.array_equal(tri.cpu().numpy().ravel(), ref["tri"])
    assert np.abs(rgba.cpu().numpy().reshape(-1, 4) - ref["rgba"]).max() <= 1e-4
