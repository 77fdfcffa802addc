"""GPU parity of the forward path (FP32) against the FP64 oracle, through the
C ABI: closest triangle id and t bit-exact, Eq. 1 slots bit-exact,
interpolated features within 1e-6, RGBA within 1e-4 max-abs."""
import numpy as np
import pytest

import oracle
from paper_2303_04086_gb300 import synth

pytestmark = pytest.mark.gpu

RGBA_TOL = 1e-4   # FP32 path vs FP64 oracle, max-abs
FEAT_TOL = 1e-6


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04086_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def tiny_obj(torch_cuda, tiny):
    from paper_2303_04086_gb300 import inolf
    return inolf.object_create(tiny)


def _render(inolf, obj, cams, W, H, prec="fp32", ws_rays=None):
    import torch
    nv = len(cams)
    tri = torch.empty((nv, H, W), dtype=torch.int32, device="cuda")
    t = torch.empty((nv, H, W), dtype=torch.float32, device="cuda")
    ws = None
    if ws_rays is not None:
        nb = inolf.render_workspace_bytes(ws_rays)
        ws = torch.empty((nb + 15) // 16 * 4, dtype=torch.int32, device="cuda")
    rgba = inolf.render(obj, cams, W, H, prec, tri_out=tri, t_out=t, workspace=ws)
    torch.cuda.synchronize()
    return rgba.cpu().numpy(), tri.cpu().numpy(), t.cpu().numpy()


def test_tiny_view_matches_oracle(torch_cuda, tiny, tiny_obj, tiny_oracle, tiny_cam):
    from paper_2303_04086_gb300 import inolf
    rgba, tri, t = _render(inolf, tiny_obj, tiny_cam[None], 128, 128)
    ref = tiny_oracle.render_pixels(tiny_cam, 128, 128)
    assert np.array_equal(tri.ravel(), ref["tri"])
    assert np.array_equal(t.ravel().view(np.int32), ref["t"].view(np.int32))
    err = np.abs(rgba.reshape(-1, 4) - ref["rgba"]).max()
    assert err <= RGBA_TOL, err
    hit = ref["tri"] >= 0
    assert 0.5 < hit.mean() < 0.65
    assert np.all(rgba.reshape(-1, 4)[~hit] == 0)


@pytest.mark.parametrize("W,H,nv", [(37, 23, 3), (1, 1, 1), (17, 129, 2)])
def test_ragged_sizes_and_views(torch_cuda, tiny, tiny_obj, tiny_oracle, W, H, nv):
    from paper_2303_04086_gb300 import inolf
    cams = synth.ring_cameras(5, 2.7)[:nv]
    rgba, tri, t = _render(inolf, tiny_obj, cams, W, H)
    for v in range(nv):
        ref = tiny_oracle.render_pixels(cams[v], W, H)
        assert np.array_equal(tri[v].ravel(), ref["tri"])
        assert np.array_equal(t[v].ravel().view(np.int32), ref["t"].view(np.int32))
        assert np.abs(rgba[v].reshape(-1, 4) - ref["rgba"]).max() <= RGBA_TOL


def test_small_workspace_chunks_views(torch_cuda, tiny, tiny_obj, tiny_oracle):
    # a workspace for 2 of the 7 views: the views are rendered in chunks, and
    # the FP32 shade runs on the CUDA cores because the workspace has no room
    # for operand tiles; with the full workspace it runs on the tensor cores
    # (split TF32).  Hits are bit-exact either way, colours agree within the
    # split-TF32 tolerance and both meet the FP32 bar against the oracle.
    from paper_2303_04086_gb300 import inolf
    cams = synth.ring_cameras(7, 3.0)
    full, tri_f, t_f = _render(inolf, tiny_obj, cams, 40, 30)
    part, tri_p, t_p = _render(inolf, tiny_obj, cams, 40, 30, ws_rays=40 * 30 * 2)  # 2 views per chunk
    assert np.array_equal(tri_f, tri_p) and np.array_equal(t_f.view(np.int32), t_p.view(np.int32))
    assert np.abs(full - part).max() <= 2e-5
    for v in range(len(cams)):
        ref = tiny_oracle.render_pixels(cams[v], 40, 30)
        assert np.abs(part[v].reshape(-1, 4) - ref["rgba"]).max() <= RGBA_TOL
        assert np.abs(full[v].reshape(-1, 4) - ref["rgba"]).max() <= RGBA_TOL


def _random_rays(n, seed, inside_frac=0.1):
    rng = np.random.default_rng(seed)
    eye = rng.normal(size=(n, 3))
    eye = 2.6 * eye / np.linalg.norm(eye, axis=1, keepdims=True)
    k = int(n * inside_frac)
    eye[:k] *= 0.2  # origins inside the proxy: the two-sided test hits the inside
    tgt = rng.uniform(-1.1, 1.1, size=(n, 3))
    d = tgt - eye
    # a few axis-aligned directions (zero components)
    if n >= k + 6:
        d[k:k + 6] = [[1, 0, 0], [0, -1, 0], [0, 0, 1], [-1, 0, 0], [0, 1, 0], [0, 0, -1]]
        eye[k:k + 6] = [[-3, 0.1, 0.2], [0.05, 3, -0.1], [0.3, 0.2, -3], [3, 0, 0], [0, -3, 0], [0, 0, 3]]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return eye.astype(np.float32), d.astype(np.float32)


@pytest.mark.parametrize("n", [1, 255, 257, 5000])
def test_explicit_rays_match_oracle(torch_cuda, tiny, tiny_obj, tiny_oracle, n):
    import torch
    from paper_2303_04086_gb300 import inolf
    o, d = _random_rays(n, n)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    tri = torch.empty(n, dtype=torch.int32, device="cuda")
    t = torch.empty(n, dtype=torch.float32, device="cuda")
    rgba = inolf.render_rays(tiny_obj, to, td, tri_out=tri, t_out=t).cpu().numpy()
    ref = tiny_oracle.render_rays(o, d)
    bt, btt, _ = oracle.hit_brute(tiny.vertices, tiny.triangles, o, d)
    assert np.array_equal(tri.cpu().numpy(), bt)
    assert np.array_equal(tri.cpu().numpy(), ref["tri"])
    assert np.array_equal(t.cpu().numpy().view(np.int32), btt.view(np.int32))
    assert np.abs(rgba - ref["rgba"]).max() <= RGBA_TOL


def test_edge_and_vertex_rays_are_counted_and_exact(torch_cuda, tiny, tiny_obj, tiny_oracle, record_property):
    # rays aimed at edge midpoints, vertices and centroids of 200 triangles:
    # the winning hit of most lies within 1e-6 (barycentric) of an edge.  They
    # are counted and reported, and the triangle id and t still match the
    # oracle bit for bit (both sides take the same FP32 test).
    import torch
    from paper_2303_04086_gb300 import inolf
    V, F = tiny.vertices.astype(np.float64), tiny.triangles
    rng = np.random.default_rng(11)
    tg = []
    for f in rng.choice(len(F), 200, replace=False):
        a, b, c = V[F[f]]
        tg += [(a + b) / 2, (b + c) / 2, (c + a) / 2, a, (a + b + c) / 3]
    tg = np.array(tg)
    eye = tg * 2.5 + rng.normal(scale=0.05, size=tg.shape)
    d = tg - eye
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o, d = eye.astype(np.float32), d.astype(np.float32)
    n = len(o)
    tri = torch.empty(n, dtype=torch.int32, device="cuda")
    t = torch.empty(n, dtype=torch.float32, device="cuda")
    rgba = inolf.render_rays(tiny_obj, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), tri_out=tri,
                             t_out=t).cpu().numpy()
    ref = tiny_oracle.render_rays(o, d)
    n_edge = int(ref["near_edge"].sum())
    record_property("near_edge_rays", n_edge)
    print(f"near-edge rays: {n_edge} of {n}")
    assert n_edge > n // 2
    assert np.array_equal(tri.cpu().numpy(), ref["tri"])
    assert np.array_equal(t.cpu().numpy().view(np.int32), ref["t"].view(np.int32))
    assert np.abs(rgba - ref["rgba"]).max() <= RGBA_TOL


def test_encode_slots_and_features(torch_cuda, tiny, tiny_obj, tiny_oracle, tiny_cam):
    import torch
    from paper_2303_04086_gb300 import inolf
    o, d = oracle.raygen(tiny_cam, 128, 128)
    r = tiny_oracle.render_rays(o, d, with_E=True)
    hit = np.nonzero(r["tri"] >= 0)[0]
    o, d = o[hit], d[hit]
    n, L = len(o), tiny.n_levels
    slots = torch.full((n, L, 8), 0xFFFFFFFF, dtype=torch.int64, device="cuda").to(torch.int32)
    feats = torch.zeros((n, L * 2), dtype=torch.float32, device="cuda")
    inolf.encode_rays(tiny_obj, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), slots, feats)
    slots = slots.cpu().numpy().view(np.uint32).astype(np.int64)
    idx, w = tiny_oracle.corners(o, d, r["t"][hit])
    assert np.all(idx >= 0)
    for l in range(L):
        h = tiny_obj.hashes[l]
        keys = synth.unpack_keys(tiny.keys[l])
        expect = oracle.psh_slots(h.phi, h.m, h.r, keys)[idx[:, l, :]]
        assert np.array_equal(slots[:, l, :], expect)
    assert np.abs(feats.cpu().numpy() - r["E"][hit, :L * 2]).max() <= FEAT_TOL


def test_fp16_tables(torch_cuda, tiny_oracle, tiny_cam):
    from paper_2303_04086_gb300 import inolf
    sc = synth.tiny_scene(seed=0, fp16=True)
    obj = inolf.object_create(sc)
    ref = oracle.Oracle(sc).render_pixels(tiny_cam, 128, 128)
    rgba, tri, t = _render(inolf, obj, tiny_cam[None], 128, 128)
    assert np.array_equal(tri.ravel(), ref["tri"])
    assert np.abs(rgba.reshape(-1, 4) - ref["rgba"]).max() <= RGBA_TOL


def test_empty_batches(torch_cuda, tiny_obj):
    import torch
    from paper_2303_04086_gb300 import inolf
    o = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    out = inolf.render_rays(tiny_obj, o, o)
    assert out.shape == (0, 4)
    with pytest.raises(inolf.InolfError):
        inolf.render(tiny_obj, np.zeros((1, 13), np.float32), 0, 4)


@pytest.mark.parametrize("views_per_chunk,pinned", [(2, True), (1, True), (3, False)])
def test_render_host_equals_device_render(torch_cuda, tiny, tiny_obj, views_per_chunk, pinned):
    # frames rendered into host memory are the device render's, bit for bit:
    # pinned memory is stored to directly by the kernels; pageable memory goes
    # through the two staging halves (the copies of chunk c overlap the
    # rendering of chunk c + 1; 7 views force slot reuse)
    import torch
    from paper_2303_04086_gb300 import inolf
    cams = synth.ring_cameras(7, 2.8)
    W, H = 37, 23
    dev = inolf.render(tiny_obj, cams, W, H).cpu().numpy()
    host = torch.empty((7, H, W, 4), dtype=torch.float32, pin_memory=pinned)
    staging = torch.empty((2 * views_per_chunk * H * W * 4,), dtype=torch.float32, device="cuda")
    out = inolf.render_host(tiny_obj, cams, W, H, "fp32", host_out=host, staging=staging)
    assert np.array_equal(out.numpy(), dev)


def test_render_host_rejects_small_staging(torch_cuda, tiny, tiny_obj):
    import torch
    from paper_2303_04086_gb300 import inolf
    cams = synth.ring_cameras(2, 2.8)
    staging = torch.empty((37 * 23 * 4,), dtype=torch.float32, device="cuda")  # one view, not two
    with pytest.raises(inolf.InolfError) as e:
        inolf.render_host(tiny_obj, cams, 37, 23, "fp32", staging=staging)
    assert e.value.status == inolf.E_INVALID
