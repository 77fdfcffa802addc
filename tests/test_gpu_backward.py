"""Backward pass (Sec. 4.2 "Training", Eq. 8) on the GPU, through the C ABI,
against the FP64 oracle: analytic gradient (global relative L2 <= 1e-4),
central finite differences of the FP64 model (per-entry relative error
<= 1e-3 where |g| > 1e-7, parameters whose +-eps crosses a ReLU kink
excluded), accumulation semantics, parameter reload, and a short training
run whose L2 loss decreases."""
import numpy as np
import pytest

import oracle
from paper_2303_04086_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(tiny):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04086_gb300 import build, inolf
    build.build()
    return torch, inolf, inolf.object_create(tiny)


def _hit_rays(orc, n, seed):
    cam = synth.camera((0.0, 0.0, 3.0))
    o, d = oracle.raygen(cam, 128, 128)
    r = orc.render_rays(o, d)
    hit = np.nonzero(r["tri"] >= 0)[0]
    sel = np.random.default_rng(seed).choice(hit, n, replace=False)
    return o[sel], d[sel]


def _gpu_grads(torch, inolf, obj, o, d, g):
    L = obj.L
    gt = [torch.zeros((obj.table_rows(l), 2), dtype=torch.float32, device="cuda") for l in range(L)]
    g1 = torch.zeros((64, obj.d_in), device="cuda")
    g2 = torch.zeros((64, 64), device="cuda")
    g3 = torch.zeros((4, 64), device="cuda")
    inolf.backward(obj, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(),
                   torch.from_numpy(np.ascontiguousarray(g, np.float32)).cuda(), gt, g1, g2, g3)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in gt], g1.cpu().numpy(), g2.cpu().numpy(), g3.cpu().numpy()


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("n,seed", [(64, 0), (3000, 1)])
def test_gradient_matches_oracle(env, tiny, tiny_oracle, n, seed):
    torch, inolf, obj = env
    o, d = _hit_rays(tiny_oracle, n, seed)
    if n > 64:  # add rays that miss
        o = np.concatenate([o, np.float32([[0, 3, 3]] * 50)])
        d = np.concatenate([d, np.float32([[0, 0, 1]] * 50)])
    target = np.random.default_rng(seed + 7).uniform(0, 1, (len(o), 4))
    y = tiny_oracle.render_rays(o, d)["rgba"]
    g = 2.0 * (y - target) / len(o)
    g[np.all(y == 0, axis=1)] = 0.0
    gt, g1, g2, g3 = _gpu_grads(torch, inolf, obj, o, d, g)
    r1, r2, r3, rf = tiny_oracle.backward(o, d, g)
    assert _rel_l2(g1, r1) <= 1e-4 and _rel_l2(g2, r2) <= 1e-4 and _rel_l2(g3, r3) <= 1e-4
    for l in range(tiny.n_levels):
        got = gt[l][obj.hashes[l].slot_of]  # slot order -> key order
        assert _rel_l2(got, rf[l]) <= 1e-4, l
        # slots no key maps to receive nothing
        mask = np.ones(len(gt[l]), bool)
        mask[obj.hashes[l].slot_of] = False
        assert np.all(gt[l][mask] == 0)


def test_gradient_against_finite_differences(env, tiny):
    torch, inolf, obj = env
    orc = oracle.Oracle(tiny)   # own copy: its parameters are perturbed
    o, d = _hit_rays(orc, 64, 3)
    rng = np.random.default_rng(4)
    target = rng.uniform(0, 1, (64, 4))

    def loss():
        y = orc.render_rays(o, d)["rgba"]
        return ((y - target) ** 2).sum() / 64

    y = orc.render_rays(o, d)["rgba"]
    gt, g1, g2, g3 = _gpu_grads(torch, inolf, obj, o, d, 2.0 * (y - target) / 64)
    z1_0, z2_0 = orc.preacts(o, d)
    params = [(0, 0, g1.ravel()), (1, 0, g2.ravel()), (2, 0, g3.ravel())]
    feat_grads = []
    for l in range(tiny.n_levels):
        feat_grads.append((3, l, gt[l][obj.hashes[l].slot_of].ravel()))
    checked = kinks = 0
    for which, level, g in params + feat_grads:
        theta = orc.param(which, level)
        idx = np.nonzero(np.abs(g) > 1e-7)[0] if which == 3 else np.arange(len(theta))
        idx = rng.choice(idx, min(40, len(idx)), replace=False)
        for i in idx:
            t0 = theta[i]
            eps = 1e-6 * max(1.0, abs(t0))
            theta[i] = t0 + eps
            lp = loss()
            zp = orc.preacts(o, d)
            theta[i] = t0 - eps
            lm = loss()
            zm = orc.preacts(o, d)
            theta[i] = t0
            if any(np.any(np.sign(a) != np.sign(b)) for a, b in [(zp[0], z1_0), (zp[1], z2_0), (zm[0], z1_0),
                                                                  (zm[1], z2_0)]):
                kinks += 1
                continue
            fd = (lp - lm) / (2 * eps)
            if abs(g[i]) > 1e-7:
                assert abs(g[i] - fd) <= 1e-3 * abs(fd) + 1e-9, (which, level, i, g[i], fd)
            checked += 1
    assert checked > 150 and kinks < checked // 5


def test_backward_accumulates(env, tiny, tiny_oracle):
    torch, inolf, obj = env
    o, d = _hit_rays(tiny_oracle, 200, 5)
    g = np.random.default_rng(6).normal(size=(200, 4)).astype(np.float32)
    L = obj.L
    gt = [torch.zeros((obj.table_rows(l), 2), device="cuda") for l in range(L)]
    gw = [torch.zeros((64, obj.d_in), device="cuda"), torch.zeros((64, 64), device="cuda"),
          torch.zeros((4, 64), device="cuda")]
    to, td, tg = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), torch.from_numpy(g).cuda()
    inolf.backward(obj, to, td, tg, gt, *gw)
    once = [t.clone() for t in gw]
    inolf.backward(obj, to, td, tg, gt, *gw)
    # atomics add the per-CTA partials in any order: equal up to FP32 rounding
    for a, b in zip(gw, once):
        assert float((a - 2 * b).norm() / (2 * b).norm()) < 1e-5


def test_load_params_round_trip(env, tiny):
    torch, inolf, _ = env
    obj = inolf.object_create(tiny)
    tables, w1, w2, w3 = obj.read_params()
    w1b = (w1 * 1.5).astype(np.float32)
    tb = [(t * -0.5).astype(np.float32) for t in tables]
    inolf.load_params(obj, [torch.from_numpy(t).cuda() for t in tb], torch.from_numpy(w1b).cuda(),
                      torch.from_numpy(w2).cuda(), torch.from_numpy(w3).cuda())
    t2, w1c, _, _ = obj.read_params()
    assert np.array_equal(w1c, w1b) and all(np.array_equal(a, b) for a, b in zip(t2, tb))
    # the render follows the new parameters (oracle with the same values)
    sc = synth.Scene(tiny.vertices, tiny.triangles, tiny.resolutions, tiny.keys,
                     [(f * -0.5).astype(np.float32) for f in tiny.features], w1b, tiny.w2, tiny.w3)
    cam = synth.camera((0.0, 0.0, 3.0))
    ref = oracle.Oracle(sc).render_pixels(cam, 64, 64)
    got = inolf.render(obj, cam[None], 64, 64).cpu().numpy().reshape(-1, 4)
    assert np.abs(got - ref["rgba"]).max() <= 1e-4


def test_training_reduces_l2_loss(env):
    torch, inolf, _ = env
    teacher = synth.tiny_scene(seed=1)
    student = synth.tiny_scene(seed=2)
    t_obj = inolf.object_create(teacher)
    field = inolf.Field(student)
    cams = synth.fibonacci_cameras(8, 3.0)
    W = H = 96
    with torch.no_grad():
        tgt = inolf.render(t_obj, cams, W, H).reshape(-1, 4)
    o_all, d_all = [], []
    for c in cams:
        o, d = oracle.raygen(c, W, H)
        o_all.append(o)
        d_all.append(d)
    o_all = torch.from_numpy(np.concatenate(o_all)).cuda()
    d_all = torch.from_numpy(np.concatenate(d_all)).cuda()
    opt = torch.optim.Adam(field.parameters(), lr=1e-2, betas=(0.9, 0.99), eps=1e-15)
    gen = torch.Generator(device="cuda").manual_seed(0)
    losses = []
    for step in range(60):
        idx = torch.randint(0, len(o_all), (1 << 14,), device="cuda", generator=gen)
        pred = field.render(o_all[idx], d_all[idx])
        loss = ((pred - tgt[idx]) ** 2).sum(1).mean()
        opt.zero_grad()
        loss.backward()
        opt.step()
        losses.append(float(loss))
    assert np.mean(losses[-5:]) < 0.5 * np.mean(losses[:5]), losses[::10]


def test_device_weight_repacking_matches_host_packing(env, tiny):
    # inolf_object_load_params repacks the weights on the device; loading the
    # object's own weights back must reproduce the host-packed BF16 / FP8
    # operand blobs and FP8 scales bit for bit (renders unchanged)
    torch, inolf, _ = env
    obj = inolf.object_create(tiny)
    cam = synth.camera((0.2, -0.1, 3.0))
    inolf.calibrate_fp8(obj, cam[None], 64, 64)
    before = {p: inolf.render(obj, cam[None], 64, 64, p).cpu().numpy() for p in ("fp32", "bf16", "fp8")}
    act0, w0 = obj.fp8_scales()
    tables, w1, w2, w3 = obj.read_params()
    inolf.load_params(obj, None, torch.from_numpy(w1).cuda(), torch.from_numpy(w2).cuda(),
                      torch.from_numpy(w3).cuda())
    act1, w1s = obj.fp8_scales()
    assert np.array_equal(w0, w1s) and np.array_equal(act0, act1)
    for p, ref in before.items():
        assert np.array_equal(inolf.render(obj, cam[None], 64, 64, p).cpu().numpy(), ref), p


def test_backward_from_forward_hits_equals_backward(env, tiny):
    # inolf_backward_hits (hit list compacted from the forward's tri / t) gives
    # the gradients inolf_backward gives after tracing again
    torch, inolf, _ = env
    obj = inolf.object_create(tiny)
    rng = np.random.default_rng(5)
    eye = rng.normal(size=(3000, 3))
    eye = 2.6 * eye / np.linalg.norm(eye, axis=1, keepdims=True)
    dd = rng.uniform(-1.1, 1.1, size=(3000, 3)) - eye
    dd /= np.linalg.norm(dd, axis=1, keepdims=True)
    o = torch.from_numpy(eye.astype(np.float32)).cuda()
    d = torch.from_numpy(dd.astype(np.float32)).cuda()
    tri = torch.empty(3000, dtype=torch.int32, device="cuda")
    t = torch.empty(3000, dtype=torch.float32, device="cuda")
    inolf.render_rays(obj, o, d, "fp32", tri_out=tri, t_out=t)
    g = torch.from_numpy(np.random.default_rng(1).normal(size=(3000, 4)).astype(np.float32)).cuda()
    out = []
    for kw in ({}, {"tri": tri, "t": t}):
        gt = [torch.zeros((obj.table_rows(l), 2), dtype=torch.float32, device="cuda") for l in range(obj.L)]
        gw = [torch.zeros(s, dtype=torch.float32, device="cuda") for s in ((64, obj.d_in), (64, 64), (4, 64))]
        inolf.backward(obj, o, d, g, gt, *gw, **kw)
        torch.cuda.synchronize()
        out.append([x.cpu().numpy() for x in gt + gw])
    # atomics add in any order: equal up to FP32 rounding of the sums
    for a, b in zip(*out):
        assert _rel_l2(a, b) < 1e-5
