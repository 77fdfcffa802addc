"""Measurement aids on the GPU: inolf_trace_stats (BVH packet statistics of
the closest-hit step) and inolf_probe_peaks (microbenchmarked roofline
denominators)."""
import numpy as np
import pytest

import oracle
from paper_2303_04086_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def inolf_mod():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04086_gb300 import build, inolf
    build.build()
    return inolf


def test_trace_stats_counts_the_oracle_hits(inolf_mod, tiny, tiny_oracle):
    inolf = inolf_mod
    obj = inolf.object_create(tiny)
    cam = synth.camera((0.3, -0.2, 3.0))
    W, H = 100, 72  # ragged: 7 x 5 tiles of 16 x 16
    st = inolf.trace_stats(obj, cam[None], W, H)
    ref = tiny_oracle.render_pixels(cam, W, H)
    assert st["rays"] == W * H
    assert st["hit_rays"] == int((ref["tri"] >= 0).sum())
    assert st["packets"] == 7 * 5 * 8
    # every packet tests the root; packets whose rays hit test triangles
    assert st["inner_node_visits"] >= st["packets"]
    assert st["triangle_tests"] > 0 and st["node_visits_per_ray"] >= 1.0


def test_trace_stats_of_a_view_that_misses(inolf_mod, tiny):
    inolf = inolf_mod
    obj = inolf.object_create(tiny)
    cam = synth.camera((0.0, 0.0, 3.0), target=(0.0, 0.0, 6.0))  # looking away from the object
    st = inolf.trace_stats(obj, cam[None], 32, 32)
    assert st["hit_rays"] == 0 and st["triangle_tests"] == 0
    assert st["inner_node_visits"] == st["packets"]  # the root box only


def test_trace_stats_rejects_density_cube_objects(inolf_mod):
    inolf = inolf_mod
    obj = inolf.object_create(synth.tiny_density_scene(seed=0))
    with pytest.raises(inolf.InolfError):
        inolf.trace_stats(obj, synth.camera((0.0, 0.0, 3.0))[None], 16, 16)


def test_probe_peaks_are_positive_and_finite(inolf_mod):
    pk = inolf_mod.probe_peaks()
    for k in ("l2_read_gbs", "l2_gather_gsps", "fp32_tflops"):
        assert np.isfinite(pk[k]) and pk[k] > 0, (k, pk)
    # an FP32 FMA rate above the unit-count peak (152 SMs x 128 lanes x 2 flop
    # x 2.07 GHz = 80.5 TFLOP/s) would mean the probe is not doing the work
    assert pk["fp32_tflops"] < 85.0
