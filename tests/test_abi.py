"""The C-ABI library loads on a host without a GPU and exports every entry
point that include/inolf.h declares; host-only calls work without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "inolf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(inolf_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2303_04086_gb300 import build, inolf
    build.build()
    return inolf.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_error_strings(lib):
    from paper_2303_04086_gb300 import inolf
    assert b"sm_103a" in lib.inolf_version()
    st = lib.inolf_build_hash(None, 5, 10, None, None)
    assert st == inolf.E_INVALID
    assert "out" in inolf.last_error()


def test_render_rejects_bad_arguments_before_any_launch(lib):
    from paper_2303_04086_gb300 import inolf
    # NULL object / negative sizes are refused on the host
    assert lib.inolf_render(None, None, 1, 4, 4, 0, None, None, None, None, 0, None) == inolf.E_INVALID
    assert lib.inolf_render_rays(None, None, None, -1, 0, None, None, None, None, 0, None) == inolf.E_INVALID
    assert lib.inolf_object_create(None, None, None) == inolf.E_INVALID
    assert lib.inolf_render_workspace_bytes(1000) >= 8000
    # the measurement aids check their arguments on the host too
    assert lib.inolf_trace_stats(None, None, 1, 4, 4, None, None, 0, None) == inolf.E_INVALID
    assert lib.inolf_probe_peaks(None, None) == inolf.E_INVALID
    assert lib.inolf_workspace_flags(None, None, None) == inolf.E_INVALID
    assert lib.inolf_set_wait_limit_ns(-1) == inolf.E_INVALID
    assert lib.inolf_set_wait_limit_ns(0) == inolf.OK
    assert lib.inolf_set_fault_injection(0) == inolf.OK


def test_render_workspace_size_follows_the_documented_layout(lib, monkeypatch):
    # header + 12 bytes per ray + operand tiles of 128 bytes per ray for at
    # most 4 Mi rays (+ 256 bytes of alignment slack); INOLF_TC_CHUNK_ROWS
    # sets the row count, read at every call
    monkeypatch.delenv("INOLF_TC_CHUNK_ROWS", raising=False)
    lib.inolf_render_workspace_bytes.restype = ctypes.c_size_t
    lib.inolf_render_workspace_bytes.argtypes = [ctypes.c_int64]

    def expect(n, rows=1 << 22):
        n1 = max(n, 1)
        return 256 + 12 * n1 + min((n1 + 255) // 256 * 256, rows) * 128 + 256

    for n in (0, 1, 1000, 300_000, 8_294_400, 530_841_600):
        assert lib.inolf_render_workspace_bytes(n) == expect(n), n
    monkeypatch.setenv("INOLF_TC_CHUNK_ROWS", "300")
    assert lib.inolf_render_workspace_bytes(100_000) == expect(100_000, 300)
    monkeypatch.setenv("INOLF_TC_CHUNK_ROWS", "0")
    assert lib.inolf_render_workspace_bytes(100_000) == 256 + 12 * 100_000 + 256


def _cube_desc_scene():
    from paper_2303_04086_gb300 import synth
    return synth.tiny_density_scene(seed=0)


def _create_status(scene, mutate_desc=None, mutate_cubes=None):
    """inolf_object_create on a density-cube description, with one field
    changed; the argument checks run before any device call."""
    from paper_2303_04086_gb300 import inolf
    L = scene.n_levels
    hashes = [inolf.build_hash(synth_unpack(k), N) for k, N in zip(scene.keys, scene.resolutions)]
    res = np.ascontiguousarray(scene.resolutions, np.int32)
    feats = [np.ascontiguousarray(f, np.float32) for f in scene.features]
    w = [np.ascontiguousarray(a, np.float32) for a in (scene.w1, scene.w2, scene.w3)]
    hp = (ctypes.POINTER(inolf.HashStruct) * L)(*[h._h for h in hashes])
    fp = (ctypes.c_void_p * L)(*[f.ctypes.data for f in feats])
    c = scene.cubes
    cells = np.ascontiguousarray(c.cells, np.int32)
    dens = np.ascontiguousarray(c.density, np.float32)
    diff = np.ascontiguousarray(c.diffuse, np.float32)
    cd = inolf.CubesDesc()
    cd.b, cd.r, cd.n_cubes = c.b, c.r, len(cells)
    cd.cells, cd.density, cd.diffuse = cells.ctypes.data, dens.ctypes.data, diff.ctypes.data
    cd.side, cd.step, cd.t_min, cd.alpha_miss = c.side, c.step, c.t_min, c.alpha_miss
    d = inolf.ObjectDesc()
    d.n_levels, d.n_features = L, 2
    d.resolution = res.ctypes.data
    d.hashes = ctypes.cast(hp, ctypes.c_void_p)
    d.features = ctypes.cast(fp, ctypes.c_void_p)
    d.w1, d.w2, d.w3 = w[0].ctypes.data, w[1].ctypes.data, w[2].ctypes.data
    d.domain_lo, d.domain_scale = -1.5, float(np.float32(1 / 3))
    d.cubes = ctypes.pointer(cd)
    keep = (cells, dens, diff)
    if mutate_cubes:
        keep = keep + (mutate_cubes(cd, cells, dens),)
    if mutate_desc:
        mutate_desc(d)
    out = ctypes.c_void_p()
    st = inolf.lib().inolf_object_create(ctypes.byref(d), None, ctypes.byref(out))
    del keep
    return st


def synth_unpack(keys):
    from paper_2303_04086_gb300 import synth
    return synth.unpack_keys(keys)


@pytest.mark.parametrize("case", ["b_not_pow2", "r_not_pow2", "fine_grid_too_large", "cell_out_of_range",
                                  "cube_twice", "negative_density", "nan_density", "zero_step", "step_too_small",
                                  "t_min_zero", "alpha_miss_one", "mesh_given", "null_cells"])
def test_cube_descriptions_are_checked_on_the_host(lib, case):
    from paper_2303_04086_gb300 import inolf
    scene = _cube_desc_scene()

    def cubes(cd, cells, dens):
        if case == "b_not_pow2":
            cd.b = 12
        elif case == "r_not_pow2":
            cd.r = 6
        elif case == "fine_grid_too_large":
            cd.b, cd.r = 512, 16
        elif case == "cell_out_of_range":
            cells[0, 1] = cd.b
        elif case == "cube_twice":
            cells[1] = cells[0]
        elif case == "negative_density":
            dens[3, 5] = -1.0
        elif case == "nan_density":
            dens[2, 0] = np.nan
        elif case == "zero_step":
            cd.step = 0.0
        elif case == "step_too_small":
            cd.step = 1e-6
        elif case == "t_min_zero":
            cd.t_min = 0.0
        elif case == "alpha_miss_one":
            cd.alpha_miss = 1.0
        elif case == "null_cells":
            cd.cells = None
        return None

    def desc(d):
        if case == "mesh_given":
            d.n_vertices, d.n_triangles = 3, 1

    st = _create_status(scene, mutate_desc=desc, mutate_cubes=cubes)
    assert st == inolf.E_INVALID, (case, st, inolf.last_error())


@pytest.mark.parametrize("case", ["no_coords", "coord_above_N", "negative_coord"])
def test_hashed_points_are_checked_on_the_host(lib, case):
    # the corner bundles are laid out from the points each hash carries:
    # a hash without them, or with a point outside [0, N], is refused before
    # any device call
    from paper_2303_04086_gb300 import inolf
    scene = _cube_desc_scene()

    def mutate(d):
        h = ctypes.cast(d.hashes, ctypes.POINTER(ctypes.POINTER(inolf.HashStruct)))[1].contents
        if case == "no_coords":
            h.coords = None
        elif case == "coord_above_N":
            h.coords[4] = int(scene.resolutions[1]) + 1
        else:
            h.coords[0] = -1

    st = _create_status(scene, mutate_desc=mutate)
    assert st == inolf.E_INVALID
    msg = inolf.last_error()
    assert ("coords" in msg) if case == "no_coords" else ("outside [0, N]" in msg)
