"""Seeded synthetic inputs for i-NOLF workloads (meshes, occupied vertex sets,
features, weights, cameras).

This module holds none of the renderer's arithmetic; it only writes the inputs
that both the CUDA path and the FP64 oracle consume.  The native part lives in
``synth.cpp`` and is compiled by :func:`build` into ``libinolf_synth.so`` next
to it.

Workloads (sizes are those of the i-NOLF speed experiments, Sec. 8.2/8.4, with
synthetic geometry in place of the paper's captured objects):

* ``tiny_scene``      level-3 icosphere (1280 triangles), L=4 levels at
                      N = 16/32/64/128, band 0.05, F=2 features, MLP 24-64-64-4;
* ``full_scene``      displaced geodesic sphere (200 000 triangles), L=16 levels
                      N_l = round(16 * 128^(l/15)), band 2 cells, MLP 48-64-64-4;
* ``tiny_density_scene`` / ``full_density_scene``  the same two objects for the
                      paper's decoupled variant: density and diffuse texture
                      cubes of a shell around the surface (Sec. 4.2) instead of
                      the mesh, PSH levels built from the voxels around every
                      possible hit point, MLP input + alpha_c (d_in + 1);
* cameras on a ring / Fibonacci sphere looking at the origin, 45 deg FOV.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.cpp")
_LIB_PATH = os.path.join(_HERE, "libinolf_synth.so")
_lib = None

DOMAIN_LO = -1.5     # scene cube [-1.5, 1.5]^3
DOMAIN_SIDE = 3.0
N_FEATURES = 2
HIDDEN = 64
D_OUT = 4
N_SH = 16


def build(force: bool = False) -> str:
    """Compile the generator (g++, OpenMP) in place; returns the .so path."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is missing: run paper_2303_04086_gb300.synth.build() first")
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.POINTER
    c_fp = P(ctypes.c_float)
    c_ip = P(ctypes.c_int32)
    lib.syn_icosphere.argtypes = [ctypes.c_int32, ctypes.c_double, P(c_fp), c_ip, P(c_ip), c_ip]
    lib.syn_geodesic.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, P(c_fp), c_ip, P(c_ip), c_ip]
    lib.syn_band_vertices.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      P(P(ctypes.c_uint64)), P(ctypes.c_int64)]
    lib.syn_features.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                                 ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
    lib.syn_xavier.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.syn_camera.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
    lib.syn_unpack_keys.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    lib.syn_free.argtypes = [ctypes.c_void_p]
    lib.syn_density_cubes.argtypes = [ctypes.c_uint64, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int32, P(c_ip), P(c_fp), P(c_fp),
                                      P(ctypes.c_int64)]
    lib.syn_live_level_vertices.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p]
    lib.syn_splitmix64.argtypes = [ctypes.c_uint64]
    lib.syn_splitmix64.restype = ctypes.c_uint64
    for name in ("syn_icosphere", "syn_geodesic", "syn_band_vertices", "syn_density_cubes",
                 "syn_live_level_vertices"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def _take_mesh(Vp, nV, Fp, nF):
    lib = _load()
    V = np.ctypeslib.as_array(Vp, shape=(nV.value * 3,)).reshape(nV.value, 3).copy()
    F = np.ctypeslib.as_array(Fp, shape=(nF.value * 3,)).reshape(nF.value, 3).copy()
    lib.syn_free(ctypes.cast(Vp, ctypes.c_void_p))
    lib.syn_free(ctypes.cast(Fp, ctypes.c_void_p))
    return V, F


def icosphere(level: int, radius: float = 1.0):
    lib = _load()
    Vp, Fp = ctypes.POINTER(ctypes.c_float)(), ctypes.POINTER(ctypes.c_int32)()
    nV, nF = ctypes.c_int32(), ctypes.c_int32()
    rc = lib.syn_icosphere(level, radius, ctypes.byref(Vp), ctypes.byref(nV), ctypes.byref(Fp), ctypes.byref(nF))
    if rc != 0:
        raise RuntimeError(f"syn_icosphere failed ({rc})")
    return _take_mesh(Vp, nV, Fp, nF)


def geodesic(freq: int, amp: float, seed: int):
    lib = _load()
    Vp, Fp = ctypes.POINTER(ctypes.c_float)(), ctypes.POINTER(ctypes.c_int32)()
    nV, nF = ctypes.c_int32(), ctypes.c_int32()
    rc = lib.syn_geodesic(freq, amp, seed, ctypes.byref(Vp), ctypes.byref(nV), ctypes.byref(Fp), ctypes.byref(nF))
    if rc != 0:
        raise RuntimeError(f"syn_geodesic failed ({rc})")
    return _take_mesh(Vp, nV, Fp, nF)


def band_vertices(V: np.ndarray, F: np.ndarray, N: int, band: float,
                  lo: float = DOMAIN_LO, side: float = DOMAIN_SIDE) -> np.ndarray:
    """Sorted packed keys of all corners of the cells within `band` (+ half a
    cell diagonal) of the mesh, at resolution N."""
    lib = _load()
    V = np.ascontiguousarray(V, np.float32)
    F = np.ascontiguousarray(F, np.int32)
    kp = ctypes.POINTER(ctypes.c_uint64)()
    n = ctypes.c_int64()
    rc = lib.syn_band_vertices(_ptr(V), len(V), _ptr(F), len(F), N, lo, side, band, ctypes.byref(kp), ctypes.byref(n))
    if rc != 0:
        raise RuntimeError(f"syn_band_vertices failed ({rc})")
    keys = np.ctypeslib.as_array(kp, shape=(max(n.value, 1),))[: n.value].copy()
    lib.syn_free(ctypes.cast(kp, ctypes.c_void_p))
    return keys


def pack_keys(coords: np.ndarray) -> np.ndarray:
    c = np.asarray(coords, np.uint64)
    return c[:, 0] | (c[:, 1] << np.uint64(21)) | (c[:, 2] << np.uint64(42))


def unpack_keys(keys: np.ndarray) -> np.ndarray:
    keys = np.ascontiguousarray(keys, np.uint64)
    out = np.empty((len(keys), 3), np.int32)
    if len(keys):
        _load().syn_unpack_keys(_ptr(keys), len(keys), _ptr(out))
    return out


def features(seed: int, level: int, keys: np.ndarray, n_features: int = N_FEATURES, fp16: bool = False) -> np.ndarray:
    keys = np.ascontiguousarray(keys, np.uint64)
    out = np.empty((len(keys), n_features), np.float32)
    if len(keys):
        _load().syn_features(seed, level, _ptr(keys), len(keys), n_features, int(fp16), _ptr(out))
    return out


def xavier(seed: int, d_in: int, hidden: int = HIDDEN, d_out: int = D_OUT):
    w1 = np.empty((hidden, d_in), np.float32)
    w2 = np.empty((hidden, hidden), np.float32)
    w3 = np.empty((d_out, hidden), np.float32)
    _load().syn_xavier(seed, d_in, hidden, d_out, _ptr(w1), _ptr(w2), _ptr(w3))
    return w1, w2, w3


def camera(eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), fovy_deg: float = 45.0) -> np.ndarray:
    """13-float pinhole record: eye, right, up, fwd (FP32) and tan(fovy/2)."""
    e = np.asarray(eye, np.float64)
    t = np.asarray(target, np.float64)
    u = np.asarray(up, np.float64)
    out = np.empty(13, np.float32)
    _load().syn_camera(_ptr(e), _ptr(t), _ptr(u), fovy_deg, _ptr(out))
    return out


def ring_cameras(n: int, radius: float, fovy_deg: float = 45.0) -> np.ndarray:
    """n cameras at r (sin th_k, 0, cos th_k), th_k = 2 pi k / n, looking at the origin."""
    cams = [camera((radius * math.sin(2 * math.pi * k / n), 0.0, radius * math.cos(2 * math.pi * k / n)),
                   fovy_deg=fovy_deg) for k in range(n)]
    return np.stack(cams)


def fibonacci_cameras(n: int, radius: float, fovy_deg: float = 45.0) -> np.ndarray:
    """n cameras on a Fibonacci sphere of the given radius, looking at the origin."""
    ga = math.pi * (3.0 - math.sqrt(5.0))
    cams = []
    for k in range(n):
        y = 1.0 - 2.0 * (k + 0.5) / n
        rr = math.sqrt(max(0.0, 1.0 - y * y))
        th = ga * k
        eye = (radius * rr * math.cos(th), radius * y, radius * rr * math.sin(th))
        up = (0.0, 1.0, 0.0) if abs(y) < 0.99 else (1.0, 0.0, 0.0)
        cams.append(camera(eye, up=up, fovy_deg=fovy_deg))
    return np.stack(cams)


@dataclass
class Cubes:
    """Density (and diffuse) texture cubes of one object (Sec. 4.2).

    Base grid of b^3 cells over the scene cube; cube i covers base cell
    cells[i] and holds the (r+1)^3 fine vertices cells[i] * r + (0..r)^3
    (x fastest) of the fine grid K = b r.  density[i] are their sigma values,
    diffuse[i] their (c_d r, g, b, tint).  The march takes samples every
    `step` from the ray's entry into the scene cube, stops once the
    transmittance falls below `t_min`, and a ray whose coarse opacity stays at
    or below `alpha_miss` is a miss."""
    b: int
    r: int
    cells: np.ndarray
    density: np.ndarray
    diffuse: Optional[np.ndarray]
    step: float
    t_min: float = 1e-4
    alpha_miss: float = 1e-4
    side: float = DOMAIN_SIDE
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.cells)


def density_cubes(seed: int, radius: float, amp: float, b: int, r: int, w: float, sigma_max: float,
                  diffuse: bool = True, lo: float = DOMAIN_LO, side: float = DOMAIN_SIDE):
    """(cells [n][3] int32, density [n][(r+1)^3] f32, diffuse [n][(r+1)^3][4] f32 or None)
    of a shell sigma = sigma_max max(0, 1 - |s| / w) around r = radius (1 + amp n(q))."""
    lib = _load()
    cp = ctypes.POINTER(ctypes.c_int32)()
    dp = ctypes.POINTER(ctypes.c_float)()
    fp = ctypes.POINTER(ctypes.c_float)()
    n = ctypes.c_int64()
    rc = lib.syn_density_cubes(seed, radius, amp, b, r, lo, side, w, sigma_max, int(diffuse), ctypes.byref(cp),
                               ctypes.byref(dp), ctypes.byref(fp), ctypes.byref(n))
    if rc != 0:
        raise RuntimeError(f"syn_density_cubes failed ({rc})")
    nv = (r + 1) ** 3
    cells = np.ctypeslib.as_array(cp, shape=(max(n.value, 1) * 3,))[: n.value * 3].reshape(n.value, 3).copy()
    dens = np.ctypeslib.as_array(dp, shape=(max(n.value * nv, 1),))[: n.value * nv].reshape(n.value, nv).copy()
    lib.syn_free(ctypes.cast(cp, ctypes.c_void_p))
    lib.syn_free(ctypes.cast(dp, ctypes.c_void_p))
    diff = None
    if diffuse:
        diff = np.ctypeslib.as_array(fp, shape=(max(n.value * nv * 4, 1),))[: n.value * nv * 4]
        diff = diff.reshape(n.value, nv, 4).copy()
        lib.syn_free(ctypes.cast(fp, ctypes.c_void_p))
    return cells, dens, diff


def live_level_vertices(cells: np.ndarray, density: np.ndarray, b: int, r: int, resolutions) -> List[np.ndarray]:
    """Sorted packed corner keys, per level, of the level cells any point of a
    live fine cell (one with a vertex of non-zero density) can fall in."""
    lib = _load()
    cells = np.ascontiguousarray(cells, np.int32)
    density = np.ascontiguousarray(density, np.float32)
    res = np.ascontiguousarray(resolutions, np.int32)
    L = len(res)
    kp = (ctypes.POINTER(ctypes.c_uint64) * L)()
    nn = (ctypes.c_int64 * L)()
    rc = lib.syn_live_level_vertices(_ptr(cells), _ptr(density), len(cells), b, r, L,
                                     _ptr(res), ctypes.cast(kp, ctypes.c_void_p), ctypes.cast(nn, ctypes.c_void_p))
    if rc != 0:
        raise RuntimeError(f"syn_live_level_vertices failed ({rc})")
    out = []
    for l in range(L):
        k = np.ctypeslib.as_array(kp[l], shape=(max(nn[l], 1),))[: nn[l]].copy()
        lib.syn_free(ctypes.cast(kp[l], ctypes.c_void_p))
        out.append(k)
    return out


@dataclass
class Scene:
    """One i-NOLF object's inputs.  keys[l] are sorted packed vertex keys of
    level l and features[l][i] belongs to keys[l][i]."""
    vertices: np.ndarray
    triangles: np.ndarray
    resolutions: List[int]
    keys: List[np.ndarray]
    features: List[np.ndarray]
    w1: np.ndarray
    w2: np.ndarray
    w3: np.ndarray
    feature_fp16: bool = False
    domain_lo: float = DOMAIN_LO
    domain_side: float = DOMAIN_SIDE
    meta: dict = field(default_factory=dict)
    cubes: Optional[Cubes] = None  # set: the decoupled variant (hit by density march, alpha_c input, diffuse)

    @property
    def n_levels(self) -> int:
        return len(self.resolutions)

    @property
    def d_in(self) -> int:
        return self.n_levels * N_FEATURES + N_SH + (1 if self.cubes is not None else 0)


def full_resolutions(n_levels: int = 16, base: int = 16, top: int = 2048) -> List[int]:
    g = top / base
    return [int(math.floor(base * g ** (l / (n_levels - 1)) + 0.5)) for l in range(n_levels)]


def _build_scene(V, F, resolutions, bands, seed, fp16, meta) -> Scene:
    keys, feats = [], []
    for l, (N, band) in enumerate(zip(resolutions, bands)):
        k = band_vertices(V, F, N, band)
        keys.append(k)
        feats.append(features(seed, l, k, fp16=fp16))
    d_in = len(resolutions) * N_FEATURES + N_SH
    w1, w2, w3 = xavier(seed, d_in)
    return Scene(V, F, list(resolutions), keys, feats, w1, w2, w3, fp16, meta=meta)


def tiny_scene(seed: int = 0, fp16: bool = False, resolutions=(16, 32, 64, 128), band: float = 0.05,
               ico_level: int = 3) -> Scene:
    """Level-3 icosphere of radius 1, L=4, band 0.05, F=2 ~ N(0, 0.1)."""
    V, F = icosphere(ico_level, 1.0)
    return _build_scene(V, F, resolutions, [band] * len(resolutions), seed, fp16,
                        {"name": "icosphere-L%d" % len(resolutions), "seed": seed})


def full_scene(seed: int = 0, freq: int = 100, n_levels: int = 16, top: int = 2048,
               band_cells: float = 2.0, amp: float = 0.1, fp16: bool = False) -> Scene:
    """Displaced geodesic sphere (20 freq^2 triangles), L levels 16..top, band
    of `band_cells` cells at each level."""
    V, F = geodesic(freq, amp, seed)
    res = full_resolutions(n_levels, 16, top)
    bands = [band_cells * DOMAIN_SIDE / N for N in res]
    return _build_scene(V, F, res, bands, seed, fp16,
                        {"name": "geodesic%d-L%d" % (freq, n_levels), "seed": seed})


def _density_scene(seed, radius, amp, b, r, resolutions, w_cells, opacity, fp16, meta) -> Scene:
    side = DOMAIN_SIDE
    K = b * r
    w = w_cells * side / K
    sigma_max = opacity / w
    cells, dens, diff = density_cubes(seed, radius, amp, b, r, w, sigma_max, True)
    step = float(np.float32(side / K))
    cubes = Cubes(b, r, cells, dens, diff, step, meta={"w": w, "sigma_max": sigma_max, "radius": radius,
                                                       "amp": amp})
    keys = live_level_vertices(cells, dens, b, r, resolutions)
    feats = [features(seed, l, k, fp16=fp16) for l, k in enumerate(keys)]
    d_in = len(resolutions) * N_FEATURES + N_SH + 1
    w1, w2, w3 = xavier(seed, d_in)
    empty_v = np.zeros((0, 3), np.float32)
    empty_f = np.zeros((0, 3), np.int32)
    return Scene(empty_v, empty_f, list(resolutions), keys, feats, w1, w2, w3, fp16, meta=meta, cubes=cubes)


def tiny_density_scene(seed: int = 0, fp16: bool = False, resolutions=(16, 32, 64, 128), b: int = 16, r: int = 8,
                       w_cells: float = 2.0, opacity: float = 12.0) -> Scene:
    """Unit sphere as a density shell (half-width w_cells fine cells, optical
    depth `opacity` across it) in b^3 base cells of r^3 fine cells (K = 128),
    L=4 levels at N = 16/32/64/128, MLP 25-64-64-4."""
    return _density_scene(seed, 1.0, 0.0, b, r, resolutions, w_cells, opacity, fp16,
                          {"name": "sphere-shell-b%d-r%d-L%d" % (b, r, len(resolutions)), "seed": seed})


def full_density_scene(seed: int = 0, n_levels: int = 16, top: int = 2048, b: int = 128, r: int = 16,
                       amp: float = 0.1, w_cells: float = 2.0, opacity: float = 12.0, fp16: bool = False) -> Scene:
    """The displaced sphere of ``full_scene`` as a density shell in 128^3 base
    cells of 16^3 fine cells (K = 2048), L levels 16..top, MLP 49-64-64-4."""
    res = full_resolutions(n_levels, 16, top)
    return _density_scene(seed, 1.0, amp, b, r, res, w_cells, opacity, fp16,
                          {"name": "displaced-shell-b%d-r%d-L%d" % (b, r, n_levels), "seed": seed})


def serving_scene(seed: int = 0, n_objects: int = 12, n_viewers: int = 32):
    """The multi-viewer serving workload: ``n_objects`` tiny scenes (seeds
    0 .. n_objects - 1) placed by translation without bounding-sphere overlap
    (centres more than 2.3 apart, uniform in [-4, 4]^3, so the r <= 1.1
    proxies stay inside a 10 m cube), and ``n_viewers`` viewers, each a unit
    direction (the viewer sits at 12 m along it, looking at the origin) with a
    resolution drawn from 1280x720 / 1920x1080 / 3840x2160.  Returns
    (scenes, translations, viewers)."""
    rng = np.random.default_rng(seed)
    places = []
    while len(places) < n_objects:
        p = rng.uniform(-4.0, 4.0, size=3)
        if all(np.linalg.norm(p - q) > 2.3 for q in places):
            places.append(p)
    scenes = [tiny_scene(seed=s) for s in range(n_objects)]
    res = [(1280, 720), (1920, 1080), (3840, 2160)]
    viewers = []
    for _ in range(n_viewers):
        d = rng.normal(size=3)
        viewers.append({"dir": d / np.linalg.norm(d), "res": res[rng.integers(0, 3)]})
    return scenes, [tuple(map(float, p)) for p in places], viewers
