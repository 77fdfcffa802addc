"""FP64 CPU oracle for the i-NOLF per-ray path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path:
its inputs are the seeded scene records of ``paper_2303_04086_gb300.synth``
(mesh, sorted vertex keys + features, weights, cameras) and it computes the
plain definition of one-query-per-ray rendering (Sec. 4.2, Eqs. 2-3):
closest triangle hit (FP32 Moller-Trumbore, lexicographic (t, id) minimum),
the Sec. 4.1 grid vertex p = floor(N x) of the hit point, a sorted-map lookup
of the 8 corner features with FP64 trilinear interpolation, FP64 real SH of
degree <= 3 of the view direction, and the FP64 MLP F_s (ReLU, ReLU,
sigmoid).  The analytic FP64 backward follows the L2 objective of Eq. 8.

The decoupled variant of Sec. 4.2 (Eqs. 4-7) is :class:`Cubes` (density
march: hit = first sample of largest weight w_i, alpha_c = accumulated weight)
plus :meth:`Oracle.render_variant_rays` (F_s with alpha_c input, c = c_d + t c_s
from the diffuse cubes).  :func:`composite` and :func:`render_scene` are the
depth fusion of several objects' renders (the frame composer of Sec. 5.1):
per ray the K nearest hits by (t, object index), straight-alpha "over" front to
back, (C / A, A) stored.

Pins (see tests/test_oracle_*.py): brute-force hits on tiny meshes, analytic
sphere intersection, a hand-checked triangle, affine-field reproduction of the
interpolation, SH closed form / orthonormality / addition theorem, a
hand-evaluated 2-ray MLP, central finite differences of the gradient, and
Eq. 1 checked for injectivity on hashes built by the library; for the
composite: one object reproduces its own render, opaque hits reduce it to a
z-buffer, back-to-front "over" gives the same pixel, a hand-worked two-object
pixel, and the K-hit cut; for the march:
homogeneous-medium transmittance in closed form, the entry-sample argmax, the
telescoping sum of the weights, affine density fields, zero density, the
analytic sphere-shell radius of hit points, and the Eq. 7 special cases.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (-ffp-contract=off, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _p(a: Optional[np.ndarray]):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        build()
    L = ctypes.CDLL(_LIB_PATH)
    vp, i32, i64, f32, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
    L.orc_raygen.argtypes = [vp, i32, i32, vp, i64, vp, vp]
    L.orc_hit_brute.argtypes = [vp, vp, i32, vp, vp, i64, vp, vp, vp, vp]
    L.orc_bvh_build.argtypes = [vp, vp, i32]
    L.orc_bvh_build.restype = vp
    L.orc_bvh_free.argtypes = [vp]
    L.orc_bvh_hit.argtypes = [vp, vp, vp, i64, vp, vp, vp]
    L.orc_cells.argtypes = [f32, f32, i32, vp, vp, vp, i64, vp, vp]
    L.orc_scene_create.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, i32, vp, vp, vp, i32, i32, i32, f32, f32]
    L.orc_scene_create.restype = vp
    L.orc_scene_free.argtypes = [vp]
    L.orc_scene_param.argtypes = [vp, i32, i32, ctypes.POINTER(i64)]
    L.orc_scene_param.restype = ctypes.POINTER(f64)
    L.orc_sh16.argtypes = [vp, vp]
    L.orc_mlp.argtypes = [vp, vp, vp, i32, i32, i32, vp, i64, vp]
    L.orc_render_rays.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp, vp]
    L.orc_render_rays.restype = i64
    L.orc_render_pixels.argtypes = [vp, vp, i32, i32, vp, i64, vp, vp, vp, vp]
    L.orc_render_pixels.restype = i64
    L.orc_corners.argtypes = [vp, vp, vp, vp, i64, vp, vp]
    L.orc_backward.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp, vp]
    L.orc_preacts.argtypes = [vp, vp, vp, i64, vp, vp]
    L.orc_psh_slots.argtypes = [vp, i32, i32, vp, i64, vp]
    L.orc_cubes_create.argtypes = [i32, i32, i64, vp, vp, vp, f32, f32, f32, f32, f32, f32]
    L.orc_cubes_create.restype = vp
    L.orc_cubes_free.argtypes = [vp]
    L.orc_density.argtypes = [vp, vp, vp, vp, i64, vp]
    L.orc_march.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
    L.orc_shade_variant_at.argtypes = [vp, vp, vp, vp, vp, vp, i64, vp]
    L.orc_render_variant_rays.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp, vp]
    L.orc_render_variant_rays.restype = i64
    L.orc_render_variant_pixels.argtypes = [vp, vp, vp, i32, i32, vp, i64, vp, vp, vp, vp]
    L.orc_render_variant_pixels.restype = i64
    L.orc_composite.argtypes = [i32, i64, vp, vp, vp, i32, vp, vp]
    L.orc_max_threads.restype = i32
    L.orc_set_threads.argtypes = [i32]
    _lib = L
    return L


def max_threads() -> int:
    return int(lib().orc_max_threads())


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, np.float32)
    return a if shape is None else a.reshape(shape)


def raygen(cam: np.ndarray, W: int, H: int, pix: Optional[np.ndarray] = None):
    """Pinhole rays of the given pixels (j*W + i; all pixels when None)."""
    cam = _f32(cam)
    n = W * H if pix is None else len(pix)
    pix = None if pix is None else np.ascontiguousarray(pix, np.int64)
    o = np.empty((n, 3), np.float32)
    d = np.empty((n, 3), np.float32)
    lib().orc_raygen(_p(cam), W, H, _p(pix), n, _p(o), _p(d))
    return o, d


def hit_brute(V, F, o, d, fp64: bool = False):
    """Closest hit over all triangles: (tri_id, t, near_edge[, fp64 tri_id])."""
    V = _f32(V); F = np.ascontiguousarray(F, np.int32)
    o = _f32(o); d = _f32(d)
    n = len(o)
    tri = np.empty(n, np.int32); t = np.empty(n, np.float32); e = np.empty(n, np.int32)
    t64 = np.empty(n, np.int32) if fp64 else None
    lib().orc_hit_brute(_p(V), _p(F), len(F), _p(o), _p(d), n, _p(tri), _p(t), _p(e), _p(t64))
    return (tri, t, e, t64) if fp64 else (tri, t, e)


class BVH:
    """The oracle's own median-split BVH (acceleration of the brute force)."""

    def __init__(self, V, F):
        self.V = _f32(V); self.F = np.ascontiguousarray(F, np.int32)
        self.h = lib().orc_bvh_build(_p(self.V), _p(self.F), len(self.F))

    def hit(self, o, d):
        o = _f32(o); d = _f32(d)
        n = len(o)
        tri = np.empty(n, np.int32); t = np.empty(n, np.float32); e = np.empty(n, np.int32)
        lib().orc_bvh_hit(self.h, _p(o), _p(d), n, _p(tri), _p(t), _p(e))
        return tri, t, e

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_bvh_free(self.h)
            self.h = None


def cells(N: int, o, d, t, lo: float = -1.5, scale: Optional[float] = None):
    """FP32 grid vertex p = floor(N x) (clamped) and fraction f of hit points."""
    scale = np.float32(1.0 / 3.0) if scale is None else np.float32(scale)
    o = _f32(o); d = _f32(d); t = _f32(t)
    n = len(o)
    c = np.empty((n, 3), np.int32); f = np.empty((n, 3), np.float32)
    lib().orc_cells(np.float32(lo), scale, N, _p(o), _p(d), _p(t), n, _p(c), _p(f))
    return c, f


def sh16(dirs) -> np.ndarray:
    dirs = np.ascontiguousarray(dirs, np.float64).reshape(-1, 3)
    out = np.empty((len(dirs), 16), np.float64)
    for i in range(len(dirs)):
        lib().orc_sh16(_p(dirs[i]), _p(out[i]))
    return out


def mlp(w1, w2, w3, x) -> np.ndarray:
    w1 = np.ascontiguousarray(w1, np.float64); w2 = np.ascontiguousarray(w2, np.float64)
    w3 = np.ascontiguousarray(w3, np.float64)
    x = np.ascontiguousarray(x, np.float64).reshape(-1, w1.shape[1])
    out = np.empty((len(x), w3.shape[0]), np.float64)
    lib().orc_mlp(_p(w1), _p(w2), _p(w3), w1.shape[1], w1.shape[0], w3.shape[0], _p(x), len(x), _p(out))
    return out


def psh_slots(phi: np.ndarray, m: int, r: int, coords: np.ndarray) -> np.ndarray:
    """Eq. 1 evaluated from an exported offset table (for checking hashes)."""
    phi = np.ascontiguousarray(phi, np.uint32)
    coords = np.ascontiguousarray(coords, np.int32)
    out = np.empty(len(coords), np.int64)
    lib().orc_psh_slots(_p(phi), m, r, _p(coords), len(coords), _p(out))
    return out


def composite(hit, t, rgba, K: int = 4):
    """Depth fusion of n_obj objects' renders of the same n rays (Sec. 5.1).

    hit [n_obj][n] (bool / int), t [n_obj][n] FP32, rgba [n_obj][n][4]
    straight RGBA.  Per ray: the hits ordered by (t, object index), the first
    K composited front to back with C += (1 - A) a c, A += (1 - A) a; returns
    ((C / A, A) or zeros as [n][4] FP64, hits used per ray)."""
    hit = np.ascontiguousarray(hit, np.int32)
    n_obj, n = hit.shape
    t = np.ascontiguousarray(t, np.float32).reshape(n_obj, n)
    rgba = np.ascontiguousarray(rgba, np.float64).reshape(n_obj, n, 4)
    out = np.empty((n, 4), np.float64)
    used = np.empty(n, np.int32)
    lib().orc_composite(n_obj, n, _p(hit), _p(t), _p(rgba), int(K), _p(out), _p(used))
    return out, used


def render_scene(orcs, translations, o, d, K: int = 4):
    """World rays o, d [n][3] (FP32) against objects placed by translation:
    each object sees the ray in its own frame (o - T, one FP32 subtraction
    per axis), renders it (closest hit + one query, or the density march of
    the decoupled variant for objects with cubes), and the results are fused
    by :func:`composite`.  Returns a dict with ``rgba`` [n][4], ``used``
    (hits composited), ``hits`` (hits before the K cut) and the per-object
    results ``per``."""
    o = _f32(o); d = _f32(d)
    per = []
    for orc, T in zip(orcs, translations):
        ol = (o - np.asarray(T, np.float32)).astype(np.float32)
        if orc.cubes is None:  # mesh proxy: closest hit, one query
            r = orc.render_rays(ol, d)
            r["hit"] = r["tri"] >= 0
        else:  # decoupled variant: density march, alpha_c input, c = c_d + t c_s
            r = orc.render_variant_rays(ol, d)
            r["hit"] = r["k"] >= 0
        per.append(r)
    hit = np.stack([r["hit"] for r in per])
    t = np.stack([r["t"] for r in per])
    rgba = np.stack([r["rgba"] for r in per])
    out, used = composite(hit, t, rgba, K)
    return {"rgba": out, "used": used, "hits": hit.sum(0), "per": per}


class Oracle:
    """FP64 renderer of one scene (a ``synth.Scene``)."""

    def __init__(self, scene):
        self.scene = scene
        s = scene
        self.L = s.n_levels
        self.nfeat = s.features[0].shape[1]
        self.d_in = s.d_in
        self.hidden = s.w1.shape[0]
        self.d_out = s.w3.shape[0]
        self._V = _f32(s.vertices); self._F = np.ascontiguousarray(s.triangles, np.int32)
        self._N = np.ascontiguousarray(s.resolutions, np.int32)
        self._keys = [np.ascontiguousarray(k, np.uint64) for k in s.keys]
        self._feats = [_f32(f) for f in s.features]
        kp = (ctypes.c_void_p * self.L)(*[k.ctypes.data for k in self._keys])
        fp = (ctypes.c_void_p * self.L)(*[f.ctypes.data for f in self._feats])
        nk = np.array([len(k) for k in self._keys], np.int64)
        self.h = lib().orc_scene_create(
            _p(self._V), _p(self._F), len(self._F), self.L, _p(self._N), kp, _p(nk), fp, self.nfeat,
            _p(_f32(s.w1)), _p(_f32(s.w2)), _p(_f32(s.w3)), self.d_in, self.hidden, self.d_out,
            np.float32(s.domain_lo), np.float32(1.0 / s.domain_side))
        if not self.h:
            raise ValueError("oracle scene rejected its inputs")
        self.cubes = None if getattr(s, "cubes", None) is None else Cubes(s.cubes, lo=s.domain_lo)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_scene_free(self.h)
            self.h = None

    def param(self, which: int, level: int = 0) -> np.ndarray:
        """Live FP64 view of W1/W2/W3 (which=0/1/2) or level features (3)."""
        cnt = ctypes.c_int64()
        ptr = lib().orc_scene_param(self.h, which, level, ctypes.byref(cnt))
        return np.ctypeslib.as_array(ptr, shape=(cnt.value,))

    def render_rays(self, o, d, with_E: bool = False):
        o = _f32(o); d = _f32(d)
        n = len(o)
        rgba = np.empty((n, self.d_out), np.float64)
        tri = np.empty(n, np.int32); t = np.empty(n, np.float32); e = np.empty(n, np.int32)
        E = np.empty((n, self.d_in), np.float64) if with_E else None
        missing = lib().orc_render_rays(self.h, _p(o), _p(d), n, _p(rgba), _p(tri), _p(t), _p(e), _p(E))
        out = {"rgba": rgba, "tri": tri, "t": t, "near_edge": e, "missing": int(missing)}
        if with_E:
            out["E"] = E
        return out

    def render_pixels(self, cam, W: int, H: int, pix: Optional[np.ndarray] = None):
        cam = _f32(cam)
        n = W * H if pix is None else len(pix)
        pix = None if pix is None else np.ascontiguousarray(pix, np.int64)
        rgba = np.empty((n, self.d_out), np.float64)
        tri = np.empty(n, np.int32); t = np.empty(n, np.float32); e = np.empty(n, np.int32)
        missing = lib().orc_render_pixels(self.h, _p(cam), W, H, _p(pix), n, _p(rgba), _p(tri), _p(t), _p(e))
        return {"rgba": rgba, "tri": tri, "t": t, "near_edge": e, "missing": int(missing)}

    def corners(self, o, d, t):
        """Key index (-1 if absent) and FP64 weight of the 8 corners per level."""
        o = _f32(o); d = _f32(d); t = _f32(t)
        n = len(o)
        idx = np.empty((n, self.L, 8), np.int64)
        w = np.empty((n, self.L, 8), np.float64)
        lib().orc_corners(self.h, _p(o), _p(d), _p(t), n, _p(idx), _p(w))
        return idx, w

    def backward(self, o, d, d_rgba):
        """Analytic FP64 gradient of sum(d_rgba * rgba): (gW1, gW2, gW3, [gfeat_l])."""
        o = _f32(o); d = _f32(d)
        d_rgba = np.ascontiguousarray(d_rgba, np.float64).reshape(len(o), self.d_out)
        g1 = np.zeros((self.hidden, self.d_in)); g2 = np.zeros((self.hidden, self.hidden))
        g3 = np.zeros((self.d_out, self.hidden))
        gf = [np.zeros((len(k), self.nfeat)) for k in self._keys]
        gp = (ctypes.c_void_p * self.L)(*[g.ctypes.data for g in gf])
        lib().orc_backward(self.h, _p(o), _p(d), len(o), _p(d_rgba), _p(g1), _p(g2), _p(g3), gp)
        return g1, g2, g3, gf

    def preacts(self, o, d):
        o = _f32(o); d = _f32(d)
        z1 = np.empty((len(o), self.hidden)); z2 = np.empty((len(o), self.hidden))
        lib().orc_preacts(self.h, _p(o), _p(d), len(o), _p(z1), _p(z2))
        return z1, z2


class Cubes:
    """The oracle's view of a ``synth.Cubes`` record: the density / diffuse
    value of a fine vertex is the one any listed cube gives it (0 if none)."""

    def __init__(self, cubes, lo: float = -1.5):
        self.c = cubes
        self._cells = np.ascontiguousarray(cubes.cells, np.int32)
        self._dens = _f32(cubes.density)
        self._diff = None if cubes.diffuse is None else _f32(cubes.diffuse)
        side = np.float32(cubes.side)
        self.h = lib().orc_cubes_create(int(cubes.b), int(cubes.r), len(self._cells), _p(self._cells),
                                        _p(self._dens), _p(self._diff), np.float32(lo),
                                        np.float32(1.0 / float(cubes.side)), side, np.float32(cubes.step),
                                        np.float32(cubes.t_min), np.float32(cubes.alpha_miss))
        if not self.h:
            raise ValueError("oracle cubes rejected their inputs")

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_cubes_free(self.h)
            self.h = None

    def density(self, o, d, t) -> np.ndarray:
        """FP32 density at o + t d."""
        o = _f32(o); d = _f32(d); t = _f32(t)
        out = np.empty(len(o), np.float32)
        lib().orc_density(self.h, _p(o), _p(d), _p(t), len(o), _p(out))
        return out

    def march(self, o, d) -> dict:
        """Hit sample k (-1 = miss), its t, alpha_c, the two largest weights
        with their samples, the samples taken and the last T before the stop."""
        o = _f32(o); d = _f32(d)
        n = len(o)
        out = {"k": np.empty(n, np.int32), "t": np.empty(n, np.float32), "alpha": np.empty(n, np.float32),
               "wmax": np.empty(n, np.float32), "k2": np.empty(n, np.int32), "w2": np.empty(n, np.float32),
               "n": np.empty(n, np.int32), "T_prev": np.empty(n, np.float32)}
        lib().orc_march(self.h, _p(o), _p(d), n, *[_p(out[k]) for k in ("k", "t", "alpha", "wmax", "k2", "w2",
                                                                          "n", "T_prev")])
        return out


def _variant_handles(orc):
    if orc.cubes is None:
        raise ValueError("the scene has no density cubes")
    return orc.h, orc.cubes.h


def _attach_variant():
    def render_variant_rays(self, o, d):
        hs, hc = _variant_handles(self)
        o = _f32(o); d = _f32(d)
        n = len(o)
        rgba = np.empty((n, 4), np.float64)
        k = np.empty(n, np.int32); t = np.empty(n, np.float32); a = np.empty(n, np.float32)
        missing = lib().orc_render_variant_rays(hs, hc, _p(o), _p(d), n, _p(rgba), _p(k), _p(t), _p(a))
        return {"rgba": rgba, "k": k, "t": t, "alpha": a, "missing": int(missing)}

    def render_variant_pixels(self, cam, W: int, H: int, pix: Optional[np.ndarray] = None):
        hs, hc = _variant_handles(self)
        cam = _f32(cam)
        n = W * H if pix is None else len(pix)
        pix = None if pix is None else np.ascontiguousarray(pix, np.int64)
        rgba = np.empty((n, 4), np.float64)
        k = np.empty(n, np.int32); t = np.empty(n, np.float32); a = np.empty(n, np.float32)
        missing = lib().orc_render_variant_pixels(hs, hc, _p(cam), W, H, _p(pix), n, _p(rgba), _p(k), _p(t),
                                                  _p(a))
        return {"rgba": rgba, "k": k, "t": t, "alpha": a, "missing": int(missing)}

    def shade_variant_at(self, o, d, t, alpha_c):
        """Variant shading (Eqs. 5, 7) at given hits (t, alpha_c)."""
        hs, hc = _variant_handles(self)
        o = _f32(o); d = _f32(d); t = _f32(t); alpha_c = _f32(alpha_c)
        rgba = np.empty((len(o), 4), np.float64)
        lib().orc_shade_variant_at(hs, hc, _p(o), _p(d), _p(t), _p(alpha_c), len(o), _p(rgba))
        return rgba

    Oracle.render_variant_rays = render_variant_rays
    Oracle.render_variant_pixels = render_variant_pixels
    Oracle.shade_variant_at = shade_variant_at


_attach_variant()
