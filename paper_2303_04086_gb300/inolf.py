"""Thin Python binding of libinolf.so (ctypes).  Argument marshalling only:
every step of the per-ray path runs in the library's CUDA kernels.  PyTorch
supplies device memory and the current stream.

Names follow the C ABI in include/inolf.h: build_hash, object_create,
render, render_rays, encode_rays, ...
"""
from __future__ import annotations

import ctypes
import os
from concurrent.futures import ThreadPoolExecutor
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libinolf.so")

OK, PENDING = 0, 1
(E_INVALID, E_OOM, E_CUDA, E_BUDGET, E_TIMEOUT, E_HASH_FAILED, E_UNKNOWN_TICKET, E_UNSUPPORTED,
 E_CANCELLED, E_DEVICE) = range(-1, -11, -1)
REQ_TEST_DROP_DESCRIPTOR = 1
FLAG_STACK_OVERFLOW, FLAG_TRAVERSAL_LIMIT, FLAG_WAIT_TIMEOUT = 1, 2, 4
INJECT_RING_STALL = 1
FP32, BF16, FP8 = 0, 1, 2
PRECISIONS = {"fp32": FP32, "bf16": BF16, "fp8": FP8}
MAX_LEVELS = 16

_lib = None


class InolfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"inolf status {status}: {msg}")
        self.status = status


class HashParams(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("slot_slack", ctypes.c_double),
                ("max_retries", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class HashStruct(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("r", ctypes.c_int32), ("n", ctypes.c_int64),
                ("phi", ctypes.POINTER(ctypes.c_uint32)), ("slot_of", ctypes.POINTER(ctypes.c_uint32)),
                ("coords", ctypes.POINTER(ctypes.c_int32))]


class CubesDesc(ctypes.Structure):
    _fields_ = [("b", ctypes.c_int32), ("r", ctypes.c_int32), ("n_cubes", ctypes.c_int64),
                ("cells", ctypes.c_void_p), ("density", ctypes.c_void_p), ("diffuse", ctypes.c_void_p),
                ("side", ctypes.c_float), ("step", ctypes.c_float), ("t_min", ctypes.c_float),
                ("alpha_miss", ctypes.c_float)]


class Peaks(ctypes.Structure):
    _fields_ = [("l2_read_gbs", ctypes.c_double), ("l2_gather_gsps", ctypes.c_double),
                ("fp32_tflops", ctypes.c_double)]


class ObjectDesc(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int32), ("n_triangles", ctypes.c_int32),
                ("vertices", ctypes.c_void_p), ("triangles", ctypes.c_void_p),
                ("n_levels", ctypes.c_int32), ("n_features", ctypes.c_int32),
                ("resolution", ctypes.c_void_p), ("hashes", ctypes.c_void_p), ("features", ctypes.c_void_p),
                ("features_fp16", ctypes.c_int32),
                ("w1", ctypes.c_void_p), ("w2", ctypes.c_void_p), ("w3", ctypes.c_void_p),
                ("fp8_act_scale", ctypes.c_float * 3),
                ("domain_lo", ctypes.c_float), ("domain_scale", ctypes.c_float),
                ("cubes", ctypes.POINTER(CubesDesc))]


def lib():
    """Load libinolf.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2303_04086_gb300.build.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    L.inolf_last_error.restype = ctypes.c_char_p
    L.inolf_version.restype = ctypes.c_char_p
    L.inolf_build_hash.argtypes = [vp, i64, i32, ctypes.POINTER(HashParams), ctypes.POINTER(ctypes.POINTER(HashStruct))]
    L.inolf_hash_free.argtypes = [ctypes.POINTER(HashStruct)]
    L.inolf_hash_free.restype = None
    L.inolf_object_create.argtypes = [ctypes.POINTER(ObjectDesc), vp, ctypes.POINTER(vp)]
    L.inolf_object_destroy.argtypes = [vp]
    L.inolf_object_destroy.restype = None
    L.inolf_object_bytes.argtypes = [vp, ctypes.POINTER(sz)]
    L.inolf_object_set_fp8_scales.argtypes = [vp, vp]
    L.inolf_object_read_params.argtypes = [vp, vp, vp, vp, vp]
    L.inolf_object_table_rows.argtypes = [vp, i32, ctypes.POINTER(i64)]
    L.inolf_render_workspace_bytes.argtypes = [i64]
    L.inolf_render_workspace_bytes.restype = sz
    L.inolf_render.argtypes = [vp, vp, i32, i32, i32, i32, vp, vp, vp, vp, sz, vp]
    L.inolf_render_rays.argtypes = [vp, vp, vp, i64, i32, vp, vp, vp, vp, sz, vp]
    L.inolf_encode_rays.argtypes = [vp, vp, vp, i64, vp, vp, vp, sz, vp]
    L.inolf_march_rays.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp, sz, vp]
    L.inolf_render_host.argtypes = [vp, vp, i32, i32, i32, i32, vp, vp, sz, vp, sz, vp]
    L.inolf_trace_stats.argtypes = [vp, vp, i32, i32, i32, vp, vp, sz, vp]
    L.inolf_probe_peaks.argtypes = [ctypes.POINTER(Peaks), vp]
    L.inolf_render_rays_noalloc.argtypes = [vp, vp, vp, i64, i32, vp, vp, vp, vp]
    L.inolf_calibrate_fp8.argtypes = [vp, vp, i32, i32, i32, vp, sz, vp]
    L.inolf_backward.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, sz, vp]
    L.inolf_backward_hits.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    L.inolf_object_load_params.argtypes = [vp, vp, vp, vp, vp, vp]
    L.inolf_object_get_fp8_scales.argtypes = [vp, vp, vp]
    L.inolf_workspace_flags.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32), vp]
    L.inolf_set_wait_limit_ns.argtypes = [i64]
    L.inolf_set_fault_injection.argtypes = [ctypes.c_uint32]
    _lib = L
    return L


def last_error() -> str:
    return lib().inolf_last_error().decode()


def _check(st: int):
    if st < 0:
        raise InolfError(st, last_error())
    return st


def _ptr(t) -> Optional[int]:
    """Device/host address of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


_check_flags = False


def check_device_flags(on: bool = True):
    """When on, every asynchronous render / backward wrapper below waits for
    its call and raises InolfError if a kernel set a failure flag (see
    workspace_flags).  Off by default: the check synchronises the stream."""
    global _check_flags
    _check_flags = bool(on)


def workspace_flags(workspace=None, stream=None) -> int:
    """inolf_workspace_flags: the INOLF_FLAG_* bits the kernels of the last
    call on `workspace` set (None = the allocation-free scratch); synchronises
    the stream.  Returns the bits; a non-zero value is not raised."""
    f = ctypes.c_uint32(0)
    st = lib().inolf_workspace_flags(_ptr(workspace), ctypes.byref(f), _stream(stream))
    if st < 0 and f.value == 0:
        raise InolfError(st, last_error())
    return int(f.value)


def _after(workspace, stream, launched=True):
    # a call without work (n = 0) launches nothing and leaves the flag word as it was
    if _check_flags and launched:
        _check(lib().inolf_workspace_flags(_ptr(workspace), ctypes.byref(ctypes.c_uint32(0)), _stream(stream)))


def set_wait_limit_ns(ns: int):
    """Limit of the warp-specialised shade kernels' hand-over waits (0 = 2 s)."""
    _check(lib().inolf_set_wait_limit_ns(int(ns)))


def set_fault_injection(mask: int):
    """Test-only fault injection (INJECT_RING_STALL), process-wide; 0 = off."""
    _check(lib().inolf_set_fault_injection(int(mask)))


# ---------------------------------------------------------------------------
# perfect spatial hash (Sec. 4.1, Eq. 1)
# ---------------------------------------------------------------------------
class Hash:
    """Handle of one level's hash; m, r, phi (r^3) and slot_of (n) as numpy views."""

    def __init__(self, handle):
        self._h = handle
        h = handle.contents
        self.m, self.r, self.n = h.m, h.r, h.n
        self.phi = np.ctypeslib.as_array(h.phi, shape=(h.r ** 3,))
        self.slot_of = np.ctypeslib.as_array(h.slot_of, shape=(max(h.n, 1),))[: h.n]

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.inolf_hash_free(self._h)
            self._h = None


def build_hash(coords: np.ndarray, grid_extent: int, sigma: float = 1.0 / 6.0, slot_slack: float = 1.0,
               max_retries: int = 8, seed: int = 0) -> Hash:
    coords = np.ascontiguousarray(coords, np.int32).reshape(-1, 3)
    out = ctypes.POINTER(HashStruct)()
    prm = HashParams(sigma, slot_slack, max_retries, seed)
    _check(lib().inolf_build_hash(ctypes.c_void_p(coords.ctypes.data), len(coords), grid_extent,
                                  ctypes.byref(prm), ctypes.byref(out)))
    return Hash(out)


# ---------------------------------------------------------------------------
# objects
# ---------------------------------------------------------------------------
class Object:
    """A device-resident i-NOLF object (inolf_object handle)."""

    def __init__(self, handle, L, d_in, hashes):
        self._h = handle
        self.L = L
        self.d_in = d_in
        self.hashes = hashes

    @property
    def handle(self):
        return self._h

    def bytes(self) -> int:
        b = ctypes.c_size_t()
        _check(lib().inolf_object_bytes(self._h, ctypes.byref(b)))
        return b.value

    def table_rows(self, level: int) -> int:
        r = ctypes.c_int64()
        _check(lib().inolf_object_table_rows(self._h, level, ctypes.byref(r)))
        return r.value

    def set_fp8_scales(self, scales: Sequence[float]):
        s = np.ascontiguousarray(scales, np.float32)
        _check(lib().inolf_object_set_fp8_scales(self._h, ctypes.c_void_p(s.ctypes.data)))

    def fp8_scales(self):
        """(activation scales of layers 1-3, weight scales of W1-W3)."""
        a = np.zeros(3, np.float32)
        w = np.zeros(3, np.float32)
        _check(lib().inolf_object_get_fp8_scales(self._h, a.ctypes.data, w.ctypes.data))
        return a, w

    def read_params(self):
        tables = [np.empty((self.table_rows(l), 2), np.float32) for l in range(self.L)]
        tp = (ctypes.c_void_p * self.L)(*[t.ctypes.data for t in tables])
        w1 = np.empty((64, self.d_in), np.float32)
        w2 = np.empty((64, 64), np.float32)
        w3 = np.empty((4, 64), np.float32)
        _check(lib().inolf_object_read_params(self._h, tp, w1.ctypes.data, w2.ctypes.data, w3.ctypes.data))
        return tables, w1, w2, w3

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.inolf_object_destroy(self._h)
            self._h = None


def build_hashes(scene, threads: int = 0, **kw) -> List[Hash]:
    """inolf_build_hash for every level of a synth.Scene, levels in parallel
    (ctypes releases the GIL during the call)."""
    from .synth import unpack_keys

    def one(l):
        return build_hash(unpack_keys(scene.keys[l]), scene.resolutions[l], **kw)

    n = threads or min(len(scene.keys), os.cpu_count() or 1)
    with ThreadPoolExecutor(max_workers=n) as ex:
        return list(ex.map(one, range(scene.n_levels)))


def object_create(scene, hashes: Optional[List[Hash]] = None, fp16: Optional[bool] = None,
                  fp8_act_scale=(0.0, 0.0, 0.0), stream=None) -> Object:
    """Upload a synth.Scene (mesh, per-level hash + features, MLP weights; or,
    for scenes with density cubes, the cubes in place of the mesh)."""
    if hashes is None:
        hashes = build_hashes(scene)
    L = scene.n_levels
    V = np.ascontiguousarray(scene.vertices, np.float32)
    F = np.ascontiguousarray(scene.triangles, np.int32)
    res = np.ascontiguousarray(scene.resolutions, np.int32)
    feats = [np.ascontiguousarray(f, np.float32) for f in scene.features]
    w1 = np.ascontiguousarray(scene.w1, np.float32)
    w2 = np.ascontiguousarray(scene.w2, np.float32)
    w3 = np.ascontiguousarray(scene.w3, np.float32)
    hp = (ctypes.POINTER(HashStruct) * L)(*[h._h for h in hashes])
    fp = (ctypes.c_void_p * L)(*[f.ctypes.data for f in feats])
    d = ObjectDesc()
    d.n_vertices, d.n_triangles = len(V), len(F)
    d.vertices, d.triangles = V.ctypes.data, F.ctypes.data
    d.n_levels, d.n_features = L, 2
    d.resolution = res.ctypes.data
    d.hashes = ctypes.cast(hp, ctypes.c_void_p)
    d.features = ctypes.cast(fp, ctypes.c_void_p)
    d.features_fp16 = int(scene.feature_fp16 if fp16 is None else fp16)
    d.w1, d.w2, d.w3 = w1.ctypes.data, w2.ctypes.data, w3.ctypes.data
    for k in range(3):
        d.fp8_act_scale[k] = float(fp8_act_scale[k])
    d.domain_lo = float(scene.domain_lo)
    d.domain_scale = float(np.float32(1.0 / scene.domain_side))
    cubes = getattr(scene, "cubes", None)
    keep = []
    if cubes is not None:
        cells = np.ascontiguousarray(cubes.cells, np.int32)
        dens = np.ascontiguousarray(cubes.density, np.float32)
        diff = np.ascontiguousarray(cubes.diffuse, np.float32)
        keep = [cells, dens, diff]
        c = CubesDesc()
        c.b, c.r, c.n_cubes = int(cubes.b), int(cubes.r), len(cells)
        c.cells, c.density, c.diffuse = cells.ctypes.data, dens.ctypes.data, diff.ctypes.data
        c.side, c.step = float(cubes.side), float(cubes.step)
        c.t_min, c.alpha_miss = float(cubes.t_min), float(cubes.alpha_miss)
        keep.append(c)
        d.cubes = ctypes.pointer(c)
    out = ctypes.c_void_p()
    _check(lib().inolf_object_create(ctypes.byref(d), _stream(stream), ctypes.byref(out)))
    del keep
    return Object(out.value, L, scene.d_in, hashes)


# ---------------------------------------------------------------------------
# rendering
# ---------------------------------------------------------------------------
def render_workspace_bytes(n_rays: int) -> int:
    return int(lib().inolf_render_workspace_bytes(int(n_rays)))


def _workspace(n_rays, device):
    import torch
    nb = render_workspace_bytes(n_rays)
    return torch.empty((nb + 15) // 16 * 4, dtype=torch.int32, device=device)


def render(obj: Object, cams: np.ndarray, W: int, H: int, prec="fp32", rgba_out=None, tri_out=None, t_out=None,
           workspace=None, stream=None):
    """Render pinhole views (cams: host [n_views, 13] float32).  Returns rgba
    [n_views, H, W, 4] (a new CUDA tensor unless rgba_out is given)."""
    import torch
    cams = np.ascontiguousarray(cams, np.float32).reshape(-1, 13)
    nv = len(cams)
    if rgba_out is None:
        rgba_out = torch.empty((nv, H, W, 4), dtype=torch.float32, device="cuda")
    if workspace is None:
        workspace = _workspace(nv * W * H, rgba_out.device)
    p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    _check(lib().inolf_render(obj.handle, cams.ctypes.data, nv, W, H, p, _ptr(rgba_out), _ptr(tri_out),
                              _ptr(t_out), _ptr(workspace), workspace.numel() * workspace.element_size(),
                              _stream(stream)))
    _after(workspace, stream, nv > 0)
    return rgba_out


def trace_stats(obj: Object, cams: np.ndarray, W: int, H: int, workspace=None, stream=None) -> dict:
    """inolf_trace_stats: rays, hit rays, BVH inner-node visits and triangle
    tests of the closest-hit packets of pinhole views (cams: host [n, 13])."""
    cams = np.ascontiguousarray(cams, np.float32).reshape(-1, 13)
    nv = len(cams)
    if workspace is None:
        workspace = _workspace(min(nv, 16) * W * H, "cuda")
    out = np.zeros(5, np.int64)
    _check(lib().inolf_trace_stats(obj.handle, cams.ctypes.data, nv, W, H, out.ctypes.data, _ptr(workspace),
                                   workspace.numel() * workspace.element_size(), _stream(stream)))
    rays, hits, inner, tests, packets = (int(v) for v in out)
    return {"rays": rays, "hit_rays": hits, "inner_node_visits": inner, "triangle_tests": tests, "packets": packets,
            "node_visits_per_ray": inner / max(packets, 1), "triangle_tests_per_ray": tests / max(packets, 1)}


def probe_peaks(stream=None) -> dict:
    """inolf_probe_peaks: L2 streaming-read GB/s, L2 random 8-byte reads
    (G/s) and packed FP32 FMA TFLOP/s measured by microbenchmarks."""
    pk = Peaks()
    _check(lib().inolf_probe_peaks(ctypes.byref(pk), _stream(stream)))
    return {"l2_read_gbs": pk.l2_read_gbs, "l2_gather_gsps": pk.l2_gather_gsps, "fp32_tflops": pk.fp32_tflops}


def render_host(obj: Object, cams: np.ndarray, W: int, H: int, prec="fp32", host_out=None, staging=None,
                workspace=None, stream=None, views_per_chunk: int = 4):
    """inolf_render_host: render pinhole views into host memory (host_out: a
    pinned CPU float32 tensor [n_views, H, W, 4], allocated when None) with the
    device-to-host copies overlapped with rendering.  Returns host_out."""
    import torch
    cams = np.ascontiguousarray(cams, np.float32).reshape(-1, 13)
    nv = len(cams)
    if host_out is None:
        host_out = torch.empty((nv, H, W, 4), dtype=torch.float32, pin_memory=True)
    if staging is None:
        staging = torch.empty((2 * max(1, views_per_chunk) * H * W * 4,), dtype=torch.float32, device="cuda")
    if workspace is None:
        workspace = _workspace(max(1, views_per_chunk) * W * H, staging.device)
    p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    _check(lib().inolf_render_host(obj.handle, cams.ctypes.data, nv, W, H, p, _ptr(host_out), _ptr(staging),
                                   staging.numel() * staging.element_size(), _ptr(workspace),
                                   workspace.numel() * workspace.element_size(), _stream(stream)))
    return host_out


def render_rays(obj: Object, o, d, prec="fp32", rgba_out=None, tri_out=None, t_out=None, workspace=None,
                stream=None):
    """Render explicit rays (o, d: CUDA float32 [n, 3])."""
    import torch
    n = o.shape[0]
    if rgba_out is None:
        rgba_out = torch.empty((n, 4), dtype=torch.float32, device=o.device)
    if workspace is None:
        workspace = _workspace(n, o.device)
    p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    _check(lib().inolf_render_rays(obj.handle, _ptr(o), _ptr(d), n, p, _ptr(rgba_out), _ptr(tri_out),
                                   _ptr(t_out), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                   _stream(stream)))
    _after(workspace, stream, n > 0)
    return rgba_out


def calibrate_fp8(obj: Object, cams: np.ndarray, W: int, H: int, workspace=None, stream=None):
    """Per-tensor FP8 activation scales (amax / 448) from the FP32 path on the
    given views; frozen in the object until the next calibration."""
    cams = np.ascontiguousarray(cams, np.float32).reshape(-1, 13)
    if workspace is None:
        workspace = _workspace(len(cams) * W * H, "cuda")
    _check(lib().inolf_calibrate_fp8(obj.handle, cams.ctypes.data, len(cams), W, H, _ptr(workspace),
                                     workspace.numel() * workspace.element_size(), _stream(stream)))
    return obj.fp8_scales()


NOALLOC_MAX_RAYS = 1048576


def render_rays_noalloc(obj: Object, o, d, prec="fp32", rgba_out=None, tri_out=None, t_out=None, stream=None):
    """inolf_render_rays_noalloc: like render_rays but with the library's fixed
    device scratch instead of a workspace (n <= NOALLOC_MAX_RAYS), for callers
    that must not allocate device memory while rendering.  Pass rgba_out to
    keep this call itself free of allocations as well."""
    import torch
    n = o.shape[0]
    if rgba_out is None:
        rgba_out = torch.empty((n, 4), dtype=torch.float32, device=o.device)
    p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    _check(lib().inolf_render_rays_noalloc(obj.handle, _ptr(o), _ptr(d), n, p, _ptr(rgba_out), _ptr(tri_out),
                                           _ptr(t_out), _stream(stream)))
    return rgba_out


def march_rays(obj: Object, o, d, k_out=None, t_out=None, alpha_out=None, workspace=None, stream=None):
    """inolf_march_rays: hit sample k (-1 = miss), its t and alpha_c of the
    density march (objects with density cubes).  Returns (k, t, alpha)."""
    import torch
    n = o.shape[0]
    if k_out is None:
        k_out = torch.empty(n, dtype=torch.int32, device=o.device)
    if t_out is None:
        t_out = torch.empty(n, dtype=torch.float32, device=o.device)
    if alpha_out is None:
        alpha_out = torch.empty(n, dtype=torch.float32, device=o.device)
    if workspace is None:
        workspace = _workspace(n, o.device)
    _check(lib().inolf_march_rays(obj.handle, _ptr(o), _ptr(d), n, _ptr(k_out), _ptr(t_out), _ptr(alpha_out),
                                  _ptr(workspace), workspace.numel() * workspace.element_size(), _stream(stream)))
    _after(workspace, stream, n > 0)
    return k_out, t_out, alpha_out


def encode_rays(obj: Object, o, d, slots_out, feat_out, workspace=None, stream=None):
    """Stage outputs: per hit ray and level the 8 corner slots and the
    interpolated features (rows of missing rays untouched)."""
    n = o.shape[0]
    if workspace is None:
        workspace = _workspace(n, o.device)
    _check(lib().inolf_encode_rays(obj.handle, _ptr(o), _ptr(d), n, _ptr(slots_out), _ptr(feat_out),
                                   _ptr(workspace), workspace.numel() * workspace.element_size(),
                                   _stream(stream)))
    _after(workspace, stream, n > 0)


# ---------------------------------------------------------------------------
# launch statistics (CUDA events around every library kernel launch)
# ---------------------------------------------------------------------------
class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("ms", ctypes.c_double)]


def stats_enable(on: bool = True):
    lib().inolf_stats_enable.argtypes = [ctypes.c_int32]
    _check(lib().inolf_stats_enable(int(bool(on))))


def stats_reset():
    _check(lib().inolf_stats_reset())


def stats_read() -> dict:
    """{kernel name: {"launches": n, "ms": summed device ms}} since the last reset."""
    L = lib()
    arr = (KernelStat * 64)()
    n = ctypes.c_int32()
    L.inolf_stats_read.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    _check(L.inolf_stats_read(ctypes.cast(arr, ctypes.c_void_p), 64, ctypes.byref(n)))
    return {arr[i].name.decode(): {"launches": int(arr[i].launches), "ms": float(arr[i].ms)}
            for i in range(min(n.value, 64))}


# ---------------------------------------------------------------------------
# training: backward, parameter updates, autograd
# ---------------------------------------------------------------------------
def backward(obj: Object, o, d, d_rgba, grad_tables, gw1, gw2, gw3, workspace=None, stream=None, tri=None,
             t=None):
    """inolf_backward: accumulate (+=) dLoss/d(tables, W1, W2, W3) for rays
    (o, d) given dLoss/dRGBA; all tensors on the device, FP32.  With the
    forward's tri / t (inolf_backward_hits) the rays are not traced again."""
    n = o.shape[0]
    if workspace is None:
        workspace = _workspace(n, o.device)
    tp = (ctypes.c_void_p * obj.L)(*[x.data_ptr() for x in grad_tables])
    if tri is not None:
        _check(lib().inolf_backward_hits(obj.handle, _ptr(o), _ptr(d), n, _ptr(tri), _ptr(t), _ptr(d_rgba),
                                         ctypes.cast(tp, ctypes.c_void_p), _ptr(gw1), _ptr(gw2), _ptr(gw3),
                                         _ptr(workspace), workspace.numel() * workspace.element_size(),
                                         _stream(stream)))
        _after(workspace, stream, n > 0)
        return
    _check(lib().inolf_backward(obj.handle, _ptr(o), _ptr(d), n, _ptr(d_rgba), ctypes.cast(tp, ctypes.c_void_p),
                                _ptr(gw1), _ptr(gw2), _ptr(gw3), _ptr(workspace),
                                workspace.numel() * workspace.element_size(), _stream(stream)))
    _after(workspace, stream, n > 0)


def load_params(obj: Object, tables=None, w1=None, w2=None, w3=None, stream=None):
    """inolf_object_load_params from device tensors (tables slot-ordered [m^3, 2])."""
    tp = None
    keep = []
    if tables is not None:
        arr = (ctypes.c_void_p * obj.L)(*[(t.data_ptr() if t is not None else None) for t in tables])
        tp = ctypes.cast(arr, ctypes.c_void_p)
        keep.append(arr)
    _check(lib().inolf_object_load_params(obj.handle, tp, _ptr(w1), _ptr(w2), _ptr(w3), _stream(stream)))


def _render_fn():
    import torch

    class _RenderRays(torch.autograd.Function):
        """Forward through inolf_render_rays, backward through inolf_backward
        (FP32 recompute).  The object's parameters are loaded from the given
        tensors before the forward."""

        @staticmethod
        def forward(ctx, o, d, field, prec, w1, w2, w3, *tables):
            load_params(field.obj, tables, w1, w2, w3)
            tri = torch.empty(o.shape[0], dtype=torch.int32, device=o.device)
            t = torch.empty(o.shape[0], dtype=torch.float32, device=o.device)
            rgba = render_rays(field.obj, o, d, prec, tri_out=tri, t_out=t)
            ctx.save_for_backward(o, d, tri, t)
            ctx.field = field
            return rgba

        @staticmethod
        def backward(ctx, g):
            o, d, tri, t = ctx.saved_tensors
            f = ctx.field
            gt = [torch.zeros_like(x) for x in f.tables]
            g1, g2, g3 = torch.zeros_like(f.w1), torch.zeros_like(f.w2), torch.zeros_like(f.w3)
            backward(f.obj, o, d, g.contiguous(), gt, g1, g2, g3, tri=tri, t=t)  # the forward's hits
            return (None, None, None, None, g1, g2, g3, *gt)

    return _RenderRays


class Field:
    """A trainable i-NOLF object: the feature tables (slot order) and MLP
    weights are torch CUDA tensors with requires_grad; ``render(o, d)`` is
    differentiable with respect to all of them."""

    def __init__(self, scene, hashes=None, fp16: bool = False):
        import torch
        self.obj = object_create(scene, hashes, fp16=fp16)
        tables, w1, w2, w3 = self.obj.read_params()
        dev = torch.device("cuda")
        self.tables = [torch.from_numpy(t).to(dev).requires_grad_() for t in tables]
        self.w1 = torch.from_numpy(w1).to(dev).requires_grad_()
        self.w2 = torch.from_numpy(w2).to(dev).requires_grad_()
        self.w3 = torch.from_numpy(w3).to(dev).requires_grad_()
        self._fn = _render_fn()

    def parameters(self):
        return [self.w1, self.w2, self.w3] + list(self.tables)

    def render(self, o, d, prec="fp32"):
        return self._fn.apply(o, d, self, prec, self.w1, self.w2, self.w3, *self.tables)


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------
class ServeParams(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_slots", ctypes.c_int32), ("max_width", ctypes.c_int32),
                ("max_height", ctypes.c_int32), ("max_hits", ctypes.c_int32), ("wait_limit_ns", ctypes.c_int64),
                ("idle_limit_ns", ctypes.c_int64), ("ctas_per_sm", ctypes.c_int32), ("policy", ctypes.c_int32),
                ("max_rays_in_flight", ctypes.c_int64)]


class Request(ctypes.Structure):
    _fields_ = [("camera", ctypes.c_float * 13), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("viewer_id", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class Result(ctypes.Structure):
    _fields_ = [("frame", ctypes.c_void_p), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("latency_ns", ctypes.c_int64), ("rays", ctypes.c_int64)]


_cudart = None


def _device_copy(dst_ptr: int, src_ptr: int, nbytes: int):
    """cudaMemcpy (default kind) through the CUDA runtime the library uses."""
    global _cudart
    if _cudart is None:
        for cand in ("/usr/local/cuda/lib64/libcudart.so.13", "libcudart.so.13", "libcudart.so"):
            try:
                _cudart = ctypes.CDLL(cand)
                break
            except OSError:
                continue
        _cudart.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    st = _cudart.cudaMemcpy(ctypes.c_void_p(dst_ptr), ctypes.c_void_p(src_ptr), nbytes, 4)  # cudaMemcpyDefault
    if st != 0:
        raise RuntimeError(f"cudaMemcpy failed ({st})")


class Server:
    """inolf_server: persistent-kernel request loop over resident objects."""

    def __init__(self, hbm_budget=4 << 30, max_slots=48, max_width=3840, max_height=2160, max_hits=4,
                 wait_limit_ns=1_000_000_000, idle_limit_ns=20_000_000, ctas_per_sm=0, policy=0,
                 max_rays_in_flight=0):
        L = lib()
        vp = ctypes.c_void_p
        L.inolf_serve_create.argtypes = [ctypes.POINTER(ServeParams), ctypes.POINTER(vp)]
        L.inolf_serve_add_object.argtypes = [vp, vp, vp]
        L.inolf_serve_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
        L.inolf_serve_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(Result)]
        L.inolf_serve_cancel.argtypes = [vp, ctypes.c_uint64]
        L.inolf_serve_release.argtypes = [vp, ctypes.c_uint64]
        L.inolf_serve_destroy.argtypes = [vp]
        L.inolf_serve_set_viewer.argtypes = [vp, ctypes.c_uint32, ctypes.c_double]
        L.inolf_serve_counters.argtypes = [vp] + [ctypes.POINTER(ctypes.c_int64)] * 4
        L.inolf_serve_profile.argtypes = [vp, vp, ctypes.c_int32]
        prm = ServeParams(hbm_budget, max_slots, max_width, max_height, max_hits, wait_limit_ns, idle_limit_ns,
                          ctas_per_sm, policy, max_rays_in_flight)
        h = vp()
        _check(L.inolf_serve_create(ctypes.byref(prm), ctypes.byref(h)))
        self._h = h.value
        self.objects = []

    def add_object(self, obj: Object, translation=(0.0, 0.0, 0.0)):
        t = np.ascontiguousarray(translation, np.float32)
        _check(lib().inolf_serve_add_object(self._h, obj.handle, t.ctypes.data))
        self.objects.append(obj)

    def submit(self, camera, width: int, height: int, prec="fp32", viewer_id: int = 0, flags: int = 0) -> int:
        r = Request()
        cam = np.ascontiguousarray(camera, np.float32).ravel()
        for k in range(13):
            r.camera[k] = float(cam[k])
        r.width, r.height = width, height
        r.precision = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        r.viewer_id, r.flags = viewer_id, flags
        t = ctypes.c_uint64()
        _check(lib().inolf_serve_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int):
        """(status, Result): status is OK, PENDING or a negative error code."""
        res = Result()
        st = lib().inolf_serve_poll(self._h, ticket, ctypes.byref(res))
        return st, res

    def wait(self, ticket: int, timeout_s: float = 60.0):
        import time
        t0 = time.monotonic()
        while True:
            st, res = self.poll(ticket)
            if st != PENDING:
                return st, res
            if time.monotonic() - t0 > timeout_s:
                raise TimeoutError(f"request {ticket} still pending after {timeout_s} s")
            time.sleep(0.0002)

    def frame(self, res: Result):
        """Copy a completed frame into a new CUDA tensor [H, W, 4]."""
        import torch
        out = torch.empty((res.height, res.width, 4), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        _device_copy(out.data_ptr(), res.frame, res.height * res.width * 16)
        return out

    def cancel(self, ticket: int):
        _check(lib().inolf_serve_cancel(self._h, ticket))

    def set_viewer(self, viewer_id: int, target_fps: float):
        _check(lib().inolf_serve_set_viewer(self._h, viewer_id, target_fps))

    def counters(self) -> dict:
        v = [ctypes.c_int64() for _ in range(4)]
        _check(lib().inolf_serve_counters(self._h, *[ctypes.byref(x) for x in v]))
        return dict(zip(("admitted", "refused", "denied", "completed"), (x.value for x in v)))

    PROFILE_KEYS = ("claim_cycles", "trace_cycles", "shade_cycles", "composite_cycles", "done_cycles", "tiles",
                    "hits", "mlp_batches", "weight_stagings", "ctas", "regs_per_thread", "static_smem",
                    "dynamic_smem", "ctas_per_sm")

    def profile(self, reset: bool = False) -> dict:
        """inolf_serve_profile: SM cycles per phase of the request loop and
        event counts, summed over the persistent CTAs (waits for the kernel to
        go idle)."""
        v = np.zeros(len(self.PROFILE_KEYS), np.int64)
        _check(lib().inolf_serve_profile(self._h, v.ctypes.data, 1 if reset else 0))
        return dict(zip(self.PROFILE_KEYS, (int(x) for x in v)))

    def release(self, ticket: int):
        _check(lib().inolf_serve_release(self._h, ticket))

    def close(self):
        if getattr(self, "_h", None):
            lib().inolf_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


# ---------------------------------------------------------------------------
# scheduling policy (Algorithm 1), host-only
# ---------------------------------------------------------------------------
class Scheduler:
    """inolf_sched: the multi-user dispatch policy; times are given in ns."""

    def __init__(self, max_rays_in_flight: int = 0):
        L = lib()
        vp, i64, u32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
        L.inolf_sched_create.argtypes = [i64, ctypes.POINTER(vp)]
        L.inolf_sched_destroy.argtypes = [vp]
        L.inolf_sched_destroy.restype = None
        L.inolf_sched_set_viewer.argtypes = [vp, u32, ctypes.c_double, i64]
        L.inolf_sched_admit.argtypes = [vp, u32, u64, i64, i64]
        L.inolf_sched_next.argtypes = [vp, i64, ctypes.POINTER(u64)]
        L.inolf_sched_complete.argtypes = [vp, u64, i64]
        L.inolf_sched_cancel.argtypes = [vp, u64]
        L.inolf_sched_state.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_int32)] + [ctypes.POINTER(i64)] * 3
        L.inolf_sched_wait_ns.argtypes = [vp, u32, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        h = vp()
        _check(L.inolf_sched_create(max_rays_in_flight, ctypes.byref(h)))
        self._h = h.value

    def set_viewer(self, viewer, fps, now):
        _check(lib().inolf_sched_set_viewer(self._h, viewer, fps, now))

    def admit(self, viewer, fid, rays, now) -> int:
        """Status: OK, or E_BUDGET when a new client is denied (starvation)."""
        return lib().inolf_sched_admit(self._h, viewer, fid, rays, now)

    def next(self, now):
        i = ctypes.c_uint64()
        st = lib().inolf_sched_next(self._h, now, ctypes.byref(i))
        return i.value if st == OK else None

    def complete(self, fid, now):
        _check(lib().inolf_sched_complete(self._h, fid, now))

    def cancel(self, fid) -> int:
        return lib().inolf_sched_cancel(self._h, fid)

    def state(self, now) -> dict:
        st = ctypes.c_int32()
        v = [ctypes.c_int64() for _ in range(3)]
        _check(lib().inolf_sched_state(self._h, now, ctypes.byref(st), *[ctypes.byref(x) for x in v]))
        return {"starving": bool(st.value), "rays_in_flight": v[0].value, "pending": v[1].value,
                "denied": v[2].value}

    def wait_ns(self, viewer):
        w, t = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().inolf_sched_wait_ns(self._h, viewer, ctypes.byref(w), ctypes.byref(t)))
        return w.value, t.value

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.inolf_sched_destroy(self._h)
            self._h = None
