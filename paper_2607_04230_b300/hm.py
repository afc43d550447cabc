"""Thin Python binding of libhm (include/hm.h): argument marshalling only.

Every step of the rendering path runs in the CUDA kernels behind the C ABI;
this module only packs structs, passes device pointers of torch tensors and
the current CUDA stream, and turns error codes into exceptions.  There is no
CPU fallback: if libhm.so is missing or cannot load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libhm.so")
_HEADER = os.path.join(os.path.dirname(_PKG), "include", "hm.h")

HM_OK = 0
STATUS_NAMES = {0: "HM_OK", 1: "HM_ERR_INVALID_ARG", 2: "HM_ERR_OOM", 3: "HM_ERR_CUDA",
                4: "HM_ERR_CAPACITY", 5: "HM_ERR_TIMEOUT", 6: "HM_ERR_NOT_READY", 7: "HM_ERR_DEVICE_CHECK"}
MAX_LIGHTS = 8
MAX_GROOMS_PER_CALL = 64


class HmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class GroomDesc(ctypes.Structure):
    _fields_ = [("num_layers", ctypes.c_int32), ("num_verts", ctypes.c_int32), ("num_faces", ctypes.c_int32),
                ("segments_per_strand", ctypes.c_int32), ("num_strands", ctypes.c_int64),
                ("layer_verts", ctypes.c_void_p), ("faces", ctypes.c_void_p), ("strand_face", ctypes.c_void_p),
                ("strand_bary", ctypes.c_void_p), ("strand_albedo", ctypes.c_void_p),
                ("bundle_delta", ctypes.c_void_p), ("strand_width_m", ctypes.c_float),
                ("roughness", ctypes.c_float), ("tilt", ctypes.c_float), ("vert_ao", ctypes.c_void_p),
                ("vert_uv", ctypes.c_void_p)]


class Camera(ctypes.Structure):
    _fields_ = [("view_proj", ctypes.c_float * 16), ("cam_pos", ctypes.c_float * 3), ("near_m", ctypes.c_float),
                ("far_m", ctypes.c_float), ("tan_half_fovy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("key_layout", ctypes.c_int32)]


KEYS_ROW_MAJOR, KEYS_BLOCK_2X2 = 0, 1


class LodParams(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_int32), ("lambda_", ctypes.c_float)]


class ShadowMap(ctypes.Structure):
    _fields_ = [("d_map", ctypes.c_void_p), ("cam", Camera), ("light", ctypes.c_int32), ("sigma", ctypes.c_float),
                ("bias_m", ctypes.c_float), ("depth_correction", ctypes.c_int32)]


class Lights(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("dir", (ctypes.c_float * 3) * MAX_LIGHTS),
                ("radiance", (ctypes.c_float * 3) * MAX_LIGHTS), ("ambient", ctypes.c_float),
                ("k_d", ctypes.c_float), ("k_s", ctypes.c_float), ("n_shadows", ctypes.c_int32),
                ("shadows", ctypes.POINTER(ShadowMap))]


class FilterParams(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_int32), ("radius", ctypes.c_int32), ("s_par", ctypes.c_float),
                ("s_perp", ctypes.c_float), ("sigma_c", ctypes.c_float), ("iso_scale", ctypes.c_float),
                ("strip_halfwidth", ctypes.c_float), ("depth_reject_m", ctypes.c_float),
                ("depth_mismatch_m", ctypes.c_float)]


class Tuning(ctypes.Structure):
    _fields_ = [("raster_precheck", ctypes.c_int32), ("raster_min_blocks", ctypes.c_int32),
                ("raster_ctas_per_sm", ctypes.c_int32), ("resolve_tile_h", ctypes.c_int32),
                ("raster_bin_w", ctypes.c_int32), ("raster_bin_h", ctypes.c_int32),
                ("raster_bin_chunk", ctypes.c_int32), ("reserved", ctypes.c_int32)]


TUNING_FIELDS = ("raster_precheck", "raster_min_blocks", "raster_ctas_per_sm", "resolve_tile_h", "raster_bin_w",
                 "raster_bin_h", "raster_bin_chunk")

STATS_FIELDS = ("strands", "segments", "bundles_culled", "covered_center", "covered_cons")


def declared_symbols() -> list:
    """Function names declared in include/hm.h."""
    txt = open(_HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:hm_status|size_t|const char \*)\s*(hm_\w+)\s*\(", txt, re.M)))


_lib = None


def lib():
    """Load libhm.so (built in-tree by paper_2607_04230_b300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"libhm.so not built ({_LIB_PATH}); run paper_2607_04230_b300.build.build()")
    L = ctypes.CDLL(_LIB_PATH)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "hm_create_groom": [P, P, P],
        "hm_destroy_groom": [P],
        "hm_set_lod": [P, P],
        "hm_update_layer_verts": [P, P, P],
        "hm_update_albedo": [P, P, P],
        "hm_render_visibility": [P, i32, P, P, P, P, i32, P, P],
        "hm_render_visibility_range": [P, i32, i32, i32, P, P, P, P, i32, P, P],
        "hm_render_visibility_multiview": [P, i32, P, i32, P, P, P, i32, P, P],
        "hm_resolve_shade": [P, i32, P, P, P, P, P, P, P, P],
        "hm_render_visibility_msaa": [P, i32, P, i32, P, i32, P, P],
        "hm_render_shadow_map": [P, i32, P, P, P, P, P],
        "hm_render_visibility_compressed": [P, i32, P, P, P, P, i32, P, P],
        "hm_resolve_compressed": [P, P, P, P, P, P, P, P],
        "hm_resolve_msaa": [P, i32, P, P, i32, P, P, P],
        "hm_shade_backward": [P, i32, P, P, P, P, P, P, P, P, P, P],
        "hm_shade_backward_noalloc": [P, i32, P, P, P, P, P, P, P, P, P],
        "hm_get_lod": [P, P, P, P],
        "hm_groom_info": [P, P, P, P, P, P],
        "hm_get_device_status": [P],
        "hm_set_phase_events": [P, i32],
        "hm_set_tuning": [P],
        "hm_get_tuning": [P],
        "hm_probe_atomic_min": [P, i64, i32, i32, P],
        "hm_probe_quotient": [P, P, P, i64, P],
    }
    for name, args in sig.items():
        if hasattr(L, name):
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
    if hasattr(L, "hm_backward_scratch_bytes"):
        L.hm_backward_scratch_bytes.argtypes = [i32, i32]
        L.hm_backward_scratch_bytes.restype = ctypes.c_size_t
        L.hm_resolve_scratch_bytes.argtypes = [i32, i32]
        L.hm_resolve_scratch_bytes.restype = ctypes.c_size_t
    if hasattr(L, "hm_vis_buffer_keys"):
        L.hm_vis_buffer_keys.argtypes = [P]
        L.hm_vis_buffer_keys.restype = ctypes.c_size_t
    L.hm_status_string.argtypes = [ctypes.c_int]
    L.hm_status_string.restype = ctypes.c_char_p
    L.hm_last_error.argtypes = []
    L.hm_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def check(status: int):
    if status != HM_OK:
        raise HmError(status, lib().hm_last_error().decode(errors="replace"))


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------
# struct packing
# ---------------------------------------------------------------------------

def camera_struct(cam) -> Camera:
    c = Camera()
    vp = np.ascontiguousarray(cam.view_proj, np.float32).reshape(16)
    for i in range(16):
        c.view_proj[i] = float(vp[i])
    for i in range(3):
        c.cam_pos[i] = float(np.float32(cam.cam_pos[i]))
    c.near_m, c.far_m, c.tan_half_fovy = cam.near, cam.far, cam.tan_half_fovy
    c.width, c.height = cam.width, cam.height
    c.key_layout = int(getattr(cam, "key_layout", KEYS_ROW_MAJOR))
    return c


def vis_buffer_keys(width: int, height: int, key_layout: int = KEYS_ROW_MAJOR) -> int:
    """Keys in one key layer (hm_vis_buffer_keys)."""
    c = Camera()
    c.width, c.height, c.key_layout = width, height, key_layout
    return int(lib().hm_vis_buffer_keys(ctypes.byref(c)))


def key_layout_index(width: int, height: int, key_layout: int) -> np.ndarray:
    """[height * width] index of each row-major pixel's key in a layer of
    the given layout (the identity for row-major)."""
    y, x = np.divmod(np.arange(width * height, dtype=np.int64), width)
    if key_layout == KEYS_ROW_MAJOR:
        return y * width + x
    wb = (width + 1) // 2
    return (((y >> 1) * wb + (x >> 1)) << 2) | ((y & 1) << 1) | (x & 1)


def keys_row_major(keys: np.ndarray, width: int, height: int, key_layout: int) -> np.ndarray:
    """A key layer of the given layout as row-major [height * width] keys."""
    return keys[key_layout_index(width, height, key_layout)]


def lights_struct(lights, shadows=None) -> Lights:
    """hm_lights of a synth.Lights; shadows: optional list of
    (synth.ShadowSpec, CUDA int64 tensor holding that light's map)."""
    L = Lights()
    n = lights.dirs.shape[0]
    if n > MAX_LIGHTS:
        raise ValueError("too many lights")
    L.count = n
    for i in range(n):
        for k in range(3):
            L.dir[i][k] = float(lights.dirs[i, k])
            L.radiance[i][k] = float(lights.radiance[i, k])
    L.ambient, L.k_d, L.k_s = lights.ambient, lights.k_d, lights.k_s
    shadows = list(shadows or [])
    arr = (ShadowMap * max(len(shadows), 1))()
    for i, (spec, t) in enumerate(shadows):
        arr[i].d_map = _dptr(t)
        arr[i].cam = camera_struct(spec.cam)
        arr[i].light = int(spec.light)
        arr[i].sigma = float(spec.sigma)
        arr[i].bias_m = float(spec.bias_m)
        arr[i].depth_correction = int(spec.depth_correction)
    L.n_shadows = len(shadows)
    L.shadows = ctypes.cast(arr, ctypes.POINTER(ShadowMap)) if shadows else None
    L._keep = arr                      # the array lives as long as the struct
    return L


def filter_struct(f) -> FilterParams:
    s = FilterParams()
    s.enabled, s.radius = int(f.enabled), int(f.radius)
    s.s_par, s.s_perp, s.sigma_c, s.iso_scale = f.s_par, f.s_perp, f.sigma_c, f.iso_scale
    s.strip_halfwidth, s.depth_reject_m, s.depth_mismatch_m = f.strip_halfwidth, f.depth_reject_m, f.depth_mismatch_m
    return s


# ---------------------------------------------------------------------------
# grooms and calls
# ---------------------------------------------------------------------------

class Groom:
    """A hair mesh uploaded to the current CUDA device (hm_create_groom)."""

    def __init__(self, g, stream=None):
        self._keep = dict(
            lv=np.ascontiguousarray(g.layer_verts, np.float32),
            faces=np.ascontiguousarray(g.faces, np.int32),
            sf=np.ascontiguousarray(g.strand_face, np.uint32),
            bary=np.ascontiguousarray(g.strand_bary, np.float32),
            alb=np.ascontiguousarray(g.strand_albedo, np.float32),
            delta=np.ascontiguousarray(g.bundle_delta, np.float32),
            ao=None if getattr(g, "vert_ao", None) is None else np.ascontiguousarray(g.vert_ao, np.float32),
            uv=None if getattr(g, "vert_uv", None) is None else np.ascontiguousarray(g.vert_uv, np.float32))
        d = GroomDesc()
        d.num_layers, d.num_verts, d.num_faces = g.num_layers, g.num_verts, g.num_faces
        d.segments_per_strand, d.num_strands = g.segments_per_strand, g.num_strands
        k = self._keep
        d.layer_verts, d.faces, d.strand_face = k["lv"].ctypes.data, k["faces"].ctypes.data, k["sf"].ctypes.data
        d.strand_bary, d.strand_albedo, d.bundle_delta = k["bary"].ctypes.data, k["alb"].ctypes.data, k["delta"].ctypes.data
        d.strand_width_m, d.roughness, d.tilt = g.strand_width_m, g.roughness, g.tilt
        d.vert_ao = None if k["ao"] is None else k["ao"].ctypes.data
        d.vert_uv = None if k["uv"] is None else k["uv"].ctypes.data
        h = ctypes.c_void_p()
        check(lib().hm_create_groom(ctypes.byref(d), _stream_ptr(stream), ctypes.byref(h)))
        self.handle = h
        self.num_faces = g.num_faces
        self.num_strands = g.num_strands
        self.num_layers = g.num_layers
        self.num_verts = g.num_verts
        self._keep = None

    def set_lod(self, enabled: int, lam: float = 3.0):
        p = LodParams(int(enabled), float(lam))
        check(lib().hm_set_lod(self.handle, ctypes.byref(p)))

    def update_layer_verts(self, t, stream=None):
        check(lib().hm_update_layer_verts(self.handle, _dptr(t), _stream_ptr(stream)))

    def update_albedo(self, t, stream=None):
        check(lib().hm_update_albedo(self.handle, _dptr(t), _stream_ptr(stream)))

    def get_lod(self, stream=None):
        n = np.zeros(self.num_faces, np.int32)
        c = np.zeros(self.num_faces, np.int32)
        check(lib().hm_get_lod(self.handle, n.ctypes.data_as(ctypes.c_void_p), c.ctypes.data_as(ctypes.c_void_p),
                               _stream_ptr(stream)))
        return n, c

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().hm_destroy_groom(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _handles(grooms):
    arr = (ctypes.c_void_p * len(grooms))(*[g.handle.value for g in grooms])
    return arr, len(grooms)


def render_visibility(grooms, cam, vis_center, vis_cons, scene_d24=None, clear=True, stats=None, stream=None):
    arr, n = _handles(grooms)
    c = camera_struct(cam)
    check(lib().hm_render_visibility(arr, n, ctypes.byref(c), _dptr(vis_center), _dptr(vis_cons), _dptr(scene_d24),
                                     int(bool(clear)), _dptr(stats), _stream_ptr(stream)))


def render_visibility_range(grooms, first, count, cam, vis_center, vis_cons, scene_d24=None, clear=True, stats=None,
                            stream=None):
    arr, n = _handles(grooms)
    c = camera_struct(cam)
    check(lib().hm_render_visibility_range(arr, n, int(first), int(count), ctypes.byref(c), _dptr(vis_center),
                                           _dptr(vis_cons), _dptr(scene_d24), int(bool(clear)), _dptr(stats),
                                           _stream_ptr(stream)))


def render_visibility_multiview(grooms, cams, vis_centers, vis_conses, clear=True, stats=None, stream=None):
    """Assemble the strands once and rasterize them into every view's layers
    (LOD from cams[0])."""
    arr, n = _handles(grooms)
    nv = len(cams)
    cs = (Camera * nv)(*[camera_struct(c) for c in cams])
    vc = (ctypes.c_void_p * nv)(*[t.data_ptr() for t in vis_centers])
    va = (ctypes.c_void_p * nv)(*[t.data_ptr() for t in vis_conses])
    for t in list(vis_centers) + list(vis_conses):
        _dptr(t)
    check(lib().hm_render_visibility_multiview(arr, n, cs, nv, vc, va, None, int(bool(clear)), _dptr(stats),
                                               _stream_ptr(stream)))


class Appearance(ctypes.Structure):
    _fields_ = [("d_table", ctypes.c_void_p), ("roughness", ctypes.c_float), ("tilt", ctypes.c_float)]


def render_visibility_compressed(grooms, cam, vis_center, vis_cons, scene_d24=None, clear=True, stats=None,
                                 stream=None):
    """hm_render_visibility with the compressed payload (tangent, uvw, AO)
    in the keys' low 40 bits."""
    arr, n = _handles(grooms)
    c = camera_struct(cam)
    check(lib().hm_render_visibility_compressed(arr, n, ctypes.byref(c), _dptr(vis_center), _dptr(vis_cons),
                                                _dptr(scene_d24), int(bool(clear)), _dptr(stats),
                                                _stream_ptr(stream)))


def resolve_compressed(cam, lights, filt, table, roughness, tilt, vis_center, vis_cons, rgba, stream=None):
    """Resolve of compressed keys; table: CUDA float32 [64][64][4]
    appearance (tip albedo rgb, root / tip ratio)."""
    c, L, f = camera_struct(cam), lights_struct(lights), filter_struct(filt)
    a = Appearance(_dptr(table).value, float(roughness), float(tilt))
    check(lib().hm_resolve_compressed(ctypes.byref(c), ctypes.byref(L), ctypes.byref(f), ctypes.byref(a),
                                      _dptr(vis_center), _dptr(vis_cons), _dptr(rgba), _stream_ptr(stream)))


def render_shadow_map(grooms, light_cam, map_center, map_cons, stats=None, stream=None):
    """Full-detail keys of every groom seen from the light (hm_render_shadow_map);
    map_cons is the map."""
    arr, n = _handles(grooms)
    c = camera_struct(light_cam)
    check(lib().hm_render_shadow_map(arr, n, ctypes.byref(c), _dptr(map_center), _dptr(map_cons), _dptr(stats),
                                     _stream_ptr(stream)))


def resolve_shade(grooms, cam, lights, filt, vis_center, vis_cons, rgba, stream=None, shadows=None,
                  tile_scratch=None):
    """tile_scratch: None, or a device tensor of resolve_scratch_bytes(W, H)
    bytes: list the tiles holding keys first and resolve only those (sparse
    frames)."""
    arr, n = _handles(grooms)
    c, L, f = camera_struct(cam), lights_struct(lights, shadows), filter_struct(filt)
    check(lib().hm_resolve_shade(arr, n, ctypes.byref(c), ctypes.byref(L), ctypes.byref(f), _dptr(vis_center),
                                 _dptr(vis_cons), _dptr(rgba), _dptr(tile_scratch), _stream_ptr(stream)))


def resolve_scratch_bytes(width: int, height: int) -> int:
    return int(lib().hm_resolve_scratch_bytes(int(width), int(height)))


def render_visibility_msaa(grooms, cam, samples: int, vis_samples, clear=True, stats=None, stream=None):
    """Multisample visibility into vis_samples, uint64 (int64 view)
    [samples][H*W]; samples in 1, 2, 4, 8."""
    arr, n = _handles(grooms)
    c = camera_struct(cam)
    check(lib().hm_render_visibility_msaa(arr, n, ctypes.byref(c), int(samples), _dptr(vis_samples),
                                          int(bool(clear)), _dptr(stats), _stream_ptr(stream)))


def resolve_msaa(grooms, cam, lights, samples: int, vis_samples, rgba, stream=None, shadows=None):
    """Shade every covered sample at its own position; rgba float32 [H*W][4]
    straight alpha (rgb mean over covered samples, alpha covered fraction)."""
    arr, n = _handles(grooms)
    c, L = camera_struct(cam), lights_struct(lights, shadows)
    check(lib().hm_resolve_msaa(arr, n, ctypes.byref(c), ctypes.byref(L), int(samples), _dptr(vis_samples),
                                _dptr(rgba), _stream_ptr(stream)))


def backward_scratch_bytes(width: int, height: int) -> int:
    return int(lib().hm_backward_scratch_bytes(int(width), int(height)))


def shade_backward(grooms, cam, lights, filt, vis_center, vis_cons, grad_rgba, grad_layer_verts, grad_albedo,
                   scratch, stream=None, shadows=None):
    arr, n = _handles(grooms)
    c, L, f = camera_struct(cam), lights_struct(lights, shadows), filter_struct(filt)
    glv = (ctypes.c_void_p * n)(*[(t.data_ptr() if t is not None else None) for t in grad_layer_verts])
    gal = (ctypes.c_void_p * n)(*[(t.data_ptr() if t is not None else None) for t in grad_albedo])
    check(lib().hm_shade_backward(arr, n, ctypes.byref(c), ctypes.byref(L), ctypes.byref(f), _dptr(vis_center),
                                  _dptr(vis_cons), _dptr(grad_rgba), glv, gal, _dptr(scratch), _stream_ptr(stream)))


def set_tuning(**kw):
    """Set launch-shape knobs (see hm_tuning in include/hm.h); unnamed ones
    keep their current value."""
    t = Tuning()
    check(lib().hm_get_tuning(ctypes.byref(t)))
    for k, v in kw.items():
        if k not in TUNING_FIELDS:
            raise KeyError(k)
        setattr(t, k, int(v))
    check(lib().hm_set_tuning(ctypes.byref(t)))


def get_tuning() -> dict:
    t = Tuning()
    check(lib().hm_get_tuning(ctypes.byref(t)))
    return {k: int(getattr(t, k)) for k in TUNING_FIELDS}


def set_phase_events(events):
    """Record torch.cuda.Event objects (enable_timing=True) at the phase
    boundaries of later calls on this thread; None turns it off."""
    if not events:
        check(lib().hm_set_phase_events(None, 0))
        return
    for e in events:
        if e is not None and not e.cuda_event:
            raise ValueError("record each torch.cuda.Event once before handing it to the library")
    arr = (ctypes.c_void_p * len(events))(*[(e.cuda_event if e is not None else None) for e in events])
    check(lib().hm_set_phase_events(arr, len(events)))


def probe_atomic_min(buf, rounds: int = 1, pattern: int = 0, stream=None):
    check(lib().hm_probe_atomic_min(_dptr(buf), buf.numel(), int(rounds), int(pattern), _stream_ptr(stream)))


def probe_quotient(num, den, out, stream=None):
    """out = the rasterizers' binary32 depth-parameter quotient num / den
    (float32 device tensors of one size; den >= 1)."""
    if not (num.numel() == den.numel() == out.numel()):
        raise ValueError("num, den and out must have the same size")
    check(lib().hm_probe_quotient(_dptr(num), _dptr(den), _dptr(out), num.numel(), _stream_ptr(stream)))


def stats_dict(stats_tensor):
    v = stats_tensor.cpu().numpy().view(np.uint64)
    return {k: int(v[i]) for i, k in enumerate(STATS_FIELDS)}


def shade_backward_noalloc(grooms, cam, lights, filt, vis_center, vis_cons, grad_rgba, grad_layer_verts,
                           grad_albedo, stream=None, shadows=None):
    """hm_shade_backward_noalloc: the adjoint without caller-allocated
    scratch (frames up to NOALLOC_MAX_PIXELS pixels)."""
    arr, n = _handles(grooms)
    c, L, f = camera_struct(cam), lights_struct(lights, shadows), filter_struct(filt)
    glv = (ctypes.c_void_p * n)(*[(t.data_ptr() if t is not None else None) for t in grad_layer_verts])
    gal = (ctypes.c_void_p * n)(*[(t.data_ptr() if t is not None else None) for t in grad_albedo])
    check(lib().hm_shade_backward_noalloc(arr, n, ctypes.byref(c), ctypes.byref(L), ctypes.byref(f),
                                          _dptr(vis_center), _dptr(vis_cons), _dptr(grad_rgba), glv, gal,
                                          _stream_ptr(stream)))


NOALLOC_MAX_PIXELS = 262144


def get_device_status(stream=None):
    check(lib().hm_get_device_status(_stream_ptr(stream)))


class Frame:
    """Device buffers of one frame: two key layers, RGBA, counters."""

    def __init__(self, width: int, height: int, device="cuda", tile_list: bool = False,
                 key_layout: int = KEYS_ROW_MAJOR):
        """tile_list: hold the resolve's tile-list scratch (sparse frames);
        key_layout: the layout of the two key layers (render() and the
        other Frame-level calls give the camera this layout)."""
        import torch
        nkeys = vis_buffer_keys(width, height, key_layout)
        if nkeys <= 0:
            raise ValueError("invalid frame size or key layout")
        self.width, self.height, self.key_layout = width, height, key_layout
        self.vis_center = torch.empty(nkeys, dtype=torch.int64, device=device)
        self.vis_cons = torch.empty(nkeys, dtype=torch.int64, device=device)
        self.rgba = torch.empty((height, width, 4), dtype=torch.float32, device=device)
        self.stats = torch.zeros(8, dtype=torch.int64, device=device)
        self.tile_scratch = None
        if tile_list:
            self.tile_scratch = torch.empty((resolve_scratch_bytes(width, height) + 3) // 4, dtype=torch.int32,
                                            device=device)

    def keys_numpy(self):
        """Both key layers as row-major [height * width] uint64 (whatever the layout)."""
        out = []
        for t in (self.vis_center, self.vis_cons):
            k = t.cpu().numpy().view(np.uint64)
            out.append(k if self.key_layout == KEYS_ROW_MAJOR else
                       keys_row_major(k, self.width, self.height, self.key_layout))
        return tuple(out)

    def camera(self, cam):
        """cam with this frame's key layout."""
        if int(getattr(cam, "key_layout", KEYS_ROW_MAJOR)) == self.key_layout:
            return cam
        import dataclasses
        return dataclasses.replace(cam, key_layout=self.key_layout)


def render(grooms, scene, frame: Frame, stream=None, shadows=None):
    """Visibility + resolve of one frame (both on the current stream);
    shadows as for lights_struct.  The camera takes the frame's key layout."""
    cam = frame.camera(scene.camera)
    render_visibility(grooms, cam, frame.vis_center, frame.vis_cons, stats=frame.stats, stream=stream)
    resolve_shade(grooms, cam, scene.lights, scene.filt, frame.vis_center, frame.vis_cons, frame.rgba,
                  stream=stream, shadows=shadows, tile_scratch=frame.tile_scratch)


def upload_scene(scene, stream=None):
    """hm grooms for every groom of a synthetic scene, LOD set from the scene."""
    gs = []
    for g in scene.grooms:
        h = Groom(g, stream=stream)
        h.set_lod(scene.lod.enabled, scene.lod.lam)
        gs.append(h)
    return gs
