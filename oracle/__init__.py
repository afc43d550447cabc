"""CPU oracle for deferred software rasterization of hair-mesh strands.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
bench.py's CPU-baseline / reference leg, never by the product package.  It
shares no code with the CUDA library (paper_2607_04230_b300/csrc); the only
common input is the seeded generator paper_2607_04230_b300/synth.py, which
holds none of the method's arithmetic.

Layers:
  * hm_oracle.c  -- FP32 decision layer (strand generation, projection, 16.8
    snap, coverage, keys, LOD, resolve masks and counts), plain C.
  * value64.py   -- FP64 value layer (shading, bilateral filter, alpha,
    reconnection blend), plain PyTorch CPU ops, differentiable for the
    reference gradient.

Functions whose result the paper does not fix (the Hermite tangent scale, the
styling function, the shading coefficients, the filter's s_par/s_perp, the
depth-threshold unit, square centre samples) follow the readings written out
in hm_oracle.c and value64.py; their agreement with the paper's own images is
"parity unpinned" (the paper ships no data or images).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hm_oracle.c")
_LIB = os.path.join(_HERE, "_hm_oracle.so")

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
PAYLOAD_MASK = np.uint64(0xFFFFFFFFFF)


def build(force: bool = False) -> str:
    """Compile the C decision layer (gcc, no contraction, SSE scalar math)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-fno-unsafe-math-optimizations",
           "-Wall", "-Wdouble-promotion", "-Wno-misleading-indentation",
           _SRC, "-o", _LIB + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class OrcGroom(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("V", ctypes.c_int32), ("F", ctypes.c_int32),
                ("segs", ctypes.c_int32), ("S", ctypes.c_int64),
                ("layer_verts", ctypes.c_void_p), ("faces", ctypes.c_void_p),
                ("strand_face", ctypes.c_void_p), ("strand_bary", ctypes.c_void_p),
                ("lod_n", ctypes.c_void_p), ("lod_c", ctypes.c_void_p),
                ("strand_base", ctypes.c_uint64), ("width_m", ctypes.c_float),
                ("vert_ao", ctypes.c_void_p), ("vert_uv", ctypes.c_void_p)]


class OrcCamera(ctypes.Structure):
    _fields_ = [("m", ctypes.c_float * 16), ("near", ctypes.c_float), ("far", ctypes.c_float),
                ("tan_half_fovy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float
        _lib.orc_lod.argtypes = [P, P, i32, f32, P, P, P]
        _lib.orc_raster.argtypes = [P, i32, P, P, P, P, i32, i32]
        _lib.orc_resolve_decisions.argtypes = [P, i32, P, i32, f32, P, P, P, i64] + [P] * 10 + [i32, i32]
        _lib.orc_oct_encode.argtypes = [P]
        _lib.orc_oct_encode.restype = ctypes.c_uint32
        _lib.orc_oct_decode.argtypes = [ctypes.c_uint32, P]
        _lib.orc_unproject.argtypes = [P, f32, f32, f32, P]
        _lib.orc_strand_control_points.argtypes = [P, i64, i32, P]
        _lib.orc_strand_tangents.argtypes = [P, i64, i32, P]
        _lib.orc_project_point.argtypes = [P, P, P, P]
        _lib.orc_segment_covers.argtypes = [i64] * 7
        _lib.orc_depth24.argtypes = [i64, i64, i64, i64, f32, f32, i64, i64]
        _lib.orc_depth24.restype = ctypes.c_uint32
        _lib.orc_center_halfwidth.argtypes = [P, f32, f32, f32]
        _lib.orc_center_halfwidth.restype = i32
        _lib.orc_screen_tangent.argtypes = [P, P, P, P]
        _lib.orc_in_strip.argtypes = [ctypes.c_int, f32, f32, ctypes.c_int, ctypes.c_int, f32]
        _lib.orc_lod_counts.argtypes = [f32, i32, f32, i32, i32, P, P]
        _lib.orc_raster_msaa.argtypes = [P, i32, P, i32, P, P, P, P, i32]
        _lib.orc_msaa_decisions.argtypes = [P, i32, P, i32, P, P, P, P, P, i32]
        _lib.orc_shadow_texels.argtypes = [P, i32, P, P, P, P, i64, P, P, i32]
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def camera_struct(cam) -> OrcCamera:
    c = OrcCamera()
    vp = np.ascontiguousarray(cam.view_proj, np.float32).reshape(16)
    for i in range(16):
        c.m[i] = float(vp[i])
    c.near, c.far, c.tan_half_fovy = cam.near, cam.far, cam.tan_half_fovy
    c.width, c.height = cam.width, cam.height
    return c


def strand_bases(grooms) -> list:
    """Global id of each groom's first strand: grooms are numbered in order."""
    out, b = [], 0
    for g in grooms:
        out.append(b)
        b += g.num_strands
    return out


class _GroomRef:
    """Keeps numpy arrays alive while C holds pointers into them."""

    def __init__(self, g, lod_n, lod_c, base):
        self.lv = np.ascontiguousarray(g.layer_verts, np.float32)
        self.faces = np.ascontiguousarray(g.faces, np.int32)
        self.sf = np.ascontiguousarray(g.strand_face, np.uint32)
        self.bary = np.ascontiguousarray(g.strand_bary, np.float32)
        self.lod_n = np.ascontiguousarray(lod_n, np.int32)
        self.lod_c = np.ascontiguousarray(lod_c, np.int32)
        s = OrcGroom()
        s.L, s.V, s.F = g.num_layers, g.num_verts, g.num_faces
        s.segs, s.S = g.segments_per_strand, g.num_strands
        s.layer_verts, s.faces = self.lv.ctypes.data, self.faces.ctypes.data
        s.strand_face, s.strand_bary = self.sf.ctypes.data, self.bary.ctypes.data
        s.lod_n, s.lod_c = self.lod_n.ctypes.data, self.lod_c.ctypes.data
        s.strand_base, s.width_m = base, g.strand_width_m
        ao, uv = getattr(g, "vert_ao", None), getattr(g, "vert_uv", None)
        self.ao = None if ao is None else np.ascontiguousarray(ao, np.float32)
        self.uv = None if uv is None else np.ascontiguousarray(uv, np.float32)
        s.vert_ao = None if self.ao is None else self.ao.ctypes.data
        s.vert_uv = None if self.uv is None else self.uv.ctypes.data
        self.s = s


def _groom_array(grooms, lods):
    bases = strand_bases(grooms)
    refs = [_GroomRef(g, l[0], l[1], b) for g, l, b in zip(grooms, lods, bases)]
    arr = (OrcGroom * len(refs))(*[r.s for r in refs])
    return arr, refs


def lod(groom, cam, lod_params):
    """Per bundle (N_LOD, C) of Eqs. 1-5 (or full detail when disabled)."""
    ref = _GroomRef(groom, np.zeros(groom.num_faces, np.int32), np.zeros(groom.num_faces, np.int32), 0)
    n = np.zeros(groom.num_faces, np.int32)
    c = np.zeros(groom.num_faces, np.int32)
    cs = camera_struct(cam)
    delta = np.ascontiguousarray(groom.bundle_delta, np.float32)
    rc = lib().orc_lod(ctypes.byref(ref.s), ctypes.byref(cs), int(lod_params.enabled),
                       float(lod_params.lam), _ptr(delta), _ptr(n), _ptr(c))
    assert rc == 0
    return n, c


def lods_for(scene):
    return [lod(g, scene.camera, scene.lod) for g in scene.grooms]


def raster(grooms, cam, lods, prefill_d24=None, nthreads: int = 0, compressed: bool = False):
    """Both visibility layers as uint64 [H*W]: (vis_center, vis_cons, counts).

    counts = (covered centre pairs, covered conservative pairs), i.e. the
    number of atomicMin operations the method performs (before any
    early-out).  compressed: the keys carry the compressed G-buffer payload
    (tangent, uvw, AO) instead of the strand-segment id."""
    arr, refs = _groom_array(grooms, lods)
    npx = cam.width * cam.height
    if prefill_d24 is None:
        vis_c = np.full(npx, EMPTY, np.uint64)
    else:
        vis_c = (np.asarray(prefill_d24, np.uint64) << np.uint64(40)) | PAYLOAD_MASK
    vis_a = vis_c.copy()
    counts = np.zeros(2, np.int64)
    rc = lib().orc_raster(arr, len(refs), ctypes.byref(camera_struct(cam)), _ptr(vis_c), _ptr(vis_a),
                          _ptr(counts), int(bool(compressed)), int(nthreads))
    assert rc == 0
    return vis_c, vis_a, counts


# Standard sample positions (1/16 px from the pixel centre, y down) for 2, 4
# and 8 samples per pixel, scaled here to 1/256 px.
MSAA_PATTERNS = {
    1: [(0, 0)],
    2: [(4, 4), (-4, -4)],
    4: [(-2, -6), (6, -2), (-6, 2), (2, 6)],
    8: [(1, -3), (-1, 3), (5, 1), (-3, -5), (-5, 5), (-7, -1), (3, 7), (7, -7)],
}


def msaa_offsets(n: int):
    pat = MSAA_PATTERNS[n]
    return (np.array([16 * p[0] for p in pat], np.int32), np.array([16 * p[1] for p in pat], np.int32))


def raster_msaa(grooms, cam, lods, n_samples: int, nthreads: int = 0):
    """Multisample visibility: uint64 [n_samples][H*W] and the number of
    covered (pixel, sample) pairs."""
    arr, refs = _groom_array(grooms, lods)
    ox, oy = msaa_offsets(n_samples)
    vis = np.full((n_samples, cam.width * cam.height), EMPTY, np.uint64)
    count = np.zeros(1, np.int64)
    rc = lib().orc_raster_msaa(arr, len(refs), ctypes.byref(camera_struct(cam)), n_samples, _ptr(ox), _ptr(oy),
                               _ptr(vis), _ptr(count), int(nthreads))
    assert rc == 0
    return vis, int(count[0])


def msaa_decisions(grooms, cam, lods, n_samples: int, vis, nthreads: int = 0):
    arr, refs = _groom_array(grooms, lods)
    ox, oy = msaa_offsets(n_samples)
    vis = np.ascontiguousarray(vis, np.uint64)
    num = np.zeros(vis.shape, np.int64)
    den = np.zeros(vis.shape, np.int64)
    rc = lib().orc_msaa_decisions(arr, len(refs), ctypes.byref(camera_struct(cam)), n_samples, _ptr(ox), _ptr(oy),
                                  _ptr(vis), _ptr(num), _ptr(den), int(nthreads))
    assert rc == 0
    return num, den


def shadow_map(grooms, spec, nthreads: int = 0):
    """The shadow map of Sec. 3.2's depth fix: every groom at full detail
    (LOD off) seen from the light's camera spec.cam; returns the
    conservative key layer uint64 [h*w] (front-most hair depth per texel)."""
    from paper_2607_04230_b300.synth import LodParams
    lods = [lod(g, spec.cam, LodParams(0)) for g in grooms]
    _, va, _ = raster(grooms, spec.cam, lods, nthreads=nthreads)
    return va


def shadow_texels(grooms, cam, lods, keys, sx, sy, light_cam, nthreads: int = 0):
    """Texel of the light's map under each key's decoded position at the
    sample point (sx, sy) in 1/256 px; -1 for none (hm_oracle.c)."""
    arr, refs = _groom_array(grooms, lods)
    keys = np.ascontiguousarray(keys, np.uint64)
    sx = np.ascontiguousarray(sx, np.int64)
    sy = np.ascontiguousarray(sy, np.int64)
    out = np.full(keys.shape, -1, np.int64)
    rc = lib().orc_shadow_texels(arr, len(refs), ctypes.byref(camera_struct(cam)), _ptr(keys), _ptr(sx), _ptr(sy),
                                 keys.size, ctypes.byref(camera_struct(light_cam)), _ptr(out), int(nthreads))
    assert rc == 0
    return out


def centre_shadow_texels(grooms, cam, lods, vis_c, maps, nthreads: int = 0):
    """Per shadow map, the texel under every centre key decoded at its pixel
    centre ([H*W] int64, -1 where none): the decisions the shadowed resolve
    takes for the shaded colours."""
    W = cam.width
    p = np.arange(vis_c.size, dtype=np.int64)
    sx, sy = 256 * (p % W) + 128, 256 * (p // W) + 128
    return [shadow_texels(grooms, cam, lods, vis_c, sx, sy, spec.cam, nthreads) for spec, _ in maps]


def sample_shadow_texels(grooms, cam, lods, n_samples: int, vis_s, maps, nthreads: int = 0):
    """Per shadow map, [n_samples][H*W] texels of each sample layer's keys
    decoded at their own sample points."""
    W = cam.width
    ox, oy = msaa_offsets(n_samples)
    p = np.arange(vis_s.shape[1], dtype=np.int64)
    out = []
    for spec, _ in maps:
        t = np.empty(vis_s.shape, np.int64)
        for k in range(n_samples):
            t[k] = shadow_texels(grooms, cam, lods, vis_s[k], 256 * (p % W) + 128 + int(ox[k]),
                                 256 * (p // W) + 128 + int(oy[k]), spec.cam, nthreads)
        out.append(t)
    return out


def resolve_decisions(grooms, cam, lods, filt, vis_c, vis_a, pixels=None, nthreads: int = 0,
                      compressed: bool = False):
    """FP32 decisions per pixel for the G (centre) and A (conservative)
    references: num/den of the pixel-centre projection (0 for compressed
    keys), isotropic flag, strip hit counts."""
    arr, refs = _groom_array(grooms, lods)
    if pixels is None:
        n = cam.width * cam.height
        pix_ptr = None
    else:
        pixels = np.ascontiguousarray(pixels, np.int64)
        n = pixels.shape[0]
        pix_ptr = _ptr(pixels)
    out = {k: np.zeros(n, np.int64) for k in ("numG", "denG", "numA", "denA")}
    out.update({k: np.zeros(n, np.uint8) for k in ("isoG", "isoA")})
    out.update({k: np.zeros(n, np.int32) for k in ("HcG", "HaG", "HcA", "HaA")})
    vc = np.ascontiguousarray(vis_c, np.uint64)
    va = np.ascontiguousarray(vis_a, np.uint64)
    rc = lib().orc_resolve_decisions(
        arr, len(refs), ctypes.byref(camera_struct(cam)), int(filt.radius), float(filt.strip_halfwidth),
        _ptr(vc), _ptr(va), pix_ptr, n,
        *[_ptr(out[k]) for k in ("numG", "denG", "numA", "denA", "isoG", "isoA", "HcG", "HaG", "HcA", "HaA")],
        int(bool(compressed)), int(nthreads))
    assert rc == 0
    return out


# ---- single-step helpers for the pin tests ---------------------------------

def oct_encode(T) -> int:
    t = np.ascontiguousarray(T, np.float32)
    return int(lib().orc_oct_encode(_ptr(t)))


def oct_decode(code: int) -> np.ndarray:
    out = np.zeros(3, np.float32)
    lib().orc_oct_decode(int(code), _ptr(out))
    return out


def unproject(cam, xs: float, ys: float, w: float) -> np.ndarray:
    out = np.zeros(3, np.float32)
    lib().orc_unproject(ctypes.byref(camera_struct(cam)), float(xs), float(ys), float(w), _ptr(out))
    return out


def strand_control_points(groom, s: int, C: int) -> np.ndarray:
    ref = _GroomRef(groom, np.zeros(groom.num_faces, np.int32), np.zeros(groom.num_faces, np.int32), 0)
    out = np.zeros((C, 3), np.float32)
    assert lib().orc_strand_control_points(ctypes.byref(ref.s), int(s), int(C), _ptr(out)) == 0
    return out


def strand_tangents(groom, s: int, C: int) -> np.ndarray:
    ref = _GroomRef(groom, np.zeros(groom.num_faces, np.int32), np.zeros(groom.num_faces, np.int32), 0)
    out = np.zeros((C, 3), np.float32)
    assert lib().orc_strand_tangents(ctypes.byref(ref.s), int(s), int(C), _ptr(out)) == 0
    return out


def project_point(cam, p):
    p = np.ascontiguousarray(p, np.float32)
    xy = np.zeros(2, np.int32)
    wz = np.zeros(4, np.float32)
    valid = lib().orc_project_point(ctypes.byref(camera_struct(cam)), _ptr(p), _ptr(xy), _ptr(wz))
    return bool(valid), int(xy[0]), int(xy[1]), wz


def segment_covers(XA, YA, XB, YB, cx, cy, h) -> bool:
    return bool(lib().orc_segment_covers(int(XA), int(YA), int(XB), int(YB), int(cx), int(cy), int(h)))


def depth24(XA, YA, XB, YB, zA, zB, cx, cy) -> int:
    return int(lib().orc_depth24(int(XA), int(YA), int(XB), int(YB), float(zA), float(zB), int(cx), int(cy)))


def center_halfwidth(cam, width_m, wA, wB) -> int:
    return int(lib().orc_center_halfwidth(ctypes.byref(camera_struct(cam)), float(width_m), float(wA), float(wB)))


def screen_tangent(cam, X, T):
    X = np.ascontiguousarray(X, np.float32)
    T = np.ascontiguousarray(T, np.float32)
    ts = np.zeros(2, np.float32)
    iso = lib().orc_screen_tangent(ctypes.byref(camera_struct(cam)), _ptr(X), _ptr(T), _ptr(ts))
    return bool(iso), ts


def in_strip(iso, tsx, tsy, dx, dy, hw) -> bool:
    return bool(lib().orc_in_strip(int(iso), float(tsx), float(tsy), int(dx), int(dy), float(hw)))


def lod_counts(Lf, n_full, delta, L, cmax):
    """(N_LOD, C) of Eqs. 1, 4, 5 for a given LOD selection value."""
    n = np.zeros(1, np.int32)
    c = np.zeros(1, np.int32)
    lib().orc_lod_counts(float(Lf), int(n_full), float(delta), int(L), int(cmax), _ptr(n), _ptr(c))
    return int(n[0]), int(c[0])


def depth_thresholds(cam, filt):
    """Depth reject / mismatch thresholds in d24 units (Sec. 3.3.1, 3.3.2).
    Reading: the paper's 1.45e-3 and 5e-4 are metres of linear view depth;
    d24 = round(m / (far - near) * 2^24), computed in double."""
    span = float(np.float32(cam.far)) - float(np.float32(cam.near))
    rej = int(np.floor(float(np.float32(filt.depth_reject_m)) / span * 16777216.0 + 0.5))
    mis = int(np.floor(float(np.float32(filt.depth_mismatch_m)) / span * 16777216.0 + 0.5))
    return rej, mis
