"""C ABI checks that need no GPU: the library loads, exports every symbol
include/hm.h declares, and rejects bad arguments before touching CUDA."""
import ctypes

import numpy as np
import pytest

from paper_2607_04230_b300 import build, hm, synth

INVALID = 1
CAPACITY = 4


@pytest.fixture(scope="module")
def L():
    build.build()
    return hm.lib()


def test_exports_every_declared_symbol(L):
    syms = hm.declared_symbols()
    assert len(syms) >= 14
    missing = [s for s in syms if not hasattr(L, s)]
    assert not missing, missing


def test_status_strings(L):
    for code, name in hm.STATUS_NAMES.items():
        assert L.hm_status_string(code).decode() == name


def _desc(g, **over):
    keep = dict(lv=np.ascontiguousarray(g.layer_verts, np.float32), faces=np.ascontiguousarray(g.faces, np.int32),
                sf=np.ascontiguousarray(g.strand_face, np.uint32), bary=np.ascontiguousarray(g.strand_bary, np.float32),
                alb=np.ascontiguousarray(g.strand_albedo, np.float32),
                delta=np.ascontiguousarray(g.bundle_delta, np.float32))
    keep.update(over.pop("arrays", {}))
    d = hm.GroomDesc()
    d.num_layers, d.num_verts, d.num_faces = g.num_layers, g.num_verts, g.num_faces
    d.segments_per_strand, d.num_strands = g.segments_per_strand, g.num_strands
    d.layer_verts, d.faces, d.strand_face = keep["lv"].ctypes.data, keep["faces"].ctypes.data, keep["sf"].ctypes.data
    d.strand_bary, d.strand_albedo = keep["bary"].ctypes.data, keep["alb"].ctypes.data
    d.bundle_delta = keep["delta"].ctypes.data
    d.strand_width_m, d.roughness, d.tilt = 1e-4, 0.15, -0.05
    for k, v in over.items():
        setattr(d, k, v)
    return d, keep


def _create(L, d):
    h = ctypes.c_void_p()
    return L.hm_create_groom(ctypes.byref(d), None, ctypes.byref(h)), h


def test_create_groom_rejects_bad_descriptors(L):
    g = synth.tiny_scene(0, num_strands=50).grooms[0]
    assert L.hm_create_groom(None, None, None) == INVALID
    for over in (dict(num_layers=1), dict(num_layers=33), dict(segments_per_strand=0),
                 dict(segments_per_strand=127), dict(num_faces=0), dict(strand_width_m=0.0),
                 dict(layer_verts=None)):
        d, keep = _desc(g, **over)
        assert _create(L, d)[0] == INVALID, over
    d, keep = _desc(g, num_strands=2 ** 31)
    assert _create(L, d)[0] == CAPACITY
    bad_faces = g.faces.copy()
    bad_faces[3, 1] = g.num_verts
    d, keep = _desc(g, arrays=dict(faces=bad_faces))
    assert _create(L, d)[0] == INVALID
    unsorted = g.strand_face.copy()
    unsorted[[0, -1]] = unsorted[[-1, 0]]
    d, keep = _desc(g, arrays=dict(sf=unsorted))
    assert _create(L, d)[0] == INVALID
    delta = g.bundle_delta.copy()
    delta[0] = 1.0
    d, keep = _desc(g, arrays=dict(delta=delta))
    assert _create(L, d)[0] == INVALID
    bary = g.strand_bary.copy()
    bary[5, 0] = -0.1
    d, keep = _desc(g, arrays=dict(bary=bary))
    assert _create(L, d)[0] == INVALID
    assert "barycentric" in L.hm_last_error().decode()


def test_render_and_resolve_reject_bad_arguments(L):
    sc = synth.tiny_scene(0, num_strands=10)
    cam = hm.camera_struct(sc.camera)
    fake = ctypes.c_void_p(1 << 20)         # never dereferenced: validation fails first
    grooms = (ctypes.c_void_p * 1)(1 << 20)
    assert L.hm_render_visibility(grooms, 1, None, fake, fake, None, 1, None, None) == INVALID
    bad = hm.camera_struct(sc.camera)
    bad.width = 0
    assert L.hm_render_visibility(grooms, 1, ctypes.byref(bad), fake, fake, None, 1, None, None) == INVALID
    bad = hm.camera_struct(sc.camera)
    bad.far_m = bad.near_m
    assert L.hm_render_visibility(grooms, 1, ctypes.byref(bad), fake, fake, None, 1, None, None) == INVALID
    bad = hm.camera_struct(sc.camera)
    bad.key_layout = 2
    assert L.hm_render_visibility(grooms, 1, ctypes.byref(bad), fake, fake, None, 1, None, None) == INVALID
    # multisample sample planes are row-major only
    blocked = hm.camera_struct(sc.camera)
    blocked.key_layout = hm.KEYS_BLOCK_2X2
    assert L.hm_render_visibility_msaa(grooms, 1, ctypes.byref(blocked), 4, fake, 1, None, None) == INVALID
    assert L.hm_render_visibility(grooms, 1, ctypes.byref(cam), None, fake, None, 1, None, None) == INVALID
    assert L.hm_render_visibility(grooms, 1, ctypes.byref(cam), ctypes.c_void_p((1 << 20) + 8), fake, None, 1,
                                  None, None) == INVALID
    assert L.hm_render_visibility(grooms, 1, ctypes.byref(cam), fake, fake, None, 1, None, None) == INVALID
    assert L.hm_render_visibility(grooms, 0, ctypes.byref(cam), fake, ctypes.c_void_p(2 << 20), None, 1, None,
                                  None) == INVALID
    assert L.hm_render_visibility(None, 1, ctypes.byref(cam), fake, ctypes.c_void_p(2 << 20), None, 1, None,
                                  None) == INVALID
    lights = hm.lights_struct(sc.lights)
    f = hm.filter_struct(synth.FilterParams(radius=9))
    assert L.hm_resolve_shade(grooms, 1, ctypes.byref(cam), ctypes.byref(lights), ctypes.byref(f), fake, fake, fake,
                              None, None) == INVALID
    lights.count = 9
    f = hm.filter_struct(synth.FilterParams())
    assert L.hm_resolve_shade(grooms, 1, ctypes.byref(cam), ctypes.byref(lights), ctypes.byref(f), fake, fake, fake,
                              None, None) == INVALID
    for n_s in (0, 3, 16):
        assert L.hm_render_visibility_msaa(grooms, 1, ctypes.byref(cam), n_s, fake, 1, None, None) == INVALID
    assert L.hm_render_visibility_msaa(grooms, 1, ctypes.byref(cam), 4, None, 1, None, None) == INVALID
    assert L.hm_render_visibility_msaa(grooms, 1, ctypes.byref(cam), 4, ctypes.c_void_p((1 << 20) + 8), 1, None,
                                       None) == INVALID
    assert L.hm_resolve_msaa(grooms, 1, ctypes.byref(cam), ctypes.byref(lights), 4, fake, fake, None) == INVALID
    lights.count = 1
    assert L.hm_resolve_msaa(grooms, 1, ctypes.byref(cam), ctypes.byref(lights), 5, fake, fake, None) == INVALID
    assert L.hm_resolve_msaa(grooms, 1, ctypes.byref(cam), ctypes.byref(lights), 4, fake, None, None) == INVALID
    assert L.hm_set_phase_events(None, 7) == INVALID
    assert L.hm_set_phase_events(None, 0) == 0
    assert L.hm_probe_atomic_min(None, 10, 1, 0, None) == INVALID


def test_tuning_and_range_arguments(L):
    t = hm.Tuning()
    assert L.hm_get_tuning(ctypes.byref(t)) == 0
    assert t.raster_min_blocks in (3, 4) and t.resolve_tile_h in (16, 32)
    assert (t.raster_bin_w, t.raster_bin_h, t.raster_bin_chunk) == (0, 0, 0)     # direct rasterizer
    for bad in ({"raster_precheck": 2}, {"raster_min_blocks": 5}, {"raster_ctas_per_sm": -1}, {"resolve_tile_h": 24},
                {"raster_bin_w": 8, "raster_bin_h": 16, "raster_bin_chunk": 256},
                {"raster_bin_w": 16, "raster_bin_h": 24, "raster_bin_chunk": 256},
                {"raster_bin_w": 16, "raster_bin_h": 16, "raster_bin_chunk": 512},
                {"raster_bin_w": 32},                                   # bin height and chunk missing
                {"raster_bin_h": 16}, {"raster_bin_chunk": 256}):       # set while the direct rasterizer is chosen
        b = hm.Tuning()
        L.hm_get_tuning(ctypes.byref(b))
        for field, v in bad.items():
            setattr(b, field, v)
        assert L.hm_set_tuning(ctypes.byref(b)) == INVALID, bad
    ok = hm.Tuning()
    L.hm_get_tuning(ctypes.byref(ok))
    ok.raster_bin_w, ok.raster_bin_h, ok.raster_bin_chunk = 32, 16, 1024
    assert L.hm_set_tuning(ctypes.byref(ok)) == 0
    assert L.hm_set_tuning(ctypes.byref(t)) == 0
    assert L.hm_set_tuning(None) == INVALID
    sc = synth.tiny_scene(0, num_strands=10)
    cam = hm.camera_struct(sc.camera)
    fake = ctypes.c_void_p(1 << 20)
    grooms = (ctypes.c_void_p * 2)(1 << 20, 2 << 20)
    for first, count in ((-1, 1), (0, 0), (1, 2), (2, 1)):
        assert L.hm_render_visibility_range(grooms, 2, first, count, ctypes.byref(cam), fake,
                                            ctypes.c_void_p(2 << 20), None, 1, None, None) == INVALID


def test_shadow_and_compressed_entries_reject_bad_arguments(L):
    """Validation of the shadow-map, compressed-payload and shadowed-lights
    arguments happens on the host before anything is launched."""
    sc = synth.tiny_scene(0, num_strands=10)
    cam = hm.camera_struct(sc.camera)
    fake, fake2 = ctypes.c_void_p(1 << 20), ctypes.c_void_p(2 << 20)
    grooms = (ctypes.c_void_p * 1)(1 << 20)
    bad = hm.camera_struct(sc.camera)
    bad.width = 0
    assert L.hm_render_shadow_map(grooms, 1, ctypes.byref(bad), fake, fake2, None, None) == INVALID
    assert L.hm_render_shadow_map(grooms, 1, ctypes.byref(cam), None, fake2, None, None) == INVALID
    assert L.hm_render_shadow_map(grooms, 1, ctypes.byref(cam), fake, fake, None, None) == INVALID
    assert L.hm_render_shadow_map(grooms, 1, ctypes.byref(cam), ctypes.c_void_p((1 << 20) + 8), fake2, None,
                                  None) == INVALID
    assert L.hm_render_visibility_compressed(grooms, 1, ctypes.byref(bad), fake, fake2, None, 1, None,
                                             None) == INVALID
    lights = hm.lights_struct(sc.lights)
    f = hm.filter_struct(synth.FilterParams())
    app = hm.Appearance(None, 0.15, -0.05)
    assert L.hm_resolve_compressed(ctypes.byref(cam), ctypes.byref(lights), ctypes.byref(f), ctypes.byref(app),
                                   fake, fake, fake, None, None) == INVALID
    app = hm.Appearance((1 << 20) + 4, 0.15, -0.05)
    assert L.hm_resolve_compressed(ctypes.byref(cam), ctypes.byref(lights), ctypes.byref(f), ctypes.byref(app),
                                   fake, fake, fake, None, None) == INVALID
    app = hm.Appearance(1 << 20, 0.0, -0.05)
    assert L.hm_resolve_compressed(ctypes.byref(cam), ctypes.byref(lights), ctypes.byref(f), ctypes.byref(app),
                                   fake, fake, fake, None, None) == INVALID
    # shadow maps on the lights: count, light index, duplicates, sigma, camera
    arr = (hm.ShadowMap * 2)()
    for i in range(2):
        arr[i].d_map = 1 << 20
        arr[i].cam = cam
        arr[i].light = 0
        arr[i].sigma = 10.0
        arr[i].bias_m = 0.0
        arr[i].depth_correction = 1
    def lights_with(n, mutate=None):
        Ls = hm.lights_struct(sc.lights)
        a = (hm.ShadowMap * 2)()
        ctypes.memmove(a, arr, ctypes.sizeof(arr))
        if mutate:
            mutate(a)
        Ls.n_shadows = n
        Ls.shadows = ctypes.cast(a, ctypes.POINTER(hm.ShadowMap))
        Ls._keep = a
        return Ls
    cases = [lights_with(2),                                               # more maps than lights
             lights_with(1, lambda a: setattr(a[0], "light", 1)),          # light out of range
             lights_with(1, lambda a: setattr(a[0], "sigma", -1.0)),
             lights_with(1, lambda a: setattr(a[0], "depth_correction", 2)),
             lights_with(1, lambda a: setattr(a[0], "d_map", (1 << 20) + 4))]
    bad_cam_map = lights_with(1)
    bad_cam_map._keep[0].cam.width = 0
    cases.append(bad_cam_map)
    for Ls in cases:
        assert L.hm_resolve_shade(grooms, 1, ctypes.byref(cam), ctypes.byref(Ls), ctypes.byref(f), fake, fake, fake,
                                  None, None) == INVALID
    # shadow maps are not taken by the compressed resolve
    app = hm.Appearance(1 << 20, 0.15, -0.05)
    Ls = lights_with(1)
    assert L.hm_resolve_compressed(ctypes.byref(cam), ctypes.byref(Ls), ctypes.byref(f), ctypes.byref(app),
                                   fake, fake, fake, None, None) == INVALID


def test_resolve_scratch_and_probe_arguments(L):
    """The tile-list scratch size covers the smallest resolve tiles (32 x 16),
    0 outside the resolution range; a misaligned scratch and an unknown probe
    pattern are rejected before anything is launched."""
    L.hm_resolve_scratch_bytes.restype = ctypes.c_size_t
    L.hm_resolve_scratch_bytes.argtypes = [ctypes.c_int32, ctypes.c_int32]
    # tile list (count and work counter, order, key counts of the 32 x 16
    # tiling, the decode pass's work counter), 16-byte aligned, then two
    # float4 per pixel for the two-pass resolve
    al = lambda b: (b + 15) // 16 * 16
    assert L.hm_resolve_scratch_bytes(1920, 1080) == al(4 * (3 + 2 * 60 * 68)) + 32 * 1920 * 1080
    assert L.hm_resolve_scratch_bytes(33, 17) == al(4 * (3 + 2 * 2 * 2)) + 32 * 33 * 17
    assert L.hm_resolve_scratch_bytes(0, 10) == 0 and L.hm_resolve_scratch_bytes(10, 16385) == 0
    # the adjoint's scratch: colour and screen-tangent gradients per pixel, then the same tile list
    L.hm_backward_scratch_bytes.restype = ctypes.c_size_t
    L.hm_backward_scratch_bytes.argtypes = [ctypes.c_int32, ctypes.c_int32]
    for w, h in ((1920, 1080), (512, 512), (33, 17)):
        assert L.hm_backward_scratch_bytes(w, h) == 32 * w * h + 4 * (3 + 2 * ((w + 31) // 32) * ((h + 15) // 16))
    assert L.hm_backward_scratch_bytes(0, 10) == 0
    sc = synth.tiny_scene(0, num_strands=10)
    cam = hm.camera_struct(sc.camera)
    fake = ctypes.c_void_p(1 << 20)
    grooms = (ctypes.c_void_p * 1)(1 << 20)
    lights = hm.lights_struct(sc.lights)
    f = hm.filter_struct(synth.FilterParams())
    for off in (2, 8):
        assert L.hm_resolve_shade(grooms, 1, ctypes.byref(cam), ctypes.byref(lights), ctypes.byref(f), fake, fake,
                                  fake, ctypes.c_void_p((1 << 20) + off), None) == INVALID
    for pattern in (-1, 3):
        assert L.hm_probe_atomic_min(fake, 16, 1, pattern, None) == INVALID
    assert L.hm_probe_atomic_min(fake, 0, 1, 0, None) == INVALID
    assert L.hm_probe_atomic_min(fake, 16, 0, 0, None) == INVALID
    assert L.hm_probe_quotient(None, None, None, -1, None) == INVALID
    assert L.hm_probe_quotient(None, fake, fake, 4, None) == INVALID
    assert L.hm_probe_quotient(None, None, None, 0, None) == 0      # empty: nothing launched


def test_key_buffer_sizes_per_layout(L):
    """hm_vis_buffer_keys: width * height row-major; 4 ceil(w/2) ceil(h/2) in
    2 x 2 blocks (odd sizes padded); 0 for an invalid layout or size.  The
    host-side index map is a bijection onto the blocked buffer's in-frame slots."""
    import numpy as np
    for w, h in ((1920, 1080), (203, 117), (1, 1), (2, 3), (16384, 16384)):
        assert hm.vis_buffer_keys(w, h, hm.KEYS_ROW_MAJOR) == w * h
        assert hm.vis_buffer_keys(w, h, hm.KEYS_BLOCK_2X2) == 4 * ((w + 1) // 2) * ((h + 1) // 2)
    assert hm.vis_buffer_keys(64, 64, 2) == 0 and hm.vis_buffer_keys(0, 64, 0) == 0
    assert hm.vis_buffer_keys(16385, 8, 0) == 0
    for w, h in ((7, 5), (8, 6), (33, 2)):
        idx = hm.key_layout_index(w, h, hm.KEYS_BLOCK_2X2)
        assert len(np.unique(idx)) == w * h and idx.max() < hm.vis_buffer_keys(w, h, hm.KEYS_BLOCK_2X2)
        # a 2 x 2 block of pixels fills one 32-byte sector (four consecutive keys)
        assert sorted(idx[[0, 1, w, w + 1]]) == [0, 1, 2, 3]
        assert np.array_equal(hm.key_layout_index(w, h, hm.KEYS_ROW_MAJOR), np.arange(w * h))
