"""GPU path vs the CPU oracle, through the C ABI.

Visibility keys and LOD results must be bit-exact; the number of covered
(pixel, layer) pairs must equal the oracle's count; RGBA must agree with the
FP64 oracle within 1e-4 (linear RGB and alpha).  Sizes span several raster
batches and resolve tiles with ragged edges; the full 1080p frame is checked
key for key and on sampled pixels for colour.
"""
import numpy as np
import pytest

import oracle
from paper_2607_04230_b300 import synth

from _parity import RGBA_TOL, assert_keys_equal, assert_rgba_close, check_full, gpu_frame, oracle_keys, oracle_rgba

pytestmark = pytest.mark.gpu


def test_tiny_256_frame():
    out, err = check_full(synth.scene_tiny_256())
    assert (out["vis_a"] != oracle.EMPTY).sum() > 5000
    assert err <= RGBA_TOL


@pytest.mark.parametrize("seed,W,H,lod", [(1, 97, 61, 0), (2, 33, 17, 1), (3, 250, 130, 1), (4, 129, 257, 0)])
def test_ragged_frames(seed, W, H, lod):
    sc = synth.tiny_scene(seed, width=W, height=H, num_strands=700, segments=7, num_layers=5,
                          length_m=0.06, dist_m=0.4, jitter_m=0.004)
    sc.lod = synth.LodParams(lod, 3.0)
    check_full(sc)


@pytest.mark.parametrize("radius,enabled", [(0, 1), (3, 1), (8, 1), (5, 0)])
def test_filter_variants(radius, enabled):
    sc = synth.tiny_scene(5, width=120, height=90, num_strands=800)
    sc.filt = synth.FilterParams(enabled=enabled, radius=radius)
    check_full(sc)


def test_lod_sweep_small_groom():
    g = synth.make_groom(7, 8, 3, 6, 0.2, 12_000, 16, curl_amp_m=0.01)
    for i in range(8):
        sc = synth.scene_lod_sweep(i, g)
        check_full(sc, sample=3000)


def test_camera_inside_groom_and_behind():
    sc = synth.tiny_scene(6, width=160, height=120, num_strands=900, dist_m=0.06)
    for lod in (0, 1):
        sc.lod = synth.LodParams(lod, 3.0)
        check_full(sc)
    # looking away: LOD culls every bundle; without LOD every segment is clipped
    ctr, _, _ = synth._aabb_center(sc.grooms)
    sc.camera = synth.make_camera(ctr + np.array([0, 0, 0.5]), ctr + np.array([0, 0, 1.5]), 40, 64, 48)
    for lod in (0, 1):
        sc.lod = synth.LodParams(lod, 3.0)
        out, _ = check_full(sc)
        assert np.all(out["vis_a"] == oracle.EMPTY)


def test_empty_groom_and_many_grooms():
    g0 = synth.tiny_scene(8, num_strands=0).grooms[0]
    g0.strand_face = g0.strand_face[:0]
    sc = synth.tiny_scene(9, width=96, height=96, num_strands=300)
    sc.grooms = [g0] + sc.grooms + [synth.tiny_scene(10, num_strands=200).grooms[0]]
    check_full(sc)


def test_crowd_small():
    gs = synth.crowd_grooms(seed=11, n_side=3, strand_scale=0.05)
    sc = synth.scene_crowd_4k(gs, width=640, height=360)
    check_full(sc, sample=20000)


def test_scene_depth_prefill():
    import torch
    from paper_2607_04230_b300 import hm
    sc = synth.tiny_scene(12, width=128, height=96, num_strands=600)
    rng = np.random.default_rng(0)
    lods, vc0, va0, _ = oracle_keys(sc)
    d = (vc0 >> np.uint64(40)).astype(np.int64)
    # a wall that hides part of the groom
    scene = np.where(rng.random(d.size) < 0.5, np.median(d[d < 2 ** 24 - 1]), 2 ** 24 - 1).astype(np.uint32)
    grooms = hm.upload_scene(sc)
    frame = hm.Frame(sc.camera.width, sc.camera.height)
    sd = torch.from_numpy(scene.view(np.int32)).cuda()
    hm.render_visibility(grooms, sc.camera, frame.vis_center, frame.vis_cons, scene_d24=sd)
    torch.cuda.synchronize()
    vc, va = frame.keys_numpy()
    ovc, ova, _ = oracle.raster(sc.grooms, sc.camera, lods, prefill_d24=scene)
    assert_keys_equal(vc, ovc, "centre layer with scene depth")
    assert_keys_equal(va, ova, "conservative layer with scene depth")


def test_deterministic_repeat():
    sc = synth.tiny_scene(13, width=200, height=150, num_strands=2000)
    a = gpu_frame(sc)
    b = gpu_frame(sc, grooms=a["grooms"])
    assert np.array_equal(a["vis_c"], b["vis_c"]) and np.array_equal(a["vis_a"], b["vis_a"])
    assert np.array_equal(a["rgba"], b["rgba"])


def test_single_groom_1080p_full_size():
    """100k strands x 16 segments at 1920x1080, the benchmark workload:
    every key of both layers; colour on 6,000 sampled pixels and on every
    promoted and depth-mismatch pixel (about 553k here); resolved as the
    benchmark resolves it (tile list, decode pass, filter pass)."""
    sc = synth.scene_single_1080p()
    out, err = check_full(sc, sample=6000, all_special=True, tile_list=True)
    assert out["stats"]["segments"] == 1_600_000
    assert out["stats"]["strands"] == 100_000


def test_crowd_4k_full_size():
    """64 grooms, 3840x2160, LOD by distance, one render call: every key;
    colour on sampled pixels and on every promoted and depth-mismatch pixel
    (about 319k here); resolved as the benchmark resolves it."""
    sc = synth.scene_crowd_4k()
    check_full(sc, sample=6000, all_special=True, tile_list=True)


def test_baked_ao_frame():
    """Per-vertex baked ambient occlusion (Sec. 3.4) interpolated along the
    strand and applied to the ambient term."""
    sc = synth.tiny_scene(14, width=200, height=160, num_strands=2500, num_layers=5, length_m=0.06)
    sc.grooms[0].vert_ao = synth.baked_ao(sc.grooms[0], seed=2)
    sc.lights.ambient = float(np.float32(0.4))
    check_full(sc)


@pytest.mark.parametrize("W,H,fovy", [(16384, 6, 0.5), (7, 16384, 170.0)])
def test_maximum_resolution_edges(W, H, fovy):
    """The largest frame side the library accepts, in either axis: the
    32-bit pixel-index and range arithmetic at its limit (a thin slice of
    the groom fills the long side)."""
    sc = synth.tiny_scene(17, width=W, height=H, num_strands=400, dist_m=0.35)
    ctr, _, _ = synth._aabb_center(sc.grooms)
    sc.camera = synth.make_camera(ctr + np.array([0.0, 0.0, 0.35]), ctr, fovy, W, H)
    out, _ = check_full(sc, sample=4000)
    assert (out["vis_a"] != oracle.EMPTY).sum() > 300


def test_degenerate_and_near_plane_segments():
    """Strands collapsed to a point (every layer at the same place: zero-length
    segments) and a camera whose near plane cuts the groom."""
    sc = synth.tiny_scene(18, width=96, height=80, num_strands=300, dist_m=0.3)
    g = sc.grooms[0]
    g.layer_verts[:] = g.layer_verts[0][None, :, :]
    out, _ = check_full(sc)
    assert (out["vis_a"] != oracle.EMPTY).sum() > 0
    sc2 = synth.tiny_scene(19, width=96, height=80, num_strands=600, dist_m=0.3)
    ctr, lo, hi = synth._aabb_center(sc2.grooms)
    sc2.camera = synth.make_camera(ctr + np.array([0.0, 0.0, 0.06]), ctr, 60, 96, 80, near=0.05)
    for lod in (0, 1):
        sc2.lod = synth.LodParams(lod, 3.0)
        check_full(sc2)


def test_segment_records_and_regeneration_agree():
    """The resolve decodes keys from the control points the visibility render
    recorded; after hm_update_layer_verts those records are stale and it
    regenerates the strands from the new layer vertices instead.  Same
    vertices: both decodes give the same image bit for bit.  New vertices
    without a new render: the image is the oracle's for the old keys and the
    new hair mesh (the records must not be used)."""
    import torch
    from paper_2607_04230_b300 import hm
    sc = synth.tiny_scene(13, width=120, height=96, num_strands=900, num_layers=5, jitter_m=0.004)
    sc.lod = synth.LodParams(1, 3.0)
    out = gpu_frame(sc)
    g, frame = out["grooms"][0], out["frame"]
    lv = torch.from_numpy(sc.grooms[0].layer_verts).cuda()
    rgba_rec = frame.rgba.clone()
    g.update_layer_verts(lv)                      # same vertices: records invalidated
    hm.resolve_shade(out["grooms"], sc.camera, sc.lights, sc.filt, frame.vis_center, frame.vis_cons, frame.rgba)
    torch.cuda.synchronize()
    assert torch.equal(frame.rgba, rgba_rec)
    # perturbed vertices, keys of the unperturbed render
    lv2 = synth.perturbed_layer_verts(sc.grooms[0], sigma_m=0.001, seed=5)
    g.update_layer_verts(torch.from_numpy(lv2).cuda())
    hm.resolve_shade(out["grooms"], sc.camera, sc.lights, sc.filt, frame.vis_center, frame.vis_cons, frame.rgba)
    torch.cuda.synchronize()
    hm.get_device_status()
    lods, vc, va, _ = oracle_keys(sc)
    sc.grooms[0].layer_verts = lv2
    ref, pix = oracle_rgba(sc, lods, vc, va)
    assert_rgba_close(frame.rgba.cpu().numpy().astype(np.float64), ref, pix)
    assert not np.allclose(frame.rgba.cpu().numpy().reshape(-1, 4)[pix], rgba_rec.cpu().numpy().reshape(-1, 4)[pix])


@pytest.mark.parametrize("tile_h", [32, 16])
def test_tile_list_resolve_bit_identical(tile_h):
    """hm_resolve_shade with the tile-list scratch (pre-pass listing the tiles
    that hold keys, persistent grid over them) writes the same image, bit for
    bit, as one CTA per tile, including the zeros of empty tiles and ragged
    edges; checked against the oracle too."""
    import torch
    from paper_2607_04230_b300 import hm
    sc = synth.tiny_scene(14, width=203, height=117, num_strands=600, dist_m=0.5)
    grooms = hm.upload_scene(sc)
    old = hm.get_tuning()
    hm.set_tuning(resolve_tile_h=tile_h)
    try:
        plain = hm.Frame(sc.camera.width, sc.camera.height)
        listed = hm.Frame(sc.camera.width, sc.camera.height, tile_list=True)
        hm.render(grooms, sc, plain)
        listed.vis_center.copy_(plain.vis_center)
        listed.vis_cons.copy_(plain.vis_cons)
        listed.rgba.fill_(float("nan"))          # every pixel must be written
        for _ in range(2):                        # the scratch is reused
            hm.resolve_shade(grooms, sc.camera, sc.lights, sc.filt, listed.vis_center, listed.vis_cons,
                             listed.rgba, tile_scratch=listed.tile_scratch)
        torch.cuda.synchronize()
        hm.get_device_status()
        assert torch.equal(plain.rgba, listed.rgba)
    finally:
        hm.set_tuning(**old)
    lods, vc, va, _ = oracle_keys(sc)
    covered = np.nonzero((va & oracle.PAYLOAD_MASK) != oracle.PAYLOAD_MASK)[0]
    ref, pix = oracle_rgba(sc, lods, vc, va, pixels=covered)
    assert_rgba_close(listed.rgba.cpu().numpy().astype(np.float64), ref, pix)


def test_tile_list_empty_frame_then_keys():
    """With the tile-list scratch, a frame without any key lists no tile: the
    decode pass's CTAs find their work counter past the end at once and every
    pixel is written RGBA 0; the same scratch then resolves a frame with keys
    exactly like one CTA per tile (the order pass resets both work counters)."""
    import torch
    from paper_2607_04230_b300 import hm
    sc = synth.tiny_scene(15, width=150, height=90, num_strands=500, dist_m=0.5)
    grooms = hm.upload_scene(sc)
    listed = hm.Frame(sc.camera.width, sc.camera.height, tile_list=True)
    listed.vis_center.fill_(-1)                # EMPTY keys everywhere
    listed.vis_cons.fill_(-1)
    listed.rgba.fill_(float("nan"))
    hm.resolve_shade(grooms, sc.camera, sc.lights, sc.filt, listed.vis_center, listed.vis_cons, listed.rgba,
                     tile_scratch=listed.tile_scratch)
    torch.cuda.synchronize()
    hm.get_device_status()
    assert torch.count_nonzero(listed.rgba).item() == 0
    plain = hm.Frame(sc.camera.width, sc.camera.height)
    hm.render(grooms, sc, plain)
    listed.vis_center.copy_(plain.vis_center)
    listed.vis_cons.copy_(plain.vis_cons)
    listed.rgba.fill_(float("nan"))
    hm.resolve_shade(grooms, sc.camera, sc.lights, sc.filt, listed.vis_center, listed.vis_cons, listed.rgba,
                     tile_scratch=listed.tile_scratch)
    torch.cuda.synchronize()
    hm.get_device_status()
    assert torch.count_nonzero(plain.vis_cons != -1).item() > 100
    assert torch.equal(plain.rgba, listed.rgba)
