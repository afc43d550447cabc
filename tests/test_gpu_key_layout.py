"""The 2 x 2-blocked key layout (hm_camera.key_layout = HM_KEYS_BLOCK_2X2) on
the GPU.

Every reader and writer of the key layers addresses them through the same
pixel -> key index, so a frame in the blocked layout must hold, at every
pixel, exactly the key the row-major layout holds there (and the oracle's),
keep its padding keys EMPTY, and resolve to the same RGBA bit for bit.  The
cases: a ragged frame with several tiles, the scene-depth pre-fill, the
1080p groom and the 4K crowd (batched and per-character calls), multiview,
the compressed payload, the binned rasterizer, shadow maps in the blocked
layout, and the adjoint.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_04230_b300 import autograd, crowd, hm, synth

from _parity import assert_keys_equal, oracle_keys

pytestmark = pytest.mark.gpu

ROW, BLK = hm.KEYS_ROW_MAJOR, hm.KEYS_BLOCK_2X2


def _render(grooms, sc, layout, tile_list=True):
    fr = hm.Frame(sc.camera.width, sc.camera.height, tile_list=tile_list, key_layout=layout)
    hm.render(grooms, sc, fr)
    torch.cuda.synchronize()
    hm.get_device_status()
    return fr


def _padding_empty(fr):
    """The blocked layer's keys outside the frame (odd sizes) stay EMPTY."""
    pad = np.ones(fr.vis_center.numel(), bool)
    pad[hm.key_layout_index(fr.width, fr.height, fr.key_layout)] = False
    for t in (fr.vis_center, fr.vis_cons):
        k = t.cpu().numpy().view(np.uint64)
        assert np.all(k[pad] == oracle.EMPTY)


def _same(a, b, what):
    for x, y, layer in zip(a.keys_numpy(), b.keys_numpy(), ("centre", "conservative")):
        assert_keys_equal(x, y, f"{layer} layer, {what}")
    assert np.array_equal(a.rgba.cpu().numpy(), b.rgba.cpu().numpy()), what


def test_blocked_keys_equal_oracle_on_a_ragged_frame():
    # 203 x 117: odd in both directions, so the last block column and row are half padding
    sc = synth.tiny_scene(41, width=203, height=117, num_strands=3000)
    lods, vc, va, counts = oracle_keys(sc)
    grooms = hm.upload_scene(sc)
    row = _render(grooms, sc, ROW)
    for tile_list in (True, False):
        blk = _render(grooms, sc, BLK, tile_list=tile_list)
        gvc, gva = blk.keys_numpy()
        assert_keys_equal(gvc, vc, "centre layer, blocked")
        assert_keys_equal(gva, va, "conservative layer, blocked")
        st = hm.stats_dict(blk.stats)
        assert (st["covered_center"], st["covered_cons"]) == (counts[0], counts[1])
        _padding_empty(blk)
        _same(blk, row, f"blocked vs row-major, tile list {tile_list}")


def test_blocked_scene_depth_prefill():
    sc = synth.tiny_scene(42, width=131, height=97, num_strands=800)
    lods, vc0, _, _ = oracle_keys(sc)
    d = (vc0 >> np.uint64(40)).astype(np.int64)
    rng = np.random.default_rng(2)
    scene = np.where(rng.random(d.size) < 0.5, np.median(d[d < 2 ** 24 - 1]), 2 ** 24 - 1).astype(np.uint32)
    ovc, ova, _ = oracle.raster(sc.grooms, sc.camera, lods, prefill_d24=scene)
    grooms = hm.upload_scene(sc)
    fr = hm.Frame(sc.camera.width, sc.camera.height, key_layout=BLK)
    sd = torch.from_numpy(scene.view(np.int32)).cuda()
    hm.render_visibility(grooms, fr.camera(sc.camera), fr.vis_center, fr.vis_cons, scene_d24=sd)
    torch.cuda.synchronize()
    gvc, gva = fr.keys_numpy()
    assert_keys_equal(gvc, ovc, "centre layer with scene depth, blocked")
    assert_keys_equal(gva, ova, "conservative layer with scene depth, blocked")
    _padding_empty(fr)


def test_blocked_equals_row_major_at_1080p():
    sc = synth.scene_single_1080p()
    grooms = hm.upload_scene(sc)
    _same(_render(grooms, sc, BLK), _render(grooms, sc, ROW), "1080p")


def test_blocked_crowd_batched_and_per_character():
    sc = synth.scene_crowd_4k()
    ref = crowd.Crowd(sc)
    ref.render_batched()
    blk = crowd.Crowd(sc, key_layout=BLK)
    blk.render_batched()
    torch.cuda.synchronize()
    _same(blk.frame, ref.frame, "crowd, one call over all grooms")
    blk.render_per_character()
    torch.cuda.synchronize()
    _same(blk.frame, ref.frame, "crowd, one call per groom")
    hm.get_device_status()


def test_blocked_multiview_compressed_and_binned():
    sc = synth.tiny_scene(43, width=160, height=121, num_strands=1500)
    grooms = hm.upload_scene(sc)
    W, H = sc.camera.width, sc.camera.height
    # multiview: two views of the same groom, both in the blocked layout
    cams = synth.view_offsets(sc.camera, [-0.02, 0.02])
    rows = [hm.Frame(W, H) for _ in cams]
    blks = [hm.Frame(W, H, key_layout=BLK) for _ in cams]
    hm.render_visibility_multiview(grooms, cams, [f.vis_center for f in rows], [f.vis_cons for f in rows])
    hm.render_visibility_multiview(grooms, [b.camera(c) for b, c in zip(blks, cams)],
                                   [f.vis_center for f in blks], [f.vis_cons for f in blks])
    torch.cuda.synchronize()
    for r, b in zip(rows, blks):
        for x, y in zip(b.keys_numpy(), r.keys_numpy()):
            assert_keys_equal(x, y, "multiview view, blocked")
    # compressed payload
    tab = torch.from_numpy(synth.appearance_table(0)).cuda()
    g0 = sc.grooms[0]
    out = []
    for layout in (ROW, BLK):
        fr = hm.Frame(W, H, key_layout=layout)
        cam = fr.camera(sc.camera)
        hm.render_visibility_compressed(grooms, cam, fr.vis_center, fr.vis_cons)
        hm.resolve_compressed(cam, sc.lights, sc.filt, tab, 0.15, -0.05, fr.vis_center, fr.vis_cons, fr.rgba)
        torch.cuda.synchronize()
        out.append(fr)
    _same(out[1], out[0], "compressed payload")
    # binned rasterizer writing the blocked layout
    saved = hm.get_tuning()
    try:
        hm.set_tuning(raster_bin_w=32, raster_bin_h=16, raster_bin_chunk=256)
        _same(_render(grooms, sc, BLK), _render(grooms, sc, ROW), "binned rasterizer")
    finally:
        hm.set_tuning(**saved)
    hm.get_device_status()


def test_blocked_shadow_map():
    sc = synth.tiny_scene(44, width=120, height=96, num_strands=1200)
    grooms = hm.upload_scene(sc)
    lcam = synth.light_camera(sc.grooms, sc.lights.dirs[0], size=151, dist_m=0.5)
    out = []
    for layout in (ROW, BLK):
        mcam = synth.Camera(**{**lcam.__dict__, "key_layout": layout})
        n = hm.vis_buffer_keys(mcam.width, mcam.height, layout)
        mc = torch.empty(n, dtype=torch.int64, device="cuda")
        ma = torch.empty(n, dtype=torch.int64, device="cuda")
        hm.render_shadow_map(grooms, mcam, mc, ma)
        spec = synth.ShadowSpec(light=0, cam=mcam, sigma=150.0, bias_m=0.0005, depth_correction=1)
        fr = hm.Frame(sc.camera.width, sc.camera.height, key_layout=layout)
        cam = fr.camera(sc.camera)
        hm.render_visibility(grooms, cam, fr.vis_center, fr.vis_cons)
        hm.resolve_shade(grooms, cam, sc.lights, sc.filt, fr.vis_center, fr.vis_cons, fr.rgba, shadows=[(spec, ma)])
        torch.cuda.synchronize()
        out.append((fr, hm.keys_row_major(ma.cpu().numpy().view(np.uint64), mcam.width, mcam.height, layout)))
    assert_keys_equal(out[1][1], out[0][1], "shadow map, blocked")
    _same(out[1][0], out[0][0], "shadowed frame")
    hm.get_device_status()


def test_blocked_gradients_equal_row_major():
    sc = synth.tiny_scene(45, width=96, height=80, num_strands=300, dist_m=0.3)
    g = sc.grooms[0]
    handle = hm.upload_scene(sc)[0]
    rng = np.random.default_rng(5)
    grad = torch.from_numpy(rng.standard_normal((80, 96, 4)).astype(np.float32)).cuda()
    res = []
    for layout in (ROW, BLK):
        lv = torch.from_numpy(g.layer_verts).cuda().requires_grad_(True)
        alb = torch.from_numpy(g.strand_albedo).cuda().requires_grad_(True)
        rgba = autograd.render(handle, sc, hm.Frame(96, 80, key_layout=layout), lv, alb)
        torch.autograd.backward(rgba, grad_tensors=grad)
        res.append((rgba.detach().cpu().numpy(), lv.grad.cpu().numpy(), alb.grad.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0])
    # the adjoint accumulates with atomics: equal up to the order of the sums
    for a, b in zip(res[0][1:], res[1][1:]):
        np.testing.assert_allclose(b, a, rtol=1e-5, atol=1e-6 * np.abs(a).max())
