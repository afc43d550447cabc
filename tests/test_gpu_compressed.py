"""Compressed G-buffer payload (Sec. 3.1.2) on the GPU against the CPU
oracle, through the C ABI: both key layers bit-exact (depth plus the
tangent / uvw / AO codes), covered-pair counts equal, RGBA of the
payload-only resolve within 1e-4 of the FP64 oracle."""
import numpy as np
import pytest

import oracle
from oracle import value64 as v64
from paper_2607_04230_b300 import synth

from _parity import RGBA_TOL, assert_keys_equal, assert_rgba_close

pytestmark = pytest.mark.gpu


def _check(scene, table_seed=0, sample=None):
    import torch
    from paper_2607_04230_b300 import hm
    grooms = hm.upload_scene(scene)
    frame = hm.Frame(scene.camera.width, scene.camera.height)
    table = synth.appearance_table(table_seed)
    tab = torch.from_numpy(table).cuda()
    g0 = scene.grooms[0]
    hm.render_visibility_compressed(grooms, scene.camera, frame.vis_center, frame.vis_cons, stats=frame.stats)
    hm.resolve_compressed(scene.camera, scene.lights, scene.filt, tab, g0.roughness, g0.tilt, frame.vis_center,
                          frame.vis_cons, frame.rgba)
    torch.cuda.synchronize()
    hm.get_device_status()
    vc, va = frame.keys_numpy()
    rgba = frame.rgba.cpu().numpy().astype(np.float64)
    stats = hm.stats_dict(frame.stats)
    lods = oracle.lods_for(scene)
    ovc, ova, cnt = oracle.raster(scene.grooms, scene.camera, lods, compressed=True)
    assert_keys_equal(vc, ovc, "compressed centre layer")
    assert_keys_equal(va, ova, "compressed conservative layer")
    assert stats["covered_center"] == cnt[0] and stats["covered_cons"] == cnt[1]
    dec = oracle.resolve_decisions(scene.grooms, scene.camera, lods, scene.filt, ovc, ova, compressed=True)
    covered = np.nonzero(ova != oracle.EMPTY)[0]
    pix = covered
    if sample is not None and covered.size > sample:
        pix = np.sort(np.random.default_rng(0).choice(covered, size=sample, replace=False))
    ref, pix = v64.resolve_cgb(scene.camera, scene.lights, scene.filt, ovc, ova, dec, table, g0.roughness, g0.tilt,
                               pixels=pix)
    err = assert_rgba_close(rgba, ref.numpy(), pix)
    empty = np.ones(ova.size, bool)
    empty[covered] = False
    assert np.all(rgba.reshape(-1, 4)[empty] == 0.0)
    return err


def test_compressed_tiny_256():
    assert _check(synth.scene_tiny_256()) <= RGBA_TOL


@pytest.mark.parametrize("seed,W,H,lod", [(51, 97, 61, 0), (52, 250, 130, 1)])
def test_compressed_ragged_lod(seed, W, H, lod):
    sc = synth.tiny_scene(seed, width=W, height=H, num_strands=900, segments=7, num_layers=5,
                          length_m=0.06, dist_m=0.4, jitter_m=0.004)
    sc.lod = synth.LodParams(lod, 3.0)
    _check(sc, table_seed=seed)


def test_compressed_baked_ao_and_filter_off():
    sc = synth.tiny_scene(53, width=160, height=128, num_strands=2000, num_layers=5, length_m=0.06)
    sc.grooms[0].vert_ao = synth.baked_ao(sc.grooms[0], seed=5)
    sc.lights.ambient = float(np.float32(0.4))
    _check(sc)
    sc.filt = synth.FilterParams(enabled=0)
    _check(sc)


def test_compressed_1080p_full_size():
    """The 100k-strand 1920x1080 groom: every key of both layers, colour on
    sampled pixels."""
    _check(synth.scene_single_1080p(), sample=6000)
