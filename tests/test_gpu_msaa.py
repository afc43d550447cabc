"""Multisample visibility and resolve (Sec. 3.3's MSAA reference) on the GPU
against the CPU oracle, through the C ABI.

Every sample layer is compared key for key with the oracle's multisample
rasterizer; the covered-sample count with the oracle's; RGBA within 1e-4 of
the FP64 multisample resolve.
"""
import numpy as np
import pytest

import oracle
from oracle import value64 as v64
from paper_2607_04230_b300 import synth

from _parity import RGBA_TOL, assert_keys_equal, assert_rgba_close

pytestmark = pytest.mark.gpu


def _gpu_msaa(scene, N):
    import torch
    from paper_2607_04230_b300 import hm
    grooms = hm.upload_scene(scene)
    cam = scene.camera
    vis = torch.empty((N, cam.width * cam.height), dtype=torch.int64, device="cuda")
    rgba = torch.empty((cam.width * cam.height, 4), dtype=torch.float32, device="cuda")
    stats = torch.zeros(8, dtype=torch.int64, device="cuda")
    hm.render_visibility_msaa(grooms, cam, N, vis, stats=stats)
    hm.resolve_msaa(grooms, cam, scene.lights, N, vis, rgba)
    torch.cuda.synchronize()
    hm.get_device_status()
    return (vis.cpu().numpy().view(np.uint64), rgba.cpu().numpy().astype(np.float64), hm.stats_dict(stats),
            [g.get_lod() for g in grooms])


def _check(scene, N, sample=None):
    vis, rgba, stats, glods = _gpu_msaa(scene, N)
    lods = oracle.lods_for(scene)
    for (n, c), (gn, gc) in zip(lods, glods):
        assert np.array_equal(n, gn) and np.array_equal(c, gc)
    ovis, cnt = oracle.raster_msaa(scene.grooms, scene.camera, lods, N)
    for k in range(N):
        assert_keys_equal(vis[k], ovis[k], f"sample layer {k} of {N}")
    assert stats["covered_center"] == cnt, (stats, cnt)
    cov = (ovis != oracle.EMPTY).sum(0)
    covered = np.nonzero(cov)[0]
    pix = covered
    if sample is not None and covered.size > sample:
        pix = np.sort(np.random.default_rng(0).choice(covered, size=sample, replace=False))
    sub = np.ascontiguousarray(ovis[:, pix])
    num, den = oracle.msaa_decisions(scene.grooms, scene.camera, lods, N, ovis)
    gts = [v64.GroomT(g, l[1], b) for g, l, b in zip(scene.grooms, lods, oracle.strand_bases(scene.grooms))]
    ref = v64.resolve_msaa(gts, scene.camera, scene.lights, sub, np.ascontiguousarray(num[:, pix]),
                           np.ascontiguousarray(den[:, pix])).numpy()
    err = assert_rgba_close(rgba, ref, pix)
    assert np.all(rgba[cov == 0] == 0.0)
    return cov, err


@pytest.mark.parametrize("N", [1, 2, 4, 8])
def test_msaa_tiny_256(N):
    sc = synth.scene_tiny_256()
    cov, err = _check(sc, N)
    assert (cov > 0).sum() > 2000 and err <= RGBA_TOL


@pytest.mark.parametrize("seed,W,H,N,lod", [(31, 97, 61, 4, 0), (32, 33, 17, 8, 1), (33, 250, 130, 2, 1)])
def test_msaa_ragged(seed, W, H, N, lod):
    sc = synth.tiny_scene(seed, width=W, height=H, num_strands=700, segments=7, num_layers=5,
                          length_m=0.06, dist_m=0.4, jitter_m=0.004)
    sc.lod = synth.LodParams(lod, 3.0)
    _check(sc, N)


def test_msaa_single_sample_equals_centre_layer():
    """One sample at the pixel centre is the centre-sample layer."""
    import torch
    from paper_2607_04230_b300 import hm
    sc = synth.tiny_scene(34, width=180, height=120, num_strands=1500)
    vis, _, _, _ = _gpu_msaa(sc, 1)
    grooms = hm.upload_scene(sc)
    frame = hm.Frame(sc.camera.width, sc.camera.height)
    hm.render_visibility(grooms, sc.camera, frame.vis_center, frame.vis_cons)
    torch.cuda.synchronize()
    vc, _ = frame.keys_numpy()
    assert_keys_equal(vis[0], vc, "1-sample layer vs centre layer")


def test_msaa_baked_ao_and_crowd():
    sc = synth.tiny_scene(35, width=160, height=128, num_strands=2000, num_layers=5, length_m=0.06)
    sc.grooms[0].vert_ao = synth.baked_ao(sc.grooms[0], seed=3)
    sc.lights.ambient = float(np.float32(0.4))
    _check(sc, 4)
    gs = synth.crowd_grooms(seed=12, n_side=2, strand_scale=0.04)
    _check(synth.scene_crowd_4k(gs, width=480, height=270), 4, sample=8000)


def test_msaa_1080p_full_size():
    """The 100k-strand 1920x1080 groom at 4 samples: every key of every
    sample layer, colour on sampled pixels."""
    sc = synth.scene_single_1080p()
    cov, _ = _check(sc, 4, sample=5000)
    assert (cov > 0).sum() > 100_000


@pytest.mark.parametrize("N", [2, 4, 8])
def test_msaa_thick_strands_largest_reach(N):
    """Strands wide enough that the sample box half-width saturates at half a
    pixel and short segments at grazing angles: the candidate columns and rows
    reach the farthest a sample box can (largest sample offset + 128/256 px),
    and every sample must still match the oracle."""
    sc = synth.tiny_scene(34, width=120, height=90, num_strands=500, segments=5, num_layers=4,
                          length_m=0.03, dist_m=0.25, jitter_m=0.004)
    sc.grooms[0].strand_width_m = np.float32(0.004)
    cov, err = _check(sc, N)
    assert (cov == N).sum() > 500 and err <= RGBA_TOL
