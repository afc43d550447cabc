"""Shadow maps with the LOD depth correction (Sec. 3.2 "Depth Comparison
Artifact Fix", queried by the shading of Sec. 3.4) on the GPU against the
CPU oracle, through the C ABI.

The map (full-detail keys seen from the light) is bit-exact; the shadowed
frame's RGBA is within 1e-4 of the FP64 oracle; the camera's LOD state is
untouched by the map pass.
"""
import numpy as np
import pytest

import oracle
from oracle import value64 as v64
from paper_2607_04230_b300 import synth

from _parity import assert_keys_equal, assert_rgba_close

pytestmark = pytest.mark.gpu


def _gpu_map(grooms, spec):
    import torch
    from paper_2607_04230_b300 import hm
    npx = spec.cam.width * spec.cam.height
    mc = torch.empty(npx, dtype=torch.int64, device="cuda")
    ma = torch.empty(npx, dtype=torch.int64, device="cuda")
    hm.render_shadow_map(grooms, spec.cam, mc, ma)
    return mc, ma


def _check_shadowed(scene, specs, map_first=True, sample=None):
    import torch
    from paper_2607_04230_b300 import hm
    grooms = hm.upload_scene(scene)
    frame = hm.Frame(scene.camera.width, scene.camera.height)
    if map_first:
        maps_gpu = [_gpu_map(grooms, s) for s in specs]
        hm.render_visibility(grooms, scene.camera, frame.vis_center, frame.vis_cons, stats=frame.stats)
    else:
        hm.render_visibility(grooms, scene.camera, frame.vis_center, frame.vis_cons, stats=frame.stats)
        maps_gpu = [_gpu_map(grooms, s) for s in specs]
    shadows = [(s, m[1]) for s, m in zip(specs, maps_gpu)]
    hm.resolve_shade(grooms, scene.camera, scene.lights, scene.filt, frame.vis_center, frame.vis_cons, frame.rgba,
                     shadows=shadows)
    torch.cuda.synchronize()
    hm.get_device_status()
    vc, va = frame.keys_numpy()
    rgba = frame.rgba.cpu().numpy().astype(np.float64)
    # maps: both layers of the full-detail light view, key for key
    maps = []
    for s, (mc, ma) in zip(specs, maps_gpu):
        lods_full = [oracle.lod(g, s.cam, synth.LodParams(0)) for g in scene.grooms]
        omc, oma, _ = oracle.raster(scene.grooms, s.cam, lods_full)
        assert_keys_equal(mc.cpu().numpy().view(np.uint64), omc, "shadow map centre layer")
        assert_keys_equal(ma.cpu().numpy().view(np.uint64), oma, "shadow map")
        maps.append((s, oma))
    # the camera's LOD and keys are those of a render without any map pass
    lods = oracle.lods_for(scene)
    for (n, c), h in zip(lods, grooms):
        gn, gc = h.get_lod()
        assert np.array_equal(n, gn) and np.array_equal(c, gc)
    ovc, ova, _ = oracle.raster(scene.grooms, scene.camera, lods)
    assert_keys_equal(vc, ovc, "centre layer")
    assert_keys_equal(va, ova, "conservative layer")
    dec = oracle.resolve_decisions(scene.grooms, scene.camera, lods, scene.filt, ovc, ova)
    dec["shadow_texels"] = oracle.centre_shadow_texels(scene.grooms, scene.camera, lods, ovc, maps)
    gts = [v64.GroomT(g, l[1], b, lod_n=l[0]) for g, l, b in zip(scene.grooms, lods, oracle.strand_bases(scene.grooms))]
    covered = np.nonzero(ova != oracle.EMPTY)[0]
    pix = covered
    if sample is not None and covered.size > sample:
        pix = np.sort(np.random.default_rng(0).choice(covered, size=sample, replace=False))
    ref, pix = v64.resolve(gts, scene.camera, scene.lights, scene.filt, ovc, ova, dec, pixels=pix, shadows=maps)
    unshadowed, _ = v64.resolve(gts, scene.camera, scene.lights, scene.filt, ovc, ova, dec, pixels=pix)
    err = assert_rgba_close(rgba, ref.numpy(), pix)
    darkened = (ref.numpy()[:, :3] < unshadowed.numpy()[:, :3] - 1e-4).any(1).mean()
    return err, darkened


@pytest.mark.parametrize("lod,corr", [(0, 0), (1, 1), (1, 0)])
def test_shadowed_frame(lod, corr):
    sc = synth.tiny_scene(41, width=160, height=128, num_strands=3000, num_layers=5, length_m=0.06, dist_m=0.35)
    sc.lod = synth.LodParams(lod, 1.0)
    lcam = synth.light_camera(sc.grooms, sc.lights.dirs[0], size=200, dist_m=0.5)
    spec = synth.ShadowSpec(light=0, cam=lcam, sigma=150.0, bias_m=0.0005, depth_correction=corr)
    _, darkened = _check_shadowed(sc, [spec])
    assert darkened > 0.05


def test_shadow_map_after_camera_render_and_two_lights():
    sc = synth.tiny_scene(42, width=128, height=96, num_strands=2000, num_layers=5, length_m=0.06, dist_m=0.4)
    sc.lights = synth.make_lights([[1.0, 1.0, 1.0], [-1.0, 0.5, 0.5]], [0.8, 0.4])
    sc.lod = synth.LodParams(1, 1.5)
    specs = [synth.ShadowSpec(light=i, cam=synth.light_camera(sc.grooms, sc.lights.dirs[i], size=150 + 20 * i,
                                                               dist_m=0.6), sigma=120.0, bias_m=0.0005)
             for i in range(2)]
    _check_shadowed(sc, specs, map_first=False)


def test_shadowed_msaa():
    import torch
    from paper_2607_04230_b300 import hm
    sc = synth.tiny_scene(43, width=96, height=80, num_strands=1500, num_layers=5, length_m=0.06, dist_m=0.35)
    spec = synth.ShadowSpec(light=0, cam=synth.light_camera(sc.grooms, sc.lights.dirs[0], size=128, dist_m=0.5),
                            sigma=150.0, bias_m=0.0005, depth_correction=0)
    grooms = hm.upload_scene(sc)
    _, ma = _gpu_map(grooms, spec)
    N = 4
    npx = sc.camera.width * sc.camera.height
    vis = torch.empty((N, npx), dtype=torch.int64, device="cuda")
    rgba = torch.empty((npx, 4), dtype=torch.float32, device="cuda")
    hm.render_visibility_msaa(grooms, sc.camera, N, vis)
    hm.resolve_msaa(grooms, sc.camera, sc.lights, N, vis, rgba, shadows=[(spec, ma)])
    torch.cuda.synchronize()
    hm.get_device_status()
    lods = oracle.lods_for(sc)
    ovis, _ = oracle.raster_msaa(sc.grooms, sc.camera, lods, N)
    for k in range(N):
        assert_keys_equal(vis[k].cpu().numpy().view(np.uint64), ovis[k], f"sample layer {k}")
    maps = [(spec, oracle.shadow_map(sc.grooms, spec))]
    num, den = oracle.msaa_decisions(sc.grooms, sc.camera, lods, N, ovis)
    tex = oracle.sample_shadow_texels(sc.grooms, sc.camera, lods, N, ovis, maps)
    gts = [v64.GroomT(g, l[1], b, lod_n=l[0]) for g, l, b in zip(sc.grooms, lods, oracle.strand_bases(sc.grooms))]
    ref = v64.resolve_msaa(gts, sc.camera, sc.lights, ovis, num, den, shadows=maps, texels=tex).numpy()
    cov = np.nonzero((ovis != oracle.EMPTY).any(0))[0]
    assert_rgba_close(rgba.cpu().numpy().astype(np.float64), ref[cov], cov)


def test_shadowed_1080p_full_size():
    """The 100k-strand 1080p groom with a 1024x1024 map on the key light:
    map key for key, colour on sampled pixels."""
    sc = synth.scene_single_1080p()
    lcam = synth.light_camera(sc.grooms, sc.lights.dirs[0], size=1024, dist_m=1.0)
    spec = synth.ShadowSpec(light=0, cam=lcam, sigma=100.0, bias_m=0.001, depth_correction=1)
    _, darkened = _check_shadowed(sc, [spec], sample=6000)
    assert darkened > 0.05
