"""Multiview rasterization (strands assembled once, projected per view):
every view's keys are bit-exact against a single-view oracle render of that
view under view 0's LOD, the covered-pair counts add up, and each view's
resolve matches the FP64 oracle within 1e-4."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_04230_b300 import hm, synth

from _parity import assert_keys_equal, assert_rgba_close, oracle_rgba

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("lod", [0, 1])
def test_multiview_equals_per_view_oracle(lod):
    sc = synth.tiny_scene(61, width=160, height=120, num_strands=1500, dist_m=0.45)
    sc.lod = synth.LodParams(lod, 3.0)
    ctr, _, _ = synth._aabb_center(sc.grooms)
    cams = synth.view_offsets(sc.camera, [-0.032, 0.032, 0.1], target=ctr)
    grooms = hm.upload_scene(sc)
    frames = [hm.Frame(c.width, c.height) for c in cams]
    stats = torch.zeros(8, dtype=torch.int64, device="cuda")
    hm.render_visibility_multiview(grooms, cams, [f.vis_center for f in frames], [f.vis_cons for f in frames],
                                   stats=stats)
    torch.cuda.synchronize()
    hm.get_device_status()
    lods = [oracle.lod(g, cams[0], sc.lod) for g in sc.grooms]
    for (n, c), g in zip(lods, grooms):
        gn, gc = g.get_lod()
        assert np.array_equal(n, gn) and np.array_equal(c, gc)
    tot = np.zeros(2, np.int64)
    for v, (cam, fr) in enumerate(zip(cams, frames)):
        ovc, ova, cnt = oracle.raster(sc.grooms, cam, lods)
        tot += cnt
        vc, va = fr.keys_numpy()
        assert_keys_equal(vc, ovc, f"view {v} centre layer")
        assert_keys_equal(va, ova, f"view {v} conservative layer")
        sv = synth.Scene(sc.grooms, cam, sc.lights, sc.filt, sc.lod)
        hm.resolve_shade(grooms, cam, sc.lights, sc.filt, fr.vis_center, fr.vis_cons, fr.rgba)
        torch.cuda.synchronize()
        ref, pix = oracle_rgba(sv, lods, ovc, ova)
        assert_rgba_close(fr.rgba.cpu().numpy().astype(np.float64), ref, pix)
    st = hm.stats_dict(stats)
    assert st["covered_center"] == tot[0] and st["covered_cons"] == tot[1]


def test_multiview_lod_off_equals_single_view_renders():
    sc = synth.tiny_scene(62, width=200, height=140, num_strands=2500)
    ctr, _, _ = synth._aabb_center(sc.grooms)
    cams = synth.view_offsets(sc.camera, [-0.05, 0.0, 0.05, 0.12], target=ctr)
    grooms = hm.upload_scene(sc)
    frames = [hm.Frame(c.width, c.height) for c in cams]
    hm.render_visibility_multiview(grooms, cams, [f.vis_center for f in frames], [f.vis_cons for f in frames])
    single = hm.Frame(cams[0].width, cams[0].height)
    for cam, fr in zip(cams, frames):
        hm.render_visibility(grooms, cam, single.vis_center, single.vis_cons)
        torch.cuda.synchronize()
        assert torch.equal(single.vis_center, fr.vis_center) and torch.equal(single.vis_cons, fr.vis_cons)
