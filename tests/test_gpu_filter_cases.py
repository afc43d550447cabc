"""The CUDA resolve on the hand-built key buffers of the closed-form filter
pins (alpha as a count ratio, promotion, the depth-mismatch blend; Sec. 3.3.2,
Sec. 3.3.3), against the FP64 oracle on every pixel, with and without the
tile-list scratch."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_04230_b300 import hm

import _filter_cases as fc
from _parity import RGBA_TOL, assert_keys_equal

pytestmark = pytest.mark.gpu


def test_crafted_filter_cases_match_the_oracle():
    sc = fc.line_scene()
    grooms = hm.upload_scene(sc)
    for tile_list in (False, True):
        frame = hm.Frame(fc.W, fc.H, tile_list=tile_list)
        hm.render_visibility(grooms, sc.camera, frame.vis_center, frame.vis_cons, stats=frame.stats)
        torch.cuda.synchronize()
        vc, va, lods = fc.raster(sc)
        gvc, gva = frame.keys_numpy()
        assert_keys_equal(gvc, vc, "centre layer")
        assert_keys_equal(gva, va, "conservative layer")
        for name, g, a in fc.crafted_cases(vc, va, sc.camera):
            frame.vis_center.copy_(torch.from_numpy(g.view(np.int64)))
            frame.vis_cons.copy_(torch.from_numpy(a.view(np.int64)))
            hm.resolve_shade(grooms, sc.camera, sc.lights, sc.filt, frame.vis_center, frame.vis_cons, frame.rgba,
                             tile_scratch=frame.tile_scratch)
            torch.cuda.synchronize()
            hm.get_device_status()
            ref, _ = fc.oracle_filter(sc, lods, g, a)
            got = frame.rgba.cpu().numpy().astype(np.float64).reshape(-1, 4)
            err = np.abs(got - ref).max()
            assert err <= RGBA_TOL, f"{name} (tile list {tile_list}): max |rgba - oracle| = {err:.3e}"
            assert np.all(got[(a & oracle.PAYLOAD_MASK) == oracle.PAYLOAD_MASK] == 0.0)
