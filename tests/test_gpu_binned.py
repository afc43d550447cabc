"""The screen-tile binned rasterizer (hm_tuning.raster_bin_w != 0, Sec. 3.1.2
with shared-memory tile binning) on the GPU.

* for every bin size and chunk size the autotuner searches, both key layers
  and the covered-pair counts equal the CPU oracle's on a ragged frame dense
  enough that tiles split into several chunks;
* RGBA through the resolve stays within tolerance of the FP64 oracle;
* several grooms in one call, accumulation into earlier keys (clear off) and
  the scene-depth pre-fill give the oracle's keys;
* at 1080p (100k strands) and on the 4K crowd the keys equal the direct
  rasterizer's (itself checked against the oracle at those sizes);
* a pair list too small for the frame reports device status bit 4 instead
  of dropping keys silently, and the workspace never grows during stream
  capture (HM_ERR_CAPACITY) but replays from a graph once it has grown.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_04230_b300 import autotune, crowd, hm, synth

from _parity import assert_keys_equal, check_full, oracle_keys

pytestmark = pytest.mark.gpu

BINNED = [c for c in autotune.candidates() if c["raster_bin_w"]]
DIRECT = {"raster_bin_w": 0, "raster_bin_h": 0, "raster_bin_chunk": 0}


def _name(c):
    return f"{c['raster_bin_w']}x{c['raster_bin_h']}_chunk{c['raster_bin_chunk']}"


@pytest.fixture
def tuning():
    saved = hm.get_tuning()
    yield hm.set_tuning
    hm.set_tuning(**saved)


def _render_keys(grooms, sc, clear=True, scene_d24=None, frame=None):
    frame = frame or hm.Frame(sc.camera.width, sc.camera.height)
    hm.render_visibility(grooms, sc.camera, frame.vis_center, frame.vis_cons, scene_d24=scene_d24, clear=clear,
                         stats=frame.stats)
    torch.cuda.synchronize()
    hm.get_device_status()
    return frame


def test_candidates_cover_bin_and_chunk_sizes():
    sizes = {(c["raster_bin_w"], c["raster_bin_h"], c["raster_bin_chunk"]) for c in BINNED}
    assert sizes == {(w, h, k) for w in (16, 32) for h in (16, 32) for k in (256, 1024)}


@pytest.mark.parametrize("cand", BINNED, ids=_name)
def test_binned_keys_and_counts_equal_oracle(tuning, cand):
    # 203 x 117: no dimension a multiple of 16; 5000 strands put thousands of
    # segments into the busiest tiles, so tiles split into several chunks
    sc = synth.tiny_scene(21, width=203, height=117, num_strands=5000)
    lods, vc, va, counts = oracle_keys(sc)
    tuning(**cand)
    frame = _render_keys(hm.upload_scene(sc), sc)
    gvc, gva = frame.keys_numpy()
    assert_keys_equal(gvc, vc, f"centre layer {_name(cand)}")
    assert_keys_equal(gva, va, f"conservative layer {_name(cand)}")
    st = hm.stats_dict(frame.stats)
    assert (st["covered_center"], st["covered_cons"]) == (counts[0], counts[1]), st


def test_binned_rgba_within_tolerance_of_oracle(tuning):
    tuning(**BINNED[0])
    check_full(synth.tiny_scene(22, width=160, height=120, num_strands=1500), tile_list=True)


def test_binned_several_grooms_and_accumulation(tuning):
    gs = synth.crowd_grooms(seed=23, n_side=2, strand_scale=0.05)
    sc = synth.scene_crowd_4k(gs, width=320, height=180)
    lods, vc, va, counts = oracle_keys(sc)
    tuning(raster_bin_w=32, raster_bin_h=16, raster_bin_chunk=256)
    grooms = hm.upload_scene(sc)
    frame = _render_keys(grooms, sc)
    gvc, gva = frame.keys_numpy()
    assert_keys_equal(gvc, vc, "centre layer, one call over 4 grooms")
    assert_keys_equal(gva, va, "conservative layer, one call over 4 grooms")
    # one call per groom, the clear only on the first: the later calls
    # accumulate into the earlier keys
    frame2 = hm.Frame(sc.camera.width, sc.camera.height)
    for i in range(len(grooms)):
        hm.render_visibility_range(grooms, i, 1, sc.camera, frame2.vis_center, frame2.vis_cons, clear=(i == 0))
    torch.cuda.synchronize()
    hm.get_device_status()
    gvc2, gva2 = frame2.keys_numpy()
    assert_keys_equal(gvc2, vc, "centre layer, per-groom calls")
    assert_keys_equal(gva2, va, "conservative layer, per-groom calls")


def test_binned_scene_depth_prefill(tuning):
    sc = synth.tiny_scene(24, width=130, height=98, num_strands=800)
    lods, vc0, _, _ = oracle_keys(sc)
    d = (vc0 >> np.uint64(40)).astype(np.int64)
    rng = np.random.default_rng(1)
    scene = np.where(rng.random(d.size) < 0.5, np.median(d[d < 2 ** 24 - 1]), 2 ** 24 - 1).astype(np.uint32)
    ovc, ova, _ = oracle.raster(sc.grooms, sc.camera, lods, prefill_d24=scene)
    tuning(raster_bin_w=16, raster_bin_h=32, raster_bin_chunk=1024)
    sd = torch.from_numpy(scene.view(np.int32)).cuda()
    frame = _render_keys(hm.upload_scene(sc), sc, scene_d24=sd)
    gvc, gva = frame.keys_numpy()
    assert_keys_equal(gvc, ovc, "centre layer with scene depth")
    assert_keys_equal(gva, ova, "conservative layer with scene depth")


def _direct_and_binned(grooms, sc, tuning, cand):
    tuning(**DIRECT)
    ref = _render_keys(grooms, sc)
    tuning(**cand)
    got = _render_keys(grooms, sc)
    for (a, b), what in zip(zip(got.keys_numpy(), ref.keys_numpy()), ("centre", "conservative")):
        assert_keys_equal(a, b, f"{what} layer, {_name(cand)} vs direct")
    assert hm.stats_dict(got.stats) == hm.stats_dict(ref.stats)


def test_binned_equals_direct_at_1080p(tuning):
    sc = synth.scene_single_1080p()
    grooms = hm.upload_scene(sc)
    for cand in (BINNED[0], BINNED[-1]):
        _direct_and_binned(grooms, sc, tuning, cand)


def test_binned_equals_direct_on_the_4k_crowd(tuning):
    sc = synth.scene_crowd_4k()
    _direct_and_binned(hm.upload_scene(sc), sc, tuning, {"raster_bin_w": 32, "raster_bin_h": 32,
                                                         "raster_bin_chunk": 1024})


def _diagonal_scene(size=512):
    """Three coincident straight strands of 6 segments along the image
    diagonal: 18 segments (one 32-slot batch, a 256-pair list) whose pixel
    boxes span several hundred 16 x 16 tiles."""
    ts = np.linspace(-0.2, 0.2, 4, dtype=np.float32)
    layers = np.zeros((4, 3, 3), np.float32)
    layers[:, :, 0] = ts[:, None]
    layers[:, :, 1] = ts[:, None]
    g = synth.Groom(layer_verts=layers, faces=np.int32([[0, 1, 2]]), strand_face=np.zeros(3, np.uint32),
                    strand_bary=np.zeros((3, 2), np.float32), strand_albedo=np.full((3, 3), 0.4, np.float32),
                    bundle_delta=np.float32([0.5]), segments_per_strand=6)
    cam = synth.make_camera([0.0, 0.0, 0.5], [0.0, 0.0, 0.0], 50.0, size, size)
    return synth.Scene([g], cam, synth.make_lights([[0.3, 1.0, 0.6]], [1.0]), name="diagonal")


def test_overfull_pair_list_sets_device_status(tuning):
    sc = _diagonal_scene()
    grooms = hm.upload_scene(sc)
    tuning(raster_bin_w=16, raster_bin_h=16, raster_bin_chunk=256)
    frame = hm.Frame(sc.camera.width, sc.camera.height)
    hm.render_visibility(grooms, sc.camera, frame.vis_center, frame.vis_cons)
    torch.cuda.synchronize()
    with pytest.raises(RuntimeError, match="DEVICE_CHECK|consistency"):
        hm.get_device_status()
    hm.get_device_status()                      # the bit was cleared by the read
    # the direct rasterizer draws the same frame without a pair list
    tuning(**DIRECT)
    _render_keys(grooms, sc)


def test_workspace_never_grows_during_capture(tuning):
    sc = synth.tiny_scene(25, width=96, height=80, num_strands=300)
    grooms = hm.upload_scene(sc)                # a fresh groom: no workspace yet
    frame = hm.Frame(sc.camera.width, sc.camera.height)
    tuning(raster_bin_w=32, raster_bin_h=32, raster_bin_chunk=256)
    g = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.graph(g):
        try:
            hm.render_visibility(grooms, sc.camera, frame.vis_center, frame.vis_cons)
        except hm.HmError as e:          # nothing was launched; the capture ends empty
            err = e
    assert err is not None and "HM_ERR_CAPACITY" in str(err), err
    # after one eager frame the workspace fits and the capture replays it
    eager = _render_keys(grooms, sc, frame=frame)
    vc, va = eager.keys_numpy()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        hm.render_visibility(grooms, sc.camera, frame.vis_center, frame.vis_cons)
    frame.vis_center.zero_()
    frame.vis_cons.zero_()
    g.replay()
    torch.cuda.synchronize()
    hm.get_device_status()
    vc2, va2 = frame.keys_numpy()
    assert_keys_equal(vc2, vc, "centre layer, graph replay")
    assert_keys_equal(va2, va, "conservative layer, graph replay")


def test_autotuner_times_binned_candidates(tuning):
    cr = crowd.Crowd(synth.scene_crowd_4k(synth.crowd_grooms(seed=26, n_side=2, strand_scale=0.05), 640, 360))
    res = autotune.autotune(cr.render_batched, n=2)
    binned_rows = [r for r in res["table"] if r["raster_bin_w"]]
    assert len(binned_rows) == len(BINNED) and all(r["ms"] > 0 for r in binned_rows)
