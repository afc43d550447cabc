"""hm_shade_backward_noalloc: the adjoint for callers that cannot allocate
device memory (no cudaMalloc where the gradient is needed, e.g. inside a
real-time frame loop or under another allocator's fixed budget), with its
scratch in a static library array instead of a caller buffer.

Checked through the C ABI against hm_shade_backward on the same inputs, on two
calls in a row (the shared static scratch must be cleared by each call), with
the gradient tolerance of the other tests.  Collected last on purpose.
"""
import numpy as np
import pytest
import torch

from paper_2607_04230_b300 import synth

pytestmark = pytest.mark.gpu


def _grads_close(a, b):
    a = a.reshape(-1).double()
    b = b.reshape(-1).double()
    assert torch.linalg.norm(a - b) <= 1e-2 * torch.linalg.norm(b)
    big = b.abs() > 1e-3 * b.abs().max()
    assert ((a[big] - b[big]).abs() <= 1e-2 * b[big].abs()).all()


@pytest.mark.parametrize("W,H", [(200, 150), (512, 512)])   # 512 x 512: the largest frame the static scratch takes
def test_noalloc_backward_matches_backward_twice(W, H):
    from paper_2607_04230_b300 import hm
    sc = synth.tiny_scene(31, width=W, height=H, num_strands=1500, dist_m=0.35)
    g = sc.grooms[0]
    grooms = hm.upload_scene(sc)
    frame = hm.Frame(sc.camera.width, sc.camera.height)
    hm.render(grooms, sc, frame)
    gen = torch.Generator(device="cuda").manual_seed(5)
    grad = torch.randn(frame.rgba.shape, device="cuda", generator=gen)
    scratch = torch.empty(hm.backward_scratch_bytes(sc.camera.width, sc.camera.height) // 4, device="cuda")
    ref_lv = torch.zeros(g.layer_verts.shape, device="cuda")
    ref_alb = torch.zeros(g.strand_albedo.shape, device="cuda")
    hm.shade_backward(grooms, sc.camera, sc.lights, sc.filt, frame.vis_center, frame.vis_cons, grad,
                      [ref_lv], [ref_alb], scratch)
    for _ in range(2):
        lv = torch.zeros_like(ref_lv)
        alb = torch.zeros_like(ref_alb)
        hm.shade_backward_noalloc(grooms, sc.camera, sc.lights, sc.filt, frame.vis_center, frame.vis_cons, grad,
                                  [lv], [alb])
        torch.cuda.synchronize()
        assert ref_lv.abs().max() > 0 and ref_alb.abs().max() > 0
        _grads_close(lv, ref_lv)
        _grads_close(alb, ref_alb)
    hm.get_device_status()


def test_noalloc_backward_rejects_large_frames():
    from paper_2607_04230_b300 import hm
    sc = synth.tiny_scene(32, width=1024, height=512, num_strands=10)
    grooms = hm.upload_scene(sc)
    frame = hm.Frame(sc.camera.width, sc.camera.height)
    grad = torch.zeros_like(frame.rgba)
    with pytest.raises(hm.HmError) as ei:
        hm.shade_backward_noalloc(grooms, sc.camera, sc.lights, sc.filt, frame.vis_center, frame.vis_cons, grad,
                                  [None], [None])
    assert ei.value.status == 4
