"""Failure detection without a GPU fault.

Host side (CPU): an allocation failure injected through HM_FAIL_ALLOC_AFTER
turns hm_create_groom into HM_ERR_OOM with nothing leaked or launched.
Device side (GPU): a key that decodes to no strand, or to a segment past the
strand's end, sets the device status word (never a trap or an out-of-bounds
access); hm_get_device_status reports HM_ERR_DEVICE_CHECK once and clears it.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import sys, ctypes
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
from paper_2607_04230_b300 import hm, synth
from test_abi import _desc
L = hm.lib()
g = synth.tiny_scene(0, num_strands=50).grooms[0]
d, keep = _desc(g)
h = ctypes.c_void_p()
rc = L.hm_create_groom(ctypes.byref(d), None, ctypes.byref(h))
print(rc, L.hm_last_error().decode(), h.value)
"""


def _run_injected(after):
    from paper_2607_04230_b300 import build
    build.build()
    code = _CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    env = dict(os.environ, HM_FAIL_ALLOC_AFTER=str(after))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    rc, rest = r.stdout.strip().split(" ", 1)
    assert int(rc) == 2, r.stdout
    assert "injected" in rest and rest.endswith("None")


def test_injected_first_allocation_failure_returns_oom():
    _run_injected(0)


@pytest.mark.gpu
@pytest.mark.parametrize("after", [3, 8])
def test_injected_later_allocation_failure_frees_and_returns_oom(after):
    # the earlier allocations succeed on a GPU and are released on failure
    _run_injected(after)


@pytest.mark.gpu
def test_corrupt_key_sets_device_status_without_fault():
    import torch
    from paper_2607_04230_b300 import hm, synth
    sc = synth.tiny_scene(51, width=96, height=80, num_strands=300)
    grooms = hm.upload_scene(sc)
    frame = hm.Frame(sc.camera.width, sc.camera.height)
    hm.render(grooms, sc, frame)
    torch.cuda.synchronize()
    hm.get_device_status()                                   # clean
    vc = frame.vis_center.cpu().numpy().view(np.uint64)
    p = int(np.nonzero((vc & np.uint64(0xFFFFFFFFFF)) != np.uint64(0xFFFFFFFFFF))[0][0])
    for bad in ((np.uint64(10 ** 6) << np.uint64(7)),        # strand beyond every groom
                (vc[p] & ~np.uint64(127)) | np.uint64(120)):  # segment past the strand's end
        corrupt = vc.copy()
        corrupt[p] = (vc[p] & ~np.uint64(0xFFFFFFFFFF)) | (bad & np.uint64(0xFFFFFFFFFF))
        frame.vis_center.copy_(torch.from_numpy(corrupt.view(np.int64)))
        hm.resolve_shade(grooms, sc.camera, sc.lights, sc.filt, frame.vis_center, frame.vis_cons, frame.rgba)
        with pytest.raises(hm.HmError) as ei:
            hm.get_device_status()
        assert ei.value.status == 7
        hm.get_device_status()                               # cleared by the read
        assert torch.isfinite(frame.rgba).all()
