"""The atomic probe behind the rasterizer's roofline denominator does the
atomics it is credited with: after `rounds` passes of pattern 0 every element
holds the smallest key written to it, (1 << 40) | index; pattern 1 and 2
leave, for every element, the smallest key any lane aimed at it (checked
against the same address maps computed on the host)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

HASH = np.uint64(0x9E3779B97F4A7C15)


def _expected(n, rounds, pattern):
    i = np.arange(n, dtype=np.uint64)
    h = (i >> np.uint64(5)) if pattern == 2 else i
    a = i if pattern == 0 else (h * HASH) % np.uint64(n)          # wraps mod 2^64 like the device
    key = (np.uint64(1) << np.uint64(40)) | i                      # the last round writes the smallest keys
    out = np.full(n, np.iinfo(np.uint64).max, dtype=np.uint64)
    np.minimum.at(out, a.astype(np.int64), key)
    return out


@pytest.mark.parametrize("pattern", [0, 1, 2])
def test_probe_writes_the_minimum_keys(pattern):
    from paper_2607_04230_b300 import hm
    n, rounds = 100_003, 3
    buf = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    hm.probe_atomic_min(buf, rounds=rounds, pattern=pattern)
    torch.cuda.synchronize()
    got = buf.cpu().numpy().view(np.uint64)
    assert np.array_equal(got, _expected(n, rounds, pattern))
