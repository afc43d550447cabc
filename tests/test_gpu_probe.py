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


def _quotient(num, den):
    from paper_2607_04230_b300 import hm
    a = torch.from_numpy(num).cuda()
    b = torch.from_numpy(den).cuda()
    out = torch.empty_like(a)
    hm.probe_quotient(a, b, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _assert_ieee(num, den):
    """The rasterizers' depth-parameter quotient equals numpy's IEEE binary32
    round-to-nearest division bit for bit (numpy on the host: no CUDA
    division involved in the expected values)."""
    got = _quotient(num, den)
    want = (num / den).astype(np.float32)
    bad = got.view(np.uint32) != want.view(np.uint32)
    assert not bad.any(), (int(bad.sum()), num[bad][:5], den[bad][:5], got[bad][:5], want[bad][:5])


def test_quotient_is_correctly_rounded_on_raster_numerators():
    """Integer depth numerators and squared lengths as the rasterizer forms
    them: 32-bit items (|num| < 2^31, den < 2^28), 64-bit items (up to 2^62),
    every denominator 1 .. 65536 with several numerators each, and numerators
    equal to the denominator (t = 1) or just below it."""
    rng = np.random.default_rng(11)
    n = 1 << 22
    cases = []
    d32 = rng.integers(1, 1 << 28, n)
    cases.append((rng.integers(-(1 << 31), 1 << 31, n), d32))
    d64 = rng.integers(1, 1 << 62, n, dtype=np.int64)
    cases.append((rng.integers(-(1 << 62), 1 << 62, n, dtype=np.int64), d64))
    dd = np.repeat(np.arange(1, 65537), 16)
    cases.append((rng.integers(0, 4, dd.size) * dd // 3 + rng.integers(-2, 3, dd.size), dd))
    cases.append((d32, d32))
    cases.append((d32 - 1, d32))
    for a, b in cases:
        num = a.astype(np.float32)          # __int2float_rn / __ll2float_rn: round to nearest
        den = b.astype(np.float32)
        ok = den >= 1
        _assert_ieee(num[ok], den[ok])


def test_quotient_is_correctly_rounded_on_hard_cases():
    """Quotients next to rounding boundaries: numerators chosen so that
    num / den lies within a few ulps of a midpoint between adjacent floats
    (where a one-ulp-accurate quotient would round the wrong way), plus
    arbitrary non-integer operands of every binade in the documented range."""
    rng = np.random.default_rng(12)
    n = 1 << 22
    den = (rng.random(n) * 2.0 ** rng.integers(0, 62, n)).astype(np.float32)
    den = np.maximum(den, np.float32(1))
    q = rng.random(n).astype(np.float32)
    mid = q.astype(np.float64) + np.spacing(q).astype(np.float64) / 2     # midpoint above q
    num = (mid * den.astype(np.float64)).astype(np.float32)
    keep = (np.abs(num) >= 1) & (np.abs(num) < 2.0 ** 63)
    _assert_ieee(num[keep], den[keep])
    num2 = (rng.standard_normal(n) * 2.0 ** rng.integers(0, 62, n)).astype(np.float32)
    keep = (np.abs(num2) >= 1) & (np.abs(num2) < 2.0 ** 63)
    _assert_ieee(num2[keep], den[keep])
    _assert_ieee(np.zeros(8, np.float32), np.arange(1, 9, dtype=np.float32))
