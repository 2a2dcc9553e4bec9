"""The integer float-float split used by the mixed-precision kernels
(ff_split in csrc/cc_device.cuh) restated with numpy integers: for every
double in its fast-path range it must return exactly hi = fl32(x) and
lo = fl32(x - hi), the pair the FP64 route produces (round to nearest
even, including ties and carries into the exponent)."""
import numpy as np
import pytest


def in_fast_range(x):
    e = ((x.view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
    return (e >= 949) & (e <= 1150)


def ff_split_int(x: np.ndarray):
    b = x.view(np.uint64)
    e = ((b >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
    assert np.all((e >= 949) & (e <= 1150))
    F = ((b & np.uint64(0xFFFFFFFFFFFFF)) | np.uint64(0x10000000000000)).astype(np.int64)
    Fr = (F + 0x0FFFFFFF + ((F >> 29) & 1)) >> 29
    d = (F - (Fr << 29)).astype(np.int32)
    s_hi = ((e - 1046 + 127) << 23).astype(np.int32).view(np.float32)
    s_lo = ((e - 1075 + 127) << 23).astype(np.int32).view(np.float32)
    h = Fr.astype(np.int32).astype(np.float32) * s_hi
    l = d.astype(np.float32) * s_lo
    neg = (b >> np.uint64(63)) != 0
    return np.where(neg, -h, h).astype(np.float32), np.where(neg, -l, l).astype(np.float32)


def reference(x):
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


@pytest.mark.parametrize("scale", [1e-20, 1e-5, 1.0, 3.7, 1e6, 1e30])
def test_random_values(scale):
    rng = np.random.default_rng(int(abs(np.log10(scale)) * 7 + 1))
    x = scale * rng.standard_normal(200000)
    x = x[in_fast_range(x)]  # the device takes the FP64 route outside
    assert x.size > 190000
    hi, lo = ff_split_int(x)
    rh, rl = reference(x)
    assert np.array_equal(hi, rh) and np.array_equal(lo, rl)


def test_ties_and_carries():
    # significands exactly halfway between two floats, and all-ones
    # significands that carry into the exponent when rounded up
    base = np.array([1.0, 1.5, 2.0, 3.0, 1234.5, 7e-10], dtype=np.float64)
    tie = base * (1.0 + 2.0 ** -24)
    tie2 = base * (1.0 + 3 * 2.0 ** -24)
    carry = np.nextafter(base * 2.0, 0.0)
    x = np.concatenate([tie, -tie, tie2, carry, -carry])
    hi, lo = ff_split_int(x)
    rh, rl = reference(x)
    assert np.array_equal(hi, rh) and np.array_equal(lo, rl)


# fl32 and f2d (csrc/cc_device.cuh): the integer forms of double -> float
# round-to-nearest-even and of float -> double, restated with numpy integers

def fl32_int(x: np.ndarray):
    b = x.view(np.uint64)
    e = ((b >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
    assert np.all((e >= 897) & (e <= 1149))
    mag = b & np.uint64(0x7FFFFFFFFFFFFFFF)
    r = mag + np.uint64(0x0FFFFFFF) + ((mag >> np.uint64(29)) & np.uint64(1))
    fb = ((r >> np.uint64(29)) - np.uint64(896 << 23)).astype(np.uint32)
    fb |= ((b >> np.uint64(32)) & np.uint64(0x80000000)).astype(np.uint32)
    return fb.view(np.float32)


def f2d_int(f: np.ndarray):
    u = f.view(np.uint32).astype(np.uint64)
    ex = (u >> np.uint64(23)) & np.uint64(0xFF)
    assert np.all((ex > 0) & (ex < 255))
    b = ((u & np.uint64(0x80000000)) << np.uint64(32)) | ((ex + np.uint64(896)) << np.uint64(52)) | \
        ((u & np.uint64(0x7FFFFF)) << np.uint64(29))
    return b.view(np.float64)


def fl32_range(x):
    e = ((x.view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
    return (e >= 897) & (e <= 1149)


@pytest.mark.parametrize("scale", [1e-36, 1e-5, 1.0, 3.7, 1e6, 1e37])
def test_fl32_random(scale):
    rng = np.random.default_rng(int(abs(np.log10(scale)) * 11 + 3))
    x = scale * rng.standard_normal(200000)
    x = x[fl32_range(x)]
    assert x.size > 150000
    assert np.array_equal(fl32_int(x).view(np.uint32), x.astype(np.float32).view(np.uint32))


def test_fl32_ties_and_carries():
    base = np.array([1.0, 1.5, 2.0, 3.0, 1234.5, 7e-10, 2.0 ** -126], dtype=np.float64)
    x = np.concatenate([base * (1.0 + 2.0 ** -24), base * (1.0 + 3 * 2.0 ** -24), np.nextafter(base * 2.0, 0.0),
                        base * (1.0 + 2.0 ** -24 + 2.0 ** -50)])
    x = np.concatenate([x, -x])
    assert np.array_equal(fl32_int(x).view(np.uint32), x.astype(np.float32).view(np.uint32))


def test_f2d_exact():
    rng = np.random.default_rng(5)
    f = (rng.standard_normal(100000) * np.exp(rng.uniform(-80, 80, 100000))).astype(np.float32)
    f = f[(np.abs(f) >= np.finfo(np.float32).tiny) & np.isfinite(f)]
    assert np.array_equal(f2d_int(f), f.astype(np.float64))


# first_level_at_or_below (csrc/cc_device.cuh): the first m >= 0 with
# h 2^-m <= tau from exponent and significand fields, against the direct
# sequence of exact halvings

def first_level_int(tau: float, h: float, levels: int) -> int:
    if not (tau < h):
        return 0
    if not (tau >= np.finfo(np.float64).tiny):
        return levels
    bt = int(np.float64(tau).view(np.int64))
    bh = int(np.float64(h).view(np.int64))
    et, eh = bt >> 52, bh >> 52
    mt, mh = bt & 0xFFFFFFFFFFFFF, bh & 0xFFFFFFFFFFFFF
    m = eh - et + (0 if mh <= mt else 1)
    return min(m, levels)


def first_level_direct(tau: float, h: float, levels: int) -> int:
    for m in range(levels):
        if not (tau < h * 2.0 ** -m):
            return m
    return levels


def test_first_level_at_or_below():
    rng = np.random.default_rng(11)
    h = 1.0 / 256
    taus = list(h * np.exp2(rng.uniform(-70, 3, 20000)))
    # thresholds hit exactly, one ulp either side, and significands equal
    for m in range(0, 64, 3):
        t = h * 2.0 ** -m
        taus += [t, np.nextafter(t, 0), np.nextafter(t, 1), 1.5 * t, 0.75 * t]
    taus += [0.0, 5e-324, np.nan, np.inf, h]
    for hh in (h, 0.3, 1.7e-5):
        for t in taus:
            for levels in (1, 20, 64):
                assert first_level_int(t, hh, levels) == first_level_direct(t, hh, levels), (t, hh, levels)
