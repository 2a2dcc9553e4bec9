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
