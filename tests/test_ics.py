"""The seeded input generators (paper_1407_7105_gb300/ics.py) against their
published definitions and the closed forms of the distributions they draw:
SplitMix64's reference outputs, the Plummer model's mass profile and
half-mass radius, N-body units (E = -1/4, the requested virial ratio,
centre-of-mass frame), the primordial-binary recipe (semi-major axes,
thermal eccentricities, mass ratios) and the independent-systems batch."""
import math

import numpy as np
import pytest

from paper_1407_7105_gb300 import ics


def _energy(m, x, v):
    T = 0.5 * float((m * (v * v).sum(axis=0)).sum())
    W = ics.potential_energy(m, x)
    return T, W


def test_splitmix64_reference_outputs():
    """SplitMix64 (Steele, Lea & Flood 2014) from state 0: the first three
    outputs are the published test vector.  ics mixes state k * golden."""
    golden = np.uint64(0x9E3779B97F4A7C15)
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    with np.errstate(over="ignore"):
        got = [int(ics._mix64(np.array([golden * np.uint64(k)], dtype=np.uint64))[0]) for k in (1, 2, 3)]
    assert got == want


def test_uniform_streams_are_uniform_and_distinct():
    u = ics.uniform(5, 1, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1 / 12) < 2e-3
    w = ics.uniform(5, 2, 200000)
    assert abs(np.corrcoef(u, w)[0, 1]) < 1e-2
    assert np.array_equal(ics.uniform(5, 1, 10, offset=7), u[7:17])  # counter-based


def test_plummer_profile_and_units():
    m, x, v = ics.plummer(8192, seed=3)
    assert abs(m.sum() - 1.0) < 1e-14
    T, W = _energy(m, x, v)
    assert abs(T + W + 0.25) < 1e-12 and abs(-T / W - 0.5) < 1e-12
    assert np.abs((x * m).sum(axis=1)).max() < 1e-15 and np.abs((v * m).sum(axis=1)).max() < 1e-15
    # Plummer: M(<r) = r^3 / (r^2 + a^2)^(3/2), a = 3 pi / 16 in N-body units;
    # the outer 0.1 % of the mass is cut, and the virial rescaling is ~1
    a = 3 * math.pi / 16
    r = np.linalg.norm(x, axis=0)
    for q in (0.5, 1.0, 2.0):
        frac = (r < q * a).mean()
        want = q ** 3 / (q * q + 1) ** 1.5
        assert abs(frac - want) < 0.02, (q, frac, want)
    assert abs(np.median(r) / (a / math.sqrt(2 ** (2 / 3) - 1)) - 1) < 0.03  # half-mass radius
    # isotropic velocities
    assert abs((v[0] ** 2).mean() / (v[2] ** 2).mean() - 1) < 0.05


def test_plummer_with_binaries_recipe():
    n = 4096
    m, x, v = ics.plummer_with_binaries(n, seed=2)
    nb = n // 4
    assert abs(m.sum() - 1.0) < 1e-12
    r = np.linalg.norm(x[:, 0:2 * nb:2] - x[:, 1:2 * nb:2], axis=0)
    dv = np.linalg.norm(v[:, 0:2 * nb:2] - v[:, 1:2 * nb:2], axis=0)
    mu = m[0:2 * nb:2] + m[1:2 * nb:2]
    # two-body orbital elements of every pair
    eps = 0.5 * dv * dv - mu / r
    assert np.all(eps < 0)  # bound
    a = -mu / (2 * eps)
    assert a.min() > 0.999e-5 and a.max() < 1.001e-2
    la = np.log(a)
    assert abs(la.mean() - 0.5 * (math.log(1e-5) + math.log(1e-2))) < 0.15  # log-uniform
    rv = ((x[:, 0:2 * nb:2] - x[:, 1:2 * nb:2]) * (v[:, 0:2 * nb:2] - v[:, 1:2 * nb:2])).sum(axis=0)
    h2 = (r * dv) ** 2 - rv ** 2
    e = np.sqrt(np.maximum(0.0, 1 - h2 / (mu * a)))
    assert abs(np.mean(e * e) - 0.5) < 0.03  # thermal: f(e) = 2e, <e^2> = 1/2
    q = m[1:2 * nb:2] / m[0:2 * nb:2]
    assert q.min() > 0.1 - 1e-12 and q.max() <= 1.0 + 1e-12


def test_box_fractal_units_and_masses():
    m, x, v = ics.box_fractal(2000, seed=4)
    assert abs(m.sum() - 1.0) < 1e-12
    T, W = _energy(m, x, v)
    assert abs(T + W + 0.25) < 1e-12 and abs(-T / W - 0.3) < 1e-12
    ratio = m.max() / m.min()
    assert ratio <= 1000.0 * (1 + 1e-12) and ratio > 50  # Salpeter on [0.1, 100]
    # Salpeter slope 2.35: the share of bodies below twice the lower limit
    lo = m.min()
    assert abs((m < 2 * lo).mean() - (1 - 2 ** -1.35) / (1 - 1000 ** -1.35)) < 0.05


@pytest.mark.parametrize("seed", [1, 2])
def test_small_systems_batch(seed):
    m, x, v, off = ics.small_systems(48, seed=seed)
    sizes = np.diff(off)
    assert sizes.min() >= 3 and sizes.max() <= 512
    for s in range(len(sizes)):
        a, b = off[s], off[s + 1]
        T, W = _energy(m[a:b], x[:, a:b], v[:, a:b])
        assert abs(m[a:b].sum() - 1.0) < 1e-12 and abs(T + W + 0.25) < 1e-10, s
