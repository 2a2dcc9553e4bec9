"""GPU parity of the OK split (Sec. 4.2; params.split = CC_SPLIT_OK, FP64):
the outer level on the level kernels (tau with the fast-pair list, the FP64
kick with the fast pairs masked), the rest of the recursion in one CTA per
set.  Against the oracle's evolve_ok: the state bit for bit (every sum in
the oracle's order, every operation an explicit IEEE one) and the oracle's
operation counts."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1407_7105_gb300 import ics

pytestmark = pytest.mark.gpu

KEYS = ("tau_pairs", "kick_pairs", "drifts", "splits", "components")


def _rel_ok(a, b, rtol=1e-12):
    scale = np.abs(b).max()
    return np.all(np.abs(a - b) <= rtol * np.abs(b) + 1e-15 * scale)


def _case(name):
    if name == "plummer1000":
        m, x, v = ics.plummer(1000, seed=1)
        return m, x, v, None, 1 / 64
    if name == "fractal1200":
        m, x, v = ics.box_fractal(1200, seed=2)
        return m, x, v, None, 1 / 64
    if name == "systems":
        m, x, v, off = ics.small_systems(60, seed=7, n_max=300)
        return m, x, v, off, 1 / 64
    if name == "plummer256":
        m, x, v = ics.plummer(256, seed=1)
        return m, x, v, None, 1 / 64
    if name == "plummer2000_long":
        # 1.27e6 fast pairs at the outer level: its nodes run GPU-wide until
        # the lists are short enough for one CTA per set
        m, x, v = ics.plummer(2000, seed=1)
        return m, x, v, None, 1 / 16
    if name == "two_systems_long":
        parts = [ics.plummer(1000, seed=s) for s in (3, 4)]
        m = np.concatenate([p[0] for p in parts])
        x = np.ascontiguousarray(np.concatenate([p[1] for p in parts], axis=1))
        v = np.ascontiguousarray(np.concatenate([p[2] for p in parts], axis=1))
        return m, x, v, np.array([0, 1000, 2000], dtype=np.int64), 1 / 16
    raise ValueError(name)


@pytest.mark.parametrize("name,steps", [("plummer1000", 1), ("fractal1200", 1), ("systems", 1), ("plummer256", 4),
                                        ("plummer2000_long", 1), ("two_systems_long", 1)])
def test_ok_matches_oracle(cclib, name, steps):
    m, x, v, off, dt = _case(name)
    c = cclib.Context(m, x, v, dt=dt, split=cclib.SPLIT_OK)
    if off is not None:
        c.set_systems(off)
    c.evolve(steps * dt)
    _, _, gx, gv = c.get_state()
    g = c.stats()
    c.close()
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=dt, split=O.SPLIT_OK), steps, sys_off=off)
    assert st.max_depth_seen >= 3
    for k in KEYS:
        assert g[k] == getattr(st, k), (k, g[k], getattr(st, k))
    assert g["max_depth_seen"] == st.max_depth_seen
    assert _rel_ok(gx, s.x3) and _rel_ok(gv, s.v3)
    # every sum runs in the oracle's order with its IEEE operations
    assert np.array_equal(gx, s.x3) and np.array_equal(gv, s.v3)


def test_ok_differs_from_cc(cclib):
    """The two splits kick different pairs at different levels."""
    m, x, v, off, dt = _case("plummer1000")
    out = {}
    for split in (cclib.SPLIT_CC, cclib.SPLIT_OK):
        c = cclib.Context(m, x, v, dt=dt, split=split)
        c.evolve(dt)
        out[split] = c.stats()["kick_pairs"]
        c.close()
    assert out[cclib.SPLIT_OK] != out[cclib.SPLIT_CC]


def test_ok_parameters_are_checked(cclib, plummer_ic):
    m, x, v = plummer_ic(64)
    for bad in (dict(split=cclib.SPLIT_OK, precision=cclib.PREC_MIXED), dict(split=cclib.SPLIT_OK, kepler=1),
                dict(split=cclib.SPLIT_OK, theta=0.5), dict(split=3)):
        with pytest.raises(cclib.CCError) as e:
            cclib.Context(m, x, v, **bad)
        assert e.value.code == -1, bad
