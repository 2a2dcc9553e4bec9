"""GPU parity of the HOLD method (Sec. 2.1, Eq. HOLD) run on the CC kernels
(params.split = CC_SPLIT_HOLD): the fast set F = {i : tau(i) < h} is the
union of the time-step graph's non-trivial components, joined into one set
after the union-find; the recursion, the drifts of S and the kicks of every
pair not inside F are the CC path's.  Against the oracle's evolve_hold,
written from Eq. HOLD with tau(i) = min_j tau(i,j) (row minima, every pair).
"""
import numpy as np
import pytest

import _bounds as B
from oracle import oracle as O
from paper_1407_7105_gb300 import ics

pytestmark = pytest.mark.gpu


def _rel_ok(a, b, rtol=1e-12):
    scale = np.abs(b).max()
    return np.all(np.abs(a - b) <= rtol * np.abs(b) + 1e-15 * scale)


def _hold(cclib, m, x, v, **kw):
    return cclib.Context(m, x, v, split=cclib.SPLIT_HOLD, **kw)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [1000, 17000])
def test_hold_split_matches_oracle(cclib, plummer_ic, prec, n):
    m, x, v = plummer_ic(n, seed=5)
    s = O.State(m, x, v)
    p = O.params(split=O.SPLIT_HOLD)
    c = _hold(cclib, m, x, v, precision=cclib.PREC_FP64 if prec == "fp64" else cclib.PREC_MIXED)
    for h in ((1 / 64, 1 / 512) if n < 5000 else (1 / 256,)):
        lab, k = c.components(h)
        olab, ok = O.hold_split(s, p, h)
        assert k == ok and np.array_equal(lab, olab), (prec, h)
    c.close()


@pytest.mark.parametrize("n,dt,s_small", [(1000, 1 / 128, 32), (2000, 1 / 32, 0)])
def test_hold_one_step_fp64(cclib, plummer_ic, n, dt, s_small):
    m, x, v = plummer_ic(n, seed=9)
    c = _hold(cclib, m, x, v, dt=dt, s_small=s_small)
    c.evolve(dt)
    _, _, gx, gv = c.get_state()
    g = c.stats()
    c.close()
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=dt, split=O.SPLIT_HOLD), 1)
    assert _rel_ok(gx, s.x3) and _rel_ok(gv, s.v3)
    for k in ("tau_pairs", "kick_pairs", "drifts", "splits", "components"):
        assert g[k] == getattr(st, k), k
    assert g["max_depth_seen"] == st.max_depth_seen


def test_hold_systems_batch_fp64_and_mixed(cclib):
    m, x, v, off = ics.small_systems(40, seed=5, n_max=96)
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=1 / 64, split=O.SPLIT_HOLD), 1, sys_off=off)
    for prec in (cclib.PREC_FP64, cclib.PREC_MIXED):
        c = _hold(cclib, m, x, v, dt=1 / 64, precision=prec, near_tol=1e-6)
        c.set_systems(off)
        c.evolve(1 / 64)
        _, _, gx, gv = c.get_state()
        g = c.stats()
        pairs, _, _ = c.near_pairs()
        c.close()
        if prec == cclib.PREC_FP64:
            assert _rel_ok(gx, s.x3) and _rel_ok(gv, s.v3)
            for k in ("tau_pairs", "kick_pairs", "drifts", "splits", "components"):
                assert g[k] == getattr(st, k), k
        else:
            S = B.abs_accel_sum(m, x, groups=B.system_index(m.shape[0], off))
            w, _ = B.check_velocity_bound(gv, s.v3, S, 1 / 64, st.max_depth_seen, exempt=B.near_bodies(pairs))
            print("HOLD systems mixed: max error / bound", w)


def test_hold_mixed_step_within_bounds(cclib, plummer_ic):
    m, x, v = plummer_ic(4096, seed=3)
    c = _hold(cclib, m, x, v, dt=1 / 256, precision=cclib.PREC_MIXED, near_tol=1e-6)
    c.evolve(1 / 256)
    _, _, gx, gv = c.get_state()
    pairs, _, _ = c.near_pairs()
    c.close()
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=1 / 256, split=O.SPLIT_HOLD), 1)
    S = B.abs_accel_sum(m, x)
    w, _ = B.check_velocity_bound(gv, s.v3, S, 1 / 256, st.max_depth_seen, exempt=B.near_bodies(pairs))
    print("HOLD mixed 4096: max error / bound", w)


def test_hold_equals_cc_on_triples(cclib):
    """A set of at most three bodies has at most one non-trivial component
    per level: there the HOLD and CC splits coincide, bit for bit."""
    parts = [ics.hierarchical_triple(7, 500 + 11 * k) for k in range(8)]
    m = np.concatenate([p[0] for p in parts])
    x = np.ascontiguousarray(np.concatenate([p[1] for p in parts], axis=1))
    v = np.ascontiguousarray(np.concatenate([p[2] for p in parts], axis=1))
    off = np.arange(0, 3 * len(parts) + 1, 3, dtype=np.int64)
    out = []
    for split in (cclib.SPLIT_CC, cclib.SPLIT_HOLD):
        c = cclib.Context(m, x, v, dt=1 / 8, split=split)
        c.set_systems(off)
        c.evolve(2 / 8)
        _, _, gx, gv = c.get_state()
        out.append((gx, gv))
        c.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_hold_rejects_kepler_mode(cclib, plummer_ic):
    m, x, v = plummer_ic(64)
    with pytest.raises(cclib.CCError) as e:
        _hold(cclib, m, x, v, kepler=1)
    assert e.value.code == -1
