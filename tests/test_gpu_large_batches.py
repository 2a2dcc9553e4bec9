"""GPU parity on batches larger than one CTA segments (more than 16384
packed elements): there the split runs the multi-block union-find
compression, the radix segmentation by root, the run bounds and the
separate classification kernel instead of the one-CTA segmentation (the
paper's reshuffle of each component into a contiguous run with start and
end pointers, Sec. 2.3 Implementation).  Every large workload (the 65536-body
fractal, the 32768-body binaries, the 4096-system batch) takes this path at
its top level.  Also the edge-record overflow: a split with more edges than
its record list holds leaves the list incomplete, and the first halves of
its components must then run a fresh split."""
import numpy as np
import pytest

import _bounds as B
from oracle import oracle as O
from paper_1407_7105_gb300 import ics

pytestmark = pytest.mark.gpu


def _rel_ok(a, b, rtol=1e-12):
    scale = np.abs(b).max()
    return np.all(np.abs(a - b) <= rtol * np.abs(b) + 1e-15 * scale)


N_BIG = 17000  # 133 tau tiles of 128 with a ragged tail of 104; > 16384 packed elements


@pytest.fixture(scope="module")
def big_plummer():
    """The 17000-body sphere, the oracle's labels at h = 1/256 and its state
    and counters after one outer step of 1/256 (about 30 s of oracle time,
    shared by the tests below)."""
    m, x, v = ics.plummer(N_BIG, seed=3)
    s = O.State(m, x, v)
    olab, ok = O.components(s, O.params(dt=1 / 256), 1 / 256)
    st = O.evolve(s, O.params(dt=1 / 256), 1)
    return m, x, v, olab, ok, s, st


def test_plummer_above_one_cta_fp64(cclib, big_plummer):
    """Components at the top-level threshold and one outer step of a
    17000-body Plummer sphere in the FP64 form: labels bit for bit, state
    within 1e-12, the oracle's split, pair and drift counts."""
    m, x, v, olab, ok, s, st = big_plummer
    c = cclib.Context(m, x, v, dt=1 / 256)
    lab, k = c.components(1 / 256)
    assert k == ok and np.array_equal(lab, olab)
    c.reset_stats()
    c.evolve(1 / 256)
    _, _, gx, gv = c.get_state()
    g = c.stats()
    c.close()
    assert _rel_ok(gx, s.x3) and _rel_ok(gv, s.v3)
    for key in ("tau_pairs", "kick_pairs", "drifts", "splits", "components"):
        assert g[key] == getattr(st, key), key
    assert g["max_depth_seen"] == st.max_depth_seen


def test_plummer_above_one_cta_mixed(cclib, big_plummer):
    """The mixed form on the same batch: its certified predicate gives the
    oracle's labels bit for bit, and after one outer step (level 0 in Morton
    order) every body is within the per-body FP32 error bound of the oracle
    (see _bounds), with the oracle's split and pair counts."""
    m, x, v, olab, ok, s, st = big_plummer
    c = cclib.Context(m, x, v, dt=1 / 256, precision=cclib.PREC_MIXED, near_tol=1e-6)
    lab, k = c.components(1 / 256)
    assert k == ok and np.array_equal(lab, olab)
    c.reset_stats()
    c.evolve(1 / 256)
    _, _, gx, gv = c.get_state()
    g = c.stats()
    pairs, _, _ = c.near_pairs()
    c.close()
    S = B.abs_accel_sum(m, x)
    ex = B.near_bodies(pairs)
    worst, _ = B.check_velocity_bound(gv, s.v3, S, 1 / 256, st.max_depth_seen, exempt=ex, what="v")
    worst_x, _ = B.check_velocity_bound(gx, s.x3, S * (1 / 256), 1 / 256, st.max_depth_seen, exempt=ex, what="x")
    print("mixed 17000: max error / bound: v", worst, "x", worst_x, "exempt", ex.size)
    if ex.size == 0:
        assert g["splits"] == st.splits and g["kick_pairs"] == st.kick_pairs


def _systems():
    # 400 systems, 19592 bodies, 20080 packed elements at the top level
    m, x, v, off = ics.small_systems(400, seed=5, n_max=512)
    return m, x, v, off


def test_systems_batch_above_one_cta_fp64(cclib):
    m, x, v, off = _systems()
    c = cclib.Context(m, x, v, dt=1 / 64)
    c.set_systems(off)
    c.evolve(1 / 64)
    _, _, gx, gv = c.get_state()
    g = c.stats()
    c.close()
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=1 / 64), 1, sys_off=off)
    assert _rel_ok(gx, s.x3) and _rel_ok(gv, s.v3)
    for key in ("tau_pairs", "kick_pairs", "drifts", "splits", "components"):
        assert g[key] == getattr(st, key), key
    assert g["max_depth_seen"] == st.max_depth_seen


def test_systems_batch_above_one_cta_mixed(cclib):
    """The same batch in the mixed form: every body within the per-body
    FP32 error bound of the oracle (see _bounds), each system's momentum
    kept (systems never interact)."""
    m, x, v, off = _systems()
    c = cclib.Context(m, x, v, dt=1 / 64, precision=cclib.PREC_MIXED, near_tol=1e-6)
    c.set_systems(off)
    c.evolve(1 / 64)
    _, _, gx, gv = c.get_state()
    g = c.stats()
    pairs, _, _ = c.near_pairs()
    c.close()
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=1 / 64), 1, sys_off=off)
    S = B.abs_accel_sum(m, x, groups=B.system_index(m.shape[0], off))
    worst, _ = B.check_velocity_bound(gv, s.v3, S, 1 / 64, st.max_depth_seen, exempt=B.near_bodies(pairs),
                                      what="systems mixed")
    print("systems mixed: max error / bound", worst)
    assert g["splits"] > 0
    for a, b in zip(off[:-1], off[1:]):
        P = (m[a:b] * gv[:, a:b]).sum(axis=1)
        assert np.abs(P).max() < 1e-8


def test_edge_record_overflow_falls_back_to_fresh_splits(cclib, plummer_ic):
    """With the record list capped, splits with more edges than the cap
    leave incomplete lists; the first halves of their components then run
    a fresh tau split instead of reusing the parent's values.  The result
    is the oracle's, with more pairs evaluated than without the cap."""
    m, x, v = plummer_ic(2000, seed=9)
    edge_rec_max = 64
    runs = {}
    for cap in (0, edge_rec_max):
        c = cclib.Context(m, x, v, dt=1 / 32, s_small=0, edge_rec_max=cap)
        c.evolve(1 / 32)
        _, _, gx, gv = c.get_state()
        runs[cap] = (gx, gv, c.stats())
        c.close()
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=1 / 32), 1)
    gx, gv, g = runs[edge_rec_max]
    assert _rel_ok(gx, s.x3) and _rel_ok(gv, s.v3)
    for key in ("tau_pairs", "kick_pairs", "drifts", "splits", "components"):
        assert g[key] == getattr(st, key), key
    # identical arithmetic either way: the FP64 form is bit for bit the same
    assert np.array_equal(gx, runs[0][0]) and np.array_equal(gv, runs[0][1])
    assert g["tau_evaluated"] > runs[0][2]["tau_evaluated"]
