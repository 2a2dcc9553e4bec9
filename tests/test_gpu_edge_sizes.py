"""Degenerate and ragged sizes on every path: 1, 2 and 3 bodies, and sizes
around the tile edges of the kernels (32 / 33, 64 / 65, 127 / 128 / 129,
255 / 257, 511 / 512 / 513: the warp tasks, the 128-body tiles, the CTA
tasks' limit), against the oracle in FP64 (state within 1e-12 and the
operation counts), bit-identical across the small-kernel limits (0: host
levels only, 32: warp tasks, 512: CTA tasks and the one-launch step), in
the mixed form within the per-body bound, in the HOLD and OK splits, and as
ragged batches of independent systems."""
import numpy as np
import pytest

import _bounds as B
from oracle import oracle as O

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 3, 5, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 257, 511, 512, 513]
KEYS = ("tau_pairs", "kick_pairs", "drifts", "splits", "components")


def _cluster(n, seed):
    """n bodies in a unit ball, equal masses 1/n, small velocities, with one
    or two circular binaries (separation 0.004 and 0.02: the recursion goes
    deep at any n >= 2 while each pair's separation stays put)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1.0, 1.0, (3, n))
    x /= np.maximum(1.0, np.linalg.norm(x, axis=0))
    v = 0.3 * rng.standard_normal((3, n))
    m = np.full(n, 1.0 / n)
    for a, sep in ((0, 0.004), (3, 0.02)):
        b = a + 1
        if b >= n:
            continue
        d = rng.standard_normal(3)
        d *= sep / np.linalg.norm(d)
        w = np.cross(d, rng.standard_normal(3))
        w *= np.sqrt((m[a] + m[b]) / sep) / np.linalg.norm(w)
        x[:, b] = x[:, a] + d
        vc = 0.5 * (v[:, a] + v[:, b])
        v[:, a] = vc - 0.5 * w
        v[:, b] = vc + 0.5 * w
    return m, np.ascontiguousarray(x), np.ascontiguousarray(v)


def _rel_ok(a, b, rtol=1e-12):
    scale = np.abs(b).max()
    return np.all(np.abs(a - b) <= rtol * np.abs(b) + 1e-15 * scale)


def _run(cclib, m, x, v, dt, off=None, steps=1, **kw):
    c = cclib.Context(m, x, v, dt=dt, **kw)
    if off is not None:
        c.set_systems(off)
    c.evolve(steps * dt)
    _, _, gx, gv = c.get_state()
    g = c.stats()
    near = c.near_pairs()[0] if kw.get("near_tol") else None
    c.close()
    return gx, gv, g, near


@pytest.mark.parametrize("n", SIZES)
def test_fp64_every_small_limit(cclib, n):
    m, x, v = _cluster(n, seed=n)
    dt = 1 / 32
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=dt), 2)
    ref = None
    for s_small in (0, 32, 512):
        gx, gv, g, _ = _run(cclib, m, x, v, dt, steps=2, s_small=s_small)
        assert _rel_ok(gx, s.x3) and _rel_ok(gv, s.v3), (n, s_small)
        for k in KEYS:
            assert g[k] == getattr(st, k), (n, s_small, k, g[k], getattr(st, k))
        assert g["max_depth_seen"] == st.max_depth_seen, (n, s_small)
        if ref is None:
            ref = (gx, gv)
        else:
            assert np.array_equal(gx, ref[0]) and np.array_equal(gv, ref[1]), (n, s_small)


@pytest.mark.parametrize("n", SIZES)
def test_mixed_within_bounds(cclib, n):
    m, x, v = _cluster(n, seed=100 + n)
    dt = 1 / 32
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=dt), 1)
    gx, gv, g, near = _run(cclib, m, x, v, dt, precision=cclib.PREC_MIXED, near_tol=1e-6)
    if near.size == 0:
        # no decision within 1e-6 of a threshold: the same splitting as the oracle
        for k in KEYS:
            assert g[k] == getattr(st, k), (n, k)
    if n == 1:
        assert np.array_equal(gv, v)
        return
    S = B.abs_accel_sum(m, x)
    ex = B.near_bodies(near)
    B.check_velocity_bound(gv, s.v3, S, dt, st.max_depth_seen, exempt=ex, what=n)
    B.check_position_bound(gx, s.x3, S, dt, st.max_depth_seen, exempt=ex, what=n)


@pytest.mark.parametrize("n", [1, 2, 3, 33, 129, 513])
@pytest.mark.parametrize("split", ["hold", "ok"])
def test_other_splits(cclib, n, split):
    m, x, v = _cluster(n, seed=200 + n)
    dt = 1 / 32
    osplit = O.SPLIT_HOLD if split == "hold" else O.SPLIT_OK
    csplit = cclib.SPLIT_HOLD if split == "hold" else cclib.SPLIT_OK
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=dt, split=osplit), 2)
    gx, gv, g, _ = _run(cclib, m, x, v, dt, steps=2, split=csplit)
    assert _rel_ok(gx, s.x3) and _rel_ok(gv, s.v3), n
    for k in KEYS:
        assert g[k] == getattr(st, k), (n, k, g[k], getattr(st, k))


@pytest.mark.parametrize("sizes", [[1, 2, 3, 33, 129, 512], [2, 2, 3, 64, 65, 300, 511, 5]])
def test_ragged_systems(cclib, sizes):
    """Ragged batches of systems: with a one-body system the outer level is
    a host level; without, every system is a task of one launch (s_small
    512); the two paths and the level-only path agree bit for bit."""
    parts = [_cluster(k, seed=300 + i) for i, k in enumerate(sizes)]
    m = np.concatenate([p[0] for p in parts])
    x = np.ascontiguousarray(np.concatenate([p[1] for p in parts], axis=1))
    v = np.ascontiguousarray(np.concatenate([p[2] for p in parts], axis=1))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    dt = 1 / 32
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=dt), 2, sys_off=off)
    ref = None
    for s_small in (0, 32, 512):
        gx, gv, g, _ = _run(cclib, m, x, v, dt, off=off, steps=2, s_small=s_small)
        assert _rel_ok(gx, s.x3) and _rel_ok(gv, s.v3), s_small
        for k in KEYS:
            assert g[k] == getattr(st, k), (s_small, k)
        if ref is None:
            ref = (gx, gv)
        else:
            assert np.array_equal(gx, ref[0]) and np.array_equal(gv, ref[1]), s_small


def test_components_of_tiny_sets(cclib):
    for n in (1, 2, 3):
        m, x, v = _cluster(n, seed=400 + n)
        c = cclib.Context(m, x, v)
        lab, k = c.components(1 / 32)
        olab, ok = O.components(O.State(m, x, v), O.params(), 1 / 32)
        assert k == ok and np.array_equal(lab, olab), n
        c.close()


def test_empty_input_is_refused(cclib):
    with pytest.raises((cclib.CCError, ValueError)):
        cclib.Context(np.zeros(0), np.zeros((3, 0)), np.zeros((3, 0)))
