"""GPU parity of the batched kernel's thread-block tasks (params.s_small >
32): components of 33..512 bodies of a host-level split, and whole systems
of up to 512 bodies, evolved by one CTA each through their full CC recursion
(split, DKD and sub-recursions on-chip; sub-components of <= 32 bodies on
the CTA's warps, larger ones in nested frames of the same CTA).

The FP64 form runs the same arithmetic as the level kernels and the
warp-per-component kernel, so its result must equal theirs bit for bit
(s_small = 512 against s_small = 32 and 0) and the oracle's to 1e-12 with
the oracle's operation counts; the mixed form stays within the per-body
FP32 bound.  When every system fits one task, an outer step is one launch.
"""
import numpy as np
import pytest

import _bounds as B
from oracle import oracle as O
from paper_1407_7105_gb300 import ics

pytestmark = pytest.mark.gpu

KEYS = ("tau_pairs", "kick_pairs", "drifts", "splits", "components")


def _rel_ok(a, b, rtol=1e-12):
    scale = np.abs(b).max()
    return np.all(np.abs(a - b) <= rtol * np.abs(b) + 1e-15 * scale)


def _case(name):
    """(m, x, v, sys_off or None, dt): where the tasks of 33..512 bodies come from"""
    if name == "plummer2000":  # a giant component shrinking below 512 a few levels down
        m, x, v = ics.plummer(2000, seed=9)
        return m, x, v, None, 1 / 32
    if name == "fractal1200":  # level 0: 93 components, three of 33..134 bodies
        m, x, v = ics.box_fractal(1200, seed=2)
        return m, x, v, None, 1 / 64
    if name == "plummer256":  # one system of 256 bodies: the whole step is one task
        m, x, v = ics.plummer(256, seed=1)
        return m, x, v, None, 1 / 64
    if name == "systems":  # 60 systems of 3..300 bodies, every one a task
        m, x, v, off = ics.small_systems(60, seed=7, n_max=300)
        return m, x, v, off, 1 / 64
    raise ValueError(name)


def _run(cclib, m, x, v, off, dt, steps=1, **kw):
    c = cclib.Context(m, x, v, dt=dt, **kw)
    if off is not None:
        c.set_systems(off)
    c.evolve(steps * dt)
    _, _, gx, gv = c.get_state()
    g = c.stats()
    c.close()
    return gx, gv, g


@pytest.mark.parametrize("name", ["plummer2000", "fractal1200", "plummer256", "systems"])
def test_batch_fp64_matches_oracle_and_level_path(cclib, name):
    m, x, v, off, dt = _case(name)
    gx, gv, g = _run(cclib, m, x, v, off, dt, s_small=512)
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=dt), 1, sys_off=off)
    assert _rel_ok(gx, s.x3) and _rel_ok(gv, s.v3)
    for k in KEYS:
        assert g[k] == getattr(st, k), k
    assert g["max_depth_seen"] == st.max_depth_seen
    for ref in (32, 0):
        rx, rv, _ = _run(cclib, m, x, v, off, dt, s_small=ref)
        assert np.array_equal(gx, rx) and np.array_equal(gv, rv), ref


def test_batch_fp64_several_steps_config_256(cclib):
    """The 256-body Plummer configuration (dt = 1/64): eight outer steps, one
    launch each, bit-identical to the level path."""
    m, x, v = ics.plummer(256, seed=1)
    gx, gv, g = _run(cclib, m, x, v, None, 1 / 64, steps=8, s_small=512)
    rx, rv, r = _run(cclib, m, x, v, None, 1 / 64, steps=8, s_small=32)
    assert np.array_equal(gx, rx) and np.array_equal(gv, rv)
    for k in KEYS:
        assert g[k] == r[k], k
    # per outer step: the padding fill and the packing of the level-0
    # state, the batched kernel, the unpacking
    assert g["launches"] <= 4 * 8, g["launches"]
    s = O.State(m, x, v)
    O.evolve(s, O.params(dt=1 / 64), 8)
    assert _rel_ok(gx, s.x3, 1e-11) and _rel_ok(gv, s.v3, 1e-11)


@pytest.mark.parametrize("name", ["fractal1200", "systems", "plummer256"])
def test_batch_mixed_within_bounds(cclib, name):
    m, x, v, off, dt = _case(name)
    c = cclib.Context(m, x, v, dt=dt, precision=cclib.PREC_MIXED, near_tol=1e-6, s_small=512)
    if off is not None:
        c.set_systems(off)
    c.evolve(dt)
    _, _, gx, gv = c.get_state()
    pairs, _, _ = c.near_pairs()
    c.close()
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=dt), 1, sys_off=off)
    if off is None:
        S = B.abs_accel_sum(m, x)
    else:
        S = B.abs_accel_sum(m, x, groups=B.system_index(m.shape[0], off))
    ex = B.near_bodies(pairs)
    w, _ = B.check_velocity_bound(gv, s.v3, S, dt, st.max_depth_seen, exempt=ex)
    wx = B.check_position_bound(gx, s.x3, S, dt, st.max_depth_seen, exempt=ex)
    print(name, "batched mixed: max error / bound", w, "positions", wx)


def test_batch_kepler_mode(cclib):
    m, x, v = ics.plummer_with_binaries(2000, seed=2)
    dt = 1 / 256
    gx, gv, g = _run(cclib, m, x, v, None, dt, kepler=1, s_small=512)
    rx, rv, r = _run(cclib, m, x, v, None, dt, kepler=1, s_small=32)
    assert np.array_equal(gx, rx) and np.array_equal(gv, rv)
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=dt, kepler=True), 1)
    for k in KEYS + ("kepler_calls",):
        assert g[k] == getattr(st, k), k
    assert _rel_ok(gx, s.x3, 1e-9)


def test_batch_kepler_systems(cclib):
    """Kepler mode with every system a task (systems of 3..300 bodies)."""
    m, x, v, off, dt = _case("systems")
    gx, gv, g = _run(cclib, m, x, v, off, dt, kepler=1, s_small=512)
    rx, rv, r = _run(cclib, m, x, v, off, dt, kepler=1, s_small=32)
    assert np.array_equal(gx, rx) and np.array_equal(gv, rv)
    for k in KEYS + ("kepler_calls",):
        assert g[k] == r[k], k


def test_batch_hold(cclib):
    m, x, v, off, dt = _case("systems")
    gx, gv, g = _run(cclib, m, x, v, off, dt, split=cclib.SPLIT_HOLD, s_small=512)
    rx, rv, _ = _run(cclib, m, x, v, off, dt, split=cclib.SPLIT_HOLD, s_small=32)
    assert np.array_equal(gx, rx) and np.array_equal(gv, rv)
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=dt, split=O.SPLIT_HOLD), 1, sys_off=off)
    for k in KEYS:
        assert g[k] == getattr(st, k), k
    assert _rel_ok(gx, s.x3) and _rel_ok(gv, s.v3)


def test_batch_depth_limit_is_an_error(cclib):
    m, x, v = ics.plummer(256, seed=1)
    c = cclib.Context(m, x, v, dt=1 / 64, max_depth=1, s_small=512)
    with pytest.raises(cclib.CCError) as e:
        c.evolve(1 / 64)
    assert e.value.code == -3
    c.close()


def test_batch_s_small_is_checked(cclib, plummer_ic):
    m, x, v = plummer_ic(64)
    with pytest.raises(cclib.CCError) as e:
        cclib.Context(m, x, v, s_small=513)
    assert e.value.code == -1


def test_batch_step_graph_replays(cclib):
    """Whole-batch mode runs each outer step as one replay of a captured CUDA
    graph; a call with another eta captures the step again.  Several calls
    and an eta change give the level path's result bit for bit (FP64)."""
    m, x, v, off, dt = _case("systems")
    out = []
    for s_small in (512, 32):
        c = cclib.Context(m, x, v, dt=dt, s_small=s_small)
        c.set_systems(off)
        c.evolve(dt)
        c.evolve(3 * dt)
        c.evolve(4 * dt, eta=0.02)
        c.evolve(5 * dt, eta=0.03)
        t, _, gx, gv = c.get_state()
        out.append((gx, gv, c.stats()))
        c.close()
        assert abs(t - 5 * dt) < 1e-15
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    for k in KEYS:
        assert out[0][2][k] == out[1][2][k], k
    # fill, pack, the batched kernel, unpack: four kernels per replayed step
    assert out[0][2]["launches"] <= 4 * 5, out[0][2]["launches"]
