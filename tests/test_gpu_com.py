"""GPU parity of the centre-of-mass approximation of V_CC (Sec. 4.1,
Discussion; params.theta > 0): in the DKD of sets of at least 33 members,
components of 2..com_max members whose radii satisfy R_a + R_b < theta
|X_a - X_b| kick each other through their centres of mass.  Against the
oracle's evolve_cc with the same theta and com_max: the FP64 form bit for
bit with the same counts (kick pairs and the pairs the approximation took),
the mixed form within the per-body FP32 bound."""
import numpy as np
import pytest

import _bounds as B
from oracle import oracle as O
from paper_1407_7105_gb300 import ics

pytestmark = pytest.mark.gpu


def _rel_ok(a, b, rtol=1e-12):
    scale = np.abs(b).max()
    return np.all(np.abs(a - b) <= rtol * np.abs(b) + 1e-15 * scale)


@pytest.mark.parametrize("case", ["fractal", "plummer"])
def test_com_one_step_fp64(cclib, case):
    if case == "fractal":
        m, x, v = ics.box_fractal(1200, seed=2)  # ~90 components of <= 32 bodies at dt = 1/64
        dt, theta, com_max = 1 / 64, 0.5, 32
    else:
        m, x, v = ics.plummer(2000, seed=9)
        dt, theta, com_max = 1 / 32, 0.8, 16
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=dt, theta=theta, com_max=com_max), 1)
    assert st.com_pairs > 0
    c = cclib.Context(m, x, v, dt=dt, theta=theta, com_max=com_max)
    c.evolve(dt)
    _, _, gx, gv = c.get_state()
    g = c.stats()
    c.close()
    assert _rel_ok(gx, s.x3) and _rel_ok(gv, s.v3)
    for key in ("tau_pairs", "kick_pairs", "com_pairs", "drifts", "splits", "components"):
        assert g[key] == getattr(st, key), key


def test_com_theta_zero_is_the_exact_path(cclib, plummer_ic):
    m, x, v = plummer_ic(1000)
    out = []
    for theta in (0.0, None):
        kw = {} if theta is None else {"theta": theta}
        c = cclib.Context(m, x, v, dt=1 / 128, **kw)
        c.evolve(1 / 128)
        _, _, gx, gv = c.get_state()
        out.append((gx, gv, c.stats()["com_pairs"]))
        c.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == 0


def test_com_mixed_within_bounds(cclib):
    m, x, v = ics.box_fractal(1200, seed=2)
    dt = 1 / 64
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=dt, theta=0.5), 1)
    c = cclib.Context(m, x, v, dt=dt, theta=0.5, precision=cclib.PREC_MIXED, near_tol=1e-6)
    c.evolve(dt)
    _, _, gx, gv = c.get_state()
    g = c.stats()
    pairs, _, _ = c.near_pairs()
    c.close()
    assert g["com_pairs"] > 0
    S = B.abs_accel_sum(m, x)
    w, _ = B.check_velocity_bound(gv, s.v3, S, dt, st.max_depth_seen, exempt=B.near_bodies(pairs))
    print("COM mixed: max error / bound", w)


def test_com_parameters_are_checked(cclib, plummer_ic):
    m, x, v = plummer_ic(64)
    for bad in (dict(theta=-1.0), dict(theta=0.5, com_max=65), dict(theta=0.5, com_max=1),
                dict(theta=0.5, split=cclib.SPLIT_HOLD), dict(theta=float("inf"))):
        with pytest.raises(cclib.CCError) as e:
            cclib.Context(m, x, v, **bad)
        assert e.value.code == -1, bad


def test_com_kepler_mode_one_step(cclib):
    """Kepler mode: the two-body components are advanced by Kepler's
    equation and, being eligible, take part in the approximation."""
    m, x, v = ics.plummer_with_binaries(2000, seed=2)
    dt = 1 / 256
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=dt, theta=0.5, kepler=True), 1)
    assert st.com_pairs > 0
    c = cclib.Context(m, x, v, dt=dt, theta=0.5, kepler=1)
    c.evolve(dt)
    _, _, gx, gv = c.get_state()
    g = c.stats()
    c.close()
    for key in ("kick_pairs", "com_pairs", "drifts", "splits", "components", "kepler_calls"):
        assert g[key] == getattr(st, key), key
    assert _rel_ok(gx, s.x3, 1e-9)
    rel = np.linalg.norm(gv - s.v3, axis=0) / np.linalg.norm(s.v3, axis=0)
    assert np.median(rel) < 1e-12 and np.quantile(rel, 0.99) < 1e-6, (np.median(rel), np.quantile(rel, 0.99))
