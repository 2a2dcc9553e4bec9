"""Pins of the oracle's CC integrator (evolve_cc, Sec. 2.2-2.3) and of its
two-body Kepler flow (CC_KEPLER, Sec. 3.2).

Anchors that do not come from the oracle itself:
  * with no edge at the threshold, one evolve_cc step is the textbook
    drift-kick-drift leapfrog of the whole system (Eq. second-order-split
    with A = T, B = V), written here independently with numpy;
  * linear and angular momentum are conserved to machine precision
    (Sec. 3.1: kicks come in symmetric pairs);
  * a two-body orbit converges to the Kepler closed form at second order
    in eta; after one period the orbit returns to its start;
  * approximate time symmetry (forward, reverse velocities, forward);
  * the Kepler solver against orbital elements advanced through the mean
    anomaly with a library root finder, and against exact rotations of a
    circular orbit.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import oracle as O
from paper_1407_7105_gb300 import ics


def _leapfrog_dkd(m, x, v, h, G=1.0, eps=0.0):
    x = x + 0.5 * h * v
    d = x[:, None, :] - x[:, :, None]           # d[:, i, j] = x_j - x_i
    r2 = (d * d).sum(axis=0) + eps * eps
    np.fill_diagonal(r2, np.inf)
    a = G * (d * (m[None, None, :] / r2 ** 1.5)).sum(axis=2)
    v = v + h * a
    x = x + 0.5 * h * v
    return x, v


def test_no_edges_is_leapfrog():
    m, x, v = ics.plummer(48, seed=2)
    s = O.State(m, x, v)
    p = O.params(eta=0.03)
    T = O.tau_matrix(s, p)
    h = 0.5 * float(T[np.isfinite(T)].min())
    st = O.evolve_cc(s, p, h)
    assert st.components == 0 and st.splits == 1
    xr, vr = _leapfrog_dkd(m, x, v, h)
    assert np.allclose(s.x3, xr, rtol=0, atol=1e-14)
    assert np.allclose(s.v3, vr, rtol=0, atol=1e-13 * np.abs(vr).max())


def test_momentum_conserved():
    m, x, v = ics.plummer(128, seed=4)
    s = O.State(m, x, v)
    E0, P0, L0 = O.energy(s)
    p = O.params(eta=0.03, dt=1.0 / 64)
    st = O.evolve(s, p, 8)
    assert st.components > 0 and st.max_depth_seen >= 2
    E1, P1, L1 = O.energy(s)
    psc = float((m * np.abs(v).sum(axis=0)).sum())
    assert np.abs(P1 - P0).max() < 64 * 2.2e-16 * psc
    lsc = float((m * np.linalg.norm(x, axis=0) * np.linalg.norm(v, axis=0)).sum())
    assert np.abs(L1 - L0).max() < 256 * 2.2e-16 * lsc
    assert abs((E1 - E0) / E0) < 1e-5


def _period(m1, m2, a):
    return 2 * math.pi * math.sqrt(a ** 3 / (m1 + m2))


def test_two_body_second_order_convergence():
    """CC on an isolated eccentric binary (no Kepler mode) is an adaptive
    power-of-two leapfrog; its error after one period falls as eta^2."""
    m1, m2, a, e = 0.6, 0.4, 1.0, 0.5
    P = _period(m1, m2, a)
    errs = []
    for eta in (0.04, 0.01, 0.0025):
        m, x, v = ics.binary(m1, m2, a, e, E_anom=0.3)
        s = O.State(m, x, v)
        p = O.params(eta=eta, dt=P / 8)
        O.evolve(s, p, 8)
        errs.append(np.abs(s.x3 - x).max())
    assert errs[0] / errs[1] > 6 and errs[1] / errs[2] > 6
    assert errs[2] < 1e-4


def test_time_symmetry():
    """Integrate forward, reverse the velocities, integrate again: the start
    is recovered with reversed velocities (tau(i,j) is only approximately
    time symmetric, so to a tolerance that shrinks with eta)."""
    devs = []
    for eta in (0.03, 0.01):
        m, x, v = ics.plummer(64, seed=5)
        s = O.State(m, x, v)
        p = O.params(eta=eta, dt=1.0 / 64)
        O.evolve(s, p, 8)
        s.v3 = -s.v3
        O.evolve(s, p, 8)
        devs.append(max(np.abs(s.x3 - x).max(), np.abs(s.v3 + v).max()))
    assert devs[0] < 1e-4
    assert devs[1] < devs[0]


def test_second_order_energy_in_eta():
    dEs = []
    for eta in (0.04, 0.01):
        m, x, v = ics.plummer(64, seed=8)
        s = O.State(m, x, v)
        E0, _, _ = O.energy(s)
        O.evolve(s, O.params(eta=eta, dt=1.0 / 32), 8)
        E1, _, _ = O.energy(s)
        dEs.append(abs((E1 - E0) / E0))
    assert dEs[0] / dEs[1] > 4


# ---------------------------------------------------------------- Kepler
def _kepler_closed_form(m1, m2, a, e, E0, t, **kw):
    mu = m1 + m2
    n = math.sqrt(mu / a ** 3)
    M0 = E0 - e * math.sin(E0)
    M = M0 + n * t
    k = math.floor(M / (2 * math.pi))
    Mr = M - 2 * math.pi * k
    E = brentq(lambda E: E - e * math.sin(E) - Mr, 0.0, 2 * math.pi, xtol=1e-15, rtol=1e-15)
    return ics.binary(m1, m2, a, e, E_anom=E, **kw)


@pytest.mark.parametrize("e", [0.0, 0.3, 0.9, 0.99])
@pytest.mark.parametrize("frac", [0.013, 0.37, 0.5, 2.71])
def test_kepler_against_mean_anomaly(e, frac):
    m1, m2, a = 0.7, 0.3, 0.02
    kw = dict(inc=0.4, node=1.1, peri=2.0)
    m, x, v = ics.binary(m1, m2, a, e, E_anom=1.0, **kw)
    P = _period(m1, m2, a)
    s = O.State(m, x, v)
    O.kepler(s, 0, 1, frac * P)
    _, xr, vr = _kepler_closed_form(m1, m2, a, e, 1.0, frac * P, **kw)
    vscale = math.sqrt((m1 + m2) / a) * math.sqrt((1 + e) / (1 - e + 1e-300))
    assert np.abs(s.x3 - xr).max() < 1e-12 * a / (1 - e) ** 0.5
    assert np.abs(s.v3 - vr).max() < 1e-12 * vscale / (1 - e) ** 0.5


def test_kepler_circular_is_rotation():
    m1, m2, a = 0.5, 0.5, 1.0
    m, x, v = ics.binary(m1, m2, a, 0.0, E_anom=0.0)
    w = math.sqrt((m1 + m2) / a ** 3)
    for t in (0.1, 1.0, 7.3):
        s = O.State(m, x, v)
        O.kepler(s, 0, 1, t)
        c, sn = math.cos(w * t), math.sin(w * t)
        R = np.array([[c, -sn, 0], [sn, c, 0], [0, 0, 1]])
        assert np.abs(s.x3 - R @ x).max() < 1e-13
        assert np.abs(s.v3 - R @ v).max() < 1e-13


def test_kepler_hyperbolic_invariants_and_reversal():
    # unbound pair: energy and angular momentum invariant; flow for -t undoes +t
    m = np.array([0.3, 0.5])
    x = np.array([[0.1, -0.2], [0.05, 0.0], [0.0, 0.01]])
    v = np.array([[0.0, 0.0], [3.0, -2.0], [0.1, 0.0]])
    s = O.State(m, x, v)
    E0, P0, L0 = O.energy(s)
    O.kepler(s, 0, 1, 0.37)
    E1, P1, L1 = O.energy(s)
    assert abs(E1 - E0) < 1e-14 * abs(E0) * 10
    assert np.abs(L1 - L0).max() < 1e-14
    O.kepler(s, 0, 1, -0.37)
    assert np.abs(s.x3 - x).max() < 1e-13 and np.abs(s.v3 - v).max() < 1e-12


def test_kepler_mode_two_body_component_exact():
    """CC_KEPLER: an isolated binary whose pair is a component is advanced
    by the Kepler flow itself, so one outer step matches the closed form to
    rounding whatever eta is."""
    m1, m2, a, e = 0.6, 0.4, 1e-3, 0.7
    m, x, v = ics.binary(m1, m2, a, e, E_anom=0.5)
    s = O.State(m, x, v)
    dt = 1.0 / 64
    st = O.evolve(s, O.params(eta=0.03, dt=dt, kepler=True), 1)
    assert st.kepler_calls == 2
    _, xr, vr = _kepler_closed_form(m1, m2, a, e, 0.5, dt)
    assert np.abs(s.x3 - xr).max() < 1e-12 * a * 50
