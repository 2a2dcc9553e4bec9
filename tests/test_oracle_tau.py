"""Pins of the oracle's interaction time step tau(i,j) (Eq. tauij, Sec. 2.2).

The paper prints no worked example of tau(i,j), so the oracle is pinned by
closed forms of special cases, by finite differences of its own T's along
the pair's motion (which checks the two time derivatives independently of
how they were derived), by exact symmetry and by exact dimensional scaling.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O

ETA = 0.03


def _tau(dx, dv, mi=0.3, mj=0.5, G=1.0, eps=0.0, eta=ETA, eta_outside=False):
    p = O.params(G=G, eps=eps, eta=eta, eta_outside=eta_outside)
    return O.tau_parts(np.asarray(dx, float), np.asarray(dv, float), mi, np.zeros(3), np.zeros(3), mj, p)


def test_rest_pair_is_free_fall_time():
    # relative velocity zero: no flyby term, dT/dt = 0, tau = eta sqrt(r^3/mu)
    r, mu = 0.25, 0.8
    t, parts = _tau([0.0, r, 0.0], [0.0, 0.0, 0.0])
    assert math.isinf(parts[2]) and math.isinf(parts[5])
    assert t == pytest.approx(ETA * math.sqrt(r ** 3 / mu), rel=1e-15)


def test_perpendicular_velocity_closed_form():
    # dx . dv = 0: both derivatives vanish, tau = eta min(sqrt(r^3/mu), r/|v|)
    r, v, mu = 1.0, 2.0, 0.8
    t, parts = _tau([r, 0.0, 0.0], [0.0, v, 0.0])
    assert parts[1] == 0.0 and parts[3] == 0.0
    assert parts[0] == pytest.approx(ETA * math.sqrt(r ** 3 / mu), rel=1e-15)
    assert parts[2] == pytest.approx(ETA * r / v, rel=1e-15)
    assert t == pytest.approx(min(parts[0], parts[2]), rel=0)
    # slow relative motion: free fall wins
    t2, p2 = _tau([r, 0.0, 0.0], [0.0, 0.01, 0.0])
    assert t2 == p2[4] == p2[0]


def test_softening_enters_r():
    eps = 0.1
    t, parts = _tau([0.3, 0.0, 0.0], [0.0, 0.0, 0.0], eps=eps)
    r = math.sqrt(0.09 + eps * eps)
    assert t == pytest.approx(ETA * math.sqrt(r ** 3 / 0.8), rel=1e-15)


def test_receding_clamp_gives_twice_T():
    # a fast receding pair with eta large enough that dT/dt >= 1 is clamped
    t, parts = _tau([1.0, 0.0, 0.0], [50.0, 0.0, 0.0], eta=2.0)
    assert parts[3] >= 1.0
    assert parts[5] == 2.0 * parts[2]


def test_approaching_pair_shortens_step():
    t, parts = _tau([1.0, 0.2, 0.0], [-3.0, 0.0, 0.0])
    assert parts[1] < 0 and parts[3] < 0
    assert parts[4] < parts[0] and parts[5] < parts[2]


@pytest.mark.parametrize("seed", range(6))
def test_time_derivatives_match_finite_differences(seed):
    """dT_ff/dt and dT_fb/dt equal the derivative of T along the pair's own
    relative motion: d(dx)/dt = dv, d(dv)/dt = -mu dx / r^3 (eps = 0)."""
    rng = np.random.default_rng(seed)
    dx = rng.normal(size=3)
    dv = rng.normal(size=3)
    mi, mj = 0.2 + rng.random(), 0.2 + rng.random()
    mu = mi + mj
    _, parts = _tau(dx, dv, mi=mi, mj=mj)
    r = np.linalg.norm(dx)
    acc = -mu * dx / r ** 3
    d = 1e-5
    _, pp = _tau(dx + d * dv, dv + d * acc, mi=mi, mj=mj)
    _, pm = _tau(dx - d * dv, dv - d * acc, mi=mi, mj=mj)
    fd_ff = (pp[0] - pm[0]) / (2 * d)
    fd_fb = (pp[2] - pm[2]) / (2 * d)
    assert parts[1] == pytest.approx(fd_ff, rel=1e-7, abs=1e-12)
    assert parts[3] == pytest.approx(fd_fb, rel=1e-7, abs=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_symmetric_bitwise(seed):
    rng = np.random.default_rng(100 + seed)
    p = O.params()
    xi, xj, vi, vj = rng.normal(size=(4, 3))
    a, _ = O.tau_parts(xi, vi, 0.3, xj, vj, 0.7, p)
    b, _ = O.tau_parts(xj, vj, 0.7, xi, vi, 0.3, p)
    assert a == b


@pytest.mark.parametrize("seed", range(4))
def test_dimensional_scaling_exact(seed):
    """x -> 4x, v -> v/2 with masses fixed multiplies every time by 8;
    all the factors are powers of two so the result is exact bitwise."""
    rng = np.random.default_rng(200 + seed)
    dx, dv = rng.normal(size=(2, 3))
    t1, p1 = _tau(dx, dv)
    t2, p2 = _tau(4.0 * dx, 0.5 * dv)
    assert t2 == 8.0 * t1
    assert p2[1] == p1[1] and p2[3] == p1[3]


def test_eta_outside_reading_differs_only_in_derivative():
    # with dx . dv = 0 the two readings coincide
    t_in, _ = _tau([1.0, 0.0, 0.0], [0.0, 2.0, 0.0])
    t_out, _ = _tau([1.0, 0.0, 0.0], [0.0, 2.0, 0.0], eta_outside=True)
    assert t_in == pytest.approx(t_out, rel=1e-15)
    t_in, _ = _tau([1.0, 0.0, 0.0], [-2.0, 0.3, 0.0])
    t_out, _ = _tau([1.0, 0.0, 0.0], [-2.0, 0.3, 0.0], eta_outside=True)
    assert t_in != t_out


def test_midpoint_property():
    """tau = T/(1 - T'/2) solves tau = T(t + tau/2) to second order: the
    step equals the (linearised) time step at its own midpoint."""
    dx = np.array([1.0, 0.3, -0.2])
    dv = np.array([-0.4, 0.1, 0.05])
    mi, mj = 0.4, 0.6
    _, parts = _tau(dx, dv, mi=mi, mj=mj)
    tau_ff = parts[4]
    mid = dx + 0.5 * tau_ff * dv
    _, pm = _tau(mid, dv, mi=mi, mj=mj)
    assert abs(pm[0] - tau_ff) / tau_ff < 50 * (ETA * 0.5) ** 2
