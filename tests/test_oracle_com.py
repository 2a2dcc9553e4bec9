"""Pins of the oracle's centre-of-mass approximation of V_CC (Sec. 4.1,
Discussion): the kick between two far components (R_a + R_b < theta
|X_a - X_b|, components of 2..com_max members) replaced by the force between
their centres of mass.

Anchors that do not come from the approximation's code itself:
  * theta = 0, or no pair of components far enough, is orc_kick bit for bit;
  * the same kick restated with numpy: exact pairs except the far ones, plus
    G M_b (X_b - X_a)/|X_b - X_a|^3 for every far component b;
  * linear and angular momentum are kept to rounding (the two forces between
    two components are opposite and along the line of their centres);
  * against the exact kick, every member of a far clump gets the clump's
    centre-of-mass acceleration, so a single body's error (the neglected
    tidal field) falls like R/d, and the error of the clump's mean
    acceleration like (R/d)^2 (the dipole about the centre of mass vanishes);
  * an evolve with the approximation conserves momentum and energy.
"""
import numpy as np

from oracle import oracle as O
from paper_1407_7105_gb300 import ics


def _clumps(k=6, per=5, spread=0.02, seed=3):
    """k tight clumps of `per` bodies on a ring of radius 1, plus 10 loose
    bodies; labels: one per clump (its smallest id), own id for the rest."""
    rng = np.random.default_rng(seed)
    xs, vs, lab = [], [], []
    nid = 0
    for c in range(k):
        ang = 2 * np.pi * c / k
        ctr = np.array([np.cos(ang), np.sin(ang), 0.1 * c])
        for q in range(per):
            xs.append(ctr + spread * rng.standard_normal(3))
            vs.append(0.1 * rng.standard_normal(3))
            lab.append(c * per)
        nid += per
    for q in range(10):
        xs.append(rng.standard_normal(3) * 2.0)
        vs.append(0.1 * rng.standard_normal(3))
        lab.append(nid + q)
    n = len(xs)
    m = rng.uniform(0.5, 1.5, n) / n
    x = np.ascontiguousarray(np.array(xs).T)
    v = np.ascontiguousarray(np.array(vs).T)
    return m, x, v, np.array(lab, dtype=np.int32)


def _kick(m, x, v, lab, h, p, com=True):
    s = O.State(m, x, v)
    st = O.Stats()
    ids = np.arange(m.shape[0], dtype=np.int32)
    if com:
        O.kick_com(s, p, ids, lab, h, stats=st)
    else:
        O.kick(s, p, ids, lab, h, stats=st)
    return s.v3, st


def test_theta_zero_and_no_far_pair_are_the_exact_kick():
    m, x, v, lab = _clumps()
    ref, _ = _kick(m, x, v, lab, 0.01, O.params(), com=False)
    for p in (O.params(theta=0.0), O.params(theta=1e-6), O.params(theta=0.5, com_max=4)):
        got, st = _kick(m, x, v, lab, 0.01, p)
        assert np.array_equal(got, ref) and st.com_pairs == 0


def test_kick_restated_with_numpy():
    m, x, v, lab = _clumps()
    theta, h, n = 0.5, 0.01, m.shape[0]
    got, st = _kick(m, x, v, lab, h, O.params(theta=theta))
    # numpy restatement
    comps = {}
    for i, l in enumerate(lab):
        comps.setdefault(int(l), []).append(i)
    comps = {l: np.array(ix) for l, ix in comps.items() if 2 <= len(ix) <= 32}
    cof = {}
    for l, ix in comps.items():
        M = m[ix].sum()
        X = (x[:, ix] * m[ix]).sum(axis=1) / M
        R = np.linalg.norm(x[:, ix] - X[:, None], axis=0).max()
        cof[l] = (M, X, R)
    far = {(a, b) for a in comps for b in comps
           if a != b and cof[a][2] + cof[b][2] < theta * np.linalg.norm(cof[a][1] - cof[b][1])}
    assert len(far) > 0
    acc = np.zeros((3, n))
    for i in range(n):
        for j in range(n):
            if i == j or lab[i] == lab[j] or (int(lab[i]), int(lab[j])) in far:
                continue
            d = x[:, j] - x[:, i]
            acc[:, i] += m[j] * d / np.linalg.norm(d) ** 3
    for (a, b) in far:
        d = cof[b][1] - cof[a][1]
        acc[:, comps[a]] += (cof[b][0] * d / np.linalg.norm(d) ** 3)[:, None]
    ref = v + h * acc
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-15)
    npairs = sum(len(comps[a]) * len(comps[b]) for (a, b) in far) // 2
    assert st.com_pairs == npairs


def test_momentum_and_angular_momentum_kept():
    m, x, v, lab = _clumps(k=8)
    got, st = _kick(m, x, v, lab, 0.05, O.params(theta=0.7))
    assert st.com_pairs > 0
    dv = got - v
    P = (m * dv).sum(axis=1)
    L = (m * np.cross(x.T, dv.T).T).sum(axis=1)
    scale = (m * np.abs(dv).sum(axis=0)).sum()
    assert np.abs(P).max() < 64 * 2.2e-16 * scale
    assert np.abs(L).max() < 256 * 2.2e-16 * scale * np.abs(x).max()


def test_error_orders_in_size_over_distance():
    """Two clumps of radius ~R at distance d: relative to the clumps' mutual
    kick, the largest error of a single body falls by ~2 when d doubles
    (first order: the tidal field is left out), the error of a clump's mean
    acceleration by ~4 (second order)."""
    rng = np.random.default_rng(5)
    base = 0.05 * rng.standard_normal((3, 8))
    errs, merrs = [], []
    for d in (1.0, 2.0, 4.0):
        x = np.concatenate([base[:, :4], base[:, 4:] + np.array([[d], [0.0], [0.0]])], axis=1)
        x = np.ascontiguousarray(x)
        m = np.full(8, 1.0 / 8)
        v = np.zeros((3, 8))
        lab = np.array([0, 0, 0, 0, 4, 4, 4, 4], dtype=np.int32)
        ex, _ = _kick(m, x, v, lab, 1.0, O.params(), com=False)
        ap, st = _kick(m, x, v, lab, 1.0, O.params(theta=0.9))
        assert st.com_pairs == 16
        errs.append(np.abs(ap - ex).max() / np.abs(ex).max())
        mean_err = np.abs((ap - ex)[:, :4].mean(axis=1)).max()
        merrs.append(mean_err / np.abs(ex[:, :4].mean(axis=1)).max())
    assert 1.6 < errs[0] / errs[1] < 2.5 and 1.6 < errs[1] / errs[2] < 2.5, errs
    assert merrs[0] / merrs[1] > 3.0 and merrs[1] / merrs[2] > 3.0, merrs


def test_evolve_with_the_approximation():
    m, x, v = ics.box_fractal(1200, seed=2)  # ~90 components of <= 32 bodies at dt = 1/64
    out = {}
    for theta in (0.0, 0.5):
        s = O.State(m, x, v)
        E0, P0, L0 = O.energy(s)
        st = O.evolve(s, O.params(dt=1 / 64, theta=theta), 1)
        E1, P1, L1 = O.energy(s)
        out[theta] = (s, st, (E1 - E0) / abs(E0), np.abs(P1 - P0).max())
    s0, st0, dE0, dP0 = out[0.0]
    s1, st1, dE1, dP1 = out[0.5]
    assert st1.com_pairs > 0.1 * st1.kick_pairs and st0.com_pairs == 0
    # the approximation's energy error stays small (the tidal field of far
    # components is left out); momentum is kept to rounding
    assert dP1 < 1e-15 and abs(dE1) < 1e-5 and abs(dE0) < 1e-6, (dP1, dE1, dE0)
