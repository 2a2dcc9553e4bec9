"""Pins of the oracle's HOLD integrator (Sec. 2.1, Eq. HOLD): the slow/fast
split by the particle time step tau(i) (read as the minimum of tau(i,j)
over the other members of the set) and the recursion
E_{h/2,H_F} D_{h/2,T_S} K_{h,V_S+V_SF} D_{h/2,T_S} E_{h/2,H_F}.

Anchors that do not come from the HOLD code itself:
  * tau(i) < h exactly when i has an edge of the time-step graph at h, so F
    is the union of the CC split's non-trivial components: the row minima
    of orc_hold_split against the breadth-first search of orc_components;
  * with no fast particle the step is the textbook leapfrog (numpy);
  * a set with at most three bodies has at most one non-trivial component
    at every level, where the CC and HOLD splits coincide: triples evolve
    bit for bit as under evolve_cc;
  * two well separated hard binaries: CC evolves each alone, HOLD kicks
    the pairs between them at the binaries' step (Sec. 2.2: the terms HOLD
    evolves inefficiently), with the same answer to the integrators' order;
  * linear and angular momentum conserved to machine precision, second
    order in eta, every pair evaluated by the HOLD split.
"""
import numpy as np

from oracle import oracle as O
from paper_1407_7105_gb300 import ics


def _leapfrog_dkd(m, x, v, h, G=1.0):
    x = x + 0.5 * h * v
    d = x[:, None, :] - x[:, :, None]
    r2 = (d * d).sum(axis=0)
    np.fill_diagonal(r2, np.inf)
    a = G * (d * (m[None, None, :] / r2 ** 1.5)).sum(axis=2)
    v = v + h * a
    x = x + 0.5 * h * v
    return x, v


def test_fast_set_is_the_union_of_cc_components():
    for seed, n in ((1, 200), (2, 350), (3, 64)):
        m, x, v = ics.plummer(n, seed=seed)
        s = O.State(m, x, v)
        p = O.params()
        for h in (1 / 16, 1 / 64, 1 / 256, 1 / 2048):
            hl, hk = O.hold_split(s, p, h)
            cl, ck = O.components(s, p, h)
            shared = np.bincount(cl, minlength=n)[cl] >= 2
            fast = hl != np.arange(n)
            fast |= np.bincount(hl, minlength=n)[hl] >= 2
            assert np.array_equal(fast, shared), (seed, h)
            assert hk == (1 if shared.any() else 0)
            if shared.any():
                assert (hl[shared] == np.flatnonzero(shared).min()).all()
                assert (hl[~shared] == np.flatnonzero(~shared)).all()


def test_no_fast_particle_is_leapfrog():
    m, x, v = ics.plummer(48, seed=2)
    s = O.State(m, x, v)
    p = O.params(split=O.SPLIT_HOLD)
    T = O.tau_matrix(s, p)
    h = 0.5 * float(T[np.isfinite(T)].min())
    st = O.evolve_hold(s, p, h)
    assert st.components == 0 and st.splits == 1
    xr, vr = _leapfrog_dkd(m, x, v, h)
    assert np.allclose(s.x3, xr, rtol=0, atol=1e-14)
    assert np.allclose(s.v3, vr, rtol=0, atol=1e-13 * np.abs(vr).max())


def test_triples_evolve_as_under_cc():
    for stream in range(6):
        m, x, v = ics.hierarchical_triple(7, 500 + 11 * stream)
        out = []
        for split in (O.SPLIT_CC, O.SPLIT_HOLD):
            s = O.State(m, x, v)
            st = O.evolve(s, O.params(dt=1 / 8, split=split), 4)
            out.append((s.x3, s.v3, st))
        (xc, vc, sc), (xh, vh, sh) = out
        assert np.array_equal(xc, xh) and np.array_equal(vc, vh), stream
        for k in ("splits", "kick_pairs", "drifts", "components", "tau_pairs", "max_depth_seen"):
            assert getattr(sc, k) == getattr(sh, k), (stream, k)
        assert sh.tau_evals == sh.tau_pairs  # HOLD evaluates every pair


def _two_binaries():
    parts = []
    for k, off in enumerate((-0.5, 0.5)):
        bm, bx, bv = ics.binary(0.25, 0.25, 1e-3, 0.3, E_anom=0.7 + k, inc=0.4 * k)
        bx = bx + np.array([[off], [0.1 * k], [0.0]])
        bv = bv + np.array([[0.0], [0.3 - 0.6 * k], [0.0]])
        parts.append((bm, bx, bv))
    m = np.concatenate([p[0] for p in parts])
    x = np.ascontiguousarray(np.concatenate([p[1] for p in parts], axis=1))
    v = np.ascontiguousarray(np.concatenate([p[2] for p in parts], axis=1))
    return m, x, v


def test_separated_binaries_hold_kicks_what_cc_does_not():
    m, x, v = _two_binaries()
    res = {}
    for split in (O.SPLIT_CC, O.SPLIT_HOLD):
        s = O.State(m, x, v)
        st = O.evolve(s, O.params(dt=1 / 32, split=split), 1)
        res[split] = (s, st)
    sc, stc = res[O.SPLIT_CC]
    sh, sth = res[O.SPLIT_HOLD]
    # CC: two components, each binary alone below the top level; HOLD: one
    # fast set of four, whose cross-binary pairs are kicked at every level
    assert stc.components > sth.components
    assert sth.kick_pairs > stc.kick_pairs
    # Both split the same flow at second order.  The binaries' centres of
    # mass move under the slow cross-binary force, integrated alike: they
    # agree to its splitting error.  Inside each binary (~700 radians per
    # step) that force acts once per step under CC and at every fast step
    # under HOLD: the relative velocities differ, by less than the
    # cross-binary kick itself, G M_other / d^2 dt.
    for i, j in ((0, 1), (2, 3)):
        M = m[i] + m[j]
        for q in ("x3", "v3"):
            ca = (m[i] * getattr(sc, q)[:, i] + m[j] * getattr(sc, q)[:, j]) / M
            cb = (m[i] * getattr(sh, q)[:, i] + m[j] * getattr(sh, q)[:, j]) / M
            assert np.abs(ca - cb).max() < (1e-8 if q == "x3" else 1e-7), (i, q)
        du = (sc.v3[:, i] - sc.v3[:, j]) - (sh.v3[:, i] - sh.v3[:, j])
        assert np.abs(du).max() < 0.5 / 1.0 ** 2 / 32


def test_momentum_conserved_and_second_order():
    m, x, v = ics.plummer(128, seed=4)
    s = O.State(m, x, v)
    E0, P0, L0 = O.energy(s)
    st = O.evolve(s, O.params(eta=0.03, dt=1.0 / 64, split=O.SPLIT_HOLD), 8)
    assert st.components > 0 and st.max_depth_seen >= 2
    assert st.tau_evals == st.tau_pairs
    E1, P1, L1 = O.energy(s)
    psc = float((m * np.abs(v).sum(axis=0)).sum())
    assert np.abs(P1 - P0).max() < 64 * 2.2e-16 * psc
    lsc = float((m * (np.abs(x) * np.abs(v).sum(axis=0)).sum(axis=0)).sum())
    assert np.abs(L1 - L0).max() < 256 * 2.2e-16 * lsc
    # energy error against eta: second order (ratio ~4 per halving)
    m, x, v = ics.plummer(64, seed=9)
    errs = []
    for eta in (0.04, 0.02, 0.01):
        s = O.State(m, x, v)
        e0, _, _ = O.energy(s)
        O.evolve(s, O.params(eta=eta, dt=1.0 / 16, split=O.SPLIT_HOLD), 4)
        e1, _, _ = O.energy(s)
        errs.append(abs((e1 - e0) / e0))
    assert errs[0] / errs[2] > 6.0, errs
