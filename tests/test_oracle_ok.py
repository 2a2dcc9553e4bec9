"""Pins of the oracle's OK split (Sec. 4.2: the interactions of a set, not its
particles, partitioned by tau(i,j) against the pivot h; reading R15 in
oracle/cc_oracle.c).

Anchors that do not come from the OK code itself:
  * with no interaction below the threshold, one step is the textbook
    drift-kick-drift leapfrog of the whole set (numpy);
  * a restatement of the reading in plain Python (recursive lists, numpy
    pair forces, tau from the pinned tau routine) on small clusters with
    several recursion levels, and interaction lists given explicitly;
  * a two-body set has one interaction, so its OK split is its CC split
    (the same leapfrog on the same power-of-two levels): bit for bit;
  * linear and angular momentum to machine precision (kicks come in
    symmetric pairs, Sec. 4.2);
  * approximate time symmetry and second-order energy error in eta;
  * the operation counts of a level (tau pairs = |I|, kick pairs = |I_S|,
    drifts = 2 |S \\ F|).
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


def test_no_fast_interaction_is_leapfrog():
    m, x, v = ics.plummer(40, seed=3)
    s = O.State(m, x, v)
    p = O.params(eta=0.03)
    T = O.tau_matrix(s, p)
    h = 0.5 * float(T[np.isfinite(T)].min())
    st = O.evolve_ok(s, p, h)
    assert st.components == 0 and st.splits == 1
    assert st.tau_pairs == 40 * 39 // 2 and st.kick_pairs == 40 * 39 // 2 and st.drifts == 2 * 40
    xr, vr = _leapfrog_dkd(m, x, v, h)
    assert np.allclose(s.x3, xr, rtol=0, atol=1e-14)
    assert np.allclose(s.v3, vr, rtol=0, atol=1e-13 * np.abs(vr).max())


class _Ref:
    """The reading of Sec. 4.2 in plain Python: evolve_ok(S, I, h) on
    particle-id lists and pair lists, tau from the oracle's pinned routine."""

    def __init__(self, s, p):
        self.s, self.p = s, p
        self.kicks = 0

    def tau(self, i, j):
        return O.tau_ids(self.s, self.p, i, j)

    def kick(self, set_ids, slow, h):
        x, v, m = self.s.x3, self.s.v3, self.s.m
        acc = {i: np.zeros(3) for i in set_ids}
        for (i, j) in slow:
            d = x[:, j] - x[:, i]
            w = 1.0 / np.dot(d, d) ** 1.5
            acc[i] += m[j] * w * d
            acc[j] -= m[i] * w * d
        for i in set_ids:
            v[:, i] += h * acc[i]
        self.kicks += len(slow)

    def drift(self, ids, dt):
        for i in ids:
            self.s.x3[:, i] += dt * self.s.v3[:, i]

    def evolve(self, set_ids, pairs, h):
        fast = [(i, j) for (i, j) in pairs if self.tau(i, j) < h]
        fs = set(fast)
        slow = [q for q in pairs if q not in fs]
        F = sorted({k for q in fast for k in q})
        rest = [i for i in set_ids if i not in set(F)]
        if fast:
            self.evolve(F, fast, 0.5 * h)
        self.drift(rest, 0.5 * h)
        self.kick(set_ids, slow, h)
        self.drift(rest, 0.5 * h)
        if fast:
            self.evolve(F, fast, 0.5 * h)


def _all_pairs(ids):
    ids = list(ids)
    return [(ids[a], ids[b]) for a in range(len(ids)) for b in range(a + 1, len(ids))]


def test_restated_in_python():
    for seed, n, dt in ((11, 12, 1 / 8), (12, 16, 1 / 16), (13, 10, 1 / 4)):
        m, x, v = ics.plummer(n, seed=seed)
        p = O.params(eta=0.05, dt=dt)
        s = O.State(m, x, v)
        st = O.evolve_ok(s, p, dt)
        assert st.max_depth_seen >= 2, (seed, st.max_depth_seen)
        r = _Ref(O.State(m, x, v), p)
        r.evolve(list(range(n)), _all_pairs(range(n)), dt)
        assert r.kicks == st.kick_pairs
        assert np.allclose(s.x3, r.s.x3, rtol=1e-13, atol=1e-15)
        assert np.allclose(s.v3, r.s.v3, rtol=1e-12, atol=1e-13 * np.abs(r.s.v3).max())


def test_explicit_interaction_list():
    """evolve_ok on a subset with an explicit (sparse) interaction list, as
    the recursion calls it."""
    m, x, v = ics.plummer(14, seed=21)
    p = O.params(eta=0.05)
    rng = np.random.default_rng(4)
    ids = np.sort(rng.choice(14, size=9, replace=False)).astype(np.int32)
    allp = _all_pairs(ids)
    pick = sorted(allp[k] for k in rng.choice(len(allp), size=20, replace=False))
    s = O.State(m, x, v)
    st = O.evolve_ok(s, p, 1 / 8, set_ids=ids, pairs=np.array(pick))
    r = _Ref(O.State(m, x, v), p)
    r.evolve(list(ids), pick, 1 / 8)
    assert r.kicks == st.kick_pairs
    assert np.allclose(s.x3, r.s.x3, rtol=1e-13, atol=1e-15)
    assert np.allclose(s.v3, r.s.v3, rtol=1e-12, atol=1e-13 * np.abs(r.s.v3).max())
    # particles outside the set are untouched
    out = np.setdiff1d(np.arange(14), ids)
    assert np.array_equal(s.x3[:, out], x[:, out]) and np.array_equal(s.v3[:, out], v[:, out])


def test_two_bodies_equal_the_cc_split():
    m, x, v = ics.binary(0.6, 0.4, 1.0, 0.7, E_anom=0.4)
    out = []
    for split in (O.SPLIT_OK, O.SPLIT_CC):
        s = O.State(m, x, v)
        st = O.evolve(s, O.params(eta=0.02, dt=1.0, split=split), 4)
        out.append((s.x3, s.v3, st.splits, st.kick_pairs, st.max_depth_seen))
    assert st.max_depth_seen >= 4
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2:] == out[1][2:]


def test_momentum_conserved():
    m, x, v = ics.plummer(96, seed=4)
    s = O.State(m, x, v)
    E0, P0, L0 = O.energy(s)
    st = O.evolve(s, O.params(eta=0.03, dt=1.0 / 64, split=O.SPLIT_OK), 6)
    assert st.components > 0 and st.max_depth_seen >= 2
    E1, P1, L1 = O.energy(s)
    psc = float((m * np.abs(v).sum(axis=0)).sum())
    assert np.abs(P1 - P0).max() < 64 * 2.2e-16 * psc
    lsc = float((m * np.linalg.norm(x, axis=0) * np.linalg.norm(v, axis=0)).sum())
    assert np.abs(L1 - L0).max() < 256 * 2.2e-16 * lsc


def test_time_symmetry():
    devs = []
    for eta in (0.03, 0.01):
        m, x, v = ics.plummer(48, seed=5)
        s = O.State(m, x, v)
        p = O.params(eta=eta, dt=1.0 / 64, split=O.SPLIT_OK)
        O.evolve(s, p, 8)
        s.v3 = -s.v3
        O.evolve(s, p, 8)
        devs.append(max(np.abs(s.x3 - x).max(), np.abs(s.v3 + v).max()))
    assert devs[0] < 1e-3
    assert devs[1] < devs[0]


def test_second_order_energy_in_eta():
    dEs = []
    for eta in (0.04, 0.01):
        m, x, v = ics.plummer(48, seed=8)
        s = O.State(m, x, v)
        E0, _, _ = O.energy(s)
        O.evolve(s, O.params(eta=eta, dt=1.0 / 32, split=O.SPLIT_OK), 8)
        E1, _, _ = O.energy(s)
        dEs.append(abs((E1 - E0) / E0))
    assert dEs[0] / dEs[1] > 4, dEs


def test_ok_kicks_slow_pairs_inside_components():
    """Where a component holds a pair that is not an edge, the CC split
    kicks it at the component's finer level, the OK split at the pivot of
    its own tau: the OK split needs fewer kick evaluations (Sec. 4.2)."""
    m, x, v = ics.plummer(64, seed=9)
    counts = {}
    for split in (O.SPLIT_CC, O.SPLIT_OK):
        s = O.State(m, x, v)
        counts[split] = O.evolve(s, O.params(eta=0.03, dt=1.0 / 16, split=split), 2)
    assert counts[O.SPLIT_OK].kick_pairs < counts[O.SPLIT_CC].kick_pairs
