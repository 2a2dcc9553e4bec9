"""GPU parity of the kick, the drift and the recursive CC integrator
(Sec. 2.2-2.3, CC pseudocode figure) against the FP64 oracle."""
import numpy as np
import pytest

import _bounds as B
from oracle import oracle as O
from paper_1407_7105_gb300 import ics

pytestmark = pytest.mark.gpu


def _rel_ok(a, b, rtol=1e-12):
    scale = np.abs(b).max()
    return np.all(np.abs(a - b) <= rtol * np.abs(b) + 1e-15 * scale)


def test_kick_bit_exact(cclib, plummer_ic):
    m, x, v = plummer_ic(300, seed=4)
    rng = np.random.default_rng(0)
    labels = rng.integers(0, 40, 300).astype(np.int32)
    c = cclib.Context(m, x, v)
    c.kick(labels, 1 / 64)
    _, _, gx, gv = c.get_state()
    s = O.State(m, x, v)
    O.kick(s, O.params(), np.arange(300), labels, 1 / 64)
    assert np.array_equal(gv, s.v3) and np.array_equal(gx, s.x3)
    c.close()


def test_drift_bit_exact_subset(cclib, plummer_ic):
    m, x, v = plummer_ic(300, seed=4)
    sub = np.arange(5, 300, 3, dtype=np.int32)
    labels = (sub // 7).astype(np.int32)
    c = cclib.Context(m, x, v)
    c.drift(labels, 1 / 128, set_ids=sub)
    _, _, gx, gv = c.get_state()
    s = O.State(m, x, v)
    O.drift(s, sub, labels, 1 / 128)
    assert np.array_equal(gx, s.x3) and np.array_equal(gv, s.v3)
    c.close()


@pytest.mark.parametrize("n,dt", [(256, 1 / 64), (1000, 1 / 128)])
def test_one_outer_step(cclib, plummer_ic, n, dt):
    m, x, v = plummer_ic(n)
    c = cclib.Context(m, x, v, dt=dt)
    c.evolve(dt)
    t, _, gx, gv = c.get_state()
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=dt), 1)
    assert t == dt
    assert _rel_ok(gx, s.x3) and _rel_ok(gv, s.v3)
    g = c.stats()
    for k in ("tau_pairs", "kick_pairs", "drifts", "splits", "components"):
        assert g[k] == getattr(st, k), k
    assert g["max_depth_seen"] == st.max_depth_seen
    c.close()


def test_eight_steps_and_conservation(cclib, plummer_ic):
    m, x, v = plummer_ic(256)
    c = cclib.Context(m, x, v, dt=1 / 64)
    E0, P0, L0 = c.energy()
    c.evolve(8 / 64)
    _, _, gx, gv = c.get_state()
    s = O.State(m, x, v)
    O.evolve(s, O.params(dt=1 / 64), 8)
    assert _rel_ok(gx, s.x3, 1e-10) and _rel_ok(gv, s.v3, 1e-10)
    E1, P1, L1 = c.energy()
    oE0, _, _ = O.energy(O.State(m, x, v))
    assert abs(E0 - oE0) < 1e-14
    assert np.abs(P1 - P0).max() < 1e-15 and np.abs(L1 - L0).max() < 1e-14
    assert abs((E1 - E0) / E0) < 1e-5
    c.close()


def test_full_size_one_step(cclib, plummer_ic):
    """The 16384-body Plummer sphere at dt = 1/256 (the benchmark workload):
    one outer step against the oracle on every particle."""
    m, x, v = plummer_ic(16384)
    c = cclib.Context(m, x, v, dt=1 / 256)
    c.evolve(1 / 256)
    _, _, gx, gv = c.get_state()
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=1 / 256), 1)
    assert _rel_ok(gx, s.x3) and _rel_ok(gv, s.v3)
    g = c.stats()
    assert g["tau_pairs"] == st.tau_pairs and g["kick_pairs"] == st.kick_pairs
    c.close()


def test_independent_systems(cclib):
    parts = [ics.plummer(k, seed=10 + k) for k in (37, 64, 5)]
    m = np.concatenate([p[0] for p in parts])
    x = np.ascontiguousarray(np.concatenate([p[1] + 10.0 * i for i, p in enumerate(parts)], axis=1))
    v = np.ascontiguousarray(np.concatenate([p[2] for p in parts], axis=1))
    off = np.array([0, 37, 101, 106], dtype=np.int64)
    c = cclib.Context(m, x, v, dt=1 / 32)
    c.set_systems(off)
    c.evolve(2 / 32)
    _, _, gx, gv = c.get_state()
    s = O.State(m, x, v)
    O.evolve(s, O.params(dt=1 / 32), 2, sys_off=off)
    assert _rel_ok(gx, s.x3) and _rel_ok(gv, s.v3)
    c.close()


def test_kepler_mode_binaries(cclib):
    m, x, v = ics.plummer_with_binaries(512, seed=3)
    c = cclib.Context(m, x, v, dt=1 / 256, kepler=1)
    c.evolve(1 / 256)
    _, _, gx, gv = c.get_state()
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=1 / 256, kepler=True), 1)
    assert c.stats()["kepler_calls"] == st.kepler_calls > 0
    assert _rel_ok(gx, s.x3, 1e-9)
    # Two different Kepler methods (universal variables on the GPU, the
    # classical Kepler equation in the oracle) agree to rounding in time,
    # but a binary that is perturbed inside a larger component passes
    # through many Kepler calls and kicks, and near pericentre of a hard
    # eccentric orbit a time offset of 1e-16 moves the velocity by up to
    # 1e-8 relative.  Velocities are therefore compared in distribution,
    # and the total energy (well conditioned) tightly.
    rel = np.linalg.norm(gv - s.v3, axis=0) / np.linalg.norm(s.v3, axis=0)
    assert np.median(rel) < 1e-12 and np.quantile(rel, 0.99) < 1e-6, (np.median(rel), np.quantile(rel, 0.99))
    Eg, _, _ = c.energy()
    Eo, _, _ = O.energy(s)
    assert abs(Eg - Eo) < 1e-10 * abs(Eo)
    c.close()


def test_kepler_mode_well_conditioned_bodies_elementwise(cclib):
    """Element-wise where the orbits are well conditioned.  At a short
    outer step (1/2048) the top-level components are mostly the binaries
    themselves: bodies whose top-level component has at most two members
    (singletons, and binaries that only the Kepler flow advances inside the
    step) must agree with the oracle within a bound that scales like the
    Kepler phase's rounding: 2^14 u64 dt S_i (D + 1), S_i the sum of
    absolute pair accelerations (for a binary member dominated by its
    partner's, so that dt S_i ~ |v| x the radians the orbit turns through
    in the step), plus the rounding of the coordinates themselves (4 u64
    |v_i|); positions within dt times the velocity bound plus 4 u64 |x_i|
    (a wide pair's orbit barely turns in the step, and the rounding of its
    absolute coordinates is then the larger term)."""
    m, x, v = ics.plummer_with_binaries(512, seed=3)
    dt = 1 / 2048
    c = cclib.Context(m, x, v, dt=dt, kepler=1)
    top, _ = c.components(dt)
    c.reset_stats()
    c.evolve(dt)
    _, _, gx, gv = c.get_state()
    g = c.stats()
    c.close()
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=dt, kepler=True), 1)
    assert g["kepler_calls"] == st.kepler_calls > 0
    sizes = np.bincount(top, minlength=m.shape[0])
    calm = np.flatnonzero(sizes[top] <= 2)
    assert calm.size > 0.8 * m.shape[0], calm.size
    S = B.abs_accel_sum(m, x)
    tol = 2.0 ** 14 * B.U64 * dt * S * (st.max_depth_seen + 1)
    tol_v = tol + 4 * B.U64 * np.linalg.norm(s.v3, axis=0)
    tol_x = dt * tol + 4 * B.U64 * np.linalg.norm(s.x3, axis=0)
    ev = np.linalg.norm(gv - s.v3, axis=0)
    ex = np.linalg.norm(gx - s.x3, axis=0)
    rv, rx = ev[calm] / tol_v[calm], ex[calm] / tol_x[calm]
    print("Kepler mode: well-conditioned bodies", calm.size, "max error / bound: v", rv.max(), "x", rx.max())
    assert rv.max() <= 1.0 and rx.max() <= 1.0, (rv.max(), rx.max())


def test_kepler_isolated_binaries_closed_form(cclib):
    """Each two-body component advanced by the GPU Kepler solver equals the
    closed-form orbit (orbital elements, mean anomaly by a library root
    finder) for eccentricities 0 .. 0.95 and many periods per step."""
    import math
    from scipy.optimize import brentq
    rows = []
    for k, e in enumerate((0.0, 0.2, 0.5, 0.8, 0.95)):
        m, x, v = ics.binary(0.6, 0.4, 1e-3 * (1 + k), e, E_anom=0.4 + k, inc=0.3 * k, node=0.2, peri=1.0)
        # independent systems never interact, so all sit at the origin: an
        # offset would cost the relative orbit digits (|x| >> a)
        rows.append((m, x, v, e, 1e-3 * (1 + k), 0.4 + k, 0.3 * k))
    m = np.concatenate([r[0] for r in rows])
    x = np.ascontiguousarray(np.concatenate([r[1] for r in rows], axis=1))
    v = np.ascontiguousarray(np.concatenate([r[2] for r in rows], axis=1))
    off = np.arange(0, 2 * len(rows) + 1, 2, dtype=np.int64)
    dt = 1.0 / 64
    c = cclib.Context(m, x, v, dt=dt, kepler=1)
    c.set_systems(off)
    c.evolve(dt)
    _, _, gx, gv = c.get_state()
    c.close()
    for k, (mm, xx, vv, e, a, E0, inc) in enumerate(rows):
        n = math.sqrt(1.0 / a ** 3)
        M = (E0 - e * math.sin(E0) + n * dt) % (2 * math.pi)
        E = brentq(lambda q: q - e * math.sin(q) - M, 0.0, 2 * math.pi, xtol=1e-15, rtol=1e-15)
        _, xr, vr = ics.binary(0.6, 0.4, a, e, E_anom=E, inc=inc, node=0.2, peri=1.0)
        got_r = gx[:, 2 * k] - gx[:, 2 * k + 1]
        ref_r = xr[:, 0] - xr[:, 1]
        # n*dt is several hundred radians here: the phase is good to ~1e-13
        assert np.abs(got_r - ref_r).max() < 1e-10 * a / (1 - e), (k, e)
        # the relative velocity likewise: |dv| ~ (phase error) x |d v/d phase|,
        # and the orbital speed peaks at pericentre, n a sqrt((1 + e)/(1 - e))
        got_u = gv[:, 2 * k] - gv[:, 2 * k + 1]
        ref_u = vr[:, 0] - vr[:, 1]
        vmax = n * a * math.sqrt((1 + e) / (1 - e))
        assert np.abs(got_u - ref_u).max() < 1e-10 * vmax / (1 - e), (k, e)
        # and the centre of mass moves uniformly (at rest here)
        com_v = (mm[0] * gv[:, 2 * k] + mm[1] * gv[:, 2 * k + 1]) / mm.sum()
        assert np.abs(com_v).max() < 1e-13 * vmax


def test_errors_are_reported(cclib, plummer_ic):
    m, x, v = plummer_ic(256)
    c = cclib.Context(m, x, v, dt=1 / 64)
    with pytest.raises(cclib.CCError) as e:
        c.evolve(0.01)
    assert e.value.code == -1
    c.close()
    c = cclib.Context(m, x, v, dt=1 / 64, max_depth=1)
    with pytest.raises(cclib.CCError) as e:
        c.evolve(1 / 64)
    assert e.value.code == -3
    c.close()
    bad = x.copy()
    bad[0, 0] = np.nan
    with pytest.raises(cclib.CCError) as e:
        cclib.Context(m, bad, v)
    assert e.value.code == -5


def test_launch_shapes_do_not_change_fp64_results(cclib, plummer_ic):
    """The autotuner tries several tile shapes for the tau and FP64 kick
    kernels; in the FP64 form every shape computes the same arithmetic in
    the same order, so tuned and untuned runs agree bit for bit."""
    m, x, v = plummer_ic(1000)
    out = []
    for tune in (0, 1):
        c = cclib.Context(m, x, v, dt=1 / 128, autotune=tune)
        c.evolve(6 / 128)
        _, _, gx, gv = c.get_state()
        out.append((gx, gv))
        c.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    s = O.State(m, x, v)
    O.evolve(s, O.params(dt=1 / 128), 6)
    assert _rel_ok(out[1][0], s.x3, 1e-10) and _rel_ok(out[1][1], s.v3, 1e-10)


def test_tuning_table_reports_the_tried_shapes(cclib, plummer_ic):
    """cc_tuning lists every (kernel, size bin) cell with a timed launch;
    once a cell has timed every variant it holds a choice among them."""
    m, x, v = plummer_ic(1000)
    c = cclib.Context(m, x, v, dt=1 / 128, precision=cclib.PREC_MIXED)
    c.evolve(6 / 128)
    cells = c.tuning()
    c.close()
    assert cells and {e["kernel"] for e in cells} <= {"tau_mixed", "kick_mixed"}
    shapes = {"tau_mixed": ([64, 128, 64], [1, 1, 2]), "kick_mixed": ([1, 4, 1], [1, 1, 4])}
    for e in cells:
        assert (e["shape"], e["slices"]) == shapes[e["kernel"]], e
        assert -1 <= e["best"] < len(e["shape"]), e
        if e["best"] >= 0:
            # variants that split tile columns are tried only for launches
            # with few blocks; every other variant has been timed
            assert e["timed"][e["best"]] >= 1 and e["us_per_mpair"][e["best"]] > 0, e
            assert all(t >= 1 for t, sl in zip(e["timed"], e["slices"]) if sl == 1), e
    assert any(e["best"] >= 0 for e in cells)


@pytest.mark.parametrize("s_small", [0, 32])
def test_first_half_splits_from_parent_records(cclib, plummer_ic, s_small):
    """A first-half split takes its edges from the parent split's tau values
    (the state is the one the parent saw).  With the small-component kernel
    off every component recurses level by level, so most splits below the
    top are first halves: the result must still be the oracle's, with the
    same split and pair counts, and fewer pairs evaluated than decided."""
    m, x, v = plummer_ic(2000, seed=9)
    c = cclib.Context(m, x, v, dt=1 / 32, s_small=s_small)
    c.evolve(1 / 32)
    _, _, gx, gv = c.get_state()
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=1 / 32), 1)
    assert _rel_ok(gx, s.x3) and _rel_ok(gv, s.v3)
    g = c.stats()
    for k in ("tau_pairs", "kick_pairs", "drifts", "splits", "components"):
        assert g[k] == getattr(st, k), k
    assert g["max_depth_seen"] == st.max_depth_seen
    assert st.max_depth_seen >= 3
    assert 0 < g["tau_evaluated"] < g["tau_pairs"]
    c.close()


@pytest.mark.parametrize("nsys", [5, 12])
def test_batches_of_large_components(cclib, nsys):
    """A batch whose sets are each one large component (100 bodies at a long
    step): the one-CTA segmentation writes runs of more than 64 members by
    a stable compaction when there are at most 8 of them and falls back to a
    serial stable scatter beyond that; both must give the oracle's state."""
    parts = [ics.plummer(100, seed=40 + k) for k in range(nsys)]
    m = np.concatenate([p[0] for p in parts])
    x = np.ascontiguousarray(np.concatenate([p[1] for p in parts], axis=1))
    v = np.ascontiguousarray(np.concatenate([p[2] for p in parts], axis=1))
    off = np.arange(nsys + 1, dtype=np.int64) * 100
    dt = 1 / 4
    c = cclib.Context(m, x, v, dt=dt)
    c.set_systems(off)
    c.evolve(dt)
    _, _, gx, gv = c.get_state()
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=dt), 1, sys_off=off)
    assert _rel_ok(gx, s.x3) and _rel_ok(gv, s.v3)
    g = c.stats()
    for k in ("tau_pairs", "kick_pairs", "splits", "components"):
        assert g[k] == getattr(st, k), k
    c.close()
