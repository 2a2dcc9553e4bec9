"""GPU parity on the other workload families of the hot path: box-fractal
clusters with a Salpeter mass spectrum, and batches of independent small
systems (hierarchical triples and Plummer clumps), at sizes the oracle
finishes in seconds."""
import numpy as np
import pytest

import _bounds as B
from oracle import oracle as O
from paper_1407_7105_gb300 import ics

pytestmark = pytest.mark.gpu


def _rel_ok(a, b, rtol=1e-12):
    scale = np.abs(b).max()
    return np.all(np.abs(a - b) <= rtol * np.abs(b) + 1e-15 * scale)


@pytest.mark.parametrize("seed", [1, 2])
def test_fractal_components_and_step_fp64(cclib, seed):
    m, x, v = ics.box_fractal(1200, seed=seed)
    c = cclib.Context(m, x, v, dt=1 / 256)
    lab, k = c.components(1 / 256)
    s = O.State(m, x, v)
    olab, ok = O.components(s, O.params(dt=1 / 256), 1 / 256)
    assert k == ok and np.array_equal(lab, olab)
    c.reset_stats()
    c.evolve(1 / 256)
    _, _, gx, gv = c.get_state()
    st = O.evolve(s, O.params(dt=1 / 256), 1)
    assert _rel_ok(gx, s.x3) and _rel_ok(gv, s.v3)
    g = c.stats()
    assert g["tau_pairs"] == st.tau_pairs and g["kick_pairs"] == st.kick_pairs and g["splits"] == st.splits
    c.close()


def test_fractal_mixed_close_to_oracle(cclib):
    m, x, v = ics.box_fractal(1200, seed=3)
    c = cclib.Context(m, x, v, dt=1 / 256, precision=cclib.PREC_MIXED, near_tol=1e-6)
    pairs = []
    for k in range(2):
        c.evolve((k + 1) / 256)
        pairs.append(c.near_pairs()[0])
    _, _, gx, gv = c.get_state()
    c.close()
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=1 / 256), 2)
    dv = np.linalg.norm(gv - s.v3, axis=0) / np.linalg.norm(s.v3, axis=0)
    assert np.median(dv) < 1e-8
    S = B.abs_accel_sum(m, x)
    ex = B.near_bodies(np.concatenate(pairs))
    w, _ = B.check_velocity_bound(gv, s.v3, S, 1 / 256, st.max_depth_seen, steps=2, exempt=ex)
    print("fractal mixed: max error / bound", w, "exempt", ex.size)


def _systems(nsys, seed):
    m, x, v, off = ics.small_systems(nsys, seed=seed, n_max=96)
    return m, x, v, off


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_small_systems_batch(cclib, prec):
    m, x, v, off = _systems(40, seed=5)
    p = cclib.PREC_FP64 if prec == "fp64" else cclib.PREC_MIXED
    c = cclib.Context(m, x, v, dt=1 / 64, precision=p, near_tol=1e-6)
    c.set_systems(off)
    pairs = []
    for k in range(2):
        c.evolve((k + 1) / 64)
        pairs.append(c.near_pairs()[0])
    _, _, gx, gv = c.get_state()
    g = c.stats()
    c.close()
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=1 / 64), 2, sys_off=off)
    if prec == "fp64":
        assert _rel_ok(gx, s.x3) and _rel_ok(gv, s.v3)
        assert g["tau_pairs"] == st.tau_pairs and g["kick_pairs"] == st.kick_pairs
        assert g["max_depth_seen"] == st.max_depth_seen
    else:
        dv = np.linalg.norm(gv - s.v3, axis=0) / np.linalg.norm(s.v3, axis=0)
        assert np.median(dv) < 1e-7, np.median(dv)
        S = B.abs_accel_sum(m, x, groups=B.system_index(m.shape[0], off))
        ex = B.near_bodies(np.concatenate(pairs))
        w, _ = B.check_velocity_bound(gv, s.v3, S, 1 / 64, st.max_depth_seen, steps=2, exempt=ex)
        print("systems mixed: max error / bound", w, "exempt", ex.size)
        # every system keeps its own momentum (they never interact)
        for a, b in zip(off[:-1], off[1:]):
            P = (m[a:b] * gv[:, a:b]).sum(axis=1)
            assert np.abs(P).max() < 1e-8


def test_small_systems_without_small_kernel_identical(cclib):
    """The persistent small-component kernel and the level-by-level path run
    the same arithmetic: with it switched off the FP64 result is the same
    bit for bit."""
    m, x, v, off = _systems(24, seed=6)
    out = []
    for s_small in (32, 0):
        c = cclib.Context(m, x, v, dt=1 / 64, s_small=s_small)
        c.set_systems(off)
        c.evolve(1 / 64)
        _, _, gx, gv = c.get_state()
        out.append((gx, gv))
        c.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_systems_energy_is_the_sum_of_the_systems(cclib):
    """With independent systems declared, cc_energy sums each system's own
    Hamiltonian (the systems overlap in space but never interact); against
    the oracle's energy of each system separately, and conserved over a
    step to the integrator's accuracy."""
    m, x, v, off = _systems(40, seed=5)
    c = cclib.Context(m, x, v, dt=1 / 64)
    c.set_systems(off)
    E, P, L = c.energy()
    ref = 0.0
    for a, b in zip(off[:-1], off[1:]):
        e, _, _ = O.energy(O.State(m[a:b], x[:, a:b], v[:, a:b]))
        ref += e
    assert abs(E - ref) < 1e-12 * abs(ref), (E, ref)
    c.evolve(2 / 64)
    E1, _, _ = c.energy()
    c.close()
    s = O.State(m, x, v)
    O.evolve(s, O.params(dt=1 / 64), 2, sys_off=off)
    ref1 = 0.0
    for a, b in zip(off[:-1], off[1:]):
        e, _, _ = O.energy(O.State(s.m[a:b], s.x3[:, a:b], s.v3[:, a:b]))
        ref1 += e
    assert abs(E1 - ref1) < 1e-10 * abs(ref1), (E1, ref1)
    assert abs((E1 - E) / E) < 1e-4
