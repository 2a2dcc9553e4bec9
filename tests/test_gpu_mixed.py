"""GPU checks of the mixed-precision form (CC_PREC_MIXED).

The certified FP32 tau pre-filter must leave the edge predicate exactly
the FP64 one: labels equal the oracle's bit for bit, including thresholds
placed within 1e-7 .. 1e-3 (relative) of individual pair time steps.  The
FP32 kick is judged by its error against the FP64 kick on the same state.
"""
import numpy as np
import pytest

import _bounds as B
from oracle import oracle as O
from paper_1407_7105_gb300 import ics

pytestmark = pytest.mark.gpu


def _mixed(cclib, m, x, v, **kw):
    return cclib.Context(m, x, v, precision=cclib.PREC_MIXED, **kw)


@pytest.mark.parametrize("n", [1000, 16384])
def test_mixed_components_equal_fp64(cclib, plummer_ic, n):
    m, x, v = plummer_ic(n)
    s = O.State(m, x, v)
    c = _mixed(cclib, m, x, v)
    for h in (1 / 64, 1 / 256, 1 / 2048):
        if n > 2000 and h != 1 / 256:
            continue
        lab, k = c.components(h)
        olab, ok = O.components(s, O.params(), h)
        assert k == ok and np.array_equal(lab, olab), h
    st = c.stats()
    assert st["tau_fp64"] < 1e-3 * st["tau_pairs"] + 100, st
    c.close()


@pytest.mark.parametrize("rel", [1e-7, -1e-7, 1e-5, -1e-5, 1e-3, -1e-3, 0.0])
def test_mixed_threshold_at_pair_tau(cclib, plummer_ic, rel):
    """Thresholds a hair above / below / at individual tau(i,j): the
    pre-filter must hand every such pair to the FP64 predicate."""
    m, x, v = plummer_ic(300, seed=9)
    s = O.State(m, x, v)
    p = O.params()
    T = O.tau_matrix(s, p)
    vals = np.sort(T[np.triu_indices(300, 1)])
    c = _mixed(cclib, m, x, v)
    for q in (0.001, 0.01, 0.1, 0.5):
        h = float(vals[int(q * (vals.size - 1))]) * (1.0 + rel)
        lab, k = c.components(h)
        olab, ok = O.components(s, p, h)
        assert k == ok and np.array_equal(lab, olab), (q, rel)
    c.close()


def test_mixed_kick_error(cclib, plummer_ic):
    m, x, v = plummer_ic(4096, seed=3)
    rng = np.random.default_rng(1)
    labels = np.arange(4096, dtype=np.int32)
    labels[rng.choice(4096, 600, replace=False)] = 7  # one 600-member group
    h = 1 / 256
    c = _mixed(cclib, m, x, v)
    c.kick(labels, h)
    _, _, _, gv = c.get_state()
    c.close()
    s = O.State(m, x, v)
    O.kick(s, O.params(), np.arange(4096), labels, h)
    da_ref = (s.v3 - v) / h
    da_gpu = (gv - v) / h
    err = np.linalg.norm(da_gpu - da_ref, axis=0) / np.linalg.norm(da_ref, axis=0)
    assert np.median(err) < 2e-7 and err.max() < 1e-5, (np.median(err), err.max())
    # per body: |da_i| <= 32 u S_i (the FP32 error model of the pair terms
    # and their grouped, compensated sum; one kick, no recursion)
    S_cross = B.abs_accel_sum(m, x, labels=labels)
    abs_err = np.linalg.norm(da_gpu - da_ref, axis=0)
    ratio = abs_err / (B.K_MIXED * B.U32 * S_cross)
    assert ratio.max() <= 1.0, (int(np.argmax(ratio)), float(ratio.max()))


def test_mixed_energy_matches_fp64(cclib, plummer_ic):
    m, x, v = plummer_ic(1024, seed=5)
    out = {}
    for name, prec in (("fp64", cclib.PREC_FP64), ("mixed", cclib.PREC_MIXED)):
        c = cclib.Context(m, x, v, dt=1 / 128, precision=prec)
        E0, P0, _ = c.energy()
        c.evolve(16 / 128)
        E1, P1, _ = c.energy()
        out[name] = ((E1 - E0) / abs(E0), np.abs(P1 - P0).max())
        c.close()
    assert abs(out["mixed"][0]) < 1e-6 and abs(out["fp64"][0]) < 1e-6, out
    assert abs(out["mixed"][0] - out["fp64"][0]) < 1e-7, out
    # FP32 pair forces are not exactly antisymmetric: momentum is kept to
    # the FP32 rounding of the forces, not to FP64 machine precision
    assert out["fp64"][1] < 1e-15 and out["mixed"][1] < 1e-10, out


def test_mixed_one_step_close_to_oracle(cclib, plummer_ic):
    m, x, v = plummer_ic(16384)
    c = _mixed(cclib, m, x, v, dt=1 / 256, near_tol=1e-6)
    c.evolve(1 / 256)
    _, _, gx, gv = c.get_state()
    pairs, _, _ = c.near_pairs()
    c.close()
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(dt=1 / 256), 1)
    dv = np.linalg.norm(gv - s.v3, axis=0) / np.linalg.norm(s.v3, axis=0)
    dx = np.linalg.norm(gx - s.x3, axis=0) / np.linalg.norm(s.x3, axis=0)
    assert np.median(dv) < 1e-8 and np.median(dx) < 1e-9, (np.median(dv), np.median(dx))
    # every body, not only the median: the per-body FP32 error bound
    S = B.abs_accel_sum(m, x)
    ex = B.near_bodies(pairs)
    wv, _ = B.check_velocity_bound(gv, s.v3, S, 1 / 256, st.max_depth_seen, exempt=ex, what="v")
    wx, _ = B.check_velocity_bound(gx, s.x3, S / 256, 1 / 256, st.max_depth_seen, exempt=ex, what="x")
    print("mixed 16384 one step: max error / bound: v", wv, "x", wx, "exempt", ex.size)


def test_mixed_spatial_order_close_to_fp64(cclib, plummer_ic):
    """A single system of >= 2048 bodies runs the mixed form with level 0
    packed in a Morton order of the positions, renewed every 8 outer steps
    (the group certificates of the tau kernel need groups that are compact
    in space): 10 steps stay close to the FP64 form, which keeps id order,
    and every particle comes back."""
    m, x, v = plummer_ic(4096, seed=6)
    out = {}
    pairs = []
    for name, prec in (("fp64", cclib.PREC_FP64), ("mixed", cclib.PREC_MIXED)):
        c = cclib.Context(m, x, v, dt=1 / 256, precision=prec, near_tol=1e-6)
        E0, _, _ = c.energy()
        # one step per call, so that every step's near-threshold pairs are read
        for k in range(10):
            c.evolve((k + 1) / 256)
            pairs.append(c.near_pairs()[0])
        E1, _, _ = c.energy()
        _, gm, gx, gv = c.get_state()
        out[name] = (gm, gx, gv, (E1 - E0) / abs(E0), c.stats())
        c.close()
    gm, gx, gv, dE, st = out["mixed"]
    assert np.array_equal(gm, m) and np.all(np.isfinite(gx)) and np.all(np.isfinite(gv))
    dv = np.linalg.norm(gv - out["fp64"][2], axis=0) / np.linalg.norm(out["fp64"][2], axis=0)
    assert np.median(dv) < 1e-7, np.median(dv)
    S = B.abs_accel_sum(m, x)
    ex = B.near_bodies(np.concatenate(pairs)) if pairs else ()
    wv, _ = B.check_velocity_bound(gv, out["fp64"][2], S, 1 / 256, st["max_depth_seen"], steps=10, exempt=ex)
    print("mixed vs FP64, 10 steps: max error / bound", wv, "exempt", len(ex))
    assert abs(dE) < 1e-6 and abs(dE - out["fp64"][3]) < 1e-7, (dE, out["fp64"][3])
    assert abs(st["splits"] - out["fp64"][4]["splits"]) <= 0.01 * out["fp64"][4]["splits"]
