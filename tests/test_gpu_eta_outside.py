"""The literal placement of eta in Eq. (tauij) (eta multiplying the min,
eta_outside = 1) on the GPU, against the oracle with the same reading:
component labels at thresholds placed among the pair time steps, in both
forms, and one outer step (the FP64 form bit for bit, the mixed form within
its force error)."""
import numpy as np
import pytest

import _bounds as B
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
def test_components_and_step_with_eta_outside(cclib, plummer_ic, prec_name):
    prec = cclib.PREC_FP64 if prec_name == "fp64" else cclib.PREC_MIXED
    m, x, v = plummer_ic(600, seed=7)
    p = O.params(eta=0.03, dt=1 / 128, eta_outside=True)
    s = O.State(m, x, v)
    T = O.tau_matrix(s, p)
    vals = np.sort(T[np.triu_indices(600, 1)])
    c = cclib.Context(m, x, v, dt=1 / 128, eta=0.03, eta_outside=1, precision=prec, near_tol=1e-6)
    for q in (0.002, 0.02, 0.2):
        h = float(vals[int(q * (vals.size - 1))]) * (1.0 + 1e-9)
        lab, k = c.components(h)
        olab, ok = O.components(s, p, h)
        assert k == ok and np.array_equal(lab, olab), (prec_name, q)
    c.reset_stats()  # the splits of the component queries above are not the step's
    c.evolve(1 / 128)
    _, _, gx, gv = c.get_state()
    st = c.stats()
    pairs, _, _ = c.near_pairs()
    c.close()
    ost = O.evolve(s, p, 1)
    assert st["splits"] == ost.splits and st["kick_pairs"] == ost.kick_pairs
    if prec == cclib.PREC_FP64:
        assert np.array_equal(gx, s.x3) and np.array_equal(gv, s.v3)
    else:
        dv = np.linalg.norm(gv - s.v3, axis=0) / np.linalg.norm(s.v3, axis=0)
        assert np.median(dv) < 1e-8, np.median(dv)
        w, _ = B.check_velocity_bound(gv, s.v3, B.abs_accel_sum(m, x), 1 / 128, ost.max_depth_seen,
                                      exempt=B.near_bodies(pairs))
        print("eta outside mixed: max error / bound", w)
