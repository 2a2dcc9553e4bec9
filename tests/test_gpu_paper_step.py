"""The first global step of the paper's smoothed Plummer test (Sec. 3.1:
1024 equal-mass bodies, eps = 1/256, eta = 0.01, one step of 700/512) on
the GPU: both forms split, kick and drift exactly as the oracle does (the
same counts of splits, kick pairs and drifts, 16 levels deep), and the FP64
form ends in the oracle's state (the oracle's counts are pinned to the
paper's printed ones in test_oracle_paper_counts.py)."""
import numpy as np
import pytest

import _bounds as B
from oracle import oracle as O
from paper_1407_7105_gb300 import ics

pytestmark = pytest.mark.gpu


def test_paper_first_global_step_counts_and_state(cclib):
    m, x, v = ics.plummer(1024, seed=1)
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(eta=0.01, eps=1.0 / 256, dt=700.0 / 512), 1)
    for prec in (cclib.PREC_FP64, cclib.PREC_MIXED):
        c = cclib.Context(m, x, v, dt=700.0 / 512, eta=0.01, eps=1.0 / 256, precision=prec, near_tol=1e-6)
        c.evolve(700.0 / 512)
        g = c.stats()
        _, _, gx, gv = c.get_state()
        pairs, _, _ = c.near_pairs()
        c.close()
        assert g["splits"] == st.splits and g["kick_pairs"] == st.kick_pairs and g["drifts"] == st.drifts, (prec, g)
        assert g["tau_pairs"] == st.tau_pairs and g["max_depth_seen"] == st.max_depth_seen
        if prec == cclib.PREC_FP64:
            assert np.array_equal(gx, s.x3) and np.array_equal(gv, s.v3)
        else:
            dv = np.linalg.norm(gv - s.v3, axis=0) / np.linalg.norm(s.v3, axis=0)
            assert np.median(dv) < 1e-7, np.median(dv)
            S = B.abs_accel_sum(m, x, eps=1.0 / 256)
            w, _ = B.check_velocity_bound(gv, s.v3, S, 700.0 / 512, st.max_depth_seen, exempt=B.near_bodies(pairs))
            print("paper step mixed: max error / bound", w)
