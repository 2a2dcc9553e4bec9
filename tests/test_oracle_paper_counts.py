"""The oracle against the operation counts the paper prints for its
smoothed Plummer test (Sec. 3.1, the figure comparing BLOCK, HOLD and CC):
one global step of the CC integrator on a softened 1024-body Plummer sphere
performs about 1.1e9 kick, 6.6e8 time-step and 5.0e6 drift evaluations.
The counts follow from the whole method at once: the scale of tau (in a
virialised cluster the flyby time eta r/|dv| sets it for most pairs; a flyby
time 1.5x too long moves the time-step count by 31 %), the lazy
breadth-first component search (Sec. 2.3), the recursion with the threshold
halved and the drift of the rest set only.  (The free-fall term and the
time-derivative correction barely move these counts; the closed-form and
finite-difference tests of tau pin them.)  A realisation of the initial
conditions moves the counts by a few per cent: seeds 1-3 give 6.5-6.7e8
time-step evaluations.  Runs the oracle for ~20 s."""
import json
import os

from oracle import oracle as O
from paper_1407_7105_gb300 import ics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_plummer1024_first_step.json")


def test_first_global_step_counts_match_the_paper():
    g = json.load(open(GOLDEN))["cc_counts_first_global_step"]
    m, x, v = ics.plummer(1024, seed=1)
    s = O.State(m, x, v)
    st = O.evolve(s, O.params(eta=0.01, eps=1.0 / 256, dt=700.0 / 512), 1)
    tau = st.tau_evals
    kick = 2 * st.kick_pairs  # each unordered cross pair kicks both bodies
    drift = st.drifts
    assert abs(tau / g["time_step_evaluations"] - 1) < 0.12, tau
    assert abs(drift / g["drift_evaluations"] - 1) < 0.12, drift
    assert abs(kick / g["kick_evaluations"] - 1) < 0.15, kick
