"""The oracle's parallel row loops (OpenMP) change no result: components,
counters and the state after outer steps are bit-identical for one thread
and for all host threads (the loops only spread independent rows; each
row's arithmetic and order are the serial ones)."""
import numpy as np

from oracle import oracle as O
from paper_1407_7105_gb300 import ics


def test_threads_give_bit_identical_results():
    m, x, v = ics.plummer(1500, seed=11)
    out = []
    for nt in (1, max(2, O.threads(0))):
        O.threads(nt)
        s = O.State(m, x, v)
        lab, k = O.components(s, O.params(), 1 / 128)
        st = O.evolve(s, O.params(dt=1 / 64), 2)
        out.append((lab, k, st.as_dict(), s.x3.copy(), s.v3.copy()))
    O.threads(0)
    a, b = out
    assert np.array_equal(a[0], b[0]) and a[1] == b[1] and a[2] == b[2]
    assert np.array_equal(a[3], b[3]) and np.array_equal(a[4], b[4])
