"""Failure detection without a GPU fault: every device wait and retry loop
of the library is bounded, and running out of either comes back to the
caller as CC_E_TIMEOUT with the context's GPU state still usable.

The test hooks of cc_params.fault_test make the bound run out on purpose:
1 = the tau kernels announce their tile copy on the mbarrier but never
issue it (a flag that nothing sets), so the wait gives up after ~2^20
cycles; 2 = the union-find hook gives up at once.  Both forms' splits run
the certified tau kernel; cc_timestep_graph runs the FP64 one.  Nothing faults, traps
or hangs: each kernel records the error word and returns, and the next
call (on the same device) gives the oracle's result."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu

CC_E_TIMEOUT = -4


@pytest.mark.parametrize("hook", [1, 2])
def test_bounded_wait_and_retry_report_timeout(cclib, plummer_ic, hook):
    m, x, v = plummer_ic(1000)
    h = 1 / 128
    for call in ("components", "timestep_graph"):
        c = cclib.Context(m, x, v, fault_test=hook)
        with pytest.raises(cclib.CCError) as e:
            getattr(c, call)(h)
        assert e.value.code == CC_E_TIMEOUT, (call, e.value)
        c.close()
    # the GPU and the library carry on: a fresh context gives the oracle's labels
    c = cclib.Context(m, x, v)
    lab, k = c.components(h)
    c.close()
    olab, ok = O.components(O.State(m, x, v), O.params(), h)
    assert k == ok and np.array_equal(lab, olab)


def test_fault_test_values_are_checked(cclib, plummer_ic):
    m, x, v = plummer_ic(64)
    with pytest.raises(cclib.CCError) as e:
        cclib.Context(m, x, v, fault_test=3)
    assert e.value.code == -1
    with pytest.raises(cclib.CCError) as e:
        cclib.Context(m, x, v, edge_rec_max=-1)
    assert e.value.code == -1
