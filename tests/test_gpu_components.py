"""GPU parity of the time-step graph and of split_cc (Sec. 2.2-2.3): edge
sets and component labels from libcc.so must equal the oracle's bit for
bit (same FP64 tau predicate, same operation order)."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _ctx(cclib, m, x, v, **kw):
    return cclib.Context(m, x, v, **kw)


@pytest.mark.parametrize("n", [256, 1000])
@pytest.mark.parametrize("hfac", [1.0, 0.25, 1 / 16])
def test_components_match_oracle(cclib, plummer_ic, n, hfac):
    m, x, v = plummer_ic(n)
    h = hfac / 64
    c = _ctx(cclib, m, x, v)
    lab, k = c.components(h)
    s = O.State(m, x, v)
    olab, ok = O.components(s, O.params(), h)
    assert k == ok
    assert np.array_equal(lab, olab)
    c.close()


def test_components_subset_and_device_pointers(cclib, plummer_ic):
    import torch
    m, x, v = plummer_ic(1000)
    rng = np.random.default_rng(3)
    sub = np.sort(rng.choice(1000, 333, replace=False)).astype(np.int32)
    c = _ctx(cclib, torch.tensor(m, device="cuda"), torch.tensor(x, device="cuda"), torch.tensor(v, device="cuda"))
    dsub = torch.tensor(sub, device="cuda")
    dlab = torch.zeros(333, dtype=torch.int32, device="cuda")
    _, k = c.components(1 / 128, set_ids=dsub, labels_out=dlab)
    olab, ok = O.components(O.State(m, x, v), O.params(), 1 / 128, set_ids=sub)
    assert k == ok and np.array_equal(dlab.cpu().numpy(), olab)
    c.close()


@pytest.mark.parametrize("n", [256, 777])
def test_timestep_graph_matches_oracle(cclib, plummer_ic, n):
    m, x, v = plummer_ic(n, seed=2)
    c = _ctx(cclib, m, x, v)
    h = 1 / 100
    E, ne, nn = c.timestep_graph(h)
    oE, onn = O.edges(O.State(m, x, v), O.params(), h)
    assert ne == oE.shape[0] and nn == onn
    assert np.array_equal(E, oE)
    # capacity shortfall reports the true count and CC_E_CAPACITY
    if ne > 2:
        E2, ne2, _ = c.timestep_graph(h, cap=2)
        assert ne2 == ne and E2.shape[0] == 2
    c.close()


def test_near_threshold_pairs_logged(cclib, plummer_ic):
    m, x, v = plummer_ic(256)
    s = O.State(m, x, v)
    p = O.params()
    tau = O.tau_ids(s, p, 3, 17)
    c = _ctx(cclib, m, x, v)
    _, _, nn = c.timestep_graph(tau)
    pairs, taus, n = c.near_pairs()
    assert nn >= 1 and n == nn
    assert [3, 17] in pairs.tolist()
    assert taus[pairs.tolist().index([3, 17])] == tau
    c.close()


def test_edge_cases(cclib, plummer_ic):
    m, x, v = plummer_ic(256)
    c = _ctx(cclib, m, x, v)
    one = np.array([5], dtype=np.int32)
    lab, k = c.components(1.0, set_ids=one)
    assert k == 0 and lab.tolist() == [5]
    lab, k = c.components(1e6)
    assert k == 1 and (lab == 0).all()
    lab, k = c.components(1e-12)
    assert k == 0 and np.array_equal(lab, np.arange(256))
    bad = np.array([4, 2], dtype=np.int32)
    with pytest.raises(cclib.CCError) as e:
        c.components(1.0, set_ids=bad)
    assert e.value.code == -1
    c.close()


def test_components_full_size(cclib, plummer_ic):
    """Top-level split of the 16384-body Plummer sphere at h = 1/256."""
    m, x, v = plummer_ic(16384)
    c = _ctx(cclib, m, x, v)
    lab, k = c.components(1 / 256)
    olab, ok = O.components(O.State(m, x, v), O.params(), 1 / 256)
    assert k == ok and np.array_equal(lab, olab)
    c.close()
