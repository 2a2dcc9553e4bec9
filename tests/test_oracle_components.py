"""Pins of the oracle's split_cc (Sec. 2.2-2.3): BFS connected components of
the time-step graph, labels = smallest id of each component.

The BFS result is checked against an independent library flood fill
(networkx) on the all-pairs edge list, against hand-built graphs whose
partition follows from geometry, and against the paper's special cases:
all interactions below the threshold give one component found with n-1
tau evaluations (Sec. 2.3); a threshold below every tau gives only the
rest set.
"""
import json
import math
import os

import networkx as nx
import numpy as np
import pytest

from oracle import oracle as O
from paper_1407_7105_gb300 import ics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _flood_fill_labels(n, edge_list, set_ids):
    g = nx.Graph()
    g.add_nodes_from(int(i) for i in set_ids)
    g.add_edges_from((int(a), int(b)) for a, b in edge_list)
    lab = {}
    for comp in nx.connected_components(g):
        mn = min(comp)
        for v in comp:
            lab[v] = mn
    return np.array([lab[int(i)] for i in set_ids], dtype=np.int32)


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("hfac", [0.3, 1.0, 3.0])
def test_bfs_matches_flood_fill(seed, hfac):
    m, x, v = ics.plummer(40, seed=seed)
    s = O.State(m, x, v)
    p = O.params(eta=0.03)
    T = O.tau_matrix(s, p)
    h = hfac * float(np.median(T[np.isfinite(T)])) * 0.05
    E, _ = O.edges(s, p, h)
    # the edge list is exactly the pairs with tau < h
    iu = np.triu_indices(40, 1)
    want = {(int(a), int(b)) for a, b in zip(*iu) if T[a, b] < h}
    assert {tuple(e) for e in E.tolist()} == want
    lab, k = O.components(s, p, h)
    ref = _flood_fill_labels(40, E, np.arange(40))
    assert np.array_equal(lab, ref)
    sizes = np.unique(lab, return_counts=True)[1]
    assert k == int((sizes >= 2).sum())


def test_subset_labels_use_set_ids():
    m, x, v = ics.plummer(30, seed=3)
    s = O.State(m, x, v)
    p = O.params()
    sub = np.array([1, 4, 5, 9, 12, 13, 20, 27], dtype=np.int32)
    T = O.tau_matrix(s, p, sub)
    h = float(np.sort(T[np.isfinite(T)])[len(sub)])
    E, _ = O.edges(s, p, h, set_ids=sub)
    lab, _ = O.components(s, p, h, set_ids=sub)
    assert np.array_equal(lab, _flood_fill_labels(30, E, sub))
    assert set(lab.tolist()) <= set(sub.tolist())


def _rest_line(n, spacing, mass=1.0):
    m = np.full(n, mass)
    x = np.zeros((3, n))
    x[0] = spacing * np.arange(n)
    return O.State(m, x, np.zeros((3, n)))


def test_chain_is_one_component():
    # pairs at rest: edge iff eta sqrt(r^3 / 2) < h.  With h between the
    # nearest- and next-nearest-neighbour thresholds only adjacent pairs
    # are edges, and the chain is one component.
    p = O.params(eta=0.03)
    s = _rest_line(9, 1.0)
    t1 = 0.03 * math.sqrt(1.0 / 2.0)
    t2 = 0.03 * math.sqrt(8.0 / 2.0)
    h = 0.5 * (t1 + t2)
    E, _ = O.edges(s, p, h)
    assert E.tolist() == [[i, i + 1] for i in range(8)]
    lab, k = O.components(s, p, h)
    assert k == 1 and (lab == 0).all()


def test_all_connected_single_sweep():
    """Sec. 2.3: with every interaction below the threshold the BFS assigns
    all particles from the first particle: exactly n - 1 tau evaluations."""
    m, x, v = ics.plummer(50, seed=7)
    s = O.State(m, x, v)
    p = O.params()
    st = O.Stats()
    lab, k = O.components(s, p, 1e6, stats=st)
    assert k == 1 and (lab == 0).all()
    assert st.tau_evals == 49
    assert st.tau_pairs == 50 * 49 // 2


def test_below_every_tau_is_rest_only():
    m, x, v = ics.plummer(50, seed=7)
    s = O.State(m, x, v)
    p = O.params()
    lab, k = O.components(s, p, 1e-12)
    assert k == 0 and np.array_equal(lab, np.arange(50))


def test_golden_partitions():
    """Hand-built systems whose partition follows from the geometry."""
    with open(os.path.join(GOLDEN, "components_handbuilt.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        m = np.array(c["m"], float)
        x = np.array(c["x"], float).T.copy()
        v = np.array(c["v"], float).T.copy()
        s = O.State(m, x, v)
        p = O.params(eta=c["eta"])
        lab, k = O.components(s, p, c["h"])
        assert lab.tolist() == c["labels"], c["name"]
        assert k == c["ncomp"], c["name"]
