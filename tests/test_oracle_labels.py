"""Pins of the oracle's Hoshen-Kopelman cluster labelling (Sec. 3,
nearest-neighbour connectivity) against a library connected-components
routine on the periodic and the open square lattice, and hand-built masks."""
import networkx as nx
import numpy as np
import pytest

import oracle as O


def components(flag, periodic):
    L = flag.shape[0]
    g = nx.grid_2d_graph(L, L, periodic=periodic)
    g.remove_nodes_from([(a, b) for a in range(L) for b in range(L) if not flag[a, b]])
    lab = -np.ones((L, L), np.int64)
    for comp in nx.connected_components(g):
        idx = min(a * L + b for a, b in comp)
        for a, b in comp:
            lab[a, b] = idx
    return lab, nx.number_connected_components(g)


@pytest.mark.parametrize("L,p,seed", [(4, 0.5, 0), (8, 0.3, 1), (16, 0.55, 2), (32, 0.6, 3), (33, 0.5, 4)])
@pytest.mark.parametrize("periodic", [True, False])
def test_labels_match_library(L, p, seed, periodic):
    rng = np.random.default_rng(seed)
    flag = (rng.random((L, L)) < p).astype(np.uint8)
    lab, n = O.label(flag, periodic)
    ref, nref = components(flag, periodic)
    assert n == nref
    np.testing.assert_array_equal(lab, ref)


def test_hand_built():
    f = np.zeros((6, 6), np.uint8)
    f[0, :] = 1           # a row touching both sides: one cluster when periodic
    f[2, 0] = f[2, 5] = 1  # joined only across the periodic boundary
    f[4, 2] = f[5, 2] = 1  # a column segment touching row 0's cluster through the wrap
    f[3, 4] = 1            # isolated
    lab, n = O.label(f, True)
    assert n == 3
    assert lab[2, 0] == lab[2, 5] == 12
    assert lab[5, 2] == lab[0, 0] == 0
    lab, n = O.label(f, False)
    assert n == 5
    assert np.all(O.label(np.zeros((5, 5), np.uint8), True)[0] == -1)
    lab, n = O.label(np.ones((5, 5), np.uint8), True)
    assert n == 1 and np.all(lab == 0)
