"""Pins of the oracle's void-plastic clusters of Sec. 3 (nearest-neighbour
clusters of voids and plastic pixels, each void-free cluster connected to
its nearest void) and of the indicators built on them: hand-built cases,
the periodic distance, ties, invariants on random inputs, and an
independent nearest-void distance from a Euclidean distance transform of
the periodically tiled lattice."""
import numpy as np
import pytest

import oracle as O

ndimage = pytest.importorskip("scipy.ndimage")


def lin(L, x2, x1):
    return x2 * L + x1


def test_detached_plastic_cluster_joins_nearest_void():
    L = 8
    m = np.zeros((L, L), np.uint8)
    p = np.zeros((L, L), np.uint8)
    m[1, 1] = 1
    m[5, 5] = 1
    p[1, 3] = 1  # distance 2 from void (1,1), far from (5,5)
    lab, st = O.void_plastic(m, p)
    assert lab[1, 3] == lab[1, 1] == lin(L, 1, 1)
    assert lab[5, 5] == lin(L, 5, 5)
    assert list(st) == [2, 2, 1, 2, 1, 2]


def test_attachment_across_the_periodic_boundary():
    L = 8
    m = np.zeros((L, L), np.uint8)
    p = np.zeros((L, L), np.uint8)
    m[4, 0] = 1  # the void at x1 = 0 is one pixel away from x1 = 7 through the boundary
    m[4, 4] = 1
    p[4, 6] = 1  # touches nothing; distance 2 to both voids...
    p[2, 7] = 1  # ...and this one: distance^2 = 1 + 4 = 5 to (4, 0), 9 + 4 = 13 to (4, 4)
    lab, st = O.void_plastic(m, p)
    assert lab[2, 7] == lab[4, 0]
    # (4, 6): distance 2 to (4, 4) and 2 to (4, 0) through the boundary: tie,
    # the void with the smaller linear index (4, 0) wins
    assert lab[4, 6] == lab[4, 0]
    assert st[0] == 2 and st[2] == 1


def test_touching_clusters_are_not_reattached_and_bridges_merge():
    L = 8
    m = np.zeros((L, L), np.uint8)
    p = np.zeros((L, L), np.uint8)
    m[2, 2] = m[2, 5] = 1
    p[2, 3] = p[2, 4] = 1  # plastic bridge between the two voids
    m[6, 6] = 1
    p[6, 7] = 1  # plastic touching its void
    lab, st = O.void_plastic(m, p)
    assert lab[2, 2] == lab[2, 3] == lab[2, 4] == lab[2, 5] == lin(L, 2, 2)
    assert lab[6, 7] == lab[6, 6] == lin(L, 6, 6)
    assert list(st[:4]) == [2, 4, 0, 3]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_invariants_and_nearest_distance(seed):
    L = 32
    rng = np.random.default_rng(seed)
    m = (rng.random((L, L)) < 0.05).astype(np.uint8)
    # plastic pixels: a dilation of the voids, thinned at random so that some
    # plastic clusters detach from their void
    near = ndimage.binary_dilation(np.tile(m, (3, 3)), iterations=2)[L:2 * L, L:2 * L]
    p = (near & (rng.random((L, L)) < 0.55) & (m == 0)).astype(np.uint8)
    lab, st = O.void_plastic(m, p)
    vp = (m | p).astype(bool)
    assert ((lab >= 0) == vp).all()
    flat = lab.ravel()
    for c in np.unique(flat[flat >= 0]):
        members = np.flatnonzero(flat == c)
        assert members.min() == c                    # canonical label
        assert m.ravel()[members].any()              # every cluster holds a void
    assert st[0] == len(np.unique(flat[flat >= 0])) and st[0] <= st[3]
    # distance of each detached plastic cluster to the void it joined equals
    # the distance transform's minimum over the cluster (periodic tiling)
    raw, _ = O.label(vp.astype(np.uint8))
    dist = ndimage.distance_transform_edt(1 - np.tile(m, (3, 3)))[L:2 * L, L:2 * L]
    for c in np.unique(raw[raw >= 0]):
        cl = raw == c
        if m[cl].any():
            continue
        dmin2 = np.round((dist[cl] ** 2).min())
        target = lab[cl][0]
        voids = np.argwhere((lab == target) & (m == 1))
        d2 = []
        for y, x in np.argwhere(cl):
            dy = np.abs(voids[:, 0] - y)
            dx = np.abs(voids[:, 1] - x)
            dy = np.minimum(dy, L - dy)
            dx = np.minimum(dx, L - dx)
            d2.append((dx * dx + dy * dy).min())
        assert min(d2) == dmin2


def test_no_voids_leaves_plastic_clusters_alone():
    L = 8
    m = np.zeros((L, L), np.uint8)
    p = np.zeros((L, L), np.uint8)
    p[1, 1] = p[5, 5] = 1
    lab, st = O.void_plastic(m, p)
    assert lab[1, 1] == lin(L, 1, 1) and lab[5, 5] == lin(L, 5, 5)
    assert list(st) == [2, 1, 0, 0, 2, 0]


def test_indicators_closed_forms():
    """sigma0 = a eps0 - b eps0^2 on an even grid: -d2 sigma0/d eps0^2 = 2b in
    the interior; n constant gives r = 0; f_p, v_max, i, n from the counts."""
    k = 9
    rec = np.zeros(k, dtype=O.RECORD_DTYPE)
    e0 = np.linspace(0.1, 0.9, k)
    s0 = 3.0 * e0 - 0.7 * e0 ** 2
    rec["eps_mean"][:, 0] = rec["eps_mean"][:, 1] = e0
    rec["sig_mean"][:, 0] = rec["sig_mean"][:, 1] = s0
    L = 10
    st = np.tile(np.array([[6, 30, 2, 8, 20, 10]], np.int32), (k, 1))
    ind = O.indicators(rec, st, L, "equibiaxial")
    np.testing.assert_allclose(ind[:, 0], e0)
    np.testing.assert_allclose(ind[:, 1], s0)
    np.testing.assert_allclose(ind[2:-2, 7], 1.4, rtol=1e-9)
    np.testing.assert_allclose(ind[:, 2], 20 / 90)
    np.testing.assert_allclose(ind[:, 3], 0.30)
    np.testing.assert_allclose(ind[:, 4], 0.25)
    np.testing.assert_allclose(ind[:, 5], 0.75)
    np.testing.assert_allclose(ind[:, 6], 0.0, atol=1e-12)
