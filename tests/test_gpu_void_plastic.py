"""Sec. 3 void-plastic clusters on the CUDA path against the oracle:
labels and counts bit-exact (integer work), on synthetic flags and on the
per-increment plastic flags of a solve, and the indicators of that solve."""
import numpy as np
import pytest

import oracle as O
from paper_0802_2488_gb300 import binding as B
from paper_0802_2488_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_0802_2488_gb300 import build
    build.build()
    c = B.Context(0)
    yield c
    c.close()


def synth(L, f, seed, keep):
    """Voids, and plastic pixels near them thinned at random (some detach)."""
    rng = np.random.default_rng(seed)
    m = O.mask(L, f, seed)
    near = np.zeros((L, L), bool)
    for dy in range(-2, 3):
        for dx in range(-2, 3):
            near |= np.roll(np.roll(m.astype(bool), dy, 0), dx, 1)
    p = (near & (rng.random((L, L)) < keep) & (m == 0)).astype(np.uint8)
    return m, p


@pytest.mark.parametrize("L,f,seed,keep", [(8, 0.1, 1, 0.5), (32, 0.05, 2, 0.5), (64, 0.02, 3, 0.4),
                                           (128, 0.1, 4, 0.6), (256, 0.01, 5, 0.3)])
def test_void_plastic_bitexact(ctx, L, f, seed, keep):
    m, p = synth(L, f, seed, keep)
    st, lab = B.epfft_void_plastic(ctx, m, p, labels=True)
    ref_lab, ref_st = O.void_plastic(m, p)
    np.testing.assert_array_equal(lab[0].cpu().numpy(), ref_lab)
    np.testing.assert_array_equal(st[0], ref_st)


def test_void_plastic_edge_cases(ctx):
    L = 16
    z = np.zeros((L, L), np.uint8)
    p = z.copy()
    p[3, 3] = p[9, 12] = 1
    for m, pl in ((z, z), (z, p), (np.ones((L, L), np.uint8), z)):
        st, lab = B.epfft_void_plastic(ctx, m, pl, labels=True)
        ref_lab, ref_st = O.void_plastic(m, pl)
        np.testing.assert_array_equal(lab[0].cpu().numpy(), ref_lab)
        np.testing.assert_array_equal(st[0], ref_st)


@pytest.mark.parametrize("load", ["equibiaxial", "shear"])
def test_solve_indicators(ctx, load):
    """Per-increment flags of a solve -> clusters and indicators."""
    L = 32
    path = inputs.load_path(load, 6, 2.0 if load == "equibiaxial" else 3.0)
    prob = B.Problem(L=L, precision="fp64", void_fraction=0.1, seed=2, max_iter=300)
    rc, rec, f = B.epfft_solve(ctx, prob, path, fields=True)
    mask = O.mask(L, 0.1, 2)
    st, lab = B.epfft_void_plastic(ctx, mask, f.plastic, labels=True)
    for k in range(len(path)):
        ref_lab, ref_st = O.void_plastic(mask, f.plastic[k])
        np.testing.assert_array_equal(lab[k].cpu().numpy(), ref_lab)
        np.testing.assert_array_equal(st[k], ref_st)
    ind = B.epfft_indicators(rec, st, L, load)
    np.testing.assert_allclose(ind, O.indicators(rec, st, L, load), rtol=1e-12, atol=1e-12)
    # every cluster holds a void once voids exist; n(eps0) starts at most 1
    assert (ind[:, 5] <= 1.0 + 1e-12).all()
