"""Pins of the oracle's void mask: the SplitMix64 stream against published
values, and the i.i.d. Bernoulli(f) statistics of Sec. 2."""
import numpy as np
import pytest

import oracle as O

# First outputs of SplitMix64 seeded with 0, as published with the reference
# generator (also java.util.SplittableRandom(0).nextLong(): -2152535657050944081).
SEED0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F,
         0xF88BB8A8724C81EC, 0x1B39896A51A8749B]


def test_splitmix64_published_stream():
    assert [O.splitmix64(0, i) for i in range(5)] == SEED0
    assert O.splitmix64(0, 0) - 2 ** 64 == -2152535657050944081


def test_threshold_edges():
    assert O.void_threshold(0.0) == 0
    assert O.void_threshold(1.0) == 2 ** 53
    assert O.void_threshold(0.5) == 2 ** 52
    assert O.void_threshold(0.1) == int(np.floor(0.1 * 2.0 ** 53))
    L = 16
    assert O.mask(L, 0.0, 3).sum() == 0
    assert O.mask(L, 1.0, 3).sum() == L * L


@pytest.mark.parametrize("f", [0.05, 0.1, 0.2, 0.35])
def test_bernoulli_statistics(f):
    L = 512
    m = O.mask(L, f, 0).astype(np.float64)
    n = L * L
    assert abs(m.mean() - f) < 5 * np.sqrt(f * (1 - f) / n)
    # no correlation between neighbouring pixels (lattice is pixelwise disordered)
    c1 = np.mean((m - f) * (np.roll(m, 1, axis=1) - f)) / (f * (1 - f))
    c2 = np.mean((m - f) * (np.roll(m, 1, axis=0) - f)) / (f * (1 - f))
    assert abs(c1) < 5 / np.sqrt(n) and abs(c2) < 5 / np.sqrt(n)
    # different seeds give independent masks
    m2 = O.mask(L, f, 1).astype(np.float64)
    cs = np.mean((m - f) * (m2 - f)) / (f * (1 - f))
    assert abs(cs) < 5 / np.sqrt(n)


def test_mask_is_nested_in_f():
    # the same uniform numbers are thresholded, so a larger f adds voids only
    a, b = O.mask(64, 0.1, 5), O.mask(64, 0.3, 5)
    assert np.all(b >= a)
