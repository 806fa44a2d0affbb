"""The library's Sec. 3 indicators (host code behind the C ABI, no GPU
needed) against the oracle's, on records and cluster counts of the shapes
a solve produces."""
import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module")
def B():
    from paper_0802_2488_gb300 import binding
    return binding


@pytest.mark.parametrize("load", ["equibiaxial", "shear"])
@pytest.mark.parametrize("k", [1, 2, 5, 20])
def test_indicators_match_oracle(B, load, k):
    rng = np.random.default_rng(k)
    rec = np.zeros(k, dtype=O.RECORD_DTYPE)
    e0 = np.cumsum(rng.uniform(0.02, 0.08, k))  # uneven increments
    rec["eps_mean"][:, :2] = e0[:, None] if load == "equibiaxial" else rng.normal(0, 1e-3, (k, 1))
    rec["eps_mean"][:, 3] = e0 if load == "shear" else 0.0
    rec["sig_mean"] = rng.normal(1.0, 0.3, (k, 4))
    st = np.stack([rng.integers(5, 50, k), rng.integers(1, 400, k), rng.integers(0, 5, k),
                   np.full(k, 40), rng.integers(0, 900, k), np.full(k, 100)], axis=1).astype(np.int32)
    L = 32
    got = B.epfft_indicators(rec, st, L, load)
    ref = O.indicators(rec, st, L, load)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("load", ["equibiaxial", "shear"])
def test_empirical_curve_matches_oracle(B, load):
    rng = np.random.default_rng(11)
    k = 15
    ind = np.zeros((k, 8))
    ind[:, 0] = np.cumsum(rng.uniform(0.03, 0.09, k))
    ind[:, 1] = np.sqrt(ind[:, 0]) + rng.normal(0, 0.01, k)
    ind[:, 2] = np.linspace(0, 0.5, k)
    ind[:, 3] = np.linspace(0.02, 0.3, k)
    ind[:, 5] = np.concatenate([[1, 1, 1], np.linspace(0.95, 0.2, k - 3)])
    st = np.zeros((k, 6), np.int32)
    st[:, 4] = rng.integers(0, 300, k)
    st[:, 5] = 64
    a, f = B.epfft_empirical_curve(ind, st, 24, 2.2, load)
    ra, rf = O.empirical_curve(ind, st, 24, 2.2, load)
    assert abs(a - ra) < 1e-12 * max(1.0, abs(ra))
    np.testing.assert_allclose(f, rf, rtol=1e-12, atol=1e-12)
