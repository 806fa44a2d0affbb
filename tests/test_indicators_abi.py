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
