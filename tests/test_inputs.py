"""The synthetic workloads of the benchmark and the tests: sizes, void
fractions, seeds, loading modes and strain paths as stated for C1-C5, and
the void-free yield strains the paths are scaled by (checked against the
oracle's Mises law: a uniform strain just below them is elastic, just above
plastic)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_0802_2488_gb300 import inputs


def test_configs_1_2_4():
    c1, c2, c4 = inputs.config1(), inputs.config2(), inputs.config4()
    assert (c1.L, c1.f, c1.seed, c1.mode, c1.n_inc) == (64, 0.10, 0, "equibiaxial", 20)
    assert (c2.L, c2.f, c2.seed, c2.mode, c2.n_inc) == (256, 0.20, 0, "shear", 40)
    assert (c4.L, c4.f, c4.seed, c4.mode, c4.n_inc) == (4096, 0.35, 0, "equibiaxial", 50)
    np.testing.assert_allclose(c1.path[-1], [1.0, 1.0, 0.0, 0.0])              # 2 x Y / (2 mu)
    np.testing.assert_allclose(c2.path[-1], [0.0, 0.0, 0.0, 3.0 / (2.0 * math.sqrt(3.0))])
    np.testing.assert_allclose(c4.path[-1], [0.75, 0.75, 0.0, 0.0])
    for c in (c1, c2, c4):
        assert c.path.shape == (c.n_inc, 4) and (c.path[:, 2] == 0).all()
        np.testing.assert_allclose(np.diff(c.path, axis=0), np.broadcast_to(c.path[0], (c.n_inc - 1, 4)), atol=1e-15)


def test_config3():
    c3 = inputs.config3()
    assert len(c3) == 64 and all(p.L == 512 and p.n_inc == 30 for p in c3)
    assert sorted({p.f for p in c3}) == [0.05, 0.10, 0.20, 0.30]
    for f in (0.05, 0.10, 0.20, 0.30):
        ps = [p for p in c3 if p.f == f]
        assert sorted(p.seed for p in ps) == list(range(16))
        assert all(p.mode == ("equibiaxial" if p.seed < 8 else "shear") for p in ps)
    assert len({p.name for p in c3}) == 64


def test_serving_stream():
    rate = 40.0
    reqs = inputs.serving_stream(4000, rate, seed=3)
    t = np.array([r.arrival_s for r in reqs])
    assert (np.diff(t) > 0).all()
    assert abs(np.mean(np.diff(t)) * rate - 1.0) < 0.05        # exponential gaps of mean 1 / rate
    assert {r.problem.L for r in reqs} == {128, 256, 512, 1024}
    assert all(0.05 <= r.problem.f <= 0.35 and 10 <= r.problem.n_inc <= 50 for r in reqs)
    assert all(r.problem.seed == r.rid == i for i, r in enumerate(reqs))
    assert 0.45 < np.mean([r.problem.mode == "shear" for r in reqs]) < 0.55
    assert inputs.serving_stream(20, rate, seed=3)[5].arrival_s == reqs[5].arrival_s


@pytest.mark.parametrize("mu,Y,lam", [(inputs.MU, inputs.YIELD, inputs.LAMBDA),
                                      (inputs.PAPER_MU, inputs.PAPER_YIELD, inputs.PAPER_LAMBDA)])
@pytest.mark.parametrize("mode", ["equibiaxial", "shear"])
def test_yield_strains(mode, mu, Y, lam):
    E = inputs.load_path(mode, 1, 1.0, mu, Y)[0]
    mat = O.material(lam=lam, mu=mu, Y=Y)
    below = O.sigma((1 - 1e-9) * E[None], np.zeros(1, np.uint8), mat)[1]
    above = O.sigma((1 + 1e-9) * E[None], np.zeros(1, np.uint8), mat)[1]
    assert below[0] == 0 and above[0] == 1


def test_paper_matrix():
    # K = lambda + 2 mu / 3 = 1 with mu = 0.4, Y = 0.5 (Sec. 2)
    assert abs(inputs.PAPER_LAMBDA + 2 * inputs.PAPER_MU / 3 - 1.0) < 1e-15
    assert (inputs.PAPER_MU, inputs.PAPER_YIELD) == (0.4, 0.5)


def test_random_strain_and_spectrum():
    E = [0.1, 0.2, 0.0, 0.05]
    e = inputs.random_strain(64, E, 0.01, seed=1)
    assert e.shape == (64, 64, 4) and np.abs(e - E).max() <= 0.01
    s = inputs.random_spectrum(16, seed=2)
    assert s.shape == (3, 16, 16)
    # Hermitian symmetry of a real field's spectrum
    m = (-np.arange(16)) % 16
    np.testing.assert_allclose(s[:, m][:, :, m], np.conj(s), atol=1e-12)
