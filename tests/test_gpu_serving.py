"""Serving (continuous batching): requests of several lattice sizes, void
fractions, loadings and increment counts are admitted as slots and budget
free up, run concurrently, and each result is the same as the solve run
alone (bit-identical records and final strain)."""
import numpy as np
import pytest

from paper_0802_2488_gb300 import binding as B
from paper_0802_2488_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_0802_2488_gb300 import build
    build.build()
    c = B.Context(0)
    yield c
    c.close()


def requests():
    out = []
    rng = np.random.default_rng(5)
    for i in range(9):
        L = int(rng.choice([32, 64, 128]))
        prec = "fp64" if i % 3 else "fp32"
        mode = "equibiaxial" if i % 2 else "shear"
        n_inc = int(rng.integers(2, 6))
        P = B.Problem(L=L, precision=prec, void_fraction=float(rng.uniform(0.05, 0.35)), seed=100 + i,
                      max_iter=int(rng.integers(20, 120)))
        out.append((P, inputs.load_path(mode, n_inc, 2.0 if mode == "equibiaxial" else 3.0)))
    return out


def serve_all(ctx, reqs, budget, slots, steps, stagger=0):
    B.epfft_serve_open(ctx, budget, slots, steps)
    try:
        tickets = {}
        results = {}
        pending = list(range(len(reqs)))
        rounds = 0
        while pending or tickets:
            # submit `stagger` new requests per round (all at once if 0)
            take = len(pending) if stagger == 0 else min(stagger, len(pending))
            for _ in range(take):
                i = pending.pop(0)
                tickets[i] = B.epfft_submit(ctx, reqs[i][0], reqs[i][1], want_eps=True)
            B.epfft_serve_step(ctx)
            rounds += 1
            for i, t in list(tickets.items()):
                r = B.epfft_poll(ctx, t, reqs[i][0], len(reqs[i][1]), want_eps=True)
                if r is not None:
                    results[i] = r
                    del tickets[i]
            assert rounds < 100000
        return results, rounds
    finally:
        B.epfft_serve_close(ctx)


def test_served_results_equal_solves_alone(ctx):
    reqs = requests()
    results, rounds = serve_all(ctx, reqs, budget=1 << 30, slots=4, steps=16, stagger=2)
    for i, (P, path) in enumerate(reqs):
        rc, rec, f = B.epfft_solve(ctx, P, path, fields=True)
        rc2, rec2, eps2, lat = results[i]
        assert rc2 == rc
        assert rec.tobytes() == rec2.tobytes(), i
        assert np.array_equal(f.eps, eps2), i
        assert lat > 0


def test_budget_admits_one_at_a_time(ctx):
    reqs = requests()[:4]
    P, path = reqs[0]
    # a budget that holds the largest single request but not two of them
    big = max(r[0].L for r in reqs)
    budget = 6 * big * big * 8 * 4
    results, rounds = serve_all(ctx, reqs, budget=budget, slots=8, steps=32)
    assert len(results) == 4
    for i, (P, path) in enumerate(reqs):
        _, rec = B.epfft_solve(ctx, P, path)
        assert rec.tobytes() == results[i][1].tobytes()


def test_request_larger_than_budget_is_refused(ctx):
    B.epfft_serve_open(ctx, 1 << 20, 4, 8)
    try:
        with pytest.raises(B.EpfftError) as e:
            B.epfft_submit(ctx, B.Problem(L=512, void_fraction=0.1), inputs.load_path("shear", 10, 3.0))
        assert e.value.code == B.EPFFT_ERR_OOM
    finally:
        B.epfft_serve_close(ctx)
