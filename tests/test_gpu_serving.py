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


def test_served_fields_equal_solves_alone(ctx):
    """Fields kept for the caller of a served solve: the plastic flags and
    cluster labels of every increment equal those of the solve run alone
    (bit for bit), the final strain too, and the final stress is the
    constitutive law of Sec. 2 at that strain (the oracle's, within 1e-12
    relative in FP64, 1e-5 in FP32).  A ticket with such fields answers
    polls until it is released."""
    import oracle as O
    reqs = [r for r in requests()[:4]]
    B.epfft_serve_open(ctx, 1 << 30, 4, 16)
    try:
        tickets = {i: B.epfft_submit(ctx, P, path, want_eps=True, want_sig=True, want_plastic=True,
                                     want_labels=True) for i, (P, path) in enumerate(reqs)}
        # nothing has run yet
        assert B.epfft_ticket_fields(ctx, tickets[0], reqs[0][0], 0, plastic=True) is None
        assert not B.epfft_release(ctx, tickets[0])
        done = {}
        rounds = 0
        while len(done) < len(reqs):
            B.epfft_serve_step(ctx)
            for i, t in tickets.items():
                if i not in done:
                    r = B.epfft_poll(ctx, t, reqs[i][0], len(reqs[i][1]), want_eps=True)
                    if r is not None:
                        done[i] = r
            rounds += 1
            assert rounds < 100000
        for i, (P, path) in enumerate(reqs):
            t, n = tickets[i], len(path)
            # still there after its final poll
            assert B.epfft_poll(ctx, t, P, n) is not None
            rc, rec, f = B.epfft_solve(ctx, P, path, fields=True)
            assert done[i][1].tobytes() == rec.tobytes()
            for k in range(n):
                g = B.epfft_ticket_fields(ctx, t, P, k, plastic=True, labels=True)
                assert np.array_equal(g["plastic"], f.plastic[k]), (i, k)
                assert np.array_equal(g["labels"], f.labels[k]), (i, k)
            g = B.epfft_ticket_fields(ctx, t, P, n - 1, eps=True, sig=True)
            assert np.array_equal(g["eps"], f.eps)
            mask = O.mask(P.L, P.void_fraction, P.seed)
            s_ref, _ = O.sigma(g["eps"].astype(np.float64), mask, O.material())
            tol = 1e-12 if P.precision == "fp64" else 1e-5
            assert np.abs(g["sig"] - s_ref).max() <= tol * np.abs(s_ref).max(), i
            # the final state only: strain and stress of an earlier increment are refused
            if n > 1:
                with pytest.raises(B.EpfftError):
                    B.epfft_ticket_fields(ctx, t, P, 0, eps=True)
            assert B.epfft_release(ctx, t)
            with pytest.raises(B.EpfftError):
                B.epfft_ticket_fields(ctx, t, P, 0, plastic=True)
    finally:
        B.epfft_serve_close(ctx)
