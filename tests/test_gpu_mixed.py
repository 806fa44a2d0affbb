"""Lattices of several sides and precisions advanced in one device loop
(S8): epfft_solve_batch groups the problems by (L, precision), runs each
group's passes on a branch of one graph body and loops while any problem is
unfinished.  Each result equals the same problem solved alone (bit-identical
records and final strain: a solve's arithmetic does not depend on the other
solves of the launch).  Serving runs every size class of a step in one such
launch; here at the serving stream's sizes (L up to 1024) under an HBM
budget that holds only part of the requests at once."""
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


def test_mixed_sizes_in_one_launch_equal_the_solves_alone(ctx):
    cases = [(128, "fp32", 0.10, "shear"), (256, "fp32", 0.25, "equibiaxial"), (512, "fp32", 0.05, "shear"),
             (64, "fp64", 0.20, "equibiaxial"), (256, "fp32", 0.15, "shear"), (32, "fp64", 0.30, "shear")]
    probs, paths = [], []
    for i, (L, prec, f, mode) in enumerate(cases):
        probs.append(B.Problem(L=L, precision=prec, void_fraction=f, seed=40 + i, max_iter=30 + 10 * i))
        paths.append(inputs.load_path(mode, 3 + i % 2, 2.0 if mode == "equibiaxial" else 3.0))
    rc, recs, flds = B.epfft_solve_batch(ctx, probs, paths, fields=True)
    st = B.epfft_last_stats(ctx)
    # one loop for all: as many steps as the longest solve needs
    need = max(len(p) * (P.max_iter + 2) for P, p in zip(probs, paths))
    assert st["loop_steps"] <= need + 8
    for i, (P, path) in enumerate(zip(probs, paths)):
        rc1, rec1, f1 = B.epfft_solve(ctx, P, path, fields=True)
        assert rec1.tobytes() == recs[i].tobytes(), i
        assert np.array_equal(f1.eps, flds[i].eps), i
        assert np.array_equal(f1.labels, flds[i].labels), i


def test_serving_stream_sizes_under_a_binding_budget(ctx):
    """Requests of L in {128, 256, 512, 1024} (FP32) with a budget that
    holds the largest one plus a little: admission waits for memory, the
    classes advance together, every result equals the solve alone."""
    rng = np.random.default_rng(9)
    reqs = []
    for i in range(8):
        L = [128, 256, 512, 1024][i % 4]
        mode = "equibiaxial" if rng.random() < 0.5 else "shear"
        P = B.Problem(L=L, precision="fp32", void_fraction=float(rng.uniform(0.05, 0.35)), seed=200 + i,
                      max_iter=12)
        reqs.append((P, inputs.load_path(mode, int(rng.integers(3, 7)), 2.0 if mode == "equibiaxial" else 3.0)))
    # footprint of the L = 1024 request: 4 state buffers, the spectrum, mask
    # and flags, i.e. about 77 + n_inc bytes per pixel in FP32
    big = 1024 * 1024 * (16 * 4 + 12 + 1 + 8)
    budget = int(1.3 * big)
    B.epfft_serve_open(ctx, budget, 4, 8)
    try:
        tickets = {i: B.epfft_submit(ctx, P, path, want_eps=True) for i, (P, path) in enumerate(reqs)}
        results, rounds, max_running = {}, 0, 0
        while tickets:
            run, queued = B.epfft_serve_step(ctx)
            max_running = max(max_running, run)
            rounds += 1
            assert rounds < 10000
            for i, t in list(tickets.items()):
                r = B.epfft_poll(ctx, t, reqs[i][0], len(reqs[i][1]), want_eps=True)
                if r is not None:
                    results[i] = r
                    del tickets[i]
    finally:
        B.epfft_serve_close(ctx)
    # the budget bound: never all eight at once
    assert 1 <= max_running < len(reqs)
    for i, (P, path) in enumerate(reqs):
        rc, rec, f = B.epfft_solve(ctx, P, path, fields=True)
        rc2, rec2, eps2, lat = results[i]
        assert rc2 == rc and rec.tobytes() == rec2.tobytes(), i
        assert np.array_equal(f.eps, eps2), i
