"""Parity at the full sizes of the batched and the large-lattice workloads, in
the launch configuration the benchmark times (tiling 0): 64 solves of
L = 512 advanced in one batch, sampled solves compared with the oracle run
one by one; and one AL iteration of the L = 4096, f = 0.35 lattice compared
with the oracle over the whole field.  FP32 tolerances as in
test_gpu_parity (a few iterations: 2e-5 relative)."""
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


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_batch_of_64_at_L512_matches_oracle(ctx):
    """The 64 lattices of the batched workload (f in {0.05, ..., 0.30} x 16
    seeds, half equibiaxial, half shear), first increment of each path, three
    iterations, one launch per pass for all 64; solves 0, 21, 42 and 63
    against the oracle."""
    B.epfft_set_tiling(ctx, 512, "fp32", 0)
    cfg = inputs.config3()
    probs = [B.Problem(L=P.L, precision="fp32", void_fraction=P.f, seed=P.seed, tol_eq=0.0, tol_macro=0.0,
                       max_iter=3) for P in cfg]
    paths = [P.path[:1] for P in cfg]
    rc, recs, fields = B.epfft_solve_batch(ctx, probs, paths, fields=True)
    assert rc == B.EPFFT_NOT_CONVERGED
    for i in (0, 21, 42, 63):
        P = cfg[i]
        ref = O.solve(O.mask(P.L, P.f, P.seed), O.material(), paths[i], tol_eq=0.0, tol_macro=0.0, max_iter=3,
                      fields=True)
        np.testing.assert_array_equal(recs[i]["iterations"], ref.records["iterations"])
        assert rel(recs[i]["sig_mean"], ref.records["sig_mean"]) < 2e-5, i
        assert rel(recs[i]["eps_mean"], ref.records["eps_mean"]) < 2e-5, i
        assert rel(fields[i].eps, ref.eps) < 2e-5, (i, rel(fields[i].eps, ref.eps))


def test_one_iteration_at_L4096_matches_oracle(ctx):
    """The large lattice (L = 4096, f = 0.35, seed 0) at the middle of its
    equibiaxial path, one AL iteration from a perturbed state."""
    if not B.epfft_supported(4096, "fp32"):
        pytest.skip("not built")
    B.epfft_set_tiling(ctx, 4096, "fp32", 0)
    P = inputs.config4()
    E = P.path[P.n_inc // 2]
    mask = O.mask(P.L, P.f, P.seed)
    eps0 = inputs.random_strain(P.L, E, 0.05, seed=4)
    ref = O.al_step(mask, O.material(), E, eps0, None)[0]
    t = torch.tensor(eps0, dtype=torch.float32, device="cuda").contiguous()
    B.epfft_iterate(ctx, B.Problem(L=P.L, precision="fp32", mask=mask), E, t, 1)
    err = rel(t.cpu().numpy(), ref)
    assert err < 2e-5, err
    # the same iteration in FP64 (tiling 1: one row per CTA) and in the
    # defect form (FP32 differences from the FP64 state, its refresh in FP64)
    B.epfft_set_tiling(ctx, 4096, "fp64", 1)
    t = torch.tensor(eps0, dtype=torch.float64, device="cuda").contiguous()
    B.epfft_iterate(ctx, B.Problem(L=P.L, precision="fp64", mask=mask), E, t, 1)
    err = rel(t.cpu().numpy(), ref)
    assert err < 1e-12, err
    t = torch.tensor(eps0, dtype=torch.float64, device="cuda").contiguous()
    B.epfft_iterate(ctx, B.Problem(L=P.L, precision="fp32_defect", mask=mask), E, t, 1)
    err = rel(t.cpu().numpy(), ref)
    assert err < 2e-5, err
