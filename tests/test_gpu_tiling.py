"""Every compiled tiling of every lattice side (S8's per-size schedules)
gives the oracle's results, and the autotuner picks one of them.  L = 512
and 2048 cover the tile shapes of the batched and large workloads (4-row
row CTAs with copies at compile-time offsets, 8 elements per thread in the
column transform at 512, one-column tiles at 2048)."""
import numpy as np
import pytest

import oracle as O
from paper_0802_2488_gb300 import binding as B
from paper_0802_2488_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TDT = {"fp64": torch.float64, "fp32": torch.float32}
TOL = {"fp64": 1e-12, "fp32": 2e-5}


@pytest.fixture(scope="module")
def ctx():
    from paper_0802_2488_gb300 import build
    build.build()
    c = B.Context(0)
    yield c
    c.close()


def rel(a, b):
    return np.linalg.norm(np.asarray(a, float) - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("L", [8, 32, 256, 512, 1024, 2048])
@pytest.mark.parametrize("variant", [0, 1, 2])
def test_each_tiling_matches_oracle(ctx, L, prec, variant):
    if not B.epfft_supported_tiling(L, prec, variant):
        pytest.skip("tiling not compiled for this size")
    B.epfft_set_tiling(ctx, L, prec, variant)
    mask = O.mask(L, 0.2, 3)
    mat = O.material()
    E = np.array([0.3, 0.2, 0.0, 0.25])
    eps0 = inputs.random_strain(L, E, 0.2, seed=L)
    k = 2
    ref, lam = eps0.copy(), None
    for _ in range(k):
        ref, lam, _, _ = O.al_step(mask, mat, E, ref, lam)
    t = torch.tensor(eps0, dtype=TDT[prec], device="cuda").contiguous()
    B.epfft_iterate(ctx, B.Problem(L=L, precision=prec, mask=mask), E, t, k)
    assert rel(t.cpu().numpy(), ref) < TOL[prec]
    B.epfft_set_tiling(ctx, L, prec, 0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autotune_chooses_a_compiled_tiling(ctx, prec):
    chosen, ms = B.epfft_autotune(ctx, 256, prec)
    built = [v for v in range(3) if B.epfft_supported_tiling(256, prec, v)]
    assert chosen in built and all(ms[v] > 0 for v in built)
    assert all(ms[v] == 0 for v in range(3) if v not in built)  # 0: not compiled
    assert ms[chosen] == min(ms[v] for v in built)
    B.epfft_set_tiling(ctx, 256, prec, 0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autotune_batch_classes(ctx, prec):
    """Small and large launches are tuned separately; set_tiling sets both."""
    c1, ms1 = B.epfft_autotune(ctx, 512, prec, n_batch=1)
    c2, ms2 = B.epfft_autotune(ctx, 512, prec, n_batch=16)
    assert c1 in (0, 1, 2) and c2 in (0, 1, 2)
    built = [v for v in range(3) if B.epfft_supported_tiling(512, prec, v)]
    assert ms1[c1] == min(ms1[v] for v in built) and ms2[c2] == min(ms2[v] for v in built)
    # the batch of 16 costs more per iteration than one solve
    assert min(ms2[v] for v in built) > min(ms1[v] for v in built)
    B.epfft_set_tiling(ctx, 512, prec, 0)
