"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and
the oracle's tests.

This module holds no arithmetic of the method: it only states workloads
(lattice size, void concentration, seed, macroscopic strain path) and draws
random test states with numpy.  The random void mask itself is part of the
method (each side generates it from the seed), so it is not produced here;
the one-void periodic cell of Fig. 1 is a fixed geometry and is.

Strain tuples are (E11, E22, E33, E12) with E33 = 0 (plane strain) and E12
the tensor shear component (the paper's simple-shear loading prescribes
eps0 = <eps_xy>, Sec. 3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Matrix of every workload: mu = 1, nu = 0.3 (lambda = 2 mu nu / (1 - 2 nu) = 1.5),
# Mises flow stress Y = 1; the augmented-Lagrangian reference medium C0 equals
# the matrix.
MU = 1.0
LAMBDA = 1.5
YIELD = 1.0

# First-yield strains of the void-free (f = 0) lattice under the two loadings,
# from the Mises criterion with the 3D deviator (plane strain, E33 = 0):
#   equibiaxial E11 = E22 = e:  |dev| = e sqrt(6)/3, 2 mu |dev| = sqrt(2/3) Y  ->  e = Y / (2 mu)
#   shear       E12 = g:        |dev| = g sqrt(2),   2 mu |dev| = sqrt(2/3) Y  ->  g = Y / (2 sqrt(3) mu)
EQUIBIAXIAL_YIELD = YIELD / (2.0 * MU)
SHEAR_YIELD = YIELD / (2.0 * math.sqrt(3.0) * MU)

# The matrix of the paper's own computations (Sec. 2): bulk modulus K = 1,
# shear modulus mu = 0.4 (so lambda = K - 2 mu / 3), flow stress Y = 0.5.
PAPER_MU = 0.4
PAPER_LAMBDA = 1.0 - 2.0 * PAPER_MU / 3.0
PAPER_YIELD = 0.5


def load_path(mode: str, n_inc: int, multiple: float, mu: float = MU, Y: float = YIELD) -> np.ndarray:
    """(n_inc, 4) prescribed mean strains ramped in equal increments to
    `multiple` x the f = 0 first-yield strain of the loading `mode`
    ('equibiaxial' or 'shear') for a matrix of shear modulus mu and flow
    stress Y (default: the workloads' matrix)."""
    n = np.arange(1, n_inc + 1, dtype=np.float64) / n_inc
    P = np.zeros((n_inc, 4))
    if mode == "equibiaxial":
        P[:, 0] = P[:, 1] = n * multiple * Y / (2.0 * mu)
    elif mode == "shear":
        P[:, 3] = n * multiple * Y / (2.0 * math.sqrt(3.0) * mu)
    else:
        raise ValueError(mode)
    return P


def one_void_cell(L: int, f: float) -> np.ndarray:
    """(L, L) uint8 mask of the periodic cell of Fig. 1: one circular void
    of area fraction about f at the centre of the cell (pixels whose centres
    lie within radius L (f / pi)^(1/2) of the cell centre are voids)."""
    c = np.arange(L) + 0.5 - L / 2.0
    r2 = f * L * L / math.pi
    return ((c[None, :] ** 2 + c[:, None] ** 2) < r2).astype(np.uint8)


@dataclass
class Problem:
    """One solve: L x L lattice, void concentration f, mask seed, strain path."""
    L: int
    f: float
    seed: int
    mode: str
    n_inc: int
    multiple: float
    name: str = ""
    path: np.ndarray = field(init=False)

    def __post_init__(self):
        self.path = load_path(self.mode, self.n_inc, self.multiple)


def config1() -> Problem:
    """L = 64, f = 0.10, seed 0, equibiaxial, 20 increments to 2x yield."""
    return Problem(64, 0.10, 0, "equibiaxial", 20, 2.0, "L64_f0.10_equibiaxial_20inc")


def config2() -> Problem:
    """L = 256, f = 0.20, seed 0, shear, 40 increments to 3x yield."""
    return Problem(256, 0.20, 0, "shear", 40, 3.0, "L256_f0.20_shear_40inc")


def config3() -> list[Problem]:
    """64 realizations of L = 512: f in {0.05, 0.10, 0.20, 0.30} x seeds 0..15;
    seeds 0-7 equibiaxial to 2x yield, 8-15 shear to 3x yield; 30 increments."""
    out = []
    for f in (0.05, 0.10, 0.20, 0.30):
        for s in range(16):
            mode = "equibiaxial" if s < 8 else "shear"
            out.append(Problem(512, f, s, mode, 30, 2.0 if s < 8 else 3.0,
                               f"L512_f{f:.2f}_s{s}_{mode}"))
    return out


def config4() -> Problem:
    """L = 4096, f = 0.35, seed 0, equibiaxial to 1.5x yield in 50 increments."""
    return Problem(4096, 0.35, 0, "equibiaxial", 50, 1.5, "L4096_f0.35_equibiaxial_50inc")


@dataclass
class Request:
    rid: int
    arrival_s: float
    problem: Problem


def serving_stream(n: int, rate_per_s: float, seed: int = 0) -> list[Request]:
    """Poisson arrivals at `rate_per_s`; per request L ~ U{128, 256, 512, 1024},
    f ~ U[0.05, 0.35], loading equibiaxial or shear with probability 1/2,
    n_inc ~ U{10..50}; the mask seed is the request id."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
    out = []
    for i in range(n):
        L = int(rng.choice([128, 256, 512, 1024]))
        f = float(rng.uniform(0.05, 0.35))
        mode = "equibiaxial" if rng.random() < 0.5 else "shear"
        n_inc = int(rng.integers(10, 51))
        mult = 2.0 if mode == "equibiaxial" else 3.0
        out.append(Request(i, float(t[i]), Problem(L, f, i, mode, n_inc, mult, f"req{i}")))
    return out


def random_strain(L: int, E, amplitude: float, seed: int) -> np.ndarray:
    """(L, L, 4) strain field: E plus i.i.d. uniform noise of the given
    amplitude on every component (a generic, non-equilibrated iterate)."""
    rng = np.random.default_rng(seed)
    return np.asarray(E, dtype=np.float64)[None, None, :] + amplitude * rng.uniform(-1.0, 1.0, size=(L, L, 4))


def random_spectrum(L: int, seed: int) -> np.ndarray:
    """(3, L, L) complex128 spectrum of three real random fields, i.e. a
    Hermitian-symmetric polarization spectrum (11, 22, 12)."""
    rng = np.random.default_rng(seed)
    p = rng.standard_normal((3, L, L))
    return np.fft.fft2(p, axes=(1, 2))
