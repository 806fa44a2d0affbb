"""Index arithmetic of the Stockham row pass's tile copies (RowIO in
csrc/passes.cuh), restated on the CPU: where the copies take the fixed
pattern (a thread's element e = E0 + k S with compile-time offsets per k),
the offsets give the same shared and global index as the general map
where(e) for every thread and step, of every compiled side, precision and
tiling; and the general map itself sends the tile's 3 M RR numbers to
distinct shared slots inside the tile and to the rows r0 .. r0 + RR - 1 of
the spectrum."""
import pytest

SIDES = [4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096]


def seq_stride(n):
    return n + n // 32 + 1 if n >= 512 else (n + n // 32 if n >= 32 else n)


def pad32(x):
    return x + (x >> 5)


def cfg(f64, L, V):
    """(M, RR, W, NT, SP) of Cfg<T, L, V> for the row pass."""
    M = L // 2
    if V == 0:
        RR = 2 if f64 else (2 if L <= 256 else (4 if L == 512 else (8 if L <= 2048 else 4)))
        W0 = (1 if L <= 256 else (2 if L <= 1024 else 1)) if f64 else (1 if L == 2048 else 2)
    else:
        RR = (1 if L <= 256 or L == 4096 else 2) if f64 else (1 if L <= 256 else 2)
        W0 = 1 if f64 else (1 if L <= 256 else (2 if L <= 1024 else (1 if L <= 2048 else 2)))
    W = min(W0, M)
    ntmax = 512 if V == 0 else 256
    if f64:
        nt0 = 256 if L > 512 else (L if L < 128 else 128)
    else:
        nt0 = L if L <= 256 else (256 if V == 0 and L == 512 else ntmax)
    return M, RR, W, max(32, nt0), seq_stride(M)


def where(e, r0, L, M, RR, W, SP):
    nbk = M // W
    c = e // (M * RR)
    rem = e - c * (M * RR)
    b = rem // (RR * W)
    rem2 = rem - b * (RR * W)
    r, w = rem2 // W, rem2 - (rem2 // W) * W
    return (c * RR + r) * SP + pad32(b * W + w), ((c * nbk + b) * L + r0 + r) * W + w


def fixed(S, M, RR, W):
    return S % (RR * W) == 0 and (M * RR) % S == 0 and (S // RR) % 32 == 0 and 3 * M * RR // S <= 24


def fixed_offsets(S, k, L, M, RR, W, SP):
    kpc = (M * RR) // S
    c, j = k // kpc, k % kpc
    return c * RR * SP + j * (S // RR + S // (32 * RR)), (c * (M // W) + j * (S // (RR * W))) * L * W


CASES = [(f64, L, V) for f64 in (False, True) for L in SIDES for V in (0, 1)]


@pytest.mark.parametrize("f64,L,V", CASES)
def test_fixed_copy_offsets_equal_the_general_map(f64, L, V):
    M, RR, W, NT, SP = cfg(f64, L, V)
    r0 = (L // RR - 1) * RR  # the last CTA of a solve
    pairs = (not f64) and (RR * W) % 2 == 0
    for S, E0, count in ((NT, lambda t: t, 3 * M * RR // NT), (2 * NT, lambda t: 2 * t, 3 * M * RR // (2 * NT))):
        if S == 2 * NT and not pairs:
            continue
        if not fixed(S, M, RR, W):
            continue
        assert (3 * M * RR) % S == 0
        for t in range(NT):
            is0, ig0 = where(E0(t), r0, L, M, RR, W, SP)
            for k in range(count):
                di, dg = fixed_offsets(S, k, L, M, RR, W, SP)
                assert (is0 + di, ig0 + dg) == where(E0(t) + k * S, r0, L, M, RR, W, SP), (t, k)


@pytest.mark.parametrize("f64,L,V", CASES)
def test_general_map_stays_in_the_tile_and_the_rows(f64, L, V):
    M, RR, W, NT, SP = cfg(f64, L, V)
    r0 = (L // RR - 1) * RR
    seen = set()
    for e in range(3 * M * RR):
        i, g = where(e, r0, L, M, RR, W, SP)
        assert 0 <= i < 3 * RR * SP and i not in seen
        seen.add(i)
        assert 0 <= g < 3 * M * L
        x2 = (g // W) % L
        assert r0 <= x2 < r0 + RR


def test_the_batched_row_tiles_take_the_fixed_pattern():
    # tiling 0 at L = 512 (the batched workload) and 1024, loads and pair
    # stores; at 2048 and 4096 (48 steps per thread) the loop stays
    for L in (512, 1024):
        M, RR, W, NT, SP = cfg(False, L, 0)
        assert fixed(NT, M, RR, W) and fixed(2 * NT, M, RR, W), L
    for L in (2048, 4096):
        M, RR, W, NT, SP = cfg(False, L, 0)
        assert not fixed(NT, M, RR, W), L
