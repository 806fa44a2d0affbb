"""Index arithmetic of the register-staged column pass (csrc/colrs.cuh),
restated on the CPU: the radix plan, the positions each thread touches in
every stage, the shared-memory swizzle, the lane mapping of a CTA and the
position -> frequency map.

* A numpy replay of the stages (in-place decimation in frequency with the
  plan's radices and twiddles, then the transposed stages in reverse order)
  gives numpy's DFT in digit-reversed order and its exact inverse.
* Every stage covers each position exactly once; the first stage holds
  positions t + m T and the last one E t + r (E = 16 elements per thread,
  8 at L = 512).
* Every warp access of eight-byte elements (half-warp phases) falls on 16
  distinct bank pairs, for the lane mapping the kernel uses (the two columns
  of a tile interleaved lane by lane when a CTA holds both).
"""
import numpy as np
import pytest

SIZES = [128, 256, 512, 1024, 2048, 4096]
E = 16  # elements per thread and sequence of the row transforms


def col_e(L):
    """Elements per thread of the column transform (RsPlan: col_e)."""
    return 8 if L == 512 else 16


def plan(L):
    ce = col_e(L)
    lc = ce.bit_length() - 1
    lg = L.bit_length() - 1
    r1 = ce if lg % lc == 0 else 1 << (lg % lc)
    S = lg // lc if lg % lc == 0 else lg // lc + 1
    radix = [r1] + [ce] * (S - 1)
    nlen = [L]
    for s in range(1, S):
        nlen.append(nlen[-1] // radix[s - 1])
    stride = [n // r for n, r in zip(nlen, radix)]
    return radix, nlen, stride


def cfg(L, W):
    """(columns per CTA, threads per CTA, interleaved) as in RsCfg."""
    T = L // col_e(L)
    cpc = max(2, 64 // T) if L <= 1024 else 1
    inter = cpc >= 2 and W == 2
    return cpc, cpc * T, inter


def sw(e):
    return e ^ ((e >> 4) & 15)


def sw8(e):
    return e ^ ((e >> 3) & 7)


def csw(L, e):
    """Swizzle of the column plan (psw): sw16, or sw8 for 8 elements."""
    return sw8(e) if col_e(L) == 8 else sw(e)


def seq_base(L, g):
    """Element offset of group g's three sequences (components at + c L)."""
    return g * (3 * L + 8)


def lane_map(L, W, tid):
    """(group, t) of thread tid of a CTA."""
    T = L // col_e(L)
    cpc, nt, inter = cfg(L, W)
    if inter:
        pair, rem = divmod(tid, 2 * T)
        return 2 * pair + (rem & 1), rem >> 1
    return divmod(tid, T)


def freq(L, p):
    radix, nlen, stride = plan(L)
    m, w = 0, 1
    for s in range(len(radix)):
        m += ((p // stride[s]) % radix[s]) * w
        w *= radix[s]
    return m


def butterflies(L, s, t):
    """(base, stride, j) of the butterflies thread t does in stage s."""
    radix, nlen, stride = plan(L)
    ce = col_e(L)
    T = L // ce
    R, N, D = radix[s], nlen[s], stride[s]
    out = []
    for i in range(ce // R):
        u = t + i * T
        b, j = divmod(u, D)
        out.append((b * N + j, D, j))
    return out


def stages_forward(L, x):
    radix, nlen, stride = plan(L)
    a = x.astype(np.complex128).copy()
    for s in range(len(radix)):
        R, N = radix[s], nlen[s]
        for t in range(L // col_e(L)):
            for base, d, j in butterflies(L, s, t):
                v = a[base + d * np.arange(R)]
                y = np.array([np.sum(v * np.exp(-2j * np.pi * np.arange(R) * k / R)) for k in range(R)])
                y *= np.exp(-2j * np.pi * j * np.arange(R) / N)
                a[base + d * np.arange(R)] = y
    return a


def stages_inverse(L, a):
    radix, nlen, stride = plan(L)
    a = a.copy()
    for s in reversed(range(len(radix))):
        R, N = radix[s], nlen[s]
        for t in range(L // col_e(L)):
            for base, d, j in butterflies(L, s, t):
                v = a[base + d * np.arange(R)] * np.exp(2j * np.pi * j * np.arange(R) / N)
                y = np.array([np.sum(v * np.exp(2j * np.pi * np.arange(R) * r / R)) for r in range(R)])
                a[base + d * np.arange(R)] = y
    return a


@pytest.mark.parametrize("L", [128, 256, 512])
def test_stages_are_the_dft_in_digit_reversed_order(L):
    rng = np.random.default_rng(L)
    x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    a = stages_forward(L, x)
    X = np.fft.fft(x)
    order = np.array([freq(L, p) for p in range(L)])
    np.testing.assert_allclose(a, X[order], rtol=0, atol=1e-9 * np.abs(X).max())
    # the transposed stages give the unnormalised inverse in natural order
    np.testing.assert_allclose(stages_inverse(L, a), L * x, rtol=0, atol=1e-9 * L * np.abs(x).max())


@pytest.mark.parametrize("L", SIZES)
def test_position_frequency_map(L):
    f = [freq(L, p) for p in range(L)]
    assert sorted(f) == list(range(L))
    # the last stage's positions E t + r hold frequencies m0(t) + r L / E
    E = col_e(L)
    T = L // E
    for t in range(T):
        m0 = freq(L, E * t)
        assert m0 < L // E
        assert [freq(L, E * t + r) for r in range(E)] == [m0 + r * (L // E) for r in range(E)]


@pytest.mark.parametrize("L", SIZES)
def test_every_stage_covers_each_position_once(L):
    radix, nlen, stride = plan(L)
    E = col_e(L)
    T = L // E
    for s in range(len(radix)):
        seen = np.zeros(L, int)
        for t in range(T):
            for base, d, j in butterflies(L, s, t):
                for r in range(radix[s]):
                    seen[base + r * d] += 1
        assert (seen == 1).all(), (L, s)
    for t in range(T):
        first = sorted(base + r * d for base, d, j in butterflies(L, 0, t) for r in range(radix[0]))
        assert first == [t + m * T for m in range(E)]
        last = sorted(base + r * d for base, d, j in butterflies(L, len(radix) - 1, t) for r in range(radix[-1]))
        assert last == [E * t + r for r in range(E)]


def phases_conflict_free(addrs):
    """Eight-byte accesses of one warp: each half-warp phase must touch
    distinct bank pairs (element index mod 16)."""
    for h in (0, 16):
        bank = [a % 16 for a in addrs[h:h + 16] if a is not None]
        if len(set(bank)) != len(bank):
            return False
    return True


@pytest.mark.parametrize("W", [1, 2])
@pytest.mark.parametrize("L", SIZES)
def test_shared_memory_accesses_are_bank_conflict_free(L, W):
    radix, nlen, stride = plan(L)
    E = col_e(L)
    T = L // E
    cpc, nt, inter = cfg(L, W)
    if E == 8 and not inter:
        pytest.skip("8 elements per thread compile for interleaved column pairs only (RsCfg)")
    assert sorted(csw(L, e) for e in range(L)) == list(range(L))  # a permutation
    for w0 in range(0, nt, 32):
        lanes = [lane_map(L, W, tid) for tid in range(w0, w0 + 32)]
        # butterfly stages
        for s in range(len(radix)):
            per = [(g, butterflies(L, s, t)) for g, t in lanes]
            for i in range(E // radix[s]):
                for r in range(radix[s]):
                    addrs = [seq_base(L, g) + csw(L, b[i][0] + r * b[i][1]) for g, b in per]
                    assert phases_conflict_free(addrs), (L, W, s, i, r)
        # the unfused Green step and the first stage: positions t + m T
        for m in range(E):
            addrs = [seq_base(L, g) + csw(L, t + m * T) for g, t in lanes]
            assert phases_conflict_free(addrs), (L, W, m)


@pytest.mark.parametrize("W", [1, 2])
@pytest.mark.parametrize("L", SIZES)
def test_global_accesses_of_a_warp_are_contiguous_runs(L, W):
    """In the first and last stage a warp reads / writes, per component and
    m, the elements x2 = t + m T of its columns; with interleaved lanes the
    two columns of a tile give one contiguous run of eight-byte numbers."""
    E = col_e(L)
    T = L // E
    cpc, nt, inter = cfg(L, W)
    for w0 in range(0, nt, 32):
        lanes = [lane_map(L, W, tid) for tid in range(w0, w0 + 32)]
        for m in range(E):
            # element index within the tiled layout: x2 W + w for column w
            # of a tile; the lanes of one tile (pair of columns) form one run
            by_tile = {}
            for g, t in lanes:
                by_tile.setdefault(g // W, []).append((t + m * T) * W + (g % W))
            for idx in by_tile.values():
                if inter:
                    assert idx == list(range(idx[0], idx[0] + len(idx))) and len(idx) >= 16, (L, W, m)


# --------------------------------------------------------------------------
# the register-staged row pass (csrc/rowrs.cuh): half-length plan, twists on
# digit-reversed positions, shared-memory banks of its patterns
# --------------------------------------------------------------------------
ROW_SIZES = [256, 512, 1024, 2048, 4096]  # lattice sides L; M = L / 2


def plan16(N, ra, rb):
    radix = [ra] + ([rb] if N > ra else [])
    while np.prod(radix) < N:
        radix.append(16)
    assert np.prod(radix) == N
    nlen = [N]
    for s in range(1, len(radix)):
        nlen.append(nlen[-1] // radix[s - 1])
    stride = [n // r for n, r in zip(nlen, radix)]
    return radix, nlen, stride


def row_plan(M):
    lg = M.bit_length() - 1
    if lg % 4 == 0:
        return plan16(M, 4, 4)
    return plan16(M, 1 << (lg % 4), 16)


def p16_freq(pl, p):
    radix, nlen, stride = pl
    m, w = 0, 1
    for s in range(len(radix)):
        m += ((p // stride[s]) % radix[s]) * w
        w *= radix[s]
    return m


def p16_pos(pl, m):
    radix, nlen, stride = pl
    p = 0
    for s in range(len(radix)):
        p += (m % radix[s]) * stride[s]
        m //= radix[s]
    return p


def p16_butterflies(pl, s, t):
    radix, nlen, stride = pl
    T = nlen[0] // E
    out = []
    for i in range(E // radix[s]):
        u = t + i * T
        b, j = divmod(u, stride[s])
        out.append((b * nlen[s] + j, stride[s], j))
    return out


def p16_forward(pl, x):
    radix, nlen, stride = pl
    a = x.astype(np.complex128).copy()
    for s in range(len(radix)):
        R, N = radix[s], nlen[s]
        for t in range(nlen[0] // E):
            for base, d, j in p16_butterflies(pl, s, t):
                idx = base + d * np.arange(R)
                v = a[idx]
                y = np.array([np.sum(v * np.exp(-2j * np.pi * np.arange(R) * k / R)) for k in range(R)])
                a[idx] = y * np.exp(-2j * np.pi * j * np.arange(R) / N)
    return a


def p16_inverse(pl, a):
    radix, nlen, stride = pl
    a = a.copy()
    for s in reversed(range(len(radix))):
        R, N = radix[s], nlen[s]
        for t in range(nlen[0] // E):
            for base, d, j in p16_butterflies(pl, s, t):
                idx = base + d * np.arange(R)
                v = a[idx] * np.exp(2j * np.pi * j * np.arange(R) / N)
                a[idx] = np.array([np.sum(v * np.exp(2j * np.pi * np.arange(R) * r / R)) for r in range(R)])
    return a


def twist(pl, L, s, fwd):
    """The pair twist of rrs_twist on the digit-reversed sequence s
    (position q holds frequency freq(q)); returns a new array."""
    M = L // 2
    T = M // E
    out = s.copy()
    done = np.zeros(M, int)
    for t in range(T):
        for j in range(E):
            q = t + j * T
            k = p16_freq(pl, q)
            if k == 0:
                z = s[q]
                out[q] = (z.real + z.imag) + 1j * (z.real - z.imag)
                done[q] += 1
                continue
            q2 = p16_pos(pl, M - k)
            if q2 < q:
                continue
            w = np.exp(-2j * np.pi * k / L)
            if not fwd:
                w = np.conj(w)
            a, b = s[q], s[q2]
            tt = w * (a - np.conj(b))
            if fwd:
                out[q] = 0.5 * ((a + np.conj(b)) - 1j * tt)
                if q2 != q:
                    out[q2] = 0.5 * ((b + np.conj(a)) - 1j * np.conj(tt))
            else:
                out[q] = (a + np.conj(b)) + 1j * tt
                if q2 != q:
                    out[q2] = (b + np.conj(a)) + 1j * np.conj(tt)
            done[q] += 1
            done[q2] += q2 != q
    assert (done == 1).all()  # every position by exactly one thread
    return out


@pytest.mark.parametrize("L", [64, 128, 256, 512, 1024])
def test_row_transform_replay_against_numpy(L):
    """Packed half spectrum of a real row, stored digit-reversed -> inverse
    twist -> inverse stages gives x(2n) + i x(2n+1) (times M); the forward
    stages and twist give the packed half spectrum back (times M)."""
    M = L // 2
    pl = row_plan(M)
    rng = np.random.default_rng(L)
    x = rng.standard_normal(L)
    X = np.fft.fft(x)
    packed = X[:M].copy()
    packed[0] = X[0].real + 1j * X[M].real
    order = np.array([p16_freq(pl, q) for q in range(M)])
    stored = packed[order]  # position q holds frequency freq(q)
    z = p16_inverse(pl, twist(pl, L, stored, fwd=False))
    # the inverse is unnormalised and its twist carries no factor 1/2, so z
    # is L (x(2n) + i x(2n+1)), as for the full-length unnormalised inverse
    np.testing.assert_allclose(z, 2 * M * (x[0::2] + 1j * x[1::2]), rtol=0, atol=1e-9 * L * np.abs(x).max())
    back = twist(pl, L, p16_forward(pl, x[0::2] + 1j * x[1::2]), fwd=True)
    np.testing.assert_allclose(back, stored, rtol=0, atol=1e-9 * np.abs(X).max())


def row_cfg(L):
    M = L // 2
    T = M // E
    RR = 16 if L <= 256 else (8 if L == 512 else (4 if L == 1024 else 2))
    return M, T, RR, (1 if L == 256 else 2), 3 * M + 16


def row_base(L, rr):
    M, T, RR, W, RS = row_cfg(L)
    return rr * RS + ((rr * (16 // RR)) & 15 if T >= 16 else (rr >> 1) + 8 * (rr & 1))


def wavefronts(addrs):
    """Shared-memory wavefronts of one warp's eight-byte accesses: per
    half-warp phase, the largest number of distinct elements on one bank
    pair."""
    n = 0
    for h in (0, 16):
        per = {}
        for a in addrs[h:h + 16]:
            if a is not None:
                per.setdefault(a % 16, set()).add(a)
        n += max((len(v) for v in per.values()), default=0)
    return n


@pytest.mark.parametrize("L", ROW_SIZES)
def test_row_pass_banks(L):
    """FFT stages, stage-1 positions, the twist's own positions and the
    transposing spectrum load and store are conflict-free; the twist
    partners (the lane order reversed) cost at most 4 wavefronts."""
    M, T, RR, W, RS = row_cfg(L)
    pl = row_plan(M)
    radix = pl[0]
    NT = RR * T
    worst_partner = 0
    for w0 in range(0, NT, 32):
        lanes = [divmod(tid, T) for tid in range(w0, w0 + 32)]
        for s in range(len(radix)):
            per = [(rr, p16_butterflies(pl, s, t)) for rr, t in lanes]
            for i in range(E // radix[s]):
                for r in range(radix[s]):
                    addrs = [row_base(L, rr) + sw(b[i][0] + r * b[i][1]) for rr, b in per]
                    assert wavefronts(addrs) == 2, (L, s, i, r)
        for j in range(E):
            own = [row_base(L, rr) + sw(t + j * T) for rr, t in lanes]
            assert wavefronts(own) == 2, (L, j)
            part = []
            for rr, t in lanes:
                k = p16_freq(pl, t + j * T)
                part.append(row_base(L, rr) + sw(p16_pos(pl, (M - k) % M)) if k else None)
            worst_partner = max(worst_partner, wavefronts(part))
    assert worst_partner <= 4, worst_partner
    # the transposing load / store: consecutive threads take consecutive
    # numbers of a tile chunk (RR rows x W columns)
    for w0 in range(0, 3 * M * RR, 32):
        addrs = []
        for e in range(w0, w0 + 32):
            chunk, within = divmod(e, RR * W)
            c, b = divmod(chunk, M // W)
            rr, w = divmod(within, W)
            addrs.append(row_base(L, rr) + c * M + sw(b * W + w))
        assert wavefronts(addrs) == 2, (L, w0, wavefronts(addrs))


@pytest.mark.parametrize("W", [1, 2])
@pytest.mark.parametrize("L", SIZES)
def test_column_pass_addresses_stay_inside_their_buffers(L, W):
    """Every shared-memory element a column-pass CTA touches (three
    components of each of its column groups, every stage's positions) lies
    inside its allocation of CPC (3 L + 8) elements, and every spectrum
    element it reads or writes, over the whole grid of L/2 / CPC CTAs, lies
    inside the 3 L (L/2) numbers of the solve's spectrum."""
    radix, nlen, stride = plan(L)
    T, M = L // col_e(L), L // 2
    cpc, nt, inter = cfg(L, W)
    smem = cpc * (3 * L + 8)
    top_s = -1
    for tid in range(nt):
        g, t = lane_map(L, W, tid)
        assert 0 <= g < cpc and 0 <= t < T
        for s in range(len(radix)):
            for base, d, j in butterflies(L, s, t):
                for r in range(radix[s]):
                    p = base + r * d
                    assert 0 <= p < L
                    top_s = max(top_s, seq_base(L, g) + 2 * L + csw(L, p))
    assert top_s < smem, (top_s, smem)
    nbk = M // W
    top_g = -1
    for bx in range(M // cpc):
        for g in range(cpc):
            p1 = bx * cpc + g
            bt, w = divmod(p1, W)
            # component 2, x2 = L - 1: the largest element of the column
            top_g = max(top_g, ((2 * nbk + bt) * L + L - 1) * W + w)
    assert top_g == 3 * L * M - 1


@pytest.mark.parametrize("L", ROW_SIZES)
def test_row_pass_addresses_stay_inside_their_buffers(L):
    """The register-staged row pass: shared-memory elements of its RR rows
    (three components of M positions each, per-row bank offset) stay inside
    RR (3 M + 16) elements, and the transposing load / store of the tile,
    over the whole grid of L / RR CTAs, stays inside the spectrum."""
    M, T, RR, W, RS = row_cfg(L)
    assert all(row_base(L, rr) - rr * RS < 16 for rr in range(RR))
    top_s = max(row_base(L, rr) + 2 * M + sw(q) for rr in range(RR) for q in range(M))
    assert top_s < RR * RS, (top_s, RR * RS)
    nbk = M // W
    top_g = -1
    for bx in range(L // RR):
        r0 = bx * RR
        e = 3 * M * RR - 1  # the largest tile element of the CTA
        chunk, within = divmod(e, RR * W)
        c, b = divmod(chunk, nbk)
        rr, w = divmod(within, W)
        assert c < 3 and b < nbk and rr < RR
        top_g = max(top_g, ((c * nbk + b) * L + r0 + rr) * W + w)
    assert top_g == 3 * L * M - 1
