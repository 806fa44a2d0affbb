// The two fused passes of one augmented-Lagrangian iteration and their
// helpers.
//
// Spectrum layout (per solve): 3 components (11, 22, 12) of the half
// spectrum along x1, packed: element m1 = 0 holds X(0) + i X(L/2) (both real
// after a real row transform), m1 = 1 .. L/2-1 hold X(m1).  After the column
// pass the same layout holds the column-transformed data.  In HBM it is
// tiled by W columns: index ((c * L/(2W) + b) * L + x2) * W + w for column
// m1 = b * W + w, so a column pass CTA reads one contiguous slab and a row
// pass CTA reads RR * W contiguous complex numbers per slab.
//
// Row pass (iteration n -> n+1, one CTA per RR rows):
//   inverse row transform of e^{n+1} -> pixelwise: sigma^n (the multiplier,
//   stored by the pass that produced eps^n), tau = sigma^n + C0:e^{n+1},
//   local step -> eps^{n+1} and its stress sigma^{n+1} (both stored),
//   p^{n+1} = sigma^{n+1} - C0:eps^{n+1} -> forward row transform.  The
//   residual of iterate n (backward divergence of Eq. 1 of sigma^n, with a
//   halo row) and the means are summed per CTA (FP64, or error-free FP32
//   pairs promoted to FP64); the last CTA of a solve finalizes the
//   indicators of Sec. 2 and advances the solve.
// Column pass (one CTA per W columns): forward column transform, the Green
//   operator of Eq. 3 per frequency (scaled by 1/L^2, mean strain at q = 0),
//   inverse column transform.
#pragma once
#include "common.cuh"
#include "fft.cuh"
#include "physics.cuh"
#include "tables.cuh"

namespace epfft {

// Tiling of one lattice size in one precision.  Two variants per size are
// compiled; the autotuner times both on the device and keeps the faster.
//   V = 0: fewer, larger CTAs (RR rows x W columns of a tile row span >= 64
//          bytes of HBM, so each CTA streams long contiguous runs);
//   V = 1: more, smaller CTAs (several per SM hide memory latency; short
//          runs rely on the L2 to merge neighbouring CTAs' accesses).
// Shared memory of a pass: its sequences (padded, fft.cuh), then its stage
// table, then (row pass) the twist octant.
template <typename T, int L, int V = 0>
struct Cfg {
  static constexpr bool F64 = sizeof(T) == 8;
  static constexpr int M = L / 2;
  using PS = PlanSel<T, L, V>;
  using PR = typename PS::PR;
  using PC = typename PS::PC;
  using TB = Tables<T, L>;
  static constexpr int RM_ROW = PS::RM_ROW, RM_COL = PS::RM_COL;
  static constexpr bool FULL = PS::FULL;
  // rows per row-pass CTA
  static constexpr int RR = V == 0 ? (F64 ? 2 : (L <= 256 ? 2 : (L == 512 ? 4 : (L <= 2048 ? 8 : 4))))
                                   : (F64 ? (L <= 256 || L == 4096 ? 1 : 2) : (L <= 256 ? 1 : 2));
  // columns per column-pass CTA (= tile width of the spectrum layout)
  static constexpr int W0 = V == 0 ? (F64 ? (L <= 256 ? 1 : (L <= 1024 ? 2 : 1))
                                          : (L == 2048 ? 1 : 2))
                                   : (F64 ? 1 : (L <= 256 ? 1 : (L <= 1024 ? 2 : (L <= 2048 ? 1 : 2))));
  static constexpr int W = W0 < M ? W0 : M;
  static constexpr int NTMAX = V == 0 ? 512 : 256;
  // resident CTAs per SM asked of the compiler: FP32 variant 1 (at most 128
  // registers per thread at 256 threads), the FP32 L = 512 row pass of
  // variant 0 (four CTAs of 4 rows and 256 threads at 64 registers, no
  // spills: 307 us at 64 x L = 512 against 337 us for two CTAs of 8 rows
  // and 512 threads, whose 16-warp barriers and tile waits overlapped
  // less) and the FP32 column
  // passes of the narrow tiles of variant 0 at L = 512 .. 2048: 768 threads
  // per SM at L = 512 (85 registers, no spills), three CTAs of 384 at
  // L = 1024 and 2048 (56 registers), so that the CTAs of an SM overlap
  // their loads with the others' transforms
  static constexpr int MINB_ROW = !F64 && (V == 1 || L == 512) ? (V == 0 ? 4 : 2) : 1;
  static constexpr int NT_ROW0 = F64 ? (L > 512 ? 256 : (L < 128 ? L : 128))
                                     : (L <= 256 ? L : (V == 0 && L == 512 ? 256 : NTMAX));
  static constexpr int NT_ROW = NT_ROW0 < 32 ? 32 : NT_ROW0;
  static constexpr int NT_COL0 = ((3 * W * L / RM_COL + 31) / 32) * 32;
  static constexpr int NT_COL = NT_COL0 < 32 ? 32 : (NT_COL0 > NTMAX ? NTMAX : NT_COL0);
  static constexpr int MINB_COL = F64 ? 1
                                      : V == 1 ? 2 : (L == 512 ? 768 / NT_COL : (L == 1024 || L == 2048 ? 3 : 1));
  // sequences transformed per call: the largest divisor of the sequence
  // count that keeps at most 16 elements per thread and stage
  static constexpr int grp(int S, int N, int NT) {
    int g = S;
    while (g > 1 && (S % g != 0 || g * N > 16 * NT)) g--;
    return g;
  }
  static constexpr int SP_R = seq_stride<M>(), SP_C = seq_stride<L>();
  static constexpr int G_R = grp(3 * RR, M, NT_ROW), G_C = grp(3 * W, L, NT_COL);
  static constexpr int ROW_DATA = (3 * RR * SP_R + 1) / 2 * 2;
  static constexpr int COL_DATA = (3 * W * SP_C + 1) / 2 * 2;
  static constexpr int ROW_TW = PR::TW_ENTRIES, COL_TW = PC::TW_ENTRIES;
  static constexpr size_t ROW_SMEM = (size_t)(ROW_DATA + ROW_TW + TB::OCT) * sizeof(C2<T>);
  static constexpr size_t COL_SMEM = (size_t)(COL_DATA + COL_TW) * sizeof(C2<T>);
  static_assert(L >= 4 && (L & (L - 1)) == 0, "L must be a power of two >= 4");
  static_assert(M % W == 0, "tile width must divide L/2");
  static_assert(L % RR == 0, "rows per CTA must divide L");
  // 227 KB per CTA, less the static arrays of the row pass
  static_assert(ROW_SMEM <= 222000 && COL_SMEM <= 230000, "shared memory per CTA");
  static_assert(NT_ROW % 32 == 0 && NT_COL % 32 == 0, "whole warps");
  static_assert(L <= NT_ROW || L % NT_ROW == 0, "pixel mapping");
  static_assert(G_R * M <= 16 * NT_ROW && G_C * L <= 16 * NT_COL, "elements per thread and stage");
};

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  static __device__ __forceinline__ void load(const float* p, float e[4]) {
    float4 v = *reinterpret_cast<const float4*>(p);
    e[0] = v.x; e[1] = v.y; e[2] = v.z; e[3] = v.w;
  }
  static __device__ __forceinline__ void store(float* p, const float e[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(e[0], e[1], e[2], e[3]);
  }
};
template <>
struct Vec4<double> {
  static __device__ __forceinline__ void load(const double* p, double e[4]) {
    double2 a = reinterpret_cast<const double2*>(p)[0];
    double2 b = reinterpret_cast<const double2*>(p)[1];
    e[0] = a.x; e[1] = a.y; e[2] = b.x; e[3] = b.y;
  }
  static __device__ __forceinline__ void store(double* p, const double e[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(e[0], e[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(e[2], e[3]);
  }
};

// ---------------------------------------------------------------------------
// Row-side helpers.  Shared memory holds 3 x RR sequences of length M
// (sequence c * RR + r = component c of row r, padded layout of fft.cuh),
// then the row plan's stage table, then the twist octant.
// ---------------------------------------------------------------------------
template <typename T, int L, int V>
struct RowIO {
  using C = Cfg<T, L, V>;
  static constexpr int M = L / 2, RR = C::RR, W = C::W, NT = C::NT_ROW, NBK = M / W;
  static constexpr int SP = C::SP_R, NSEQ = 3 * RR;
  static constexpr int SZ = C::ROW_DATA;

  // shared index of element n of component c of row r
  static __device__ __forceinline__ int at(int c, int r, int n) { return (c * RR + r) * SP + pad32(n); }

  // Chunk element e (c, b, r, w) of the RR rows: shared and global index.
  // For e < 3 M RR (c < 3, b < M / W, r < RR, w < W) and rows r0 + r < L
  // (a pass over L rows has L / RR CTAs per solve), is < 3 RR SP <= SZ and
  // ig < 3 M L; builds with self-checks verify both at every access.
  static __device__ __forceinline__ void where(int e, int r0, int& is, size_t& ig) {
    const int c = e / (M * RR);
    const int rem = e - c * (M * RR);
    const int b = rem / (RR * W);
    const int rem2 = rem - b * (RR * W);
    const int r = rem2 / W, w = rem2 - r * W;
    is = at(c, r, b * W + w);
    ig = ((size_t)(c * NBK + b) * L + r0 + r) * W + w;
  }
  // FP32 complex numbers are stored two at a time (16-byte accesses) when a
  // tile chunk (RR x W numbers, contiguous in HBM) has even length.
  static constexpr bool PAIRS = sizeof(C2<T>) == 8 && (RR * W) % 2 == 0;

  // Issues the asynchronous copies of the RR rows' spectrum into shared
  // memory (complete with cp_async_wait_all() and a barrier): consecutive
  // threads take consecutive numbers of the tile chunks, so a warp reads
  // 32 consecutive numbers of HBM, and the whole tile is in flight at once.
  // Fixed pattern of the copies: when a step of S consecutive elements
  // (S = NT numbers, or 2 NT numbers for the pair stores) covers whole tile
  // chunks and divides a component's M RR numbers, and S / RR is a multiple
  // of 32, element e = E0 + k S of a thread (E0 = tid, or 2 tid) has
  // c = k / KPC and b = E0 / (RR W) + (k mod KPC) S / (RR W) (KPC = M RR / S),
  // while r and w depend on E0 alone; so where(e) is where(E0) plus
  // c RR SP + j (S / RR + S / (32 RR)) in shared memory (pad32 adds one slot
  // per 32 elements) and (c NBK + j S / (RR W)) L W in the spectrum
  // (j = k mod KPC), offsets known at compile time.  The steps are unrolled
  // completely, so the pattern is taken up to 24 steps per thread (64 x
  // L = 512: 307 -> 300 us; at L = 4096, 48 steps, the loop measured faster).
  template <int S>
  static __host__ __device__ constexpr bool fixed() {
    return S % (RR * W) == 0 && (M * RR) % S == 0 && (S / RR) % 32 == 0 && 3 * M * RR / S <= 24;
  }
  template <int S, int k>
  static __host__ __device__ constexpr int fixed_is() {
    return (k / ((M * RR) / S)) * RR * SP + (k % ((M * RR) / S)) * (S / RR + S / (32 * RR));
  }
  template <int S, int k>
  static __host__ __device__ constexpr size_t fixed_ig() {
    return ((size_t)(k / ((M * RR) / S)) * NBK + (size_t)(k % ((M * RR) / S)) * (S / (RR * W))) * L * W;
  }
  static __device__ __forceinline__ void load_async(C2<T>* sp, const C2<T>* __restrict__ spec, int r0) {
    if constexpr (fixed<NT>()) {
      int is0;
      size_t ig0;
      where(threadIdx.x, r0, is0, ig0);
      load_fixed<0>(sp, spec, is0, ig0);
    } else {
#pragma unroll 4
      for (int e = threadIdx.x; e < 3 * M * RR; e += NT) {
        int is;
        size_t ig;
        where(e, r0, is, ig);
        if (ECHK(is, SZ, 1) && ECHK(ig, (size_t)3 * M * L, 2)) cp_async_c2(sp + is, spec + ig);
      }
    }
  }
  template <int k>
  static __device__ __forceinline__ void load_fixed(C2<T>* sp, const C2<T>* __restrict__ spec, int is0, size_t ig0) {
    if constexpr (k < 3 * M * RR / NT) {
      const int is = is0 + fixed_is<NT, k>();
      const size_t ig = ig0 + fixed_ig<NT, k>();
      if (ECHK(is, SZ, 1) && ECHK(ig, (size_t)3 * M * L, 2)) cp_async_c2(sp + is, spec + ig);
      load_fixed<k + 1>(sp, spec, is0, ig0);
    }
  }
  // the pair of numbers at shared index is0 and global index ig0 (see store)
  static __device__ __forceinline__ void store_pair(const C2<T>* sp, C2<T>* __restrict__ spec, int is0, size_t ig0) {
    // the pair's second number: w + 1 of the same row (W >= 2, w even,
    // so b W + w + 1 is no multiple of 32 and the padding adds nothing)
    // or, for W = 1, the same column of the next row
    const int is1 = is0 + (W >= 2 ? 1 : SP);
    if (ECHK(is0, SZ, 3) && ECHK(is1, SZ, 3) && ECHK(ig0 + 1, (size_t)3 * M * L, 4) && ECHK(ig0 & 1, 1, 5)) {
      const float2 a = reinterpret_cast<const float2*>(sp)[is0];
      const float2 b = reinterpret_cast<const float2*>(sp)[is1];
      *reinterpret_cast<float4*>(spec + ig0) = make_float4(a.x, a.y, b.x, b.y);
    }
  }
  template <int k>
  static __device__ __forceinline__ void store_fixed(const C2<T>* sp, C2<T>* __restrict__ spec, int is0, size_t ig0) {
    if constexpr (k < 3 * M * RR / (2 * NT)) {
      store_pair(sp, spec, is0 + fixed_is<2 * NT, k>(), ig0 + fixed_ig<2 * NT, k>());
      store_fixed<k + 1>(sp, spec, is0, ig0);
    }
  }
  static __device__ __forceinline__ void store(const C2<T>* sp, C2<T>* __restrict__ spec, int r0) {
    if constexpr (PAIRS && fixed<2 * NT>()) {
      int is0;
      size_t ig0;
      where(2 * threadIdx.x, r0, is0, ig0);
      store_fixed<0>(sp, spec, is0, ig0);
    } else if constexpr (PAIRS) {
#pragma unroll 4
      for (int e2 = threadIdx.x; e2 < 3 * M * RR / 2; e2 += NT) {
        int is0;
        size_t ig0;
        where(2 * e2, r0, is0, ig0);
        store_pair(sp, spec, is0, ig0);
      }
    } else {
#pragma unroll 4
      for (int e = threadIdx.x; e < 3 * M * RR; e += NT) {
        int is;
        size_t ig;
        where(e, r0, is, ig);
        if (ECHK(is, SZ, 3) && ECHK(ig, (size_t)3 * M * L, 4)) spec[ig] = sp[is];
      }
    }
  }
  // Half spectrum (packed) -> Z for the half-length inverse transform:
  // Z(k) = (Y(k) + Y*(M-k)) + i exp(+2 pi i k / L) (Y(k) - Y*(M-k)),
  // with Y(0) = Re S(0), Y(M) = Im S(0).  Unnormalised: the inverse
  // half-length transform of Z then yields x(2n) + i x(2n+1) of
  // x(x1) = sum_m Y(m) exp(+2 pi i m x1 / L).  Consecutive threads take
  // consecutive k of one sequence.
  static __device__ __forceinline__ void c2r_twist(C2<T>* sp, const C2<T>* __restrict__ oct) {
    auto pair = [&](int k, int sq0, int ds) {
      const int kk = M - k;
      const int ik = pad32(k), ikk = pad32(kk);  // 0 < k, kk < M
      const C2<T> wk = conj(twist_tw<T, L>(oct, k));
      for (int sq = sq0; sq < NSEQ; sq += ds) {
        C2<T>* s = sp + sq * SP;
        if (!ECHK(sq * SP + ikk, SZ, 38) || !ECHK(sq * SP + ik, SZ, 38)) continue;
        const C2<T> a = s[ik], b = s[ikk];
        // the partner's product conj(wk) (b - conj(a)) equals -conj(t)
        const C2<T> t = wk * (a - conj(b));
        s[ik] = (a + conj(b)) + mul_i(t);
        if (kk != k) s[ikk] = (b + conj(a)) + mul_i(conj(t));
      }
    };
    visit_pairs(pair);
    pack0(sp);
  }
  // Z = transform of z(n) = x(2n) + i x(2n+1) -> packed half spectrum of x:
  // X(k) = [(Z(k) + Z*(M-k)) - i exp(-2 pi i k / L) (Z(k) - Z*(M-k))] / 2,
  // S(0) = X(0) + i X(M).
  static __device__ __forceinline__ void r2c_twist(C2<T>* sp, const C2<T>* __restrict__ oct) {
    auto pair = [&](int k, int sq0, int ds) {
      const int kk = M - k;
      const int ik = pad32(k), ikk = pad32(kk);  // 0 < k, kk < M
      const C2<T> wk = twist_tw<T, L>(oct, k);
      for (int sq = sq0; sq < NSEQ; sq += ds) {
        C2<T>* s = sp + sq * SP;
        if (!ECHK(sq * SP + ikk, SZ, 38) || !ECHK(sq * SP + ik, SZ, 38)) continue;
        const C2<T> a = s[ik], b = s[ikk];
        // the partner's product conj(wk) (b - conj(a)) equals -conj(t)
        const C2<T> t = wk * (a - conj(b));
        s[ik] = T(0.5) * ((a + conj(b)) - mul_i(t));
        if (kk != k) s[ikk] = T(0.5) * ((b + conj(a)) - mul_i(conj(t)));
      }
    };
    visit_pairs(pair);
    pack0(sp);
  }
  // Calls pair(k, sq0, ds) so that every (sequence, k), k = 1 .. M/2, is
  // visited once: a thread keeps one k (its twiddle read once) and walks
  // the sequences sq0, sq0 + ds, ...; consecutive threads take consecutive
  // k of one sequence.
  template <typename F>
  static __device__ __forceinline__ void visit_pairs(F&& pair) {
    constexpr int HK = M / 2;
    if constexpr (NT >= HK) {
      pair(1 + (int)(threadIdx.x % HK), (int)(threadIdx.x / HK), NT / HK);
    } else {
#pragma unroll 1
      for (int k = 1 + (int)threadIdx.x; k <= HK; k += NT) pair(k, 0, 1);
    }
  }
  // Element 0 of each sequence, both ways: (a, b) -> (a + b, a - b) (the
  // packed X(0), X(M) of the half spectrum and the Z(0) of the transform).
  // It touches no element of visit_pairs, so no barrier separates them.
  static __device__ __forceinline__ void pack0(C2<T>* sp) {
    for (int sq = threadIdx.x; sq < NSEQ; sq += NT) {
      C2<T>* s = sp + sq * SP;
      const C2<T> z = s[0];
      s[0] = mk(z.re + z.im, z.re - z.im);
    }
  }
  // Half-length transforms of all 3 RR sequences, C::G_R per call.
  template <bool INV>
  static __device__ __forceinline__ void fft(C2<T>* sp, const C2<T>* __restrict__ stw) {
    constexpr int G = C::G_R;
#pragma unroll 1
    for (int g = 0; g < NSEQ / G; g++)
      fft_seq<T, M, C::RM_ROW, C::FULL, G, NT, INV>(sp + g * G * SP, stw);
  }
  // Stage table and twist octant: global -> shared, asynchronously (complete
  // with cp_async_wait_all() and a barrier).  Returns the shared stage
  // table; the octant follows it.
  static __device__ __forceinline__ const C2<T>* load_tables(C2<T>* sp, const C2<T>* __restrict__ tab) {
    C2<T>* stw = sp + SZ;
    copy_table<T, NT>(stw, tab + C::TB::off_row(V), C::ROW_TW);
    copy_table<T, NT>(stw + C::ROW_TW, tab, C::TB::OCT);
    return stw;
  }
  static __device__ __forceinline__ const C2<T>* octant(const C2<T>* stw) { return stw + C::ROW_TW; }
  // real value of pixel x1 < L of component c < 3, row r < RR (inside the
  // data region by construction: x1 / 2 < M)
  static __device__ __forceinline__ T& px(C2<T>* sp, int c, int r, int x1) {
    return reinterpret_cast<T*>(sp)[2 * at(c, r, x1 >> 1) + (x1 & 1)];
  }
};

template <typename T>
__device__ __forceinline__ void load_E(const double* p, T E[4]) {
  E[0] = T(p[0]); E[1] = T(p[1]); E[2] = T(p[2]); E[3] = T(p[3]);
}

// FP64 sums of N_ACC values over the first NW warps of the CTA, in a fixed
// order; every thread of the CTA calls it (it holds a barrier), the threads
// i < N_ACC write sum i to out[i].  Within a warp the values (padded to 16)
// are summed by recursive halving: at the levels h = 8, 4, 2, 1 a lane keeps
// the half of its values selected by lane bit h and adds the partner's
// (lane ^ h) copy of that half; after that lane l holds value l & 15 summed
// over the 16 lanes that share bit 16, and one more exchange with lane ^ 16
// completes the warp sum.  That is 16 FP64 adds per lane, where one shuffle
// tree per value costs 5 N_ACC; FP64 adds are scarce on GB300 (about two
// per clock and SM).  Thread i then adds the warps' sums in warp order.
template <int NW>
__device__ __forceinline__ void block_sum_f64(const double* v, double* out) {
  static_assert(N_ACC <= 16, "values per reduction");
  __shared__ double red[NW][16];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid < NW) {
    double a[16];
#pragma unroll
    for (int i = 0; i < 16; i++) a[i] = i < N_ACC ? v[i] : 0.0;
#pragma unroll
    for (int h = 8; h >= 1; h >>= 1) {
      const bool up = (lane & h) != 0;
#pragma unroll
      for (int k = 0; k < h; k++) {
        const double keep = up ? a[k + h] : a[k];
        const double send = up ? a[k] : a[k + h];
        a[k] = keep + __shfl_xor_sync(0xffffffffu, send, h);
      }
    }
    const double s = a[0] + __shfl_xor_sync(0xffffffffu, a[0], 16);
    if (lane < 16) red[wid][lane] = s;
  }
  __syncthreads();
  if (threadIdx.x < N_ACC) {
    double t = red[0][threadIdx.x];
#pragma unroll
    for (int w = 1; w < NW; w++) t += red[w][threadIdx.x];
    out[threadIdx.x] = t;
  }
}

// CTA sums of the per-thread accumulators.  FP64: block_sum_f64.  FP32:
// values are added as FP32 (hi, lo) pairs with the error-free TwoSum of
// Knuth/Moller (s = a + b, e = exact rounding error of the add), first
// within each warp by the same recursive halving as block_sum_f64, then
// across the warps in warp order, so the CTA total carries about twice
// FP32 precision without FP64 work; thread i promotes the final pair of
// value i to FP64 (hi + lo).
template <int NT>
__device__ __forceinline__ void block_reduce_acc(double acc[N_ACC], double* out) {
  block_sum_f64<NT / 32>(acc, out);
}
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float bh, float bl) {
  const float sum = hi + bh;
  const float bb = sum - hi;
  const float err = (hi - (sum - bb)) + (bh - bb);
  hi = sum;
  lo = lo + bl + err;
}
template <int NT>
__device__ __forceinline__ void block_reduce_acc(float acc[N_ACC], double* out) {
  constexpr int NW = NT / 32;
  static_assert(N_ACC <= 16, "values per reduction");
  __shared__ float red2[NW][16][2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // recursive halving over 16 slots (as block_sum_f64), each add a TwoSum
  // of (hi, lo) pairs: lane l ends with slot l & 15 of the warp
  float hi[16], lo[16];
#pragma unroll
  for (int i = 0; i < 16; i++) {
    hi[i] = i < N_ACC ? acc[i] : 0.0f;
    lo[i] = 0.0f;
  }
#pragma unroll
  for (int h = 8; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int k = 0; k < h; k++) {
      const float kh = up ? hi[k + h] : hi[k], kl = up ? lo[k + h] : lo[k];
      const float sh = up ? hi[k] : hi[k + h], sl = up ? lo[k] : lo[k + h];
      const float bh = __shfl_xor_sync(0xffffffffu, sh, h);
      const float bl = __shfl_xor_sync(0xffffffffu, sl, h);
      hi[k] = kh;
      lo[k] = kl;
      two_sum_add(hi[k], lo[k], bh, bl);
    }
  }
  {
    const float bh = __shfl_xor_sync(0xffffffffu, hi[0], 16);
    const float bl = __shfl_xor_sync(0xffffffffu, lo[0], 16);
    two_sum_add(hi[0], lo[0], bh, bl);
  }
  if (lane < 16) {
    red2[wid][lane][0] = hi[0];
    red2[wid][lane][1] = lo[0];
  }
  __syncthreads();
  if (threadIdx.x < N_ACC) {
    float h = red2[0][threadIdx.x][0], l = red2[0][threadIdx.x][1];
#pragma unroll
    for (int w = 1; w < NW; w++) two_sum_add(h, l, red2[w][threadIdx.x][0], red2[w][threadIdx.x][1]);
    out[threadIdx.x] = (double)h + (double)l;
  }
}

// Sums of the NREC per-CTA partial records of a solve, computed by the last
// CTA: the first NWA warps (enough for one record per thread, at most all
// warps) take records t, t + 32 NWA, ..., loading up to two records per
// thread before adding them, then block_sum_f64 combines the threads; the
// order is fixed, so the result does not depend on timing.
template <int NT, int NREC>
__device__ __forceinline__ void sum_partials(const double* partials, double* out) {
  constexpr int NW = NT / 32, NWR = (NREC + 31) / 32;
  constexpr int NWA = NWR < NW ? NWR : NW, NTA = 32 * NWA;
  constexpr int K = (NREC + NTA - 1) / NTA, KC = K < 2 ? K : 2, NV = (N_ACC + 1) / 2;
  static_assert(PART_STRIDE % 2 == 0 && PART_STRIDE >= 2 * NV, "record layout");
  double v[N_ACC];
#pragma unroll
  for (int i = 0; i < N_ACC; i++) v[i] = 0.0;
  if (threadIdx.x < NTA) {
#pragma unroll 1
    for (int k0 = 0; k0 < K; k0 += KC) {
      double2 x[KC][NV];
#pragma unroll
      for (int k = 0; k < KC; k++) {
        const int b = threadIdx.x + (k0 + k) * NTA;
#pragma unroll
        for (int i = 0; i < NV; i++)
          x[k][i] = b < NREC ? __ldcg(reinterpret_cast<const double2*>(partials + (size_t)b * PART_STRIDE) + i)
                             : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int k = 0; k < KC; k++)
#pragma unroll
        for (int i = 0; i < N_ACC; i++) v[i] += (i & 1) ? x[k][i / 2].y : x[k][i / 2].x;
    }
  }
  block_sum_f64<NWA>(v, out);
}

// Last CTA of a solve's row pass: indicators of Sec. 2 and the state
// machine.  Runs on one thread; A holds the sums of the partials (ITER).
// The indicators are eta1 = sqrt(div2 / ss), eta2 = sqrt(dd / ss) and
// eta3 = sqrt(comp / EE); the stopping tests compare the squares scaled by
// the denominators (div2 < tol^2 ss, ...), so an iteration takes no FP64
// division or root, and the roots are formed once, for the record.
template <int L>
__device__ __forceinline__ void finalize_solve(Solve& S, int phase, const double* A) {
  constexpr double inv = 1.0 / ((double)L * (double)L);  // exact: L is a power of two
  if (phase == PH_INIT) {
    const double* E = S.path + 4 * S.inc;
    for (int c = 0; c < 4; c++) {
      S.Eprev[c] = E[c];
      S.epsm_next[c] = A[A_E11 + c] * inv;
    }
    S.npl_next = A[A_NPL];
    S.cur = 1 - S.cur;
    S.iter = 0;
    S.phase = PH_ITER;
    return;
  }
  if (phase == PH_FINAL) {
    S.phase = PH_DONE;
    return;
  }
  // A holds sigma sums and the residual of iterate n, and the strain sums,
  // plastic count and fixed-point residual of iterate n + 1 (the pass
  // produced it); <eps> and the plastic count of iterate n come from the
  // previous pass
  double sig[4];
  for (int c = 0; c < 4; c++) sig[c] = A[A_S11 + c] * inv;
  const double div2 = A[A_DIV2] * inv, comp = A[A_COMP] * inv;
  const int n = S.iter;
  S.total_iters += 1;
  if (n >= 1) {
    const double* E = S.path + 4 * S.inc;
    double EE = E[0] * E[0] + E[1] * E[1] + E[2] * E[2] + 2.0 * E[3] * E[3];
    if (EE == 0.0) EE = 1.0;
    const double ss = sig[0] * sig[0] + sig[1] * sig[1] + 2.0 * sig[3] * sig[3];
    double ds[4];
    for (int c = 0; c < 4; c++) ds[c] = sig[c] - S.sig_prev[c];
    const double dd = ds[0] * ds[0] + ds[1] * ds[1] + 2.0 * ds[3] * ds[3];
    const double comp_n = S.comp_cur;
    // eta1 and eta2 are finite when ss > 0, and 0 (else infinite) when
    // ss = 0 and the numerator is 0
    const bool finite = isfinite(div2) && isfinite(dd) && isfinite(sig[0]) && isfinite(sig[1]) &&
                        isfinite(sig[3]) && (ss > 0.0 || (div2 == 0.0 && dd == 0.0));
    const double te2 = S.tol_eq * S.tol_eq, tm2 = S.tol_macro * S.tol_macro;
    const bool pos = ss > 0.0;
    // equilibrium test: eta1 for the operators of Eq. 3; the continuum and
    // symmetrized operators are not Green operators of Eq. 1, so there (and
    // for every operator when the caller asks for one criterion) the
    // fixed-point residual eta3 of the iterate takes its place
    const bool eq_ok = S.eq_fixed_point
                           ? (comp_n < te2 * EE && S.tol_eq > 0.0)
                           : (pos ? div2 < te2 * ss : S.tol_eq > 0.0);
    const bool conv = finite && eq_ok && (pos ? dd < tm2 * ss : S.tol_macro > 0.0);
    if (!finite || conv || n >= S.max_iter) {
      double eta1, eta2;
      if (pos) {
        eta1 = sqrt(div2 / ss);
        eta2 = sqrt(dd / ss);
      } else {
        eta1 = div2 == 0.0 ? 0.0 : CUDART_INF;
        eta2 = dd == 0.0 ? 0.0 : CUDART_INF;
      }
      Record& R = S.rec[S.inc];
      for (int c = 0; c < 4; c++) {
        R.sig_mean[c] = sig[c];
        R.eps_mean[c] = S.epsm_next[c];
      }
      R.eta1 = eta1;
      R.eta2 = eta2;
      R.eta3 = sqrt(comp_n / EE);
      R.iterations = n;
      R.n_plastic = (int32_t)S.npl_next;
      R.n_clusters = 0;
      R.status = !finite ? 2 : (conv ? 0 : 1);
      if (!finite) {
        S.status = 2;
        S.phase = PH_DONE;
      } else if (S.inc + 1 < S.n_inc) {
        S.inc += 1;
        S.phase = PH_INIT;  // eps^n (buffer cur) is the accepted state
      } else {
        S.phase = PH_FINAL;
      }
      return;
    }
  }
  for (int c = 0; c < 4; c++) {
    S.sig_prev[c] = sig[c];
    S.epsm_next[c] = A[A_E11 + c] * inv;
  }
  S.npl_next = A[A_NPL];
  S.comp_cur = comp;
  S.iter = n + 1;
  S.cur = 1 - S.cur;
}

// After every CTA of the row pass: the last one decides whether the
// device-side loop runs another step (condition of the graph's while node).
__device__ __forceinline__ void batch_arrive(Solve* solves, int nb, BatchCtl* bc,
                                             cudaGraphConditionalHandle cond, int use_cond) {
  __threadfence();
  const unsigned total = gridDim.x * gridDim.y;
  const unsigned prev = atomicAdd(&bc->arrive, 1u);
  if (prev == total - 1) {
    __threadfence();
    int active = 0, waiting = 0;
    for (int i = 0; i < nb; i++) {
      const int ph = *(volatile int32_t*)&solves[i].phase;
      active += ph != PH_DONE;
      waiting += ph == PH_REF;
    }
    bc->active = active;
    bc->waiting = waiting;
    bc->body_iters += 1;
    // a solve waiting for its refresh stops the loop (the host runs it)
    const bool go = active > 0 && waiting == 0 && bc->body_iters < bc->max_body_iters;
    if (active > 0 && waiting == 0 && bc->body_iters >= bc->max_body_iters) bc->timed_out = 1;
    if (use_cond) cudaGraphSetConditional(cond, go ? 1u : 0u);
    bc->arrive = 0;
    __threadfence();
  }
}

// ---------------------------------------------------------------------------
// Row pass
// ---------------------------------------------------------------------------
template <typename T, int L, int V>
__global__ void __launch_bounds__(Cfg<T, L, V>::NT_ROW, Cfg<T, L, V>::MINB_ROW)
row_pass(Solve* __restrict__ solves, int nb, BatchCtl* bc, const C2<T>* __restrict__ tw,
         cudaGraphConditionalHandle cond, int use_cond) {
  using C = Cfg<T, L, V>;
  constexpr int RR = C::RR, W = C::W, NT = C::NT_ROW, M = C::M;
  constexpr int P = L >= NT ? L / NT : 1;
  using IO = RowIO<T, L, V>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C2<T>* sp = reinterpret_cast<C2<T>*>(smraw);
  __shared__ bool s_last;

  // Every index of the pass is in range when the grid has L / RR CTAs per
  // solve (see RowIO::where; pixel x = (r0 + r) L + x1 < L^2 for x1 < L).
  if (!ECHK(gridDim.x - 1, L / RR, 27)) return;
  Solve& S = solves[blockIdx.y];
  // The mutable control fields are rewritten by the last CTA of this launch
  // (finalize_solve); every thread reads them exactly once, through
  // volatile loads, so no later re-load can observe the new values.
  const volatile Solve& Sv = S;
  const int phase = Sv.phase;
  const int cur = Sv.cur;
  const int inc = Sv.inc;
  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  // pixel j of this thread in a row: each warp owns a contiguous run of
  // 32 P pixels, lane-fastest (L < 32: one short row per warp)
  auto xmap = [&](int j) { return L >= 32 ? wid * (32 * P) + j * 32 + lane : tid; };
  if (phase != PH_DONE) {
    const int r0 = blockIdx.x * RR;
    const T* __restrict__ ein = reinterpret_cast<const T*>(S.eps[cur]);
    T* __restrict__ eout = reinterpret_cast<T*>(S.eps[1 - cur]);
    // sigma of eps^n (read) and of the iterate this pass produces (written)
    const T* __restrict__ sin_ = reinterpret_cast<const T*>(S.sig[cur]);
    T* __restrict__ sout = reinterpret_cast<T*>(S.sig[1 - cur]);
    C2<T>* spec = reinterpret_cast<C2<T>*>(S.spec);
    const uint8_t* __restrict__ mask = S.mask;
    const Mat<T> m = make_mat<T>(S);
    const size_t LL = (size_t)L * L;
    // stage table and twist octant, in flight until the first barrier after
    // cp_async_wait_all() (INIT, ITER; the other phases do not read them)
    const C2<T>* stw = sp + C::ROW_DATA;
    if (phase == PH_INIT || phase == PH_ITER) IO::load_tables(sp, tw);
    T acc[N_ACC];
#pragma unroll
    for (int i = 0; i < N_ACC; i++) acc[i] = T(0);

    if (phase == PH_FINAL) {
      // plastic flags of the accepted state of the last increment
      uint8_t* fl = S.flags ? S.flags + (size_t)(S.n_inc - 1) * LL : nullptr;  // inc == n_inc - 1
      for (int r = 0; r < RR && fl; r++)
        for (int j = 0; j < P; j++) {
          const int x1 = xmap(j);
          if (x1 >= L) continue;
          const size_t x = (size_t)(r0 + r) * L + x1;
          T e[4];
          Vec4<T>::load(ein + 4 * x, e);
          fl[x] = is_plastic(e, mask[x] != 0, m);
        }
    } else if (phase == PH_INIT) {
      // warm start: eps^0 = accepted state + (E_inc - E_{inc-1}); p^0 -> spectrum
      T dE[4];
      const double* E = S.path + 4 * (ECHK(inc, S.n_inc, 26) ? inc : 0);
      for (int c = 0; c < 4; c++) dE[c] = T(E[c] - Sv.Eprev[c]);
      uint8_t* fl = (S.flags && inc > 0) ? S.flags + (size_t)(inc - 1) * LL : nullptr;
      for (int r = 0; r < RR; r++)
        for (int j = 0; j < P; j++) {
          const int x1 = xmap(j);
          if (x1 >= L) continue;
          const size_t x = (size_t)(r0 + r) * L + x1;
          if (!ECHK(x, LL, 20)) continue;
          const bool v = mask[x] != 0;
          T e[4], s[4], c0[4];
          Vec4<T>::load(ein + 4 * x, e);
          if (fl) fl[x] = is_plastic(e, v, m);
          for (int c = 0; c < 4; c++) e[c] += dE[c];
          Vec4<T>::store(eout + 4 * x, e);
          const bool pl = sigma(e, v, m, s);
          Vec4<T>::store(sout + 4 * x, s);
          // <eps^0> and its plastic pixels (the stats of iterate 0)
#pragma unroll
          for (int c = 0; c < 4; c++) acc[A_E11 + c] += e[c];
          acc[A_NPL] += pl ? T(1) : T(0);
          c0_apply(e, m, c0);
          IO::px(sp, 0, r, x1) = s[0] - c0[0];
          IO::px(sp, 1, r, x1) = s[1] - c0[1];
          IO::px(sp, 2, r, x1) = s[3] - c0[3];
        }
    } else {  // PH_ITER
      T E[4];
      load_E(S.path + 4 * inc, E);
      IO::load_async(sp, spec, r0);
      // sigma of the RR rows and of the halo row, and the void flags, are
      // brought into the L2 while the spectrum is transformed (16 KB pieces,
      // one per lane of warp 0, issued after the spectrum copies so that
      // those go first)
      if constexpr (L >= 64) {
        constexpr unsigned RB = (unsigned)(L * 4 * sizeof(T)), PB = RB < 16384u ? RB : 16384u;
        constexpr int NPR = (int)(RB / PB), NPC = (RR + 1) * NPR;
        if (wid == 0) {
          const int xh = (r0 + L - 1) & (L - 1);
          for (int i = lane; i < NPC; i += 32) {
            const int k = i / NPR, row = k < RR ? r0 + k : xh;
            if (ECHK(row, L, 39)) prefetch_l2(reinterpret_cast<const char*>(sin_ + (size_t)4 * row * L) + (size_t)(i % NPR) * PB, PB);
          }
          if (lane == 31) prefetch_l2(mask + (size_t)r0 * L, (unsigned)(RR * L));
        }
      }
      // halo row x2 = r0 - 1: sigma12 and sigma22 of iterate n for the
      // backward difference along x2; loaded while the spectrum is in
      // flight when the registers allow (few pixels per thread), else after
      // the transform
      T prev12[P], prev22[P];
      auto load_halo = [&]() {
        const int xh = (r0 + L - 1) & (L - 1);
#pragma unroll
        for (int j = 0; j < P; j++) {
          const int x1 = xmap(j);
          prev12[j] = prev22[j] = T(0);
          if (x1 >= L) continue;
          const size_t x = (size_t)xh * L + x1;
          if (!ECHK(x, LL, 22)) continue;
          T s[4];
          Vec4<T>::load(sin_ + 4 * x, s);
          prev12[j] = s[3];
          prev22[j] = s[1];
        }
      };
      constexpr bool EARLY_HALO = P <= 2;
      if constexpr (EARLY_HALO) load_halo();
      cp_async_wait_all();
      __syncthreads();
      IO::c2r_twist(sp, IO::octant(stw));
      __syncthreads();
      IO::template fft<true>(sp, stw);
      if constexpr (!EARLY_HALO) load_halo();
      // Pixel update of the AL iteration at (r, x1), given the stress sj of
      // iterate n (the multiplier) and the left neighbour's sigma11, sigma12
      // (x - e^1).
      auto update = [&](int r, int j, int x1, bool v, const T (&sj)[4], T l11, T l12) {
        if (x1 >= L) return;
        const size_t x = (size_t)(r0 + r) * L + x1;
        // Eq. 1: div_i = sum_j sigma_ij(x) - sigma_ij(x - e^j)
        const T d1 = (sj[0] - l11) + (sj[3] - prev12[j]);
        const T d2 = (sj[3] - l12) + (sj[1] - prev22[j]);
        prev12[j] = sj[3];
        prev22[j] = sj[1];
#pragma unroll
        for (int c = 0; c < 4; c++) acc[A_S11 + c] += sj[c];
        acc[A_DIV2] += d1 * d1 + d2 * d2;
        // augmented-Lagrangian update of this pixel
        T e[4] = {IO::px(sp, 0, r, x1), IO::px(sp, 1, r, x1), E[2], IO::px(sp, 2, r, x1)};
        T c0[4], tau[4], e1[4], s1[4], p1[3];
        c0_apply(e, m, c0);
#pragma unroll
        for (int c = 0; c < 4; c++) tau[c] = sj[c] + c0[c];
        local_solve_p(tau, v, m, e1, s1, p1);
        Vec4<T>::store(eout + 4 * x, e1);
        Vec4<T>::store(sout + 4 * x, s1);
        // <eps^{n+1}> and its plastic pixels (stats of the next iterate)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[A_E11 + c] += e1[c];
        acc[A_NPL] += is_plastic(e1, v, m) ? T(1) : T(0);
        const T q0 = e1[0] - e[0], q1 = e1[1] - e[1], q2 = e1[2] - e[2], q3 = e1[3] - e[3];
        acc[A_COMP] += q0 * q0 + q1 * q1 + q2 * q2 + T(2) * q3 * q3;
        // next polarization sigma(eps^{n+1}) - C0:eps^{n+1} (in-plane)
        IO::px(sp, 0, r, x1) = p1[0];
        IO::px(sp, 1, r, x1) = p1[1];
        IO::px(sp, 2, r, x1) = p1[2];
      };
      // stress of iterate n and voids of row r, group j
      auto load_px = [&](int r, int j, T (&sg)[4], bool& v) {
        const int x1 = xmap(j);
        const size_t x = (size_t)(r0 + r) * L + x1;
        const bool act = x1 < L && ECHK(x, LL, 23);
        v = act ? mask[x] != 0 : true;
        if (act) Vec4<T>::load(sin_ + 4 * x, sg);
        else sg[0] = sg[1] = sg[2] = sg[3] = T(0);
      };
      // Left neighbours: the previous lane by a warp shuffle; lane 0 takes
      // lane 31 of the previous pixel group of its warp (the run is
      // contiguous), and at the start of a run reads sigma at x - e^1
      // (periodic) from memory.
      // A row is processed in chunks of PC pixels per thread (j = j0 ..
      // j0 + PC - 1); run11, run12 carry sigma11, sigma12 of lane 31 of the
      // previous pixel group from chunk to chunk.
      constexpr int PC = P < 8 ? P : 8;
      auto row = [&](int r, int j0, T (&sg)[PC][4], bool (&vv)[PC], T& run11, T& run12) {
#pragma unroll
        for (int jj = 0; jj < PC; jj++) {
          const int j = j0 + jj;
          const int x1 = xmap(j);
          T l11, l12;
          if constexpr (L < 32) {
            const int src = (lane + L - 1) & (L - 1);
            l11 = __shfl_sync(0xffffffffu, sg[jj][0], src);
            l12 = __shfl_sync(0xffffffffu, sg[jj][3], src);
          } else {
            l11 = __shfl_up_sync(0xffffffffu, sg[jj][0], 1);
            l12 = __shfl_up_sync(0xffffffffu, sg[jj][3], 1);
            if (lane == 0) {
              if (j > 0) {
                l11 = run11;
                l12 = run12;
              } else {
                const size_t xl = (size_t)(r0 + r) * L + ((x1 + L - 1) & (L - 1));
                if (ECHK(xl, LL, 24)) {
                  T sl[4];
                  Vec4<T>::load(sin_ + 4 * xl, sl);
                  l11 = sl[0];
                  l12 = sl[3];
                }
              }
            }
            run11 = __shfl_sync(0xffffffffu, sg[jj][0], 31);
            run12 = __shfl_sync(0xffffffffu, sg[jj][3], 31);
          }
          update(r, j, x1, vv[jj], sg[jj], l11, l12);
        }
      };
      // When the rows' stresses fit in fewer than 32 registers per thread,
      // all of them are loaded before the first row is processed (their
      // latencies overlap); otherwise a row is loaded chunk by chunk (PC
      // loads in flight per thread, from the L2 where the prefetch above
      // put them).
      constexpr bool PRE = RR * P * 4 * (int)sizeof(T) < 128;
      if constexpr (PRE) {
        static_assert(PC == P, "one chunk per row");
        T pen[RR][P][4];
        bool pvv[RR][P];
#pragma unroll
        for (int r = 0; r < RR; r++)
#pragma unroll
          for (int j = 0; j < P; j++) load_px(r, j, pen[r][j], pvv[r][j]);
#pragma unroll
        for (int r = 0; r < RR; r++) {
          T run11 = T(0), run12 = T(0);
          row(r, 0, pen[r], pvv[r], run11, run12);
        }
      } else {
        for (int r = 0; r < RR; r++) {
          T run11 = T(0), run12 = T(0);
#pragma unroll
          for (int j0 = 0; j0 < P; j0 += PC) {
            T en[PC][4];
            bool vv[PC];
#pragma unroll
            for (int jj = 0; jj < PC; jj++) load_px(r, j0 + jj, en[jj], vv[jj]);
            row(r, j0, en, vv, run11, run12);
          }
        }
      }
    }

    if (phase == PH_ITER || phase == PH_INIT) {
      cp_async_wait_all();  // the tables (INIT)
      __syncthreads();
      IO::template fft<false>(sp, stw);
      IO::r2c_twist(sp, IO::octant(stw));
      __syncthreads();
      IO::store(sp, spec, r0);
    }
    if (phase == PH_ITER || phase == PH_INIT) {
      if (ECHK(blockIdx.x, L / RR, 25)) block_reduce_acc<NT>(acc, S.partials + (size_t)blockIdx.x * PART_STRIDE);
    }
    // every thread of this CTA is done with the solve state before the CTA
    // counts itself in
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      const unsigned prev = atomicAdd(&S.arrive, 1u);
      s_last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
      __shared__ double tot[N_ACC];
      __threadfence();
      if (phase == PH_ITER || phase == PH_INIT) {
        sum_partials<NT, L / RR>(S.partials, tot);
        __syncthreads();
      }
      if (tid == 0) {
        finalize_solve<L>(S, phase, tot);
        S.arrive = 0;
      }
    }
  }
  if (tid == 0) batch_arrive(solves, nb, bc, cond, use_cond);
}

// ---------------------------------------------------------------------------
// Column pass
// ---------------------------------------------------------------------------
// GEN = false: the Eq. 3 operator only (every solve of the launch uses it);
// GEN = true: the operator each solve names (GreenMode).
template <typename T, int L, int V, bool GEN>
__global__ void __launch_bounds__(Cfg<T, L, V>::NT_COL, Cfg<T, L, V>::MINB_COL)
col_pass(Solve* __restrict__ solves, const C2<T>* __restrict__ tw, const C2<T>* __restrict__ ktab,
         cudaGraphConditionalHandle cond, int use_cond, int succ) {
  using C = Cfg<T, L, V>;
  constexpr int W = C::W, NT = C::NT_COL, M = C::M, NBK = M / W, SP = C::SP_C, SZ = C::COL_DATA;
  extern __shared__ __align__(16) unsigned char smraw[];
  // 3 W sequences of length L (sequence c * W + w = component c of column
  // w, padded layout of fft.cuh), then the column plan's stage table
  C2<T>* sp = reinterpret_cast<C2<T>*>(smraw);
  C2<T>* stw = sp + SZ;
  auto at = [](int c, int w, int x2) { return (c * W + w) * SP + pad32(x2); };
  const int tid = threadIdx.x;
  // Every index of the pass is in range when the grid has M / W CTAs per
  // solve: b < M / W, c < 3, w < W and x2 < L give at(c, w, x2) < 3 W SP <=
  // SZ and a global index below 3 M L.
  if (!ECHK(gridDim.x - 1, NBK, 33)) return;
  // The row pass that follows re-arms the loop; a body that never reaches
  // it must not loop again.
  if (use_cond && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) cudaGraphSetConditional(cond, 0u);
  Solve& S = solves[blockIdx.y];
  const volatile Solve& Sv = S;
  if (Sv.phase != PH_ITER) return;
  const int inc = Sv.inc;
  const int b = blockIdx.x;
  C2<T>* spec = reinterpret_cast<C2<T>*>(S.spec);
  copy_table<T, NT>(stw, tw + C::TB::off_col(V), C::COL_TW);
  // the slab of each component is contiguous in HBM: consecutive threads
  // copy consecutive numbers, asynchronously, the whole slab in flight
#pragma unroll 4
  for (int e = tid; e < 3 * L * W; e += NT) {
    const int c = e / (L * W);
    const int rem = e - c * (L * W);
    const int x2 = rem / W, w = rem - x2 * W;
    const int i = at(c, w, x2);
    const size_t g = (size_t)(c * NBK + b) * L * W + rem;
    if (ECHK(i, SZ, 30) && ECHK(g, (size_t)3 * M * L, 34)) cp_async_c2(sp + i, spec + g);
  }
  // the slab of the CTA that follows this one on an SM (succ = the CTAs the
  // GPU holds at once, counted in launch order) is asked of the L2 while
  // this CTA transforms its own, in 16 KB pieces by warp 0
  if (tid < 32 && succ > 0) {
    const long long nxt = (long long)blockIdx.y * gridDim.x + blockIdx.x + succ;
    if (nxt < (long long)gridDim.x * gridDim.y) {
      const int bs = (int)(nxt % gridDim.x), ss = (int)(nxt / gridDim.x);
      const volatile Solve& Sn = solves[ss];
      if (Sn.phase == PH_ITER) {
        constexpr unsigned SB = (unsigned)(L * W * sizeof(C2<T>)), PB = SB < 16384u ? SB : 16384u;
        constexpr int NPS = (int)(SB / PB);
        const char* sn = reinterpret_cast<const char*>(solves[ss].spec);
        for (int k = tid; k < 3 * NPS; k += 32) {
          const int c = k / NPS;
          if (ECHK(bs, NBK, 35)) prefetch_l2(sn + ((size_t)(c * NBK + bs) * L * W) * sizeof(C2<T>) + (size_t)(k % NPS) * PB, PB);
        }
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
  constexpr int G = C::G_C;
#pragma unroll 1
  for (int g = 0; g < 3 * W / G; g++) fft_seq<T, L, C::RM_COL, C::FULL, G, NT, false>(sp + g * G * SP, stw);

  const T lam0 = T(S.lam0), mu0 = T(S.mu0);
  const T scale = T(1.0 / ((double)L * (double)L));
  const int gm = GEN ? S.green : (int)GM_EQ3;
  const C2<T>* __restrict__ qtab = ktab + L;  // continuum momenta follow k(m)
  // frequencies with m1 = b*W + w != 0 (consecutive threads: consecutive m2)
  for (int f = tid; f < W * L; f += NT) {
    const int w = f / L, m2 = f - w * L;
    const int m1 = b * W + w;
    if (m1 == 0) continue;
    const int i0 = at(0, w, m2), i1 = i0 + W * SP, i2 = i0 + 2 * W * SP;  // components 11, 22, 12
    if (!ECHK(i0, SZ, 31) || !ECHK(i1, SZ, 31) || !ECHK(i2, SZ, 31) || !ECHK(m1, L, 35) || !ECHK(m2, L, 35)) continue;
    C2<T> p11 = sp[i0], p22 = sp[i1], p12 = sp[i2];
    if (GEN) green_op(gm, ktab, qtab, L, m1, m2, lam0, mu0, scale, p11, p22, p12);
    else green_apply(ktab[m1], ktab[m2], lam0, mu0, scale, p11, p22, p12);
    sp[i0] = p11;
    sp[i1] = p22;
    sp[i2] = p12;
  }
  if (b == 0) {
    // packed column: Z = A + i B with A the m1 = 0 column and B the
    // m1 = L/2 column, both transforms of real sequences (Hermitian)
    const double* Ep = S.path + 4 * inc;
    for (int m2 = tid; m2 <= L / 2; m2 += NT) {
      const int mp = (L - m2) & (L - 1);
      C2<T> A[3], B[3], Ap[3], Bp[3];
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const C2<T> z = sp[at(c, 0, m2)], zp = sp[at(c, 0, mp)];
        A[c] = T(0.5) * (z + conj(zp));
        const C2<T> d = z - conj(zp);  // B = d / (2i)
        B[c] = mk(T(0.5) * d.im, T(-0.5) * d.re);
        Ap[c] = conj(A[c]);
        Bp[c] = conj(B[c]);
      }
      if (m2 == 0) {
        // the mean strain, or 0 where it is added in FP64 after the
        // transforms (the defect form and its reference)
        const T z = S.zero_mean ? T(0) : T(1);
        A[0] = mk(z * T(Ep[0]), T(0));
        A[1] = mk(z * T(Ep[1]), T(0));
        A[2] = mk(z * T(Ep[3]), T(0));
      } else {
        green_op(gm, ktab, qtab, L, 0, m2, lam0, mu0, scale, A[0], A[1], A[2]);
        green_op(gm, ktab, qtab, L, 0, mp, lam0, mu0, scale, Ap[0], Ap[1], Ap[2]);
      }
      green_op(gm, ktab, qtab, L, M, m2, lam0, mu0, scale, B[0], B[1], B[2]);
      green_op(gm, ktab, qtab, L, M, mp, lam0, mu0, scale, Bp[0], Bp[1], Bp[2]);
#pragma unroll
      for (int c = 0; c < 3; c++) {
        sp[at(c, 0, m2)] = A[c] + mul_i(B[c]);
        if (mp != m2) sp[at(c, 0, mp)] = Ap[c] + mul_i(Bp[c]);
      }
    }
  }
  __syncthreads();
#pragma unroll 1
  for (int g = 0; g < 3 * W / G; g++) fft_seq<T, L, C::RM_COL, C::FULL, G, NT, true>(sp + g * G * SP, stw);
  if constexpr (sizeof(C2<T>) == 8) {
#pragma unroll 4
    for (int e2 = tid; e2 < 3 * L * W / 2; e2 += NT) {
      const int e = 2 * e2;
      const int c = e / (L * W);
      const int rem = e - c * (L * W);
      const int xa = rem / W, wa = rem - xa * W;
      // the pair's second number: column wa + 1 of the same row (W >= 2,
      // rem even) or row xa + 1 of the column (W = 1, xa even, so xa + 1 is
      // no multiple of 32 and the padding adds nothing)
      const int ia = at(c, wa, xa), ib = ia + (W >= 2 ? SP : 1);
      if (ECHK(ia, SZ, 32) && ECHK(ib, SZ, 32) && ECHK((size_t)(c * NBK + b) * L * W + rem + 1, (size_t)3 * M * L, 36)) {
        const float2 u = reinterpret_cast<const float2*>(sp)[ia];
        const float2 v = reinterpret_cast<const float2*>(sp)[ib];
        *reinterpret_cast<float4*>(spec + (size_t)(c * NBK + b) * L * W + rem) = make_float4(u.x, u.y, v.x, v.y);
      }
    }
  } else {
#pragma unroll 4
    for (int e = tid; e < 3 * L * W; e += NT) {
      const int c = e / (L * W);
      const int rem = e - c * (L * W);
      const int x2 = rem / W, w = rem - x2 * W;
      const int i = at(c, w, x2);
      if (ECHK(i, SZ, 32)) spec[(size_t)(c * NBK + b) * L * W + rem] = sp[i];
    }
  }
}

// ---------------------------------------------------------------------------
// Row transforms alone (compatible-strain projection of a given field)
// ---------------------------------------------------------------------------
template <typename T, int L, int V>
__global__ void __launch_bounds__(Cfg<T, L, V>::NT_ROW)
row_forward(const T* __restrict__ p, C2<T>* __restrict__ spec, const C2<T>* __restrict__ tw) {
  using C = Cfg<T, L, V>;
  constexpr int RR = C::RR, W = C::W, NT = C::NT_ROW, P = L >= NT ? L / NT : 1;
  using IO = RowIO<T, L, V>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C2<T>* sp = reinterpret_cast<C2<T>*>(smraw);
  if (!ECHK(gridDim.x - 1, L / RR, 28)) return;  // indices: see RowIO::where
  const int r0 = blockIdx.x * RR;
  const size_t LL = (size_t)L * L;
  const C2<T>* stw = IO::load_tables(sp, tw);
  for (int r = 0; r < RR; r++)
    for (int j = 0; j < P; j++) {
      const int x1 = threadIdx.x + j * NT;
      if (x1 >= L) continue;
      const size_t x = (size_t)(r0 + r) * L + x1;
      for (int c = 0; c < 3; c++) IO::px(sp, c, r, x1) = p[c * LL + x];
    }
  cp_async_wait_all();
  __syncthreads();
  IO::template fft<false>(sp, stw);
  IO::r2c_twist(sp, IO::octant(stw));
  __syncthreads();
  IO::store(sp, spec, r0);
}

template <typename T, int L, int V>
__global__ void __launch_bounds__(Cfg<T, L, V>::NT_ROW)
row_inverse(const C2<T>* __restrict__ spec, T* __restrict__ e, const C2<T>* __restrict__ tw) {
  using C = Cfg<T, L, V>;
  constexpr int RR = C::RR, W = C::W, NT = C::NT_ROW, P = L >= NT ? L / NT : 1;
  using IO = RowIO<T, L, V>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C2<T>* sp = reinterpret_cast<C2<T>*>(smraw);
  if (!ECHK(gridDim.x - 1, L / RR, 28)) return;  // indices: see RowIO::where
  const int r0 = blockIdx.x * RR;
  const size_t LL = (size_t)L * L;
  const C2<T>* stw = IO::load_tables(sp, tw);
  IO::load_async(sp, spec, r0);
  cp_async_wait_all();
  __syncthreads();
  IO::c2r_twist(sp, IO::octant(stw));
  __syncthreads();
  IO::template fft<true>(sp, stw);
  for (int r = 0; r < RR; r++)
    for (int j = 0; j < P; j++) {
      const int x1 = threadIdx.x + j * NT;
      if (x1 >= L) continue;
      const size_t x = (size_t)(r0 + r) * L + x1;
      for (int c = 0; c < 3; c++) e[c * LL + x] = IO::px(sp, c, r, x1);
    }
}

}  // namespace epfft
