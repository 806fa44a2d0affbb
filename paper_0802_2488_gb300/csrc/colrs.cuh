// Register-staged column pass (FP32, lattice sides 128 .. 4096).
//
// The same work as col_pass (forward column transform of the three
// polarization components, the Green operator of Eq. 3 per frequency,
// inverse column transform), organised so that the column transforms cost
// few shared-memory accesses and little index arithmetic:
//
//   * a column of length L is transformed by T = L / E threads, each of
//     which owns E = 16 elements per stage and component (E = 8 at
//     L = 512: three radix-8 stages, half the registers of 2 x 16 x 16 with
//     as many stages, so twice the resident warps): an in-place
//     decimation-in-frequency (DIF) transform, a first stage of radix
//     R1 = 2, 4, 8 or 16 followed by radix-E stages, leaves the spectrum in
//     digit-reversed order; the inverse runs the transposed stages in
//     reverse order (decimation in time), so it takes the digit-reversed
//     spectrum and returns natural order.  The Green operator is pointwise
//     in frequency, so no reordering is ever needed: a position's frequency
//     follows from its digits (RsPlan in tables.cuh);
//   * the first forward stage reads its elements straight from HBM and the
//     last inverse stage writes them straight back; the last forward stage,
//     the Green operator and the first inverse stage run in registers on the
//     three components at once; the other stages exchange through shared
//     memory, one read and one write per element and stage;
//   * a thread keeps the same butterflies for the three components, so the
//     twiddles of a stage are loaded once (read-only path, a per-size table
//     rounded once from extended precision) and used three times; the
//     Fourier symbols of the last stage's frequencies come from a table in
//     the order the threads read them; every address is a compile-time
//     offset from one per-thread base.
//
// Stage s (1-based): N_s = L / (R_1 ... R_{s-1}) is the length of its
// sub-transforms, D_s = N_s / R_s their stride; butterfly (b, j),
// b < L / N_s, j < D_s, reads positions b N_s + j + r D_s (r < R_s), forms
// y_k = sum_r v_r exp(-2 pi i r k / R_s) and writes y_k exp(-2 pi i j k / N_s)
// back to position b N_s + j + k D_s.  Thread t does butterflies
// u = t + i T (i < E / R_s), (b, j) = (u / D_s, u mod D_s); in the first
// stage it holds positions t + m T, in the last one E t + r, which carry
// frequencies m0(t) + r L / E.
//
// Shared memory: per column group g, three sequences of L elements from
// g (3 L + 8); element e of a sequence sits at sw16(e) = e XOR ((e / 16) mod
// 16), which keeps every access pattern of the transform on distinct bank
// pairs per half-warp (runs of consecutive positions, the stride-16 reads of
// the last stage); when a CTA holds both columns of a two-column tile, its
// lanes alternate between them (one contiguous HBM run per warp), and the
// offset of 8 between groups keeps the two columns' accesses apart in the
// banks.  With E = 8 the element sits at sw8(e) = e XOR ((e / 8) mod 8)
// instead: the last stage's stride-8 reads of the eight lanes of a column
// in a half-warp then fall on eight distinct bank pairs, and the other
// column's lanes on the other eight.  tests/test_colrs_layout.py models
// these banks and runs.
#pragma once
#include "fft.cuh"
#include "passes.cuh"
#include "physics.cuh"
#include "tables.cuh"

namespace epfft {

__host__ __device__ constexpr int sw16(int e) { return e ^ ((e >> 4) & 15); }
__host__ __device__ constexpr int sw8(int e) { return e ^ ((e >> 3) & 7); }
// the swizzle of plan P: sw16 for 16 elements per thread, sw8 for 8
template <typename P>
__host__ __device__ constexpr int psw(int e) { return P::E == 8 ? sw8(e) : sw16(e); }

// CTA shape of the register-staged column pass for tile width W.
template <int L, int W>
struct RsCfg {
  using P = RsPlan<L>;
  static constexpr int T = P::T;
  // columns per CTA: two (a tile) or more, 64 threads per CTA up to L = 512
  // (eight CTAs per SM), 128 at L = 1024; one column above
  // (two CTAs per SM at L = 4096; a CTA that held both columns of a tile
  // would read whole sectors but fill the SM alone, which measured slower)
  static constexpr int CPC = L <= 1024 ? (64 / T > 2 ? 64 / T : 2) : 1;
  static constexpr int NT = CPC * T;
  // the two columns of a tile alternate lane by lane
  static constexpr bool INTER = CPC >= 2 && W == 2;
  static constexpr int GSTRIDE = 3 * L + 8;  // elements between column groups
  // register cap: 128 for 16 elements per thread (the fused stage holds
  // 3 x 16 complex numbers), 72 for 8 (seven CTAs of 128 threads per SM;
  // measured at 64 x L = 512: 103 us against 104 us at 80 registers and
  // 127 us at 64, where the fused stage spills)
  static constexpr int RCAP = P::E == 16 ? 128 : 72;
  static constexpr int MINB = 65536 / (NT * RCAP) > 0 ? 65536 / (NT * RCAP) : 1;
  static constexpr size_t SMEM = (size_t)CPC * GSTRIDE * sizeof(C2<float>);
  static_assert(NT >= 32 && NT % 32 == 0, "whole warps");
  static_assert(!INTER || CPC % 2 == 0, "column pairs");
  // sw8 keeps the stride-8 reads of the last stage apart in the banks only
  // when the two columns of a tile alternate lane by lane
  static_assert(P::E == 16 || INTER, "8 elements per thread need interleaved column pairs");
  static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
};

// Twiddles of stage s of plan P for thread t (all of its butterflies), from
// the read-only path.
template <typename P, int s>
__device__ __forceinline__ void p16_twiddles(const C2<float>* __restrict__ tws, int t, C2<float> (&w)[16][15]) {
  constexpr int R = P::radix(s), D = P::stride(s), K = P::E / R;
  if constexpr (D > 1) {
    const float2* tb = reinterpret_cast<const float2*>(tws + P::tw_off(s));
#pragma unroll
    for (int i = 0; i < K; i++) {
      const int j = (t + i * P::T) % D;
#pragma unroll
      for (int k = 1; k < R; k++) {
        const float2 x = __ldg(tb + (k - 1) * D + j);
        w[i][k - 1] = mk(x.x, x.y);
      }
    }
  }
}

// Twiddles of butterfly i of stage s of plan P for thread t (w[k - 1],
// k = 1 .. radix - 1), from the read-only path.
template <typename P, int s>
__device__ __forceinline__ void p16_twiddles_i(const C2<float>* __restrict__ tws, int t, int i, C2<float> (&w)[15]) {
  constexpr int R = P::radix(s), D = P::stride(s);
  if constexpr (D > 1) {
    const float2* tb = reinterpret_cast<const float2*>(tws + P::tw_off(s));
    const int j = (t + i * P::T) % D;
#pragma unroll
    for (int k = 1; k < R; k++) {
      const float2 x = __ldg(tb + (k - 1) * D + j);
      w[k - 1] = mk(x.x, x.y);
    }
  }
}

// One forward (DIF) or inverse (DIT) stage s of plan P on the three
// sequences sq, sq + SSTR, sq + 2 SSTR in shared memory, for thread t of the
// sequence's T threads.
template <typename P, int s, bool INV, int SSTR>
__device__ __forceinline__ void p16_stage(C2<float>* sq, int t, const C2<float>* __restrict__ tws) {
  constexpr int R = P::radix(s), N = P::nlen(s), D = P::stride(s), K = P::E / R;
  C2<float> w[16][15];
  p16_twiddles<P, s>(tws, t, w);
#pragma unroll 1
  for (int c = 0; c < 3; c++) {
    C2<float>* q = sq + c * SSTR;
#pragma unroll
    for (int i = 0; i < K; i++) {
      const int u = t + i * P::T;
      const int base = (u / D) * N + u % D;
      C2<float> v[R];
#pragma unroll
      for (int r = 0; r < R; r++) v[r] = q[psw<P>(base + r * D)];
      if constexpr (!INV) {
        Bfly<float, R, false, true>::run(v);
        if constexpr (D > 1) {
#pragma unroll
          for (int k = 1; k < R; k++) v[k] = v[k] * w[i][k - 1];
        }
      } else {
        if constexpr (D > 1) {
#pragma unroll
          for (int k = 1; k < R; k++) v[k] = v[k] * conj(w[i][k - 1]);
        }
        Bfly<float, R, true, true>::run(v);
      }
#pragma unroll
      for (int r = 0; r < R; r++) q[psw<P>(base + r * D)] = v[r];
    }
  }
}

// Forward stages s .. S-1 of plan P (each preceded by a barrier).
template <typename P, int SSTR, int s = 2>
__device__ __forceinline__ void p16_forward_mid(C2<float>* sq, int t, const C2<float>* __restrict__ tws) {
  if constexpr (s < P::S) {
    __syncthreads();
    p16_stage<P, s, false, SSTR>(sq, t, tws);
    p16_forward_mid<P, SSTR, s + 1>(sq, t, tws);
  }
}
// Inverse stages s .. 2 of plan P (each followed by a barrier).
template <typename P, int SSTR, int s = P::S - 1>
__device__ __forceinline__ void p16_inverse_mid(C2<float>* sq, int t, const C2<float>* __restrict__ tws) {
  if constexpr (s >= 2) {
    p16_stage<P, s, true, SSTR>(sq, t, tws);
    __syncthreads();
    p16_inverse_mid<P, SSTR, s - 1>(sq, t, tws);
  }
}

// The column pass.  Grid: (L/2 / CPC, solves); stored column p1 of the
// tiled spectrum layout (tile width W) per group of T threads; it holds
// frequency m1 = p1, or, with DREV (the layout of the register-staged row
// pass, rowrs.cuh), the frequency the row transform's digit-reversed order
// puts there, m1 = RowPlan<L/2>::freq(p1) (p1 = 0 holds the packed
// m1 = 0 and L/2 columns either way).  The launch shape is checked on
// entry; for that shape every index below is in range (positions < L,
// components < 3, columns < L/2, groups < CPC).
template <int L, int W, bool GEN, bool DREV>
__global__ void __launch_bounds__(RsCfg<L, W>::NT, RsCfg<L, W>::MINB)
col_pass_rs(Solve* __restrict__ solves, const C2<float>* __restrict__ ktab, const C2<float>* __restrict__ tws,
            cudaGraphConditionalHandle cond, int use_cond) {
  using P = RsPlan<L>;
  using CF = RsCfg<L, W>;
  constexpr int T = P::T, E = P::E, M = L / 2, NBK = M / W, CPC = CF::CPC, S = P::S;
  extern __shared__ __align__(16) unsigned char smraw[];
  if (!ECHK(blockDim.x - 1, CF::NT, 40) || !ECHK(gridDim.x - 1, M / CPC, 40)) return;
  if (use_cond && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
  Solve& Sol = solves[blockIdx.y];
  const volatile Solve& Sv = Sol;
  if (Sv.phase != PH_ITER) return;
  const int inc = Sv.inc;
  int g, t;
  if constexpr (CF::INTER) {
    const int pr = threadIdx.x / (2 * T), rm = threadIdx.x % (2 * T);
    g = 2 * pr + (rm & 1);
    t = rm >> 1;
  } else {
    g = threadIdx.x / T;
    t = threadIdx.x % T;
  }
  const int p1 = blockIdx.x * CPC + g;
  const int bt = p1 / W, w = p1 % W;
  const int m1 = DREV ? RowPlan<M>::freq_d(p1) : p1;
  C2<float>* sq = reinterpret_cast<C2<float>*>(smraw) + g * CF::GSTRIDE;
  C2<float>* spec = reinterpret_cast<C2<float>*>(Sol.spec);
  // element x2 of component c of this column: spec[gbase(c) + x2 W]
  auto gbase = [&](int c) { return ((size_t)(c * NBK + bt) * L) * W + w; };
  const float lam0 = float(Sol.lam0), mu0 = float(Sol.mu0);
  const float scale = float(1.0 / ((double)L * (double)L));
  const int gm = GEN ? Sol.green : (int)GM_EQ3;
  const C2<float>* __restrict__ qtab = ktab + L;  // continuum momenta follow k(m)

  // forward stage 1 straight from HBM: positions t + m T
  {
    constexpr int R = P::R1, D = P::stride(1), K = E / R;
    C2<float> tv[16][15];
    p16_twiddles<P, 1>(tws, t, tv);
#pragma unroll 1
    for (int c = 0; c < 3; c++) {
      const float2* src = reinterpret_cast<const float2*>(spec + gbase(c));
      C2<float> v[E];
#pragma unroll
      for (int m = 0; m < E; m++) {
        const float2 x = __ldcg(src + (size_t)(t + m * T) * W);
        v[m] = mk(x.x, x.y);
      }
      C2<float>* q = sq + c * L;
#pragma unroll
      for (int i = 0; i < K; i++) {
        // butterfly u = t + i T: positions u + r D = t + (i + r K) T
        C2<float> a[R];
#pragma unroll
        for (int r = 0; r < R; r++) a[r] = v[i + r * K];
        Bfly<float, R, false, true>::run(a);
        if constexpr (D > 1) {
#pragma unroll
          for (int k = 1; k < R; k++) a[k] = a[k] * tv[i][k - 1];
        }
#pragma unroll
        for (int k = 0; k < R; k++) q[psw<P>(t + (i + k * K) * T)] = a[k];
      }
    }
  }
  p16_forward_mid<P, L>(sq, t, tws);
  __syncthreads();

  if (blockIdx.x != 0) {
    // last forward stage, the Green operator of Eq. 3 (scaled by 1/L^2) and
    // the first inverse stage, in registers: positions 16 t + r carry
    // frequencies m0 + r L / 16 (no column here is the packed one, m1 > 0)
    C2<float> a0[E], a1[E], a2[E];
#pragma unroll
    for (int r = 0; r < E; r++) {
      a0[r] = sq[psw<P>(E * t + r)];
      a1[r] = sq[L + psw<P>(E * t + r)];
      a2[r] = sq[2 * L + psw<P>(E * t + r)];
    }
    Bfly<float, E, false, true>::run(a0);
    Bfly<float, E, false, true>::run(a1);
    Bfly<float, E, false, true>::run(a2);
    const C2<float> k1 = ktab[m1];
    const float2* kq = reinterpret_cast<const float2*>(tws + P::KQOFF) + t;
    const int m0 = P::freq_d(E * t);
#pragma unroll
    for (int r = 0; r < E; r++) {
      if (GEN) {
        green_op(gm, ktab, qtab, L, m1, m0 + r * (L / E), lam0, mu0, scale, a0[r], a1[r], a2[r]);
      } else {
        const float2 k2 = __ldg(kq + r * T);
        green_apply(k1, mk(k2.x, k2.y), lam0, mu0, scale, a0[r], a1[r], a2[r]);
      }
    }
    Bfly<float, E, true, true>::run(a0);
    Bfly<float, E, true, true>::run(a1);
    Bfly<float, E, true, true>::run(a2);
#pragma unroll
    for (int r = 0; r < E; r++) {
      sq[psw<P>(E * t + r)] = a0[r];
      sq[L + psw<P>(E * t + r)] = a1[r];
      sq[2 * L + psw<P>(E * t + r)] = a2[r];
    }
  } else {
    // the CTA that holds the packed column (m1 = 0): the last stage through
    // shared memory, then the Green operator position by position
    p16_stage<P, S, false, L>(sq, t, tws);
    __syncthreads();
    if (m1 != 0) {
      const C2<float> k1 = ktab[m1];
      for (int m = 0; m < E; m++) {
        const int p = t + m * T;
        const int m2 = P::freq_d(p);
        const int ip = psw<P>(p);
        C2<float> p11 = sq[ip], p22 = sq[L + ip], p12 = sq[2 * L + ip];
        if (GEN) green_op(gm, ktab, qtab, L, m1, m2, lam0, mu0, scale, p11, p22, p12);
        else green_apply(k1, ktab[m2], lam0, mu0, scale, p11, p22, p12);
        sq[ip] = p11;
        sq[L + ip] = p22;
        sq[2 * L + ip] = p12;
      }
    } else {
      // packed column: Z = A + i B with A the m1 = 0 column and B the
      // m1 = L/2 column, both transforms of real sequences (Hermitian)
      const double* Ep = Sol.path + 4 * inc;
      for (int m2 = t; m2 <= L / 2; m2 += T) {
        const int mp = (L - m2) & (L - 1);
        const int ia = psw<P>(P::pos_d(m2)), ib = psw<P>(P::pos_d(mp));
        C2<float> A[3], B[3], Ap[3], Bp[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
          const C2<float> z = sq[c * L + ia], zp = sq[c * L + ib];
          A[c] = 0.5f * (z + conj(zp));
          const C2<float> d = z - conj(zp);  // B = d / (2i)
          B[c] = mk(0.5f * d.im, -0.5f * d.re);
          Ap[c] = conj(A[c]);
          Bp[c] = conj(B[c]);
        }
        if (m2 == 0) {
          // the mean strain, or 0 for the defect form (added in FP64 there)
          const float z = Sol.zero_mean ? 0.f : 1.f;
          A[0] = mk(z * float(Ep[0]), 0.f);
          A[1] = mk(z * float(Ep[1]), 0.f);
          A[2] = mk(z * float(Ep[3]), 0.f);
        } else {
          green_op(gm, ktab, qtab, L, 0, m2, lam0, mu0, scale, A[0], A[1], A[2]);
          green_op(gm, ktab, qtab, L, 0, mp, lam0, mu0, scale, Ap[0], Ap[1], Ap[2]);
        }
        green_op(gm, ktab, qtab, L, M, m2, lam0, mu0, scale, B[0], B[1], B[2]);
        green_op(gm, ktab, qtab, L, M, mp, lam0, mu0, scale, Bp[0], Bp[1], Bp[2]);
#pragma unroll
        for (int c = 0; c < 3; c++) {
          sq[c * L + ia] = A[c] + mul_i(B[c]);
          if (mp != m2) sq[c * L + ib] = Ap[c] + mul_i(Bp[c]);
        }
      }
    }
    __syncthreads();
    p16_stage<P, S, true, L>(sq, t, tws);
  }
  __syncthreads();
  p16_inverse_mid<P, L>(sq, t, tws);

  // inverse stage 1 straight to HBM
  {
    constexpr int R = P::R1, D = P::stride(1), K = E / R;
    C2<float> tv[16][15];
    p16_twiddles<P, 1>(tws, t, tv);
#pragma unroll 1
    for (int c = 0; c < 3; c++) {
      const C2<float>* q = sq + c * L;
      C2<float> v[E];
#pragma unroll
      for (int i = 0; i < K; i++) {
        C2<float> a[R];
#pragma unroll
        for (int k = 0; k < R; k++) a[k] = q[psw<P>(t + (i + k * K) * T)];
        if constexpr (D > 1) {
#pragma unroll
          for (int k = 1; k < R; k++) a[k] = a[k] * conj(tv[i][k - 1]);
        }
        Bfly<float, R, true, true>::run(a);
#pragma unroll
        for (int r = 0; r < R; r++) v[i + r * K] = a[r];
      }
      float2* dst = reinterpret_cast<float2*>(spec + gbase(c));
#pragma unroll
      for (int m = 0; m < E; m++) __stcg(dst + (size_t)(t + m * T) * W, make_float2(v[m].re, v[m].im));
    }
  }
}

}  // namespace epfft
