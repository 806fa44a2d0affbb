// Per-size transform plans and the device tables they read.
//
// Every (real type, lattice side) has one table in device memory, built on
// the host in extended precision and rounded once to T, shared by both
// tiling variants.  Layout in complex units:
//   [0, OCT)              exp(-2 pi i k / L), k = 0 .. L/8 (row twists)
//   [OFF_R[v], +TW_R[v])  stage table of the row plan of variant v
//   [OFF_C[v], +TW_C[v])  stage table of the column plan of variant v
//   [KOFF, KOFF + L)      k(m) = (sin q, 2 sin^2(q/2)), q = 2 pi m / L, the
//                         symbol of the forward difference of Eq. 1
//                         (i k = exp(i q) - 1)
//   [QOFF, QOFF + L)      (q~(m), 0), the continuum momentum 2 pi m~ / L with
//                         m~ = m folded into (-L/2, L/2] (CG1 operator)
//   [RSOFF, + RS_ENTRIES) the stage twiddles of the register-staged column
//                         transform of length L and the Fourier symbols in
//                         the order its last stage reads them (RsPlan)
//   [RROFF, + RR_ENTRIES) the stage twiddles of the register-staged row
//                         transform of length L/2 and its twists (RowPlan)
// Variants with the same plans share their stage tables.
#pragma once
#include <vector>

#include "fft.cuh"

namespace epfft {

// Radix plans of the register-staged transforms (colrs.cuh, rowrs.cuh): a
// thread owns E = 16 (or 8) elements per stage and sequence; stage 1 has
// radix RA, stage 2 radix RB, later stages radix E, and N = RA RB E^(S - 2).
// Stage s (1-based) works on sub-transforms of length nlen(s) with stride
// stride(s) = nlen(s) / radix(s); its twiddles exp(-2 pi i j k / nlen(s)),
// j < stride(s), k = 1 .. radix(s) - 1, sit at tw_off(s) + (k - 1) stride(s)
// + j; the last stage (stride 1) has none.  After the forward
// (decimation-in-frequency) stages, position p = sum_s p_s stride(s) holds
// frequency freq(p) = p_1 + RA (p_2 + RB (p_3 + E (...))); pos() inverts it.
template <int N, int RA, int RB, int E_ = 16>
struct Plan16 {
  static constexpr int E = E_;
  static constexpr int T = N / E;  // threads per sequence
  static constexpr int S = N == RA ? 1 : 2 + ilog2c(N / (RA * RB)) / ilog2c(E);
  static __host__ __device__ constexpr int radix(int s) { return s == 1 ? RA : (s == 2 ? RB : E); }
  static __host__ __device__ constexpr int nlen(int s) { return s == 1 ? N : nlen(s - 1) / radix(s - 1); }
  static __host__ __device__ constexpr int stride(int s) { return nlen(s) / radix(s); }
  static __host__ __device__ constexpr int tw_count(int s) { return stride(s) > 1 ? (radix(s) - 1) * stride(s) : 0; }
  static __host__ __device__ constexpr int tw_off(int s) { return s <= 1 ? 0 : tw_off(s - 1) + tw_count(s - 1); }
  static constexpr int TW_END = tw_off(S + 1);
  static __host__ __device__ constexpr int freq(int p) {
    int m = 0, w = 1;
    for (int s = 1; s <= S; s++) {
      m += ((p / stride(s)) % radix(s)) * w;
      w *= radix(s);
    }
    return m;
  }
  static __host__ __device__ constexpr int pos(int m) {
    int p = 0;
    for (int s = 1; s <= S; s++) {
      p += (m % radix(s)) * stride(s);
      m /= radix(s);
    }
    return p;
  }
  // device forms of freq and pos: every radix and stride is a power of two,
  // so the digits are shifts and masks by compile-time amounts
  static __host__ __device__ constexpr int lg_stride(int s) { return ilog2c(stride(s)); }
  static __host__ __device__ constexpr int lg_weight(int s) { return s <= 1 ? 0 : lg_weight(s - 1) + ilog2c(radix(s - 1)); }
  template <int s = 1>
  static __device__ __forceinline__ int freq_d(int p) {
    if constexpr (s > S) {
      return 0;
    } else {
      return (((p >> lg_stride(s)) & (radix(s) - 1)) << lg_weight(s)) | freq_d<s + 1>(p);
    }
  }
  template <int s = 1>
  static __device__ __forceinline__ int pos_d(int m) {
    if constexpr (s > S) {
      return 0;
    } else {
      return (((m >> lg_weight(s)) & (radix(s) - 1)) << lg_stride(s)) | pos_d<s + 1>(m);
    }
  }
  static_assert(E == 8 || E == 16, "elements per thread");
  static_assert(N >= E && RA * (S >= 2 ? RB : 1) * (1 << (ilog2c(E) * (S > 2 ? S - 2 : 0))) == N, "radix plan");
  static_assert(E % RA == 0 && E % RB == 0, "radices divide the elements per thread");
};

// elements per thread of the register-staged column transform of length L:
// 8 at L = 512 (three radix-8 stages: half the registers of 16 elements,
// with the same number of stages as 2 x 16 x 16), else 16
template <int L>
constexpr int col_e() { return L == 512 ? 8 : 16; }
template <int N, int E = 16>
constexpr int col_ra() { return ilog2c(N) % ilog2c(E) == 0 ? E : (1 << (ilog2c(N) % ilog2c(E))); }
// the column transform of length L: a first stage of radix 2, 4, 8 or 16,
// then radix E
template <int L>
struct RsPlan : Plan16<L, col_ra<L, col_e<L>()>(), col_e<L>(), col_e<L>()> {
  using B = Plan16<L, col_ra<L, col_e<L>()>(), col_e<L>(), col_e<L>()>;
  static constexpr int R1 = col_ra<L, col_e<L>()>();
  // after the stage twiddles: the Fourier symbols of the frequencies the
  // last stage's positions carry, entry r T + t = k(m) of position E t + r
  static constexpr int KQOFF = B::TW_END;
  static constexpr int TW_ENTRIES = KQOFF + L;
};
// the half-length row transform of length M: a first stage of radix 2, 4 or
// 8 (radix 4 twice when log2 M is a multiple of 4), so that the pixel step,
// which sits between the last inverse and the first forward stage, holds
// few numbers per thread
template <int M>
constexpr int row_ra() { return ilog2c(M) % 4 == 0 ? 4 : (1 << (ilog2c(M) % 4)); }
template <int M>
constexpr int row_rb() { return ilog2c(M) % 4 == 0 ? 4 : 16; }
template <int M>
struct RowPlan : Plan16<M, row_ra<M>(), row_rb<M>()> {
  using B = Plan16<M, row_ra<M>(), row_rb<M>()>;
  static constexpr int R1 = row_ra<M>();
  // after the stage twiddles: exp(-2 pi i freq(q) / (2 M)) per position q,
  // the twists between the half-length transform and the real one
  static constexpr int TQOFF = B::TW_END;
  static constexpr int TW_ENTRIES = TQOFF + M;
};

// Transform plans of tiling variant V for (T, L): largest radix of the row
// (length L/2) and column (length L) transforms, and the twiddle format
// (full tables when they fit beside the data in shared memory).
template <typename T, int L, int V>
struct PlanSel {
  static constexpr bool F64 = sizeof(T) == 8;
  // FP64 at L = 4096: radix 16 and compact twiddles in both tilings (the
  // 4096-point column of three components takes 203 KB of shared memory)
  static constexpr int RM_ROW = F64 ? (L <= 512 ? 4 : (V == 0 || L == 4096 ? 16 : 8)) : 16;
  static constexpr int RM_COL = F64 ? (L <= 512 ? 4 : (V == 0 || L == 4096 ? 16 : 8)) : 16;
  static constexpr bool FULL = L <= 2048;
  using PR = FftPlan<L / 2, RM_ROW, FULL>;
  using PC = FftPlan<L, RM_COL, FULL>;
};

template <typename T, int L>
struct Tables {
  using S0 = PlanSel<T, L, 0>;
  using S1 = PlanSel<T, L, 1>;
  static constexpr bool SAME = S0::RM_ROW == S1::RM_ROW && S0::RM_COL == S1::RM_COL && S0::FULL == S1::FULL;
  static constexpr int OCT = L / 8 + 1;
  static constexpr int TW_R0 = S0::PR::TW_ENTRIES, TW_C0 = S0::PC::TW_ENTRIES;
  static constexpr int TW_R1 = S1::PR::TW_ENTRIES, TW_C1 = S1::PC::TW_ENTRIES;
  static constexpr int OFF_R0 = OCT, OFF_C0 = OFF_R0 + TW_R0;
  static constexpr int OFF_R1 = SAME ? OFF_R0 : OFF_C0 + TW_C0;
  static constexpr int OFF_C1 = SAME ? OFF_C0 : OFF_R1 + TW_R1;
  static constexpr int KOFF = SAME ? OFF_C0 + TW_C0 : OFF_C1 + TW_C1;
  static constexpr int QOFF = KOFF + L;
  static constexpr int RSOFF = QOFF + L;
  static constexpr int RS_ENTRIES = L >= 32 ? RsPlan<(L >= 32 ? L : 32)>::TW_ENTRIES : 0;
  static constexpr int RROFF = RSOFF + RS_ENTRIES;
  static constexpr int RR_ENTRIES = L >= 64 ? RowPlan<(L >= 64 ? L / 2 : 32)>::TW_ENTRIES : 0;
  static constexpr int TOTAL = RROFF + RR_ENTRIES;
  static __host__ __device__ constexpr int off_row(int v) { return v == 0 ? OFF_R0 : OFF_R1; }
  static __host__ __device__ constexpr int off_col(int v) { return v == 0 ? OFF_C0 : OFF_C1; }
};

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
// exp(-2 pi i n / d) in extended precision, rounded once (real, imag).
template <typename T>
inline void host_expi(long n, long d, T* out) {
  const long double pi = 3.141592653589793238462643383279502884L;
  const long double a = 2.0L * pi * (long double)(n % d) / (long double)d;
  out[0] = (T)cosl(a);
  out[1] = (T)(-sinl(a));
}

// Stage table of plan P at h (complex entries, interleaved reals).
template <typename T, typename P>
inline void host_stage_table(T* h) {
  for (int k = 1; k < P::NSTAGES; k++) {
    const int R = P::radix(k), NS = P::ns(k);
    for (int p = 0; p < P::NP; p++) {
      const int pw = P::NP == R - 1 ? p + 1 : (1 << p);  // full: w^(p+1); compact: w^(2^p)
      for (int jm = 0; jm < NS; jm++) host_expi<T>((long)jm * pw, (long)NS * R, h + 2 * (P::tw_off(k) + p * NS + jm));
    }
  }
}

// Stage twiddles of a Plan16 at h (complex entries, interleaved reals).
template <typename T, typename P>
inline void host_plan16_twiddles(T* h) {
  for (int st = 1; st <= P::S; st++)
    for (int k = 1; k < P::radix(st) && P::stride(st) > 1; k++)
      for (int j = 0; j < P::stride(st); j++)
        host_expi<T>((long)j * k, P::nlen(st), h + 2 * (P::tw_off(st) + (k - 1) * P::stride(st) + j));
}

template <typename T, int L>
inline void host_tables_L(std::vector<T>& h) {
  using TB = Tables<T, L>;
  h.assign((size_t)2 * TB::TOTAL, T(0));
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < TB::OCT; k++) host_expi<T>(k, L, h.data() + 2 * k);
  host_stage_table<T, typename TB::S0::PR>(h.data() + 2 * TB::OFF_R0);
  host_stage_table<T, typename TB::S0::PC>(h.data() + 2 * TB::OFF_C0);
  if (!TB::SAME) {
    host_stage_table<T, typename TB::S1::PR>(h.data() + 2 * TB::OFF_R1);
    host_stage_table<T, typename TB::S1::PC>(h.data() + 2 * TB::OFF_C1);
  }
  for (int m = 0; m < L; m++) {
    const long double q = 2.0L * pi * (long double)m / (long double)L;
    const long double hs = sinl(pi * (long double)m / (long double)L);
    h[2 * (TB::KOFF + m)] = (T)sinl(q);
    h[2 * (TB::KOFF + m) + 1] = (T)(2.0L * hs * hs);
    const int mf = m > L / 2 ? m - L : m;
    h[2 * (TB::QOFF + m)] = (T)(2.0L * pi * (long double)mf / (long double)L);
    h[2 * (TB::QOFF + m) + 1] = T(0);
  }
  if constexpr (L >= 32) {
    using RP = RsPlan<L>;
    host_plan16_twiddles<T, RP>(h.data() + 2 * TB::RSOFF);
    for (int t = 0; t < RP::T; t++)
      for (int r = 0; r < RP::E; r++) {
        const int m = RP::freq(RP::E * t + r);
        T* o = h.data() + 2 * (TB::RSOFF + RP::KQOFF + r * RP::T + t);
        o[0] = h[2 * (TB::KOFF + m)];
        o[1] = h[2 * (TB::KOFF + m) + 1];
      }
  }
  if constexpr (L >= 64) {
    using RW = RowPlan<L / 2>;
    host_plan16_twiddles<T, RW>(h.data() + 2 * TB::RROFF);
    for (int q = 0; q < L / 2; q++) host_expi<T>(RW::freq(q), L, h.data() + 2 * (TB::RROFF + RW::TQOFF + q));
  }
}

// Runtime dispatch over the supported sides: fills h and returns the
// offset of k(m) (complex units), or -1 for an unsupported L.
template <typename T>
inline int host_tables(int L, std::vector<T>& h) {
  switch (L) {
#define EPFFT_TAB(n)              \
  case n:                         \
    host_tables_L<T, n>(h);       \
    return Tables<T, n>::KOFF;
    EPFFT_TAB(4) EPFFT_TAB(8) EPFFT_TAB(16) EPFFT_TAB(32) EPFFT_TAB(64) EPFFT_TAB(128) EPFFT_TAB(256)
    EPFFT_TAB(512) EPFFT_TAB(1024) EPFFT_TAB(2048) EPFFT_TAB(4096)
#undef EPFFT_TAB
    default:
      return -1;
  }
}

}  // namespace epfft
