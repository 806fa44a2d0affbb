// Shared-memory Stockham FFT used by the row and column passes.
//
// A CTA transforms NSEQ sequences of length N that live in shared memory,
// sequence s at s * seq_stride<N>() with element x at pad32(x) = x + x / 32
// (one unused slot per 32 elements).  A stage of radix R (NS = product of
// the earlier radices) gives each thread one butterfly index j (consecutive
// threads take consecutive j of one sequence): it reads x[j + r N/R],
// applies the twiddles exp(-+2 pi i (j mod NS) r / (NS R)), a radix-R DFT
// in registers, and writes y[(j / NS) NS R + (j mod NS) + r NS] (autosort),
// in place between two barriers.  With the padding, both the contiguous
// reads and the stride-R writes of a warp touch each bank no more often
// than the data size requires, and for fixed j the R addresses differ by
// compile-time constants.
//
// Radix plan (FftPlan): one smaller radix first when needed, then stages of
// the largest radix RM (4, 8 or 16).  Twiddles come from a shared-memory
// copy of a table generated on the host in extended precision and rounded
// once, per stage and per j mod NS: either every power w^r (full), or
// w, w^2, w^4, w^8 (compact; the other powers are products of at most three
// of these, within a few units of rounding), w = exp(-2 pi i (j mod NS) /
// (NS R)).
#pragma once
#include "common.cuh"

namespace epfft {

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

// Padded layout of one sequence of length N.  From N = 512 on, every warp
// of a stage works inside one sequence, and the stride between sequences is
// made odd so that accesses that step across sequences (the transposing
// loads and stores of the passes) spread over the banks too.
template <int N>
__host__ __device__ constexpr int seq_stride() { return N >= 512 ? N + N / 32 + 1 : (N >= 32 ? N + N / 32 : N); }
__device__ __forceinline__ int pad32(int x) { return x + (x >> 5); }

// Radix plan of a length-N transform with largest radix RM (4, 8 or 16):
// log2(N) mod log2(RM) first (when not 0), then radix-RM stages.  The stage
// table holds, for every stage k >= 1, NP arrays of ns(k) entries:
// compact (NP = log2 R): w, w^2, w^4, ...; full (NP = R - 1): w .. w^(R-1).
template <int N, int RM, bool FULL>
struct FftPlan {
  static constexpr int LG = ilog2c(N), LR = ilog2c(RM);
  static constexpr int R0 = LG % LR == 0 ? (N < RM ? N : RM) : (1 << (LG % LR));
  static constexpr int NSTAGES = N <= 1 ? 0 : (LG % LR == 0 ? LG / LR : LG / LR + 1);
  static constexpr int NP = FULL ? RM - 1 : LR;
  static __host__ __device__ constexpr int radix(int k) { return k == 0 ? R0 : RM; }
  static __host__ __device__ constexpr int ns(int k) { return k == 0 ? 1 : R0 * (1 << (LR * (k - 1))); }
  static __host__ __device__ constexpr int tw_off(int k) { return k <= 1 ? 0 : tw_off(k - 1) + NP * ns(k - 1); }
  static constexpr int TW_ENTRIES = tw_off(NSTAGES);  // complex entries of the stage table
};

// Radix-R DFT in registers: forward kernel exp(-2 pi i r k / R), inverse
// exp(+2 pi i r k / R); unnormalised.
template <typename T, int R, bool INV, bool PK = false>
struct Bfly;

template <typename T, bool INV, bool PK>
struct Bfly<T, 2, INV, PK> {
  static __device__ __forceinline__ void run(C2<T>* v) {
    C2<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  }
};

template <typename T, bool INV, bool PK>
struct Bfly<T, 4, INV, PK> {
  static __device__ __forceinline__ void run(C2<T>* v) {
    C2<T> a0 = v[0] + v[2], a1 = v[0] - v[2];
    C2<T> a2 = v[1] + v[3], a3 = mul_mi<T, INV>(v[1] - v[3]);
    v[0] = a0 + a2;
    v[2] = a0 - a2;
    v[1] = a1 + a3;
    v[3] = a1 - a3;
  }
};

// FP32 (PK): the same butterflies on packed pairs (re, im) with GB300's two-wide
// FP32 instructions (one add or FMA on both parts).  A difference x - y is
// fma(y, -1, x) and the rotation by -+i enters as fma(swap(d), (+-1, -+1), a),
// each rounded once exactly as the scalar add, so the results are bit-for-bit
// those of the generic code with about half the arithmetic instructions.
__device__ __forceinline__ float2 f2(C2<float> a) { return make_float2(a.re, a.im); }
__device__ __forceinline__ C2<float> c2(float2 a) { return mk(a.x, a.y); }

template <bool INV>
struct Bfly<float, 2, INV, true> {
  static __device__ __forceinline__ void run(C2<float>* v) {
    const float2 a = f2(v[0]), b = f2(v[1]), m1 = make_float2(-1.0f, -1.0f);
    v[0] = c2(__fadd2_rn(a, b));
    v[1] = c2(__ffma2_rn(b, m1, a));
  }
};

template <bool INV>
struct Bfly<float, 4, INV, true> {
  static __device__ __forceinline__ void run(C2<float>* v) {
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 x0 = f2(v[0]), x1 = f2(v[1]), x2 = f2(v[2]), x3 = f2(v[3]);
    const float2 a0 = __fadd2_rn(x0, x2), a1 = __ffma2_rn(x2, m1, x0);
    const float2 a2 = __fadd2_rn(x1, x3), d = __ffma2_rn(x3, m1, x1);
    // a3 = (v1 - v3) times -i (forward: (d.im, -d.re)) or +i (inverse:
    // (-d.im, d.re)): the swapped d times a sign pair
    const float2 ds = make_float2(d.y, d.x);
    const float2 sp = INV ? make_float2(-1.0f, 1.0f) : make_float2(1.0f, -1.0f);
    const float2 sn = INV ? make_float2(1.0f, -1.0f) : make_float2(-1.0f, 1.0f);
    v[0] = c2(__fadd2_rn(a0, a2));
    v[2] = c2(__ffma2_rn(a2, m1, a0));
    v[1] = c2(__ffma2_rn(ds, sp, a1));
    v[3] = c2(__ffma2_rn(ds, sn, a1));
  }
};

template <typename T, bool INV, bool PK>
struct Bfly<T, 8, INV, PK> {
  static __device__ __forceinline__ void run(C2<T>* v) {
    C2<T> e[4] = {v[0], v[2], v[4], v[6]};
    C2<T> o[4] = {v[1], v[3], v[5], v[7]};
    Bfly<T, 4, INV, PK>::run(e);
    Bfly<T, 4, INV, PK>::run(o);
    const T h = T(0.70710678118654752440084436210485);
    // o[k] times exp(-+ i pi k / 4), k = 1, 2, 3
    C2<T> t1 = INV ? mk(h * (o[1].re - o[1].im), h * (o[1].re + o[1].im))
                   : mk(h * (o[1].re + o[1].im), h * (o[1].im - o[1].re));
    C2<T> t2 = mul_mi<T, INV>(o[2]);
    C2<T> t3 = INV ? mk(-h * (o[3].re + o[3].im), h * (o[3].re - o[3].im))
                   : mk(h * (o[3].im - o[3].re), -h * (o[3].re + o[3].im));
    v[0] = e[0] + o[0];
    v[4] = e[0] - o[0];
    v[1] = e[1] + t1;
    v[5] = e[1] - t1;
    v[2] = e[2] + t2;
    v[6] = e[2] - t2;
    v[3] = e[3] + t3;
    v[7] = e[3] - t3;
  }
};

// a times exp(-+ i t) given c = cos t and sn = sin t of the forward kernel
template <typename T, bool INV>
__device__ __forceinline__ C2<T> rot_k(C2<T> a, T c, T sn) {
  const T s = INV ? sn : -sn;  // imaginary part of exp(-+ i t)
  return mk(a.re * c - a.im * s, a.re * s + a.im * c);
}

// Radix 16 as 4 x 4: DFT4 over n1 of x[4 n1 + n2], multiplication by
// exp(-+2 pi i n2 k1 / 16), DFT4 over n2; output index k1 + 4 k2.
template <typename T, bool INV, bool PK>
struct Bfly<T, 16, INV, PK> {
  static __device__ __forceinline__ void run(C2<T>* v) {
    C2<T> y[4][4];  // y[n2][k1]
#pragma unroll
    for (int n2 = 0; n2 < 4; n2++) {
      y[n2][0] = v[n2];
      y[n2][1] = v[4 + n2];
      y[n2][2] = v[8 + n2];
      y[n2][3] = v[12 + n2];
      Bfly<T, 4, INV, PK>::run(y[n2]);
    }
    const T c1 = T(0.92387953251128675612818318939678828682);  // cos(pi/8)
    const T s1 = T(0.38268343236508977172845998403039886676);  // sin(pi/8)
    const T h = T(0.70710678118654752440084436210485);         // cos(pi/4)
    // angle 2 pi m / 16: (cos, sin) for m = 1, 2, 3, 6, 9
    y[1][1] = rot_k<T, INV>(y[1][1], c1, s1);    // m = 1
    y[1][2] = rot_k<T, INV>(y[1][2], h, h);      // m = 2
    y[1][3] = rot_k<T, INV>(y[1][3], s1, c1);    // m = 3
    y[2][1] = rot_k<T, INV>(y[2][1], h, h);      // m = 2
    y[2][2] = mul_mi<T, INV>(y[2][2]);           // m = 4
    y[2][3] = rot_k<T, INV>(y[2][3], -h, h);     // m = 6
    y[3][1] = rot_k<T, INV>(y[3][1], s1, c1);    // m = 3
    y[3][2] = rot_k<T, INV>(y[3][2], -h, h);     // m = 6
    y[3][3] = rot_k<T, INV>(y[3][3], -c1, -s1);  // m = 9
#pragma unroll
    for (int k1 = 0; k1 < 4; k1++) {
      C2<T> z[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
      Bfly<T, 4, INV, PK>::run(z);
#pragma unroll
      for (int k2 = 0; k2 < 4; k2++) v[k1 + 4 * k2] = z[k2];
    }
  }
};

// Twiddles w^r, r = 1 .. R-1 (conjugated for the inverse kernel), from the
// stage block tb: full tables hold w^r at tb[(r - 1) NS + jm]; compact ones
// hold w^(2^p) at tb[p NS + jm], and the other powers are products of at
// most three of those.
template <typename T, int R, int NS, bool INV, bool FULL>
__device__ __forceinline__ void stage_twiddles(const C2<T>* __restrict__ tb, int jm, C2<T> (&w)[16]) {
  if constexpr (FULL) {
#pragma unroll
    for (int r = 1; r < R; r++) {
      const C2<T> t = tb[(r - 1) * NS + jm];
      w[r] = INV ? conj(t) : t;
    }
  } else {
    C2<T> p1 = tb[jm];
    C2<T> p2 = p1, p4 = p1, p8 = p1;
    if (R > 2) p2 = tb[NS + jm];
    if (R > 4) p4 = tb[2 * NS + jm];
    if (R > 8) p8 = tb[3 * NS + jm];
    if (INV) {
      p1 = conj(p1);
      p2 = conj(p2);
      p4 = conj(p4);
      p8 = conj(p8);
    }
    w[1] = p1;
    if (R > 2) {
      w[2] = p2;
      w[3] = p1 * p2;
    }
    if (R > 4) {
      w[4] = p4;
      w[5] = p1 * p4;
      w[6] = p2 * p4;
      w[7] = w[3] * p4;
    }
    if (R > 8) {
      w[8] = p8;
#pragma unroll
      for (int r = 1; r < 8; r++) w[8 + r] = w[r] * p8;
    }
  }
}

// Offsets (in elements) of the r-th read and write of a butterfly from its
// base address; compile-time for unrolled r.  Reads are N/R apart, writes
// NS apart; the padding adds one slot per 32 elements crossed (see the
// derivation in the layout comment of stockham_stage).
template <int N, int R, int NS>
__host__ __device__ constexpr int read_off(int r) {
  return N < 32 ? r * (N / R) : r * (N / R) + (r * (N / R)) / 32;
}
template <int N, int R, int NS>
__host__ __device__ constexpr int write_off(int r) {
  return N < 32 ? r * NS : r * NS + (r * NS) / 32;
}

// One Stockham stage K of the length-N plan over NSEQ sequences at
// s + sq * seq_stride<N>(); tw = shared stage table of N.  Ends with a
// barrier.
//   Read base: pad32(j).  For N/R >= 32, pad32(j + r N/R) = pad32(j) +
//   r N/R (33/32); for N/R < 32, j < N/R and N/R divides 32, so
//   pad32(j + r N/R) = j + r N/R + (r N/R) / 32.
//   Write base: with a = (j / NS) NS R, jm = j mod NS < NS: for NS <= 32,
//   NS divides 32 and a is a multiple of NS R, so pad32(a + jm + r NS) =
//   a + a/32 + jm + r NS + (r NS)/32; for NS > 32 (a multiple of 32),
//   pad32(a + jm + r NS) = pad32(a + jm) + r NS (33/32) = pad32(a + jm) +
//   r NS + (r NS) / 32.
template <typename T, int N, int RM, bool FULL, int NSEQ, int NT, int K, bool INV>
__device__ __forceinline__ void stockham_stage(C2<T>* s, const C2<T>* __restrict__ tw) {
  using P = FftPlan<N, RM, FULL>;
  constexpr int R = P::radix(K), NS = P::ns(K);
  constexpr int NJ = N / R;                // butterflies per sequence
  constexpr int NBF = NSEQ * NJ;           // butterflies in this stage
  constexpr int KB = (NBF + NT - 1) / NT;  // per thread
  constexpr int SP = seq_stride<N>();
  C2<T> v[KB][R];
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < KB; q++) {
    const int g = tid + q * NT;
    if (NBF % NT == 0 || g < NBF) {
      const int j = g % NJ, sq = g / NJ;
      const int rb = sq * SP + (NJ >= 32 ? pad32(j) : j);
#pragma unroll
      for (int r = 0; r < R; r++) v[q][r] = s[rb + read_off<N, R, NS>(r)];
      if constexpr (NS > 1) {
        C2<T> w[16];
        stage_twiddles<T, R, NS, INV, FULL>(tw + P::tw_off(K), j % NS, w);
#pragma unroll
        for (int r = 1; r < R; r++) v[q][r] = v[q][r] * w[r];
      }
      // packed FP32 pairs for transforms up to 2048 points (at 4096 the
      // scalar form schedules better; both give the same bits)
      Bfly<T, R, INV, sizeof(T) == 4 && N <= 2048>::run(v[q]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < KB; q++) {
    const int g = tid + q * NT;
    if (NBF % NT == 0 || g < NBF) {
      const int j = g % NJ, sq = g / NJ;
      const int jm = j % NS, a = (j / NS) * NS * R;
      const int wb = sq * SP + (N < 32 ? a + jm : (NS <= 32 ? a + (a >> 5) + jm : pad32(a + jm)));
      // a + jm + r NS < N for every r (a is a multiple of NS R below N), so
      // every write stays inside sequence sq
#pragma unroll
      for (int r = 0; r < R; r++) s[wb + write_off<N, R, NS>(r)] = v[q][r];
    }
  }
  __syncthreads();
}

template <typename T, int N, int RM, bool FULL, int NSEQ, int NT, bool INV, int K = 0>
__device__ __forceinline__ void fft_stages(C2<T>* s, const C2<T>* __restrict__ tw) {
  if constexpr (K < FftPlan<N, RM, FULL>::NSTAGES) {
    stockham_stage<T, N, RM, FULL, NSEQ, NT, K, INV>(s, tw);
    fft_stages<T, N, RM, FULL, NSEQ, NT, INV, K + 1>(s, tw);
  }
}

// Transforms NSEQ sequences of length N (layout above) in place with the
// plan FftPlan<N, RM, FULL> and its stage table tw (shared memory).  The
// caller has completed the data and the table (barrier) before the call;
// the call ends with a barrier.
template <typename T, int N, int RM, bool FULL, int NSEQ, int NT, bool INV>
__device__ __forceinline__ void fft_seq(C2<T>* s, const C2<T>* __restrict__ tw) {
  fft_stages<T, N, RM, FULL, NSEQ, NT, INV>(s, tw);
}

// Asynchronous global -> shared copy of one complex number (cp.async: the
// copy holds no register and any number can be in flight): 8 bytes through
// L1 for FP32, 16 bytes past L1 for FP64.  Both addresses are aligned to the
// element size.  The copies of a thread complete at cp_async_wait_all();
// a barrier after it publishes them to the CTA.
template <typename T>
__device__ __forceinline__ void cp_async_c2(C2<T>* dst, const C2<T>* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(C2<T>) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Asks the L2 to fetch bytes [p, p + n) from HBM (a bulk prefetch: a hint
// that completes on its own and changes no data); p and n are multiples of
// 16 bytes.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned n) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(n) : "memory");
}

// Copies n table entries from global to shared memory asynchronously
// (complete with cp_async_wait_all() and a barrier).
template <typename T, int NT>
__device__ __forceinline__ void copy_table(C2<T>* dst, const C2<T>* __restrict__ src, int n) {
  for (int i = threadIdx.x; i < n; i += NT) cp_async_c2(dst + i, src + i);
}

// exp(-2 pi i k / L) for 0 <= k <= L/4 from the octant t[0 .. L/8]:
// for k > L/8, exp(-i (pi/2 - a)) = (sin a, -cos a) with a = 2 pi (L/4 - k) / L.
template <typename T, int L>
__device__ __forceinline__ C2<T> twist_tw(const C2<T>* __restrict__ t, int k) {
  if (k <= L / 8) return t[k];
  const C2<T> b = t[L / 4 - k];
  return mk(-b.im, -b.re);
}

}  // namespace epfft
