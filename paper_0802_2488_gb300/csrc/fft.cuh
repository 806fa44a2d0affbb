// Shared-memory Stockham FFT used by the row and column passes.
//
// A CTA transforms NB sequences of length N that live in shared memory in
// "batch-interleaved" order: element x of sequence b is s[x * XS + b]
// (XS >= NB; XS > NB when only some of the interleaved sequences are
// transformed by one call).  Each
// stage reads R elements spaced N/R apart into registers, applies the stage
// twiddles, a radix-R butterfly, and writes them back in autosort (Stockham)
// order; after the last stage the sequences are in natural order, in place.
// Radix plan: one radix-2 or radix-4 stage first when log2(N) is not a
// multiple of 3, then radix-8 stages.
//
// Twiddles come from a table tw[k] = exp(-2 pi i k / Ltw) (k < Ltw), with
// Ltw = twstride * N; the table is generated on the host in extended
// precision and rounded once to T.
#pragma once
#include "common.cuh"

namespace epfft {

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

template <int N, int NS>
__host__ __device__ constexpr int stage_radix() {
  return NS == 1 ? (ilog2c(N) % 3 == 0 ? 8 : (ilog2c(N) % 3 == 1 ? 2 : 4)) : 8;
}

// Radix-R DFT in registers: forward kernel exp(-2 pi i r k / R), inverse
// exp(+2 pi i r k / R); unnormalised.
template <typename T, int R, bool INV>
struct Bfly;

template <typename T, bool INV>
struct Bfly<T, 2, INV> {
  static __device__ __forceinline__ void run(C2<T>* v) {
    C2<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  }
};

template <typename T, bool INV>
struct Bfly<T, 4, INV> {
  static __device__ __forceinline__ void run(C2<T>* v) {
    C2<T> a0 = v[0] + v[2], a1 = v[0] - v[2];
    C2<T> a2 = v[1] + v[3], a3 = mul_mi<T, INV>(v[1] - v[3]);
    v[0] = a0 + a2;
    v[2] = a0 - a2;
    v[1] = a1 + a3;
    v[3] = a1 - a3;
  }
};

template <typename T, bool INV>
struct Bfly<T, 8, INV> {
  static __device__ __forceinline__ void run(C2<T>* v) {
    C2<T> e[4] = {v[0], v[2], v[4], v[6]};
    C2<T> o[4] = {v[1], v[3], v[5], v[7]};
    Bfly<T, 4, INV>::run(e);
    Bfly<T, 4, INV>::run(o);
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

// One Stockham stage (radix R, NS = product of the earlier radices).
// Must be entered with the data complete in shared memory; ends with a
// barrier.  blockDim.x == NT.
template <typename T, int N, int NB, int XS, int NT, int R, int NS, bool INV>
__device__ __forceinline__ void stockham_stage(C2<T>* s, const C2<T>* __restrict__ tw,
                                               int twstride) {
  constexpr int NBF = NB * (N / R);  // butterflies in this stage
  constexpr int K = (NBF + NT - 1) / NT;
  C2<T> v[K][R];
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < K; q++) {
    const int g = tid + q * NT;
    if (NBF % NT == 0 || g < NBF) {
      const int b = g % NB, j = g / NB;
#pragma unroll
      for (int r = 0; r < R; r++) {
        const int ix = (j + r * (N / R)) * XS + b;
        v[q][r] = ECHK(ix, N * XS, 101) ? s[ix] : v[q][r];
      }
      if (NS > 1) {
        const int jm = j % NS;
#pragma unroll
        for (int r = 1; r < R; r++) {
          const int it = (jm * r * (N / (NS * R))) * twstride;
          C2<T> w = ECHK(it, N * twstride, 102) ? tw[it] : mk(T(1), T(0));
          if (INV) w.im = -w.im;
          v[q][r] = v[q][r] * w;
        }
      }
      Bfly<T, R, INV>::run(v[q]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; q++) {
    const int g = tid + q * NT;
    if (NBF % NT == 0 || g < NBF) {
      const int b = g % NB, j = g / NB;
      const int jm = j % NS;
      const int base = (j / NS) * NS * R + jm;
#pragma unroll
      for (int r = 0; r < R; r++) {
        const int ix = (base + r * NS) * XS + b;
        if (ECHK(ix, N * XS, 103)) s[ix] = v[q][r];
      }
    }
  }
  __syncthreads();
}

template <typename T, int N, int NB, int XS, int NT, bool INV, int NS = 1>
__device__ __forceinline__ void fft_stages(C2<T>* s, const C2<T>* __restrict__ tw, int twstride) {
  if constexpr (NS < N) {
    constexpr int R = stage_radix<N, NS>();
    stockham_stage<T, N, NB, XS, NT, R, NS, INV>(s, tw, twstride);
    fft_stages<T, N, NB, XS, NT, INV, NS * R>(s, tw, twstride);
  }
}

// NG groups of NB sequences; element x of sequence b of group g is at
// s[x * XS + g * NB + b] (XS >= NG * NB; XS is chosen odd by the callers so
// that element strides do not fold onto few shared-memory banks).  The groups
// are transformed together when every thread holds at most 16 elements per
// stage, else one group at a time.
template <typename T, int N, int NG, int NB, int XS, int NT, bool INV>
__device__ __forceinline__ void fft_block(C2<T>* s, const C2<T>* __restrict__ tw, int twstride) {
  static_assert(XS >= NG * NB, "element stride too small");
  if constexpr ((NG * NB * N + NT - 1) / NT <= 16) {
    fft_stages<T, N, NG * NB, XS, NT, INV>(s, tw, twstride);
  } else {
#pragma unroll 1
    for (int g = 0; g < NG; g++) fft_stages<T, N, NB, XS, NT, INV>(s + g * NB, tw, twstride);
  }
}

}  // namespace epfft
