// Reference of the defect-correction form (FP64 state, FP32 transforms).
//
// The Green operator is linear, so for any reference polarization p_ref
//   E + Gamma(p) = E + Gamma(p_ref) + Gamma(p - p_ref).
// The defect form keeps the strain and stress of every iterate in FP64,
// computes g_ref = Gamma(p_ref) in FP64 here, and lets the iteration's own
// passes transform only p - p_ref in FP32 (row_pass<double, L, V, true>
// with the FP32 column pass, zero_mean set).  The FP32 rounding of the
// transforms then scales with |p - p_ref| instead of |p|: refreshing p_ref
// to the current polarization from time to time lets the iteration reach
// the equilibrium tolerances of the FP64 scheme (Sec. 2, eta1 and eta2),
// which the plain FP32 transforms cannot.
//
// A refresh, for every solve of a batch in its iteration phase:
//   ref_forward   p_ref = sigma - C0:eps of the current iterate (in-plane
//                 components 11, 22, 12; FP64), stored, and its FP64 row
//                 transform written to the solve's FP64 spectrum; the FP32
//                 spectrum is cleared (the next column pass then transforms
//                 p - p_ref = 0);
//   col_pass<double, L, V> on the shadow solves (spec = the FP64 spectrum,
//                 zero_mean = 1): Eq. 3 per frequency, 0 at q = 0;
//   ref_inverse   the FP64 inverse row transform into g_ref.
// Solves in other phases are skipped and keep their reference (p_ref = 0,
// g_ref = 0 at the start of a solve: the first iterations transform the whole
// polarization in FP32).
#pragma once
#include "passes.cuh"

namespace epfft {

// Forward half of a refresh.  Grid: (L / RR, solves) with the FP64 tiling V.
// shadow[i] mirrors phase, increment and buffer index of solves[i] for the
// column pass that follows (block (0, i) writes them).  The launch shape is
// checked on entry; then every index is in range (rows r0 + r < L, pixels
// x1 < L, RowIO::where for the spectrum, the FP32 spectrum's 12 L^2 bytes
// split into L / RR equal pieces of 12 L RR bytes, a multiple of 16).
template <int L, int V>
__global__ void __launch_bounds__(Cfg<double, L, V>::NT_ROW)
ref_forward(Solve* __restrict__ solves, Solve* __restrict__ shadow, const C2<double>* __restrict__ tw) {
  using C = Cfg<double, L, V>;
  constexpr int RR = C::RR, NT = C::NT_ROW, P = L >= NT ? L / NT : 1;
  using IO = RowIO<double, L, V>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C2<double>* sp = reinterpret_cast<C2<double>*>(smraw);
  if (!ECHK(gridDim.x - 1, L / RR, 60) || !ECHK(blockDim.x - 1, NT, 60)) return;
  Solve& S = solves[blockIdx.y];
  const volatile Solve& Sv = S;
  const int phase = Sv.phase, cur = Sv.cur, inc = Sv.inc;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Solve& Z = shadow[blockIdx.y];
    Z.phase = phase;
    Z.inc = inc;
    Z.cur = cur;
  }
  if (phase != PH_ITER) return;
  const int r0 = blockIdx.x * RR;
  const size_t LL = (size_t)L * L;
  const double* __restrict__ eps = reinterpret_cast<const double*>(S.eps[cur]);
  const double* __restrict__ sig = reinterpret_cast<const double*>(S.sig[cur]);
  double* __restrict__ pref = reinterpret_cast<double*>(S.pref);
  const Mat<double> m = make_mat<double>(S);
  const C2<double>* stw = IO::load_tables(sp, tw);
  for (int r = 0; r < RR; r++)
    for (int j = 0; j < P; j++) {
      const int x1 = (int)threadIdx.x + j * NT;
      if (x1 >= L) continue;
      const size_t x = (size_t)(r0 + r) * L + x1;
      double e[4], s[4], c0[4];
      Vec4<double>::load(eps + 4 * x, e);
      Vec4<double>::load(sig + 4 * x, s);
      c0_apply(e, m, c0);
      const double p11 = s[0] - c0[0], p22 = s[1] - c0[1], p12 = s[3] - c0[3];
      pref[x] = p11;
      pref[LL + x] = p22;
      pref[2 * LL + x] = p12;
      IO::px(sp, 0, r, x1) = p11;
      IO::px(sp, 1, r, x1) = p22;
      IO::px(sp, 2, r, x1) = p12;
    }
  // this CTA's piece of the FP32 spectrum
  {
    constexpr size_t PIECE = (size_t)12 * L * RR / 16;  // float4 per CTA
    static_assert((12 * L * RR) % 16 == 0, "16-byte pieces");
    float4* f = reinterpret_cast<float4*>(S.spec) + (size_t)blockIdx.x * PIECE;
    for (size_t i = threadIdx.x; i < PIECE; i += NT) f[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  cp_async_wait_all();
  __syncthreads();
  IO::template fft<false>(sp, stw);
  IO::r2c_twist(sp, IO::octant(stw));
  __syncthreads();
  IO::store(sp, reinterpret_cast<C2<double>*>(S.spec64), r0);
}

// Inverse half of a refresh: g_ref from the FP64 spectrum the column pass
// left.  Grid and checks as ref_forward.
template <int L, int V>
__global__ void __launch_bounds__(Cfg<double, L, V>::NT_ROW)
ref_inverse(Solve* __restrict__ solves, const C2<double>* __restrict__ tw) {
  using C = Cfg<double, L, V>;
  constexpr int RR = C::RR, NT = C::NT_ROW, P = L >= NT ? L / NT : 1;
  using IO = RowIO<double, L, V>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C2<double>* sp = reinterpret_cast<C2<double>*>(smraw);
  if (!ECHK(gridDim.x - 1, L / RR, 61) || !ECHK(blockDim.x - 1, NT, 61)) return;
  Solve& S = solves[blockIdx.y];
  const volatile Solve& Sv = S;
  if (Sv.phase != PH_ITER) return;
  const int r0 = blockIdx.x * RR;
  const size_t LL = (size_t)L * L;
  double* __restrict__ gref = reinterpret_cast<double*>(S.gref);
  const C2<double>* stw = IO::load_tables(sp, tw);
  IO::load_async(sp, reinterpret_cast<const C2<double>*>(S.spec64), r0);
  cp_async_wait_all();
  __syncthreads();
  IO::c2r_twist(sp, IO::octant(stw));
  __syncthreads();
  IO::template fft<true>(sp, stw);
  for (int r = 0; r < RR; r++)
    for (int j = 0; j < P; j++) {
      const int x1 = (int)threadIdx.x + j * NT;
      if (x1 >= L) continue;
      const size_t x = (size_t)(r0 + r) * L + x1;
      for (int c = 0; c < 3; c++) gref[c * LL + x] = IO::px(sp, c, r, x1);
    }
}

}  // namespace epfft
