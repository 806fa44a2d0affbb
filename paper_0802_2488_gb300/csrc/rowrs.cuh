// Register-staged row pass (FP32, lattice sides 256 .. 4096) and the row
// transforms alone (projection, displacement), tiling variant 2.
//
// The same work as row_pass (inverse row transform of e^{n+1}, the pixel
// update of the augmented Lagrangian, forward row transform of the next
// polarization, residual partial sums), organised like the register-staged
// column pass (colrs.cuh): a row's half-length transform (M = L/2 points) is
// done by T = M/16 threads that keep the same 16 positions for the three
// components, in stages whose addresses are compile-time offsets.
//
// Spectrum order.  The forward row transform is a decimation-in-frequency
// transform, whose output is in digit-reversed order (RowPlan in
// tables.cuh), and the spectrum is stored in that order along m1: stored
// column p holds frequency m1 = RowPlan<M>::freq(p) (the column pass takes
// that map, colrs.cuh with DREV).  The inverse row transform is then the
// transposed, decimation-in-time one, which takes the digit-reversed
// spectrum and returns natural order; so neither direction reorders.
//
// The pixel update sits between the last inverse stage and the first
// forward stage, in registers: the first stage (radix R1 = 2, 4 or 8) leaves
// thread t with positions n = t + m T of z(n) = x(2n) + i x(2n+1), a
// butterfly at a time (R1 positions, three components), i.e. the pixels
// 2n and 2n+1; their update reads sigma^n of the two pixels, of the left
// neighbour (from the previous lane, or from memory at the start of a run)
// and of the row above (from memory; the L1 or L2 holds it, since the
// thread of the row above reads it too), and writes eps^{n+1}, sigma^{n+1}
// and the next polarization, which enters the forward butterfly at once.
//
// The real-to-complex twists of the half-length transforms pair frequencies
// k and M - k, which sit at scattered positions of the digit-reversed order;
// each pair is done by the thread holding the smaller of its two positions
// (reads both, writes both), so a twist needs no barrier between its reads
// and its writes.
//
// Shared memory: row r's three sequences (components 11, 22, 12) from
// r (3 M + 16) + off(r), element q of a sequence at sw16(q) (colrs.cuh).
// The bank offset off(r) spreads the rows of the transposing spectrum load
// and store over the banks (a half-warp takes 16 consecutive numbers of the
// tile chunks, RR rows x W columns each): off(r) = 16 r / RR; with 8 threads
// per row (L = 256: two rows per half-warp in the transform stages)
// off(r) = r / 2 + 8 (r mod 2), which also keeps the two rows of a phase 8
// bank pairs apart.  Spectrum tile width W (2, or 1 at L = 256): a CTA
// reads and writes contiguous runs of RR W complex numbers (16 at L = 256
// and 512, 8 at 1024, 4 above) per component and tile.
#pragma once
#include "colrs.cuh"

namespace epfft {

template <int L>
struct RowRsCfg {
  static constexpr int M = L / 2;
  using P = RowPlan<M>;
  static constexpr int T = P::T;  // threads per row
  static constexpr int RR = L <= 256 ? 16 : (L == 512 ? 8 : (L == 1024 ? 4 : 2));  // rows per CTA
  static constexpr int NT = RR * T;
  // tile width of the spectrum layout: two columns (the register-staged
  // column pass reads a two-column tile with whole sectors per warp), one at
  // L = 256 (16 rows per CTA make 128-byte runs already)
  static constexpr int W = L == 256 ? 1 : 2;
  static constexpr int RSTRIDE = 3 * M + 16;  // elements between rows in shared memory
  static constexpr size_t SMEM = (size_t)RR * RSTRIDE * sizeof(C2<float>);
  // bank offset of row r (below 16, inside the row's stride)
  static __device__ __forceinline__ int base(int r) {
    return r * RSTRIDE + (T >= 16 ? (r * (16 / RR)) & 15 : (r >> 1) + 8 * (r & 1));
  }
  static constexpr int MINB = 65536 / (NT * 128) > 0 ? 65536 / (NT * 128) : 1;
  static_assert(L >= 256 && L <= 4096, "lattice sides of the register-staged row pass");
  static_assert(NT % 32 == 0 && T >= 8, "whole warps; rows of at least 8 threads");
  static_assert((M / W) * W == M && L % RR == 0, "tiles");
  static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
};

// Spectrum tile element e of the CTA's RR rows (consecutive e: consecutive
// numbers in HBM): component c, tile b, row rr, column w of the tile.
template <int L>
__device__ __forceinline__ void rrs_where(int e, int& c, int& b, int& rr, int& w) {
  using CF = RowRsCfg<L>;
  constexpr int CH = CF::RR * CF::W, NBK = CF::M / CF::W;  // numbers per tile chunk, tiles per component
  const int chunk = e / CH, in = e % CH;
  c = chunk / NBK;
  b = chunk % NBK;
  rr = in / CF::W;
  w = in % CF::W;
}

// Asynchronous copies of the CTA's spectrum rows into shared memory
// (complete with cp_async_wait_all() and a barrier).
template <int L>
__device__ __forceinline__ void rrs_load(C2<float>* sm, const C2<float>* __restrict__ spec, int r0) {
  using CF = RowRsCfg<L>;
  constexpr int TOT = 3 * CF::M * CF::RR, NBK = CF::M / CF::W;
#pragma unroll 4
  for (int e = threadIdx.x; e < TOT; e += CF::NT) {
    int c, b, rr, w;
    rrs_where<L>(e, c, b, rr, w);
    const size_t g = ((size_t)(c * NBK + b) * L + r0 + rr) * CF::W + w;
    cp_async_c2(sm + CF::base(rr) + c * CF::M + sw16(b * CF::W + w), spec + g);
  }
}

// Stores the CTA's spectrum rows, two numbers (16 bytes) per store: the
// pair (w, w + 1) of a tile row, or for W = 1 the same column of rows rr and
// rr + 1.
template <int L>
__device__ __forceinline__ void rrs_store(const C2<float>* sm, C2<float>* __restrict__ spec, int r0) {
  using CF = RowRsCfg<L>;
  constexpr int TOT = 3 * CF::M * CF::RR, NBK = CF::M / CF::W;
#pragma unroll 4
  for (int e2 = threadIdx.x; e2 < TOT / 2; e2 += CF::NT) {
    int c, b, rr, w;
    rrs_where<L>(2 * e2, c, b, rr, w);
    const size_t g = ((size_t)(c * NBK + b) * L + r0 + rr) * CF::W + w;
    const C2<float>* s0 = sm + CF::base(rr) + c * CF::M;
    C2<float> a, z;
    if constexpr (CF::W >= 2) {
      a = s0[sw16(b * CF::W + w)];
      z = s0[sw16(b * CF::W + w + 1)];
    } else {
      a = s0[sw16(b)];
      z = sm[CF::base(rr + 1) + c * CF::M + sw16(b)];
    }
    *reinterpret_cast<float4*>(spec + g) = make_float4(a.re, a.im, z.re, z.im);
  }
}

// The twist between the packed half spectrum Y of a real row and the
// half-length transform Z of z(n) = x(2n) + i x(2n+1), in place on the
// three sequences of row sequence base sq (digit-reversed positions).
// Inverse direction (before the inverse transform):
//   Z(k) = (Y(k) + Y*(M-k)) + i exp(+2 pi i k / L) (Y(k) - Y*(M-k)),
// forward direction (after the forward transform):
//   X(k) = [(Z(k) + Z*(M-k)) - i exp(-2 pi i k / L) (Z(k) - Z*(M-k))] / 2,
// and at k = 0 the packed pair (a, b) -> (a + b, a - b) both ways.  The
// partner of position q (frequency k) is pos(M - k); the thread holding the
// smaller position does the pair.
template <int L, bool FWD>
__device__ __forceinline__ void rrs_twist(C2<float>* sq, int t, const C2<float>* __restrict__ twr) {
  using CF = RowRsCfg<L>;
  using P = typename CF::P;
  constexpr int M = CF::M, T = CF::T;
  const float2* tq = reinterpret_cast<const float2*>(twr + P::TQOFF);
#pragma unroll 2
  for (int j = 0; j < P::E; j++) {
    const int q = t + j * T;
    const int k = P::freq_d(q);
    if (k == 0) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const C2<float> z = sq[c * M + sw16(q)];
        sq[c * M + sw16(q)] = mk(z.re + z.im, z.re - z.im);
      }
      continue;
    }
    const int q2 = P::pos_d(M - k);
    if (q2 < q) continue;
    const float2 x = __ldg(tq + q);  // exp(-2 pi i k / L)
    const C2<float> wk = FWD ? mk(x.x, x.y) : mk(x.x, -x.y);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const C2<float> a = sq[c * M + sw16(q)], b = sq[c * M + sw16(q2)];
      const C2<float> tt = wk * (a - conj(b));
      if (FWD) {
        sq[c * M + sw16(q)] = 0.5f * ((a + conj(b)) - mul_i(tt));
        if (q2 != q) sq[c * M + sw16(q2)] = 0.5f * ((b + conj(a)) - mul_i(conj(tt)));
      } else {
        sq[c * M + sw16(q)] = (a + conj(b)) + mul_i(tt);
        if (q2 != q) sq[c * M + sw16(q2)] = (b + conj(a)) + mul_i(conj(tt));
      }
    }
  }
}

// Forward stage 1 butterfly i of thread t on z[c][k] (positions
// t + (i + k K1) T, natural order, three components), written to shared
// memory; tw = the butterfly's twiddles.
template <int L>
__device__ __forceinline__ void rrs_forward1(C2<float>* sq, int t, int i, C2<float> (&z)[3][RowPlan<L / 2>::R1],
                                             const C2<float> (&tw)[15]) {
  using CF = RowRsCfg<L>;
  using P = typename CF::P;
  constexpr int R1 = P::R1, K1 = P::E / R1, D = P::stride(1), M = CF::M, T = CF::T;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    Bfly<float, R1, false, true>::run(z[c]);
    if constexpr (D > 1) {
#pragma unroll
      for (int k = 1; k < R1; k++) z[c][k] = z[c][k] * tw[k - 1];
    }
#pragma unroll
    for (int k = 0; k < R1; k++) sq[c * M + sw16(t + (i + k * K1) * T)] = z[c][k];
  }
}

// Forward stages 2 .. S, the forward twist and the store (each step
// preceded by a barrier), after forward stage 1 has written shared memory.
template <int L>
__device__ __forceinline__ void rrs_forward_tail(C2<float>* sm, C2<float>* sq, int t, const C2<float>* __restrict__ twr,
                                                 C2<float>* __restrict__ spec, int r0) {
  using CF = RowRsCfg<L>;
  using P = typename CF::P;
  p16_forward_mid<P, CF::M>(sq, t, twr);
  if constexpr (P::S >= 2) {
    __syncthreads();
    p16_stage<P, P::S, false, CF::M>(sq, t, twr);
  }
  __syncthreads();
  rrs_twist<L, true>(sq, t, twr);
  __syncthreads();
  rrs_store<L>(sm, spec, r0);
}

// Pixel pair (2n, 2n+1) of row x2: the augmented-Lagrangian update of the
// row pass (see row_pass in passes.cuh), in registers.  zc[c] holds
// e_c(2n) + i e_c(2n+1) of the compatible strain of iterate n+1 and receives
// p_c(2n) + i p_c(2n+1) of the next polarization.  lane_left: the thread
// holding n - 1 is the previous lane of this warp (else sigma at x - e1 is
// read from memory).
template <int L>
__device__ __forceinline__ void rrs_pixel_pair(int x2, int n, bool lane_left, C2<float> (&zc)[3], const float E[4],
                                               const float* __restrict__ sin_, float* __restrict__ eout,
                                               float* __restrict__ sout, const uint8_t* __restrict__ mask,
                                               const Mat<float>& m, float (&acc)[N_ACC]) {
  const size_t row = (size_t)x2 * L, up = (size_t)((x2 + L - 1) & (L - 1)) * L;
  const int x1 = 2 * n;
  const float4 s0 = __ldg(reinterpret_cast<const float4*>(sin_) + row + x1);
  const float4 s1 = __ldg(reinterpret_cast<const float4*>(sin_) + row + x1 + 1);
  const float4 u0 = __ldg(reinterpret_cast<const float4*>(sin_) + up + x1);
  const float4 u1 = __ldg(reinterpret_cast<const float4*>(sin_) + up + x1 + 1);
  const uint16_t mv = __ldg(reinterpret_cast<const unsigned short*>(mask + row + x1));
  // sigma11, sigma12 of pixel 2n - 1 (periodic)
  float l11 = __shfl_up_sync(0xffffffffu, s1.x, 1);
  float l12 = __shfl_up_sync(0xffffffffu, s1.w, 1);
  if (!lane_left) {
    const float4 sl = __ldg(reinterpret_cast<const float4*>(sin_) + row + ((x1 + L - 1) & (L - 1)));
    l11 = sl.x;
    l12 = sl.w;
  }
  const float sg[2][4] = {{s0.x, s0.y, s0.z, s0.w}, {s1.x, s1.y, s1.z, s1.w}};
  const float up12[2] = {u0.w, u1.w}, up22[2] = {u0.y, u1.y};
  const float left11[2] = {l11, s0.x}, left12[2] = {l12, s0.w};
  float pr[2][3];
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const bool v = ((mv >> (8 * h)) & 0xff) != 0;
    // Eq. 1: div_i = sum_j sigma_ij(x) - sigma_ij(x - e^j)
    const float d1 = (sg[h][0] - left11[h]) + (sg[h][3] - up12[h]);
    const float d2 = (sg[h][3] - left12[h]) + (sg[h][1] - up22[h]);
#pragma unroll
    for (int c = 0; c < 4; c++) acc[A_S11 + c] += sg[h][c];
    acc[A_DIV2] += d1 * d1 + d2 * d2;
    const float e[4] = {h ? zc[0].im : zc[0].re, h ? zc[1].im : zc[1].re, E[2], h ? zc[2].im : zc[2].re};
    float c0[4], tau[4], e1[4], s1v[4], p1[3];
    c0_apply(e, m, c0);
#pragma unroll
    for (int c = 0; c < 4; c++) tau[c] = sg[h][c] + c0[c];
    local_solve_p(tau, v, m, e1, s1v, p1);
    *reinterpret_cast<float4*>(eout + 4 * (row + x1 + h)) = make_float4(e1[0], e1[1], e1[2], e1[3]);
    *reinterpret_cast<float4*>(sout + 4 * (row + x1 + h)) = make_float4(s1v[0], s1v[1], s1v[2], s1v[3]);
#pragma unroll
    for (int c = 0; c < 4; c++) acc[A_E11 + c] += e1[c];
    acc[A_NPL] += is_plastic(e1, v, m) ? 1.f : 0.f;
    const float q0 = e1[0] - e[0], q1 = e1[1] - e[1], q2 = e1[2] - e[2], q3 = e1[3] - e[3];
    acc[A_COMP] += q0 * q0 + q1 * q1 + q2 * q2 + 2.f * q3 * q3;
    pr[h][0] = p1[0];
    pr[h][1] = p1[1];
    pr[h][2] = p1[2];
  }
#pragma unroll
  for (int c = 0; c < 3; c++) zc[c] = mk(pr[0][c], pr[1][c]);
}

// Warm start of pixel pair (2n, 2n+1) of row x2 (phase INIT, see row_pass):
// eps^0 = accepted state + dE, its stress, the plastic flags of the accepted
// state (increments after the first), and the polarization into zc.
template <int L>
__device__ __forceinline__ void rrs_init_pair(int x2, int n, C2<float> (&zc)[3], const float dE[4],
                                              const float* __restrict__ ein, float* __restrict__ eout,
                                              float* __restrict__ sout, const uint8_t* __restrict__ mask,
                                              uint8_t* __restrict__ fl, const Mat<float>& m, float (&acc)[N_ACC]) {
  const size_t x = (size_t)x2 * L + 2 * n;
  float pr[2][3];
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const bool v = mask[x + h] != 0;
    float e[4], s[4], c0[4];
    Vec4<float>::load(ein + 4 * (x + h), e);
    if (fl) fl[x + h] = is_plastic(e, v, m);
#pragma unroll
    for (int c = 0; c < 4; c++) e[c] += dE[c];
    Vec4<float>::store(eout + 4 * (x + h), e);
    const bool pl = sigma(e, v, m, s);
    Vec4<float>::store(sout + 4 * (x + h), s);
#pragma unroll
    for (int c = 0; c < 4; c++) acc[A_E11 + c] += e[c];
    acc[A_NPL] += pl ? 1.f : 0.f;
    c0_apply(e, m, c0);
    pr[h][0] = s[0] - c0[0];
    pr[h][1] = s[1] - c0[1];
    pr[h][2] = s[3] - c0[3];
  }
#pragma unroll
  for (int c = 0; c < 3; c++) zc[c] = mk(pr[0][c], pr[1][c]);
}

// The row pass, tiling variant 2.  Grid: (L / RR, solves).  The launch
// shape is checked on entry; for that shape every index below is in range
// (rows r0 + rr < L, positions < M, pixels < L, tiles < M / W).
template <int L>
__global__ void __launch_bounds__(RowRsCfg<L>::NT, RowRsCfg<L>::MINB)
row_pass_rs(Solve* __restrict__ solves, int nb, BatchCtl* bc, const C2<float>* __restrict__ twr,
            cudaGraphConditionalHandle cond, int use_cond) {
  using CF = RowRsCfg<L>;
  using P = typename CF::P;
  constexpr int M = CF::M, T = CF::T, RR = CF::RR, NT = CF::NT, R1 = P::R1, K1 = P::E / R1;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ bool s_last;
  if (!ECHK(blockDim.x - 1, NT, 50) || !ECHK(gridDim.x - 1, L / RR, 50)) return;
  Solve& S = solves[blockIdx.y];
  const volatile Solve& Sv = S;
  const int phase = Sv.phase;
  const int cur = Sv.cur;
  const int inc = Sv.inc;
  const int tid = threadIdx.x, rr = tid / T, t = tid % T, lane = tid & 31;
  const int r0 = blockIdx.x * RR, x2 = r0 + rr;
  C2<float>* sm = reinterpret_cast<C2<float>*>(smraw);
  C2<float>* sq = sm + CF::base(rr);
  float acc[N_ACC];
#pragma unroll
  for (int i = 0; i < N_ACC; i++) acc[i] = 0.f;
  if (phase != PH_DONE) {
    const float* __restrict__ ein = reinterpret_cast<const float*>(S.eps[cur]);
    float* __restrict__ eout = reinterpret_cast<float*>(S.eps[1 - cur]);
    const float* __restrict__ sin_ = reinterpret_cast<const float*>(S.sig[cur]);
    float* __restrict__ sout = reinterpret_cast<float*>(S.sig[1 - cur]);
    C2<float>* spec = reinterpret_cast<C2<float>*>(S.spec);
    const uint8_t* __restrict__ mask = S.mask;
    const Mat<float> m = make_mat<float>(S);
    const size_t LL = (size_t)L * L;
    if (phase == PH_FINAL) {
      // plastic flags of the accepted state of the last increment
      uint8_t* fl = S.flags ? S.flags + (size_t)(S.n_inc - 1) * LL : nullptr;
      for (int j = 0; j < P::E && fl; j++) {
        const size_t x = (size_t)x2 * L + 2 * (t + j * T);
#pragma unroll
        for (int h = 0; h < 2; h++) {
          float e[4];
          Vec4<float>::load(ein + 4 * (x + h), e);
          fl[x + h] = is_plastic(e, mask[x + h] != 0, m);
        }
      }
    } else {
      if (phase == PH_INIT) {
        float dE[4];
        const double* Ep = S.path + 4 * (ECHK(inc, S.n_inc, 51) ? inc : 0);
        for (int c = 0; c < 4; c++) dE[c] = float(Ep[c] - Sv.Eprev[c]);
        uint8_t* fl = (S.flags && inc > 0) ? S.flags + (size_t)(inc - 1) * LL : nullptr;
#pragma unroll 1
        for (int i = 0; i < K1; i++) {
          C2<float> tw[15];
          p16_twiddles_i<P, 1>(twr, t, i, tw);
          C2<float> z[3][R1];
#pragma unroll
          for (int k = 0; k < R1; k++) {
            C2<float> zc[3];
            rrs_init_pair<L>(x2, t + (i + k * K1) * T, zc, dE, ein, eout, sout, mask, fl, m, acc);
#pragma unroll
            for (int c = 0; c < 3; c++) z[c][k] = zc[c];
          }
          rrs_forward1<L>(sq, t, i, z, tw);
        }
      } else {  // PH_ITER
        float E[4];
        load_E(S.path + 4 * inc, E);
        rrs_load<L>(sm, spec, r0);
        // sigma of the RR rows and of the row above them, and the void
        // flags, are asked of the L2 (16 KB pieces, one per lane of warp 0)
        // while the spectrum is transformed, after its copies were issued
        if (tid < 32) {
          constexpr unsigned RB = (unsigned)(L * 16), PB = RB < 16384u ? RB : 16384u;
          constexpr int NPR = (int)(RB / PB), NPC = (RR + 1) * NPR;
          const int xh = (r0 + L - 1) & (L - 1);
          for (int i = tid; i < NPC; i += 32) {
            const int k = i / NPR, row = k < RR ? r0 + k : xh;
            prefetch_l2(reinterpret_cast<const char*>(sin_ + (size_t)4 * row * L) + (size_t)(i % NPR) * PB, PB);
          }
          if (tid == 31) prefetch_l2(mask + (size_t)r0 * L, (unsigned)(RR * L));
        }
        cp_async_wait_all();
        __syncthreads();
        rrs_twist<L, false>(sq, t, twr);
        __syncthreads();
        // inverse stages S .. 2 (the first one after the twist's barrier)
        if constexpr (P::S >= 2) {
          p16_stage<P, P::S, true, M>(sq, t, twr);
          __syncthreads();
          p16_inverse_mid<P, M>(sq, t, twr);
        }
        // inverse stage 1, the pixel update and forward stage 1, a butterfly
        // (R1 positions, three components) at a time
        const bool lane_left = t > 0 && lane > 0;
#pragma unroll 1
        for (int i = 0; i < K1; i++) {
          C2<float> tw[15];
          p16_twiddles_i<P, 1>(twr, t, i, tw);
          C2<float> z[3][R1];
#pragma unroll
          for (int c = 0; c < 3; c++) {
#pragma unroll
            for (int k = 0; k < R1; k++) z[c][k] = sq[c * M + sw16(t + (i + k * K1) * T)];
            if constexpr (P::stride(1) > 1) {
#pragma unroll
              for (int k = 1; k < R1; k++) z[c][k] = z[c][k] * conj(tw[k - 1]);
            }
            Bfly<float, R1, true, true>::run(z[c]);
          }
#pragma unroll
          for (int k = 0; k < R1; k++) {
            C2<float> zc[3] = {z[0][k], z[1][k], z[2][k]};
            rrs_pixel_pair<L>(x2, t + (i + k * K1) * T, lane_left, zc, E, sin_, eout, sout, mask, m, acc);
#pragma unroll
            for (int c = 0; c < 3; c++) z[c][k] = zc[c];
          }
          rrs_forward1<L>(sq, t, i, z, tw);
        }
      }
      rrs_forward_tail<L>(sm, sq, t, twr, spec, r0);
      block_reduce_acc<NT>(acc, S.partials + (size_t)blockIdx.x * PART_STRIDE);
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

// Row transforms alone (tiling variant 2): the forward transform of three
// planes p (p11, p22, p12, L x L reals each) into the stored spectrum, and
// the inverse of the stored spectrum into three planes e.
template <int L>
__global__ void __launch_bounds__(RowRsCfg<L>::NT)
row_forward_rs(const float* __restrict__ p, C2<float>* __restrict__ spec, const C2<float>* __restrict__ twr) {
  using CF = RowRsCfg<L>;
  using P = typename CF::P;
  constexpr int T = CF::T, RR = CF::RR, NT = CF::NT, R1 = P::R1, K1 = P::E / R1;
  extern __shared__ __align__(16) unsigned char smraw[];
  if (!ECHK(blockDim.x - 1, NT, 52) || !ECHK(gridDim.x - 1, L / RR, 52)) return;
  const int tid = threadIdx.x, rr = tid / T, t = tid % T;
  const int r0 = blockIdx.x * RR, x2 = r0 + rr;
  C2<float>* sm = reinterpret_cast<C2<float>*>(smraw);
  C2<float>* sq = sm + CF::base(rr);
  const size_t LL = (size_t)L * L;
#pragma unroll 1
  for (int i = 0; i < K1; i++) {
    C2<float> tw[15];
    p16_twiddles_i<P, 1>(twr, t, i, tw);
    C2<float> z[3][R1];
#pragma unroll
    for (int k = 0; k < R1; k++) {
      const size_t x = (size_t)x2 * L + 2 * (t + (i + k * K1) * T);
#pragma unroll
      for (int c = 0; c < 3; c++) z[c][k] = mk(p[c * LL + x], p[c * LL + x + 1]);
    }
    rrs_forward1<L>(sq, t, i, z, tw);
  }
  rrs_forward_tail<L>(sm, sq, t, twr, spec, r0);
}

template <int L>
__global__ void __launch_bounds__(RowRsCfg<L>::NT)
row_inverse_rs(const C2<float>* __restrict__ spec, float* __restrict__ e, const C2<float>* __restrict__ twr) {
  using CF = RowRsCfg<L>;
  using P = typename CF::P;
  constexpr int M = CF::M, T = CF::T, RR = CF::RR, NT = CF::NT, R1 = P::R1, K1 = P::E / R1;
  extern __shared__ __align__(16) unsigned char smraw[];
  if (!ECHK(blockDim.x - 1, NT, 53) || !ECHK(gridDim.x - 1, L / RR, 53)) return;
  const int tid = threadIdx.x, rr = tid / T, t = tid % T;
  const int r0 = blockIdx.x * RR, x2 = r0 + rr;
  C2<float>* sm = reinterpret_cast<C2<float>*>(smraw);
  C2<float>* sq = sm + CF::base(rr);
  const size_t LL = (size_t)L * L;
  rrs_load<L>(sm, spec, r0);
  cp_async_wait_all();
  __syncthreads();
  rrs_twist<L, false>(sq, t, twr);
  __syncthreads();
  if constexpr (P::S >= 2) {
    p16_stage<P, P::S, true, M>(sq, t, twr);
    __syncthreads();
    p16_inverse_mid<P, M>(sq, t, twr);
  }
#pragma unroll 1
  for (int i = 0; i < K1; i++) {
    C2<float> tw[15];
    p16_twiddles_i<P, 1>(twr, t, i, tw);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      C2<float> z[R1];
#pragma unroll
      for (int k = 0; k < R1; k++) z[k] = sq[c * M + sw16(t + (i + k * K1) * T)];
      if constexpr (P::stride(1) > 1) {
#pragma unroll
        for (int k = 1; k < R1; k++) z[k] = z[k] * conj(tw[k - 1]);
      }
      Bfly<float, R1, true, true>::run(z);
#pragma unroll
      for (int k = 0; k < R1; k++) {
        const size_t x = (size_t)x2 * L + 2 * (t + (i + k * K1) * T);
        e[c * LL + x] = z[k].re;
        e[c * LL + x + 1] = z[k].im;
      }
    }
  }
}

}  // namespace epfft
