// On-chip schedule for small FP32 lattices (tiling 3, L = 16, 32, 64): one
// CTA runs a whole solve (every increment and iteration of the
// augmented-Lagrangian scheme, Sec. 1-2) without leaving the kernel.  The
// spectrum lives in shared memory in two layouts, rows (the half-length row
// transforms) and columns (the column transforms and the Green operator of
// Eq. 3); a transpose in shared memory joins them.  Strain and stress of the
// iterates stay in their global ping-pong buffers (a few hundred KB per
// solve, L2-resident).  Each step does what one step of the two-pass loop
// does, [column pass, row pass], with the same pixel update, residual,
// reductions and state machine (finalize_solve); a batch is one CTA per
// solve.  The per-CTA sums run in another order than the two-pass loop's, so
// the results agree with it to FP32 rounding, not bit for bit.
#pragma once
#include "passes.cuh"

namespace epfft {

template <int L>
struct OnChip {
  // threads: enough for one call per transform (16 elements per thread and
  // stage), few enough that the transforms and the pixel update keep their
  // registers (170 at 384 threads)
  static constexpr int M = L / 2, NT = L == 64 ? 384 : 256;
  using PS = PlanSel<float, L, 0>;
  using PR = FftPlan<M, PS::RM_ROW, PS::FULL>;
  using PC = FftPlan<L, PS::RM_COL, PS::FULL>;
  using TB = Tables<float, L>;
  static constexpr int SPR = seq_stride<M>(), SPC = seq_stride<L>();
  static constexpr int RSZ = 3 * L * SPR;  // rows: sequence c L + x2, element k at pad32(k)
  static constexpr int CSZ = 3 * M * SPC;  // columns: sequence c M + m1, element x2 at pad32(x2)
  static constexpr int RTW = PR::TW_ENTRIES, CTW = PC::TW_ENTRIES, OCT = TB::OCT;
  static constexpr int OFF_C = RSZ, OFF_RT = RSZ + CSZ, OFF_CT = OFF_RT + RTW, OFF_OCT = OFF_CT + CTW;
  static constexpr size_t SMEM = (size_t)(OFF_OCT + OCT) * sizeof(C2<float>);
  static_assert(L >= 16 && L <= 64, "on-chip sides");
  static_assert(3 * L * M <= 16 * NT, "row and column transforms in one call each");
  static_assert(SMEM <= 200 * 1024, "shared memory per CTA");
  // index of element k of row sequence (c, x2) / element x2 of column (c, m1)
  static __device__ __forceinline__ int ri(int c, int x2, int k) { return (c * L + x2) * SPR + pad32(k); }
  static __device__ __forceinline__ int ci(int c, int m1, int x2) { return OFF_C + (c * M + m1) * SPC + pad32(x2); }
  // real value of pixel x1 of component c, row x2 (row layout)
  static __device__ __forceinline__ float& px(C2<float>* s, int c, int x2, int x1) {
    return reinterpret_cast<float*>(s)[2 * ri(c, x2, x1 >> 1) + (x1 & 1)];
  }
};

// Half spectrum <-> z transforms of the half-length row transforms (the twists
// of RowIO) over all 3 L row sequences; oct: twist octant.
template <int L, bool FWD>
__device__ __forceinline__ void oc_twist(C2<float>* s, const C2<float>* __restrict__ oct) {
  using O = OnChip<L>;
  constexpr int M = O::M, HK = M / 2, NSEQ = 3 * L;
  for (int i = threadIdx.x; i < HK * NSEQ; i += O::NT) {
    const int k = 1 + i % HK, sq = i / HK, kk = M - k;
    C2<float>* q = s + sq * O::SPR;
    const int ik = pad32(k), ikk = pad32(kk);
    const C2<float> a = q[ik], b = q[ikk];
    if (FWD) {
      const C2<float> wk = twist_tw<float, L>(oct, k);
      const C2<float> t = wk * (a - conj(b));
      q[ik] = 0.5f * ((a + conj(b)) - mul_i(t));
      if (kk != k) q[ikk] = 0.5f * ((b + conj(a)) - mul_i(conj(t)));
    } else {
      const C2<float> wk = conj(twist_tw<float, L>(oct, k));
      const C2<float> t = wk * (a - conj(b));
      q[ik] = (a + conj(b)) + mul_i(t);
      if (kk != k) q[ikk] = (b + conj(a)) + mul_i(conj(t));
    }
  }
  for (int sq = threadIdx.x; sq < NSEQ; sq += O::NT) {
    C2<float>* q = s + sq * O::SPR;
    const C2<float> z = q[0];
    q[0] = mk(z.re + z.im, z.re - z.im);
  }
  __syncthreads();
}

// Transposes between the row and the column layout (R -> C when TO_COL).
template <int L, bool TO_COL>
__device__ __forceinline__ void oc_transpose(C2<float>* s) {
  using O = OnChip<L>;
  constexpr int M = O::M;
  for (int e = threadIdx.x; e < 3 * L * M; e += O::NT) {
    const int c = e / (L * M), rem = e - c * (L * M);
    const int x2 = rem / M, m1 = rem - x2 * M;
    if (TO_COL) s[O::ci(c, m1, x2)] = s[O::ri(c, x2, m1)];
    else s[O::ri(c, x2, m1)] = s[O::ci(c, m1, x2)];
  }
  __syncthreads();
}

// Whole solves on chip.  Grid: one CTA of OnChip<L>::NT threads per solve.
// bound: loop steps a solve may take (n_inc (max_iter + 2) + 9); a solve
// that reaches it stops and sets bc->timed_out.
template <int L>
__global__ void __launch_bounds__(OnChip<L>::NT, 1)
solve_onchip(Solve* __restrict__ solves, BatchCtl* bc, const C2<float>* __restrict__ tw,
             const C2<float>* __restrict__ ktab) {
  using O = OnChip<L>;
  constexpr int M = O::M, NT = O::NT;
  constexpr size_t LL = (size_t)L * L;
  extern __shared__ __align__(16) unsigned char smraw[];
  C2<float>* s = reinterpret_cast<C2<float>*>(smraw);
  const C2<float>* rtw = s + O::OFF_RT;
  const C2<float>* ctw = s + O::OFF_CT;
  const C2<float>* oct = s + O::OFF_OCT;
  __shared__ int s_phase;
  __shared__ double tot[N_ACC];
  if (!ECHK(blockDim.x - 1, NT, 80)) return;
  Solve& S = solves[blockIdx.x];
  const int tid = threadIdx.x;
  copy_table<float, NT>(s + O::OFF_RT, tw + O::TB::off_row(0), O::RTW);
  copy_table<float, NT>(s + O::OFF_CT, tw + O::TB::off_col(0), O::CTW);
  copy_table<float, NT>(s + O::OFF_OCT, tw, O::OCT);
  cp_async_wait_all();
  const Mat<float> m = make_mat<float>(S);
  const uint8_t* __restrict__ mask = S.mask;
  const float lam0 = float(S.lam0), mu0 = float(S.mu0), scale = float(1.0 / ((double)L * (double)L));
  const C2<float>* __restrict__ qtab = ktab + L;
  const int64_t bound = (int64_t)S.n_inc * ((int64_t)S.max_iter + 2) + 9;
  __syncthreads();
  for (int64_t step = 0;; step++) {
    if (tid == 0) s_phase = *(volatile int32_t*)&S.phase;
    __syncthreads();
    const int phase = s_phase;
    if (phase == PH_DONE) break;
    if (step >= bound) {
      if (tid == 0) atomicOr(&bc->timed_out, 1);
      break;
    }
    const int cur = *(volatile int32_t*)&S.cur, inc = *(volatile int32_t*)&S.inc;
    // ---- column phase (ITER): forward column transforms, Eq. 3, inverse ----
    if (phase == PH_ITER) {
      oc_transpose<L, true>(s);
      fft_seq<float, L, O::PS::RM_COL, O::PS::FULL, 3 * M, NT, false>(s + O::OFF_C, ctw);
      const int gm = S.green;
      for (int f = tid; f < (M - 1) * L; f += NT) {
        const int m1 = 1 + f / L, m2 = f % L;
        C2<float>& p11 = s[O::ci(0, m1, m2)];
        C2<float>& p22 = s[O::ci(1, m1, m2)];
        C2<float>& p12 = s[O::ci(2, m1, m2)];
        green_op(gm, ktab, qtab, L, m1, m2, lam0, mu0, scale, p11, p22, p12);
      }
      // packed column: Z = A + i B, A the m1 = 0 column, B the m1 = L/2 one
      const double* Ep = S.path + 4 * inc;
      for (int m2 = tid; m2 <= L / 2; m2 += NT) {
        const int mp = (L - m2) & (L - 1);
        C2<float> A[3], Bq[3], Ap[3], Bp[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
          const C2<float> z = s[O::ci(c, 0, m2)], zp = s[O::ci(c, 0, mp)];
          A[c] = 0.5f * (z + conj(zp));
          const C2<float> d = z - conj(zp);
          Bq[c] = mk(0.5f * d.im, -0.5f * d.re);
          Ap[c] = conj(A[c]);
          Bp[c] = conj(Bq[c]);
        }
        if (m2 == 0) {
          const float z = S.zero_mean ? 0.0f : 1.0f;
          A[0] = mk(z * float(Ep[0]), 0.0f);
          A[1] = mk(z * float(Ep[1]), 0.0f);
          A[2] = mk(z * float(Ep[3]), 0.0f);
        } else {
          green_op(gm, ktab, qtab, L, 0, m2, lam0, mu0, scale, A[0], A[1], A[2]);
          green_op(gm, ktab, qtab, L, 0, mp, lam0, mu0, scale, Ap[0], Ap[1], Ap[2]);
        }
        green_op(gm, ktab, qtab, L, M, m2, lam0, mu0, scale, Bq[0], Bq[1], Bq[2]);
        green_op(gm, ktab, qtab, L, M, mp, lam0, mu0, scale, Bp[0], Bp[1], Bp[2]);
#pragma unroll
        for (int c = 0; c < 3; c++) {
          s[O::ci(c, 0, m2)] = A[c] + mul_i(Bq[c]);
          if (mp != m2) s[O::ci(c, 0, mp)] = Ap[c] + mul_i(Bp[c]);
        }
      }
      __syncthreads();
      fft_seq<float, L, O::PS::RM_COL, O::PS::FULL, 3 * M, NT, true>(s + O::OFF_C, ctw);
      oc_transpose<L, false>(s);
    }
    // ---- row phase ----
    const float* __restrict__ ein = reinterpret_cast<const float*>(S.eps[cur]);
    float* __restrict__ eout = reinterpret_cast<float*>(S.eps[1 - cur]);
    const float* __restrict__ sin_ = reinterpret_cast<const float*>(S.sig[cur]);
    float* __restrict__ sout = reinterpret_cast<float*>(S.sig[1 - cur]);
    float acc[N_ACC];
#pragma unroll
    for (int i = 0; i < N_ACC; i++) acc[i] = 0.0f;
    if (phase == PH_FINAL) {
      uint8_t* fl = S.flags ? S.flags + (size_t)(S.n_inc - 1) * LL : nullptr;
      for (int x = tid; x < (int)LL && fl; x += NT) {
        float e[4];
        Vec4<float>::load(ein + 4 * x, e);
        fl[x] = is_plastic(e, mask[x] != 0, m);
      }
    } else if (phase == PH_INIT) {
      float dE[4];
      const double* E = S.path + 4 * (ECHK(inc, S.n_inc, 81) ? inc : 0);
      for (int c = 0; c < 4; c++) dE[c] = float(E[c] - S.Eprev[c]);
      uint8_t* fl = (S.flags && inc > 0) ? S.flags + (size_t)(inc - 1) * LL : nullptr;
      for (int x = tid; x < (int)LL; x += NT) {
        const bool v = mask[x] != 0;
        float e[4], sg[4], c0[4];
        Vec4<float>::load(ein + 4 * x, e);
        if (fl) fl[x] = is_plastic(e, v, m);
        for (int c = 0; c < 4; c++) e[c] += dE[c];
        Vec4<float>::store(eout + 4 * x, e);
        const bool pl = sigma(e, v, m, sg);
        Vec4<float>::store(sout + 4 * x, sg);
#pragma unroll
        for (int c = 0; c < 4; c++) acc[A_E11 + c] += e[c];
        acc[A_NPL] += pl ? 1.0f : 0.0f;
        c0_apply(e, m, c0);
        const int x2 = x / L, x1 = x % L;
        O::px(s, 0, x2, x1) = sg[0] - c0[0];
        O::px(s, 1, x2, x1) = sg[1] - c0[1];
        O::px(s, 2, x2, x1) = sg[3] - c0[3];
      }
    } else {  // PH_ITER
      float E[4];
      load_E(S.path + 4 * inc, E);
      oc_twist<L, false>(s, oct);
      fft_seq<float, M, O::PS::RM_ROW, O::PS::FULL, 3 * L, NT, true>(s, rtw);
      for (int x = tid; x < (int)LL; x += NT) {
        const int x2 = x / L, x1 = x % L;
        const int xl = x2 * L + ((x1 + L - 1) & (L - 1)), xu = ((x2 + L - 1) & (L - 1)) * L + x1;
        const bool v = mask[x] != 0;
        float sj[4], sl[4], su[4];
        Vec4<float>::load(sin_ + 4 * x, sj);
        Vec4<float>::load(sin_ + 4 * xl, sl);
        Vec4<float>::load(sin_ + 4 * xu, su);
        // Eq. 1: div_i = sum_j sigma_ij(x) - sigma_ij(x - e^j)
        const float d1 = (sj[0] - sl[0]) + (sj[3] - su[3]);
        const float d2 = (sj[3] - sl[3]) + (sj[1] - su[1]);
#pragma unroll
        for (int c = 0; c < 4; c++) acc[A_S11 + c] += sj[c];
        acc[A_DIV2] += d1 * d1 + d2 * d2;
        float e[4] = {O::px(s, 0, x2, x1), O::px(s, 1, x2, x1), E[2], O::px(s, 2, x2, x1)};
        float c0[4], tau[4], e1[4], s1[4], p1[3];
        c0_apply(e, m, c0);
#pragma unroll
        for (int c = 0; c < 4; c++) tau[c] = sj[c] + c0[c];
        local_solve_p(tau, v, m, e1, s1, p1);
        Vec4<float>::store(eout + 4 * x, e1);
        Vec4<float>::store(sout + 4 * x, s1);
#pragma unroll
        for (int c = 0; c < 4; c++) acc[A_E11 + c] += e1[c];
        acc[A_NPL] += is_plastic(e1, v, m) ? 1.0f : 0.0f;
        const float q0 = e1[0] - e[0], q1 = e1[1] - e[1], q2 = e1[2] - e[2], q3 = e1[3] - e[3];
        acc[A_COMP] += q0 * q0 + q1 * q1 + q2 * q2 + 2.0f * q3 * q3;
        O::px(s, 0, x2, x1) = p1[0];
        O::px(s, 1, x2, x1) = p1[1];
        O::px(s, 2, x2, x1) = p1[2];
      }
    }
    __syncthreads();
    if (phase == PH_ITER || phase == PH_INIT) {
      fft_seq<float, M, O::PS::RM_ROW, O::PS::FULL, 3 * L, NT, false>(s, rtw);
      oc_twist<L, true>(s, oct);
      block_reduce_acc<NT>(acc, S.partials);
      __syncthreads();
      sum_partials<NT, 1>(S.partials, tot);
    }
    __syncthreads();
    if (tid == 0) finalize_solve<L>(S, phase, tot);
    __syncthreads();
  }
}

}  // namespace epfft
