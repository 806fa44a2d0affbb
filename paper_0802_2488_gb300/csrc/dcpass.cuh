// The defect-correction form (EPFFT_FP32_DEFECT): FP32 iterations on the
// differences from an FP64 reference state.
//
// Every ref_every iterations of a solve (and after each warm start) a
// refresh, in FP64, makes the current iterate the reference: eps_ref, sigma_ref = sigma(eps_ref)
// from the law, p_ref = sigma_ref - C0:eps_ref, the compatible strain
// e_ref = E + Gamma(p_ref) (Eqs. 2-3) and tau_ref = sigma_ref + C0:eps_ref,
// which the local step maps back to eps_ref.  Between refreshes an iterate
// is eps = eps_ref + d_eps, sigma = sigma_ref + d_sig with FP32 differences,
// and one augmented-Lagrangian iteration (Sec. 1, the steps of the other
// passes) becomes, exactly in real arithmetic:
//   e^{n+1} - eps_ref = a_ref + Gamma(p^n - p_ref),  a_ref = e_ref - eps_ref,
//   p^n - p_ref = d_sig^n - C0:d_eps^n,
//   tau^{n+1} = tau_ref + d_tau,  d_tau = d_sig^n + C0:(e^{n+1} - eps_ref),
//   d_eps^{n+1} = LS(tau_ref + d_tau) - LS(tau_ref),  LS the local step,
//   d_sig^{n+1} = sigma(eps_ref + d_eps^{n+1}) - sigma_ref,
//   div sigma^n = div sigma_ref + div d_sig^n.
// The FP32 transforms carry only p - p_ref, the local step is evaluated as a
// difference with formulas that keep FP32 accuracy relative to the
// difference (delta_step), and the reference terms a_ref, div sigma_ref
// are per-pixel FP32 numbers that shrink with the residual.  So the rounding
// of every FP32 quantity scales with how far the iterate moved since the
// last refresh, and the iteration reaches the FP64 scheme's tolerances
// (eta1, eta2 of Sec. 2); the indicators and means add the FP64 reference
// sums to FP32 (hi, lo) sums of the differences.
#pragma once
#include "passes.cuh"

namespace epfft {

// FP32 constants of the delta step.
struct DcConst {
  float ce;       // 1 / (2 (mu + mu0)): elastic deviator of the local step
  float cp;       // 1 / (2 mu0): plastic and void deviator
  float ge;       // mu / (mu + mu0): elastic stress deviator per unit tau'
  float ylim;     // sqrt(2/3) Y
  float ry;       // sqrt(2/3) Y / (2 mu0)
  float jc;       // mu / ((mu + mu0) 2 mu0)
  float tstar;    // |tau'| of the plastic threshold
  float tstar2;
  float two_mu0, lam0;
  float k3;       // 3 K
  float cm, cv;   // 1 / (3 (K + K0)), 1 / (3 K0): mean part of the local step
};

__device__ __forceinline__ DcConst dc_consts(const Solve& S) {
  const float* c = S.mcf;
  DcConst k;
  k.ce = c[MC_INV_2MUMU0];
  k.cp = c[MC_INV_2MU0];
  k.ge = c[MC_GSC_EL];
  k.ylim = c[MC_YLIM];
  k.ry = c[MC_RY];
  k.jc = c[MC_JC];
  k.tstar = c[MC_TSTAR];
  k.tstar2 = c[MC_TSTAR2];
  k.two_mu0 = c[MC_TWO_MU0];
  k.lam0 = c[MC_LAM0];
  k.k3 = c[MC_3K];
  k.cm = c[MC_INV_3KK0];
  k.cv = c[MC_INV_3K0];
  return k;
}

// Differences of the local step (local_solve_p) and of the stress of its
// solution between tau_ref and tau_ref + dt, in FP32.  t: the deviator of
// tau_ref (11, 22, 33, 12), h = |t|^2 - T*^2 (formed in FP64, so exact to
// FP32 rounding even near the threshold T* = sqrt(2/3) Y (mu + mu0) / mu).
// The deviatoric map is phi(s) = s ce (elastic, mu |s| / (mu + mu0) <=
// sqrt(2/3) Y) or s cp - ry n(s) (plastic), n(s) = s / |s|; its stress is
// psi(s) = ge s or ylim n(s).  With a = |t|, b = |t + dt|:
//   n(t + dt) - n(t) = dt / b - t (2 t.dt + |dt|^2) / (a b (a + b)),
//   |t + dt|^2 - T*^2 = h + 2 t.dt + |dt|^2,
// and across the threshold phi_P - phi_E = J, psi_P - psi_E = -2 mu0 J with
//   J(s) = n(s) jc (|s| - T*),  |s| - T* = (|s|^2 - T*^2) / (|s| + T*),
// all of them differences formed without cancellation.  Voids: phi = s cp,
// psi = 0.  The mean part is linear.  Returns the branch at tau_ref + dt.
__device__ __forceinline__ bool delta_step(const float t[4], float h, const float dt[4], bool is_void,
                                           const DcConst& k, float de[4], float ds[4]) {
  const float dm = (dt[0] + dt[1] + dt[2]) * (1.0f / 3.0f);
  const float d[4] = {dt[0] - dm, dt[1] - dm, dt[2] - dm, dt[3]};
  if (is_void) {
    const float em = dm * k.cv;
#pragma unroll
    for (int i = 0; i < 4; i++) {
      de[i] = d[i] * k.cp + (i < 3 ? em : 0.0f);
      ds[i] = 0.0f;
    }
    return false;
  }
  const float em = dm * k.cm, sm = k.k3 * em;
  const float tdt = t[0] * d[0] + t[1] * d[1] + t[2] * d[2] + 2.0f * t[3] * d[3];
  const float dd2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + 2.0f * d[3] * d[3];
  const float w = 2.0f * tdt + dd2;  // |t + dt|^2 - |t|^2
  const float hb = h + w;
  const bool pa = h > 0.0f, pb = hb > 0.0f;
  float e[4], s[4];
  if (!pa && !pb) {
#pragma unroll
    for (int i = 0; i < 4; i++) {
      e[i] = d[i] * k.ce;
      s[i] = d[i] * k.ge;
    }
  } else {
    const float b2 = fmaxf((h + k.tstar2) + w, 0.0f);
    const float rb = b2 > 0.0f ? rsqrtf(b2) : 0.0f;
    const float b = b2 * rb;
    if (pa && b2 <= 1e-12f * (h + k.tstar2)) {
      // t + dt = 0 (to rounding) from the plastic branch: phi(0) - phi(t),
      // psi(0) - psi(t), with n(t) = t / a
      const float ra = rsqrtf(h + k.tstar2);
#pragma unroll
      for (int i = 0; i < 4; i++) {
        e[i] = -(t[i] * k.cp - k.ry * (t[i] * ra));
        s[i] = -k.ylim * (t[i] * ra);
      }
    } else {
      float J[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      if (pa != pb) {
        const float jf = k.jc * hb * __fdividef(rb, b + k.tstar);
#pragma unroll
        for (int i = 0; i < 4; i++) J[i] = (t[i] + d[i]) * jf;
      }
      if (!pa) {  // elastic -> plastic
#pragma unroll
        for (int i = 0; i < 4; i++) {
          e[i] = d[i] * k.ce + J[i];
          s[i] = d[i] * k.ge - k.two_mu0 * J[i];
        }
      } else {  // plastic -> plastic or plastic -> elastic
        const float a2 = h + k.tstar2;
        const float ra = rsqrtf(a2);
        const float a = a2 * ra;
        const float q = __fdividef(w * ra * rb, a + b);
        float dn[4];
#pragma unroll
        for (int i = 0; i < 4; i++) dn[i] = d[i] * rb - t[i] * q;
#pragma unroll
        for (int i = 0; i < 4; i++) {
          e[i] = d[i] * k.cp - k.ry * dn[i] - J[i];
          s[i] = k.ylim * dn[i] + k.two_mu0 * J[i];
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 3; i++) {
    de[i] = e[i] + em;
    ds[i] = s[i] + sm;
  }
  de[3] = e[3];
  ds[3] = s[3];
  return pb;
}

__device__ __forceinline__ void ld4(const float* p, float v[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = a.z;
  v[3] = a.w;
}
__device__ __forceinline__ void st4(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// The row pass of the defect form.  Tiles, transforms and pixel mapping of
// the FP32 row pass of tiling V (RowIO<float, L, V>); grid (L / RR, solves).
// ITER: the iteration above in FP32 on the differences; INIT: the warm start
// in FP64 (flags of the accepted state, eps_ref = accepted + (E_k - E_{k-1}),
// sigma_ref = sigma(eps_ref), differences zero), after which the solve waits
// for a refresh (PH_REF); FINAL: flags of the accepted state, which becomes
// the reference (the fields of the solve are read from eps_ref, sigma_ref).
// Every index is in range for that grid (RowIO::where; pixels x < L^2).
// Loop control of a defect batch (the last CTA of the launch): as
// batch_arrive, and the condition of the loop body's refresh node, set when
// some solve waits for its refresh (PH_REF).
__device__ __forceinline__ void batch_arrive_dc(Solve* solves, int nb, BatchCtl* bc, cudaGraphConditionalHandle cond,
                                                int use_cond, cudaGraphConditionalHandle rcond, int use_rcond) {
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
    const bool go = active > 0 && bc->body_iters < bc->max_body_iters;
    if (active > 0 && bc->body_iters >= bc->max_body_iters) bc->timed_out = 1;
    if (use_cond) cudaGraphSetConditional(cond, go ? 1u : 0u);
    if (use_rcond) {
      cudaGraphSetConditional(rcond, waiting > 0 ? 1u : 0u);
      bc->refresh_runs += waiting > 0;
    }
    bc->arrive = 0;
    __threadfence();
  }
}

// Resident CTAs per SM asked of the compiler: at L = 512 four CTAs of 256
// threads in tiling 0, two in tiling 1 (64 and 128 registers, no spills),
// one elsewhere (the 1024- and 2048-point rows spill at 64).
template <int L, int V>
constexpr int dc_minb() { return L == 512 ? (V == 0 ? 4 : 2) : 1; }

template <int L, int V>
__global__ void __launch_bounds__(Cfg<float, L, V>::NT_ROW, dc_minb<L, V>())
row_pass_dc(Solve* __restrict__ solves, int nb, BatchCtl* bc, const C2<float>* __restrict__ tw,
            cudaGraphConditionalHandle cond, int use_cond, cudaGraphConditionalHandle rcond, int use_rcond) {
  using C = Cfg<float, L, V>;
  constexpr int RR = C::RR, NT = C::NT_ROW;
  constexpr int P = L >= NT ? L / NT : 1;
  using IO = RowIO<float, L, V>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C2<float>* sp = reinterpret_cast<C2<float>*>(smraw);
  __shared__ bool s_last;
  if (!ECHK(gridDim.x - 1, L / RR, 70) || !ECHK(blockDim.x - 1, NT, 70)) return;
  Solve& S = solves[blockIdx.y];
  const volatile Solve& Sv = S;
  const int phase = Sv.phase;
  const int cur = Sv.cur;
  const int inc = Sv.inc;
  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  auto xmap = [&](int j) { return L >= 32 ? wid * (32 * P) + j * 32 + lane : tid; };
  if (phase == PH_INIT || phase == PH_ITER || phase == PH_FINAL) {
    const int r0 = blockIdx.x * RR;
    const size_t LL = (size_t)L * L;
    double* __restrict__ eref = reinterpret_cast<double*>(S.eref);
    double* __restrict__ sref = reinterpret_cast<double*>(S.sref);
    const float* __restrict__ de_in = reinterpret_cast<const float*>(S.deps[cur]);
    float* __restrict__ de_out = reinterpret_cast<float*>(S.deps[1 - cur]);
    const float* __restrict__ ds_in = reinterpret_cast<const float*>(S.dsig[cur]);
    float* __restrict__ ds_out = reinterpret_cast<float*>(S.dsig[1 - cur]);
    const uint8_t* __restrict__ mask = S.mask;
    const C2<float>* stw = sp + C::ROW_DATA;
    if (phase == PH_ITER) IO::load_tables(sp, tw);
    float acc[N_ACC];
#pragma unroll
    for (int i = 0; i < N_ACC; i++) acc[i] = 0.0f;

    if (phase == PH_FINAL || phase == PH_INIT) {
      // FP64: the accepted state eps_ref + d_eps^n
      const Mat<double> m = make_mat<double>(S);
      double dE[4] = {0.0, 0.0, 0.0, 0.0};
      uint8_t* fl = nullptr;
      if (phase == PH_FINAL) {
        fl = S.flags ? S.flags + (size_t)(S.n_inc - 1) * LL : nullptr;
      } else {
        const double* E = S.path + 4 * (ECHK(inc, S.n_inc, 71) ? inc : 0);
        for (int c = 0; c < 4; c++) dE[c] = E[c] - Sv.Eprev[c];
        fl = (S.flags && inc > 0) ? S.flags + (size_t)(inc - 1) * LL : nullptr;
      }
      for (int r = 0; r < RR; r++)
        for (int j = 0; j < P; j++) {
          const int x1 = xmap(j);
          if (x1 >= L) continue;
          const size_t x = (size_t)(r0 + r) * L + x1;
          if (!ECHK(x, LL, 72)) continue;
          const bool v = mask[x] != 0;
          double e[4], s[4];
          float d[4];
          Vec4<double>::load(eref + 4 * x, e);
          ld4(de_in + 4 * x, d);
#pragma unroll
          for (int c = 0; c < 4; c++) e[c] += (double)d[c];
          if (fl) fl[x] = is_plastic(e, v, m);
          const float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
          if (phase == PH_FINAL) {
            // the final state becomes the reference (its fields are read
            // there), with its stress from the law in FP64
            sigma(e, v, m, s);
            Vec4<double>::store(eref + 4 * x, e);
            Vec4<double>::store(sref + 4 * x, s);
          } else {
#pragma unroll
            for (int c = 0; c < 4; c++) e[c] += dE[c];
            const bool pl = sigma(e, v, m, s);
            Vec4<double>::store(eref + 4 * x, e);
            Vec4<double>::store(sref + 4 * x, s);
            // the buffers the iterations read after this pass
            st4(de_out + 4 * x, z);
            st4(ds_out + 4 * x, z);
            // plastic pixels of iterate 0 (its mean strain comes from the
            // refresh, in FP64)
            acc[A_NPL] += pl ? 1.0f : 0.0f;
          }
        }
    } else {  // PH_ITER
      const DcConst k = dc_consts(S);
      const float* __restrict__ b0 = reinterpret_cast<const float*>(S.base[0]);
      const float* __restrict__ b1 = reinterpret_cast<const float*>(S.base[1]);
      const float* __restrict__ b2 = reinterpret_cast<const float*>(S.base[2]);
      C2<float>* spec = reinterpret_cast<C2<float>*>(S.spec);
      IO::load_async(sp, spec, r0);
      // the rows' differences, the halo row and their reference data are
      // asked of the L2 while the spectrum is transformed
      if constexpr (L >= 64) {
        if (wid == 0) {
          const int xh = (r0 + L - 1) & (L - 1);
          constexpr unsigned RB = (unsigned)(L * 16), PB = RB < 16384u ? RB : 16384u;
          constexpr int NPR = (int)(RB / PB);
          for (int i = lane; i < (RR + 1) * NPR; i += 32) {
            const int kr = i / NPR, row = kr < RR ? r0 + kr : xh;
            prefetch_l2(reinterpret_cast<const char*>(ds_in + (size_t)4 * row * L) + (size_t)(i % NPR) * PB, PB);
          }
          for (int i = lane; i < 2 * RR * NPR; i += 32) {
            const int kr = (i / NPR) % RR;
            const float* bb = i < RR * NPR ? b0 : b1;
            prefetch_l2(reinterpret_cast<const char*>(bb + (size_t)4 * (r0 + kr) * L) + (size_t)(i % NPR) * PB, PB);
          }
          // div sigma_ref of the rows: RR L float2, contiguous
          constexpr unsigned QB = (unsigned)(RR * L * 8), QP = QB < 16384u ? QB : 16384u;
          for (int i = lane; i < (int)(QB / QP); i += 32)
            prefetch_l2(reinterpret_cast<const char*>(b2 + (size_t)2 * r0 * L) + (size_t)i * QP, QP);
          if (lane == 31) prefetch_l2(mask + (size_t)r0 * L, (unsigned)(RR * L));
        }
      }
      float prev12[P], prev22[P];
      auto load_halo = [&]() {
        const int xh = (r0 + L - 1) & (L - 1);
#pragma unroll
        for (int j = 0; j < P; j++) {
          const int x1 = xmap(j);
          prev12[j] = prev22[j] = 0.0f;
          if (x1 >= L) continue;
          const size_t x = (size_t)xh * L + x1;
          if (!ECHK(x, LL, 73)) continue;
          float s[4];
          ld4(ds_in + 4 * x, s);
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
      // one pixel: sj = d_sig^n, (l11, l12) = d_sig^n at x - e^1
      auto update = [&](int r, int j, int x1, bool v, const float (&sj)[4], float l11, float l12) {
        if (x1 >= L) return;
        const size_t x = (size_t)(r0 + r) * L + x1;
        float tb[4], ab[4];
        ld4(b0 + 4 * x, tb);
        ld4(b1 + 4 * x, ab);
        const float2 rb = reinterpret_cast<const float2*>(b2)[x];
        // Eq. 1 (backward differences): div sigma_ref + div d_sig^n
        const float d1 = rb.x + ((sj[0] - l11) + (sj[3] - prev12[j]));
        const float d2 = rb.y + ((sj[3] - l12) + (sj[1] - prev22[j]));
        prev12[j] = sj[3];
        prev22[j] = sj[1];
#pragma unroll
        for (int c = 0; c < 4; c++) acc[A_S11 + c] += sj[c];
        acc[A_DIV2] += d1 * d1 + d2 * d2;
        // e^{n+1} - eps_ref = a_ref + (the transformed difference)
        const float u[4] = {ab[0] + IO::px(sp, 0, r, x1), ab[1] + IO::px(sp, 1, r, x1), ab[2],
                            ab[3] + IO::px(sp, 2, r, x1)};
        const float lu = k.lam0 * (u[0] + u[1] + u[2]);
        const float dtau[4] = {sj[0] + (lu + k.two_mu0 * u[0]), sj[1] + (lu + k.two_mu0 * u[1]),
                               sj[2] + (lu + k.two_mu0 * u[2]), sj[3] + k.two_mu0 * u[3]};
        const float t[4] = {tb[0], tb[1], -(tb[0] + tb[1]), tb[2]};
        float de[4], ds[4];
        const bool pl = delta_step(t, tb[3], dtau, v, k, de, ds);
        st4(de_out + 4 * x, de);
        st4(ds_out + 4 * x, ds);
#pragma unroll
        for (int c = 0; c < 4; c++) acc[A_E11 + c] += de[c];
        acc[A_NPL] += pl ? 1.0f : 0.0f;
        // eps^{n+1} - e^{n+1}
        const float q0 = de[0] - u[0], q1 = de[1] - u[1], q2 = de[2] - u[2], q3 = de[3] - u[3];
        acc[A_COMP] += q0 * q0 + q1 * q1 + q2 * q2 + 2.0f * q3 * q3;
        // p^{n+1} - p_ref = d_sig - C0:d_eps (in-plane)
        const float le = k.lam0 * (de[0] + de[1] + de[2]);
        IO::px(sp, 0, r, x1) = ds[0] - (le + k.two_mu0 * de[0]);
        IO::px(sp, 1, r, x1) = ds[1] - (le + k.two_mu0 * de[1]);
        IO::px(sp, 2, r, x1) = ds[3] - k.two_mu0 * de[3];
      };
      auto load_px = [&](int r, int j, float (&sg)[4], bool& v) {
        const int x1 = xmap(j);
        const size_t x = (size_t)(r0 + r) * L + x1;
        const bool act = x1 < L && ECHK(x, LL, 74);
        v = act ? mask[x] != 0 : true;
        if (act) ld4(ds_in + 4 * x, sg);
        else sg[0] = sg[1] = sg[2] = sg[3] = 0.0f;
      };
      // left neighbours as in row_pass: the previous lane by a shuffle, lane
      // 31 of the previous pixel group for lane 0, and at the start of a
      // run d_sig at x - e^1 (periodic) from memory
      constexpr int PC = P < 8 ? P : 8;
      auto row = [&](int r, int j0, float (&sg)[PC][4], bool (&vv)[PC], float& run11, float& run12) {
#pragma unroll
        for (int jj = 0; jj < PC; jj++) {
          const int j = j0 + jj;
          const int x1 = xmap(j);
          float l11, l12;
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
                if (ECHK(xl, LL, 75)) {
                  float sl[4];
                  ld4(ds_in + 4 * xl, sl);
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
      constexpr bool PRE = RR * P * 16 < 128;
      if constexpr (PRE) {
        static_assert(PC == P, "one chunk per row");
        float pen[RR][P][4];
        bool pvv[RR][P];
#pragma unroll
        for (int r = 0; r < RR; r++)
#pragma unroll
          for (int j = 0; j < P; j++) load_px(r, j, pen[r][j], pvv[r][j]);
#pragma unroll
        for (int r = 0; r < RR; r++) {
          float run11 = 0.0f, run12 = 0.0f;
          row(r, 0, pen[r], pvv[r], run11, run12);
        }
      } else {
        for (int r = 0; r < RR; r++) {
          float run11 = 0.0f, run12 = 0.0f;
#pragma unroll
          for (int j0 = 0; j0 < P; j0 += PC) {
            float en[PC][4];
            bool vv[PC];
#pragma unroll
            for (int jj = 0; jj < PC; jj++) load_px(r, j0 + jj, en[jj], vv[jj]);
            row(r, j0, en, vv, run11, run12);
          }
        }
      }
      __syncthreads();
      IO::template fft<false>(sp, stw);
      IO::r2c_twist(sp, IO::octant(stw));
      __syncthreads();
      IO::store(sp, spec, r0);
    }
    if (phase == PH_ITER || phase == PH_INIT) {
      if (ECHK(blockIdx.x, L / RR, 76)) block_reduce_acc<NT>(acc, S.partials + (size_t)blockIdx.x * PART_STRIDE);
    }
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
        if (phase == PH_ITER) {
          // sums of sigma^n and eps^{n+1}: the reference's and the differences'
          for (int c = 0; c < 4; c++) {
            tot[A_S11 + c] += S.ref_sum[c];
            tot[A_E11 + c] += S.ref_sum[4 + c];
          }
        }
        finalize_solve<L>(S, phase, tot);
        // after a warm start, and every ref_every iterations, the solve waits
        // for the refresh of its reference (the loop body's next node)
        if (phase == PH_INIT) S.phase = PH_REF;
        else if (phase == PH_ITER && S.phase == PH_ITER && ++S.since_ref >= S.ref_every) S.phase = PH_REF;
        S.arrive = 0;
      }
    }
  }
  if (tid == 0) batch_arrive_dc(solves, nb, bc, cond, use_cond, rcond, use_rcond);
}

// Refresh, forward half (FP64 tiling V; grid (L / RR, solves)), for the
// solves waiting in PH_REF: the latest iterate eps_ref + d_eps becomes the
// reference (after a warm start d_eps is zero) and the differences read
// next are cleared; sigma_ref = sigma(eps_ref) from the law; p_ref
// into the FP64 spectrum, the row transform, tau_ref's deviator and
// |tau_ref'|^2 - T*^2 into base[0], the CTA's sums of sigma_ref and eps_ref
// (refpart), the CTA's piece of the FP32 spectrum cleared.  shadow[i] takes
// the phase (PH_ITER for both), increment and buffer of solves[i] for the
// FP64 column pass.  Every index is in range for that grid.
template <int L, int V>
__global__ void __launch_bounds__(Cfg<double, L, V>::NT_ROW)
dc_ref_forward(Solve* __restrict__ solves, Solve* __restrict__ shadow, const C2<double>* __restrict__ tw) {
  using C = Cfg<double, L, V>;
  constexpr int RR = C::RR, NT = C::NT_ROW, P = L >= NT ? L / NT : 1;
  using IO = RowIO<double, L, V>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C2<double>* sp = reinterpret_cast<C2<double>*>(smraw);
  if (!ECHK(gridDim.x - 1, L / RR, 77) || !ECHK(blockDim.x - 1, NT, 77)) return;
  Solve& S = solves[blockIdx.y];
  const volatile Solve& Sv = S;
  const int phase = Sv.phase, cur = Sv.cur, inc = Sv.inc;
  const bool live = phase == PH_REF;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Solve& Z = shadow[blockIdx.y];
    Z.phase = live ? (int32_t)PH_ITER : (int32_t)PH_DONE;
    Z.inc = inc;
    Z.cur = cur;
  }
  if (!live) return;
  const int r0 = blockIdx.x * RR;
  const size_t LL = (size_t)L * L;
  double* __restrict__ eref = reinterpret_cast<double*>(S.eref);
  double* __restrict__ sref = reinterpret_cast<double*>(S.sref);
  float* __restrict__ de = reinterpret_cast<float*>(S.deps[cur]);
  float* __restrict__ ds = reinterpret_cast<float*>(S.dsig[cur]);
  float* __restrict__ b0 = reinterpret_cast<float*>(S.base[0]);
  const uint8_t* __restrict__ mask = S.mask;
  const Mat<double> m = make_mat<double>(S);
  const double tst2 = S.mcd[MC_TSTAR2];
  const C2<double>* stw = IO::load_tables(sp, tw);
  double acc[N_ACC];
#pragma unroll
  for (int i = 0; i < N_ACC; i++) acc[i] = 0.0;
  for (int r = 0; r < RR; r++)
    for (int j = 0; j < P; j++) {
      const int x1 = (int)threadIdx.x + j * NT;
      if (x1 >= L) continue;
      const size_t x = (size_t)(r0 + r) * L + x1;
      double e[4], s[4], c0[4];
      Vec4<double>::load(eref + 4 * x, e);
      {
        // the new reference: eps_ref + d_eps, and sigma of it from the law in
        // FP64 (not sigma_ref + d_sig: the FP32 rounding of the differences
        // would otherwise accumulate over the refreshes into a multiplier
        // that is no longer sigma(eps))
        float q[4];
        ld4(de + 4 * x, q);
#pragma unroll
        for (int c = 0; c < 4; c++) e[c] += (double)q[c];
        sigma(e, mask[x] != 0, m, s);
        Vec4<double>::store(eref + 4 * x, e);
        Vec4<double>::store(sref + 4 * x, s);
        const float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        st4(de + 4 * x, z);
        st4(ds + 4 * x, z);
      }
      c0_apply(e, m, c0);
      IO::px(sp, 0, r, x1) = s[0] - c0[0];
      IO::px(sp, 1, r, x1) = s[1] - c0[1];
      IO::px(sp, 2, r, x1) = s[3] - c0[3];
      // tau_ref = sigma_ref + C0:eps_ref, its deviator and distance to the
      // plastic threshold
      const double t0 = s[0] + c0[0], t1 = s[1] + c0[1], t2 = s[2] + c0[2], t3 = s[3] + c0[3];
      const double tm = (t0 + t1 + t2) * (1.0 / 3.0);
      const double u0 = t0 - tm, u1 = t1 - tm, u2 = t2 - tm;
      const double h = (u0 * u0 + u1 * u1 + u2 * u2 + 2.0 * t3 * t3) - tst2;
      const float tb[4] = {(float)u0, (float)u1, (float)t3, (float)h};
      st4(b0 + 4 * x, tb);
#pragma unroll
      for (int c = 0; c < 4; c++) {
        acc[A_S11 + c] += s[c];
        acc[A_E11 + c] += e[c];
      }
    }
  {
    constexpr size_t PIECE = (size_t)12 * L * RR / 16;  // float4 of the FP32 spectrum per CTA
    static_assert((12 * L * RR) % 16 == 0, "16-byte pieces");
    float4* f = reinterpret_cast<float4*>(S.spec) + (size_t)blockIdx.x * PIECE;
    for (size_t i = threadIdx.x; i < PIECE; i += NT) f[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
  block_reduce_acc<NT>(acc, S.refpart + (size_t)blockIdx.x * PART_STRIDE);
  cp_async_wait_all();
  __syncthreads();
  IO::template fft<false>(sp, stw);
  IO::r2c_twist(sp, IO::octant(stw));
  __syncthreads();
  IO::store(sp, reinterpret_cast<C2<double>*>(S.spec64), r0);
}

// Refresh, inverse half: g_ref = Gamma(p_ref) from the FP64 spectrum the
// column pass left, a_ref = E + g_ref - eps_ref into base[1] (e33 = E33),
// div sigma_ref (backward differences of Eq. 1) into base[2].  Grid and
// checks as dc_ref_forward.
template <int L, int V>
__global__ void __launch_bounds__(Cfg<double, L, V>::NT_ROW)
dc_ref_inverse(Solve* __restrict__ solves, const C2<double>* __restrict__ tw) {
  using C = Cfg<double, L, V>;
  constexpr int RR = C::RR, NT = C::NT_ROW, P = L >= NT ? L / NT : 1;
  using IO = RowIO<double, L, V>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C2<double>* sp = reinterpret_cast<C2<double>*>(smraw);
  if (!ECHK(gridDim.x - 1, L / RR, 78) || !ECHK(blockDim.x - 1, NT, 78)) return;
  Solve& S = solves[blockIdx.y];
  const volatile Solve& Sv = S;
  const int phase = Sv.phase, inc = Sv.inc;
  if (phase != PH_REF) return;
  const int r0 = blockIdx.x * RR;
  const size_t LL = (size_t)L * L;
  const double* __restrict__ eref = reinterpret_cast<const double*>(S.eref);
  const double* __restrict__ sref = reinterpret_cast<const double*>(S.sref);
  float* __restrict__ b1 = reinterpret_cast<float*>(S.base[1]);
  float2* __restrict__ b2 = reinterpret_cast<float2*>(S.base[2]);
  const double* E = S.path + 4 * (ECHK(inc, S.n_inc, 79) ? inc : 0);
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
      const int x2 = r0 + r;
      const size_t x = (size_t)x2 * L + x1;
      const size_t xl = (size_t)x2 * L + ((x1 + L - 1) & (L - 1));
      const size_t xu = (size_t)((x2 + L - 1) & (L - 1)) * L + x1;
      double e[4], s[4], sl[4], su[4];
      Vec4<double>::load(eref + 4 * x, e);
      const float a[4] = {(float)((E[0] + IO::px(sp, 0, r, x1)) - e[0]), (float)((E[1] + IO::px(sp, 1, r, x1)) - e[1]),
                          (float)(E[2] - e[2]), (float)((E[3] + IO::px(sp, 2, r, x1)) - e[3])};
      st4(b1 + 4 * x, a);
      Vec4<double>::load(sref + 4 * x, s);
      Vec4<double>::load(sref + 4 * xl, sl);
      Vec4<double>::load(sref + 4 * xu, su);
      const double d1 = (s[0] - sl[0]) + (s[3] - su[3]);
      const double d2 = (s[3] - sl[3]) + (s[1] - su[1]);
      b2[x] = make_float2((float)d1, (float)d2);
    }
}

// Refresh, last step (one CTA of NT threads per solve): the sums of
// sigma_ref and eps_ref over the CTA records of dc_ref_forward, in a fixed
// order; the solve takes the mean strain of its latest iterate (the new
// reference) from them and continues its iterations.
template <int L, int V, int NT>
__global__ void __launch_bounds__(NT) dc_ref_sums(Solve* __restrict__ solves) {
  constexpr int NREC = L / Cfg<double, L, V>::RR;
  Solve& S = solves[blockIdx.x];
  const volatile Solve& Sv = S;
  const int phase = Sv.phase;
  if (phase != PH_REF) return;
  __shared__ double tot[N_ACC];
  sum_partials<NT, NREC>(S.refpart, tot);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < 4; c++) {
      S.ref_sum[c] = tot[A_S11 + c];
      S.ref_sum[4 + c] = tot[A_E11 + c];
    }
    constexpr double inv = 1.0 / ((double)L * (double)L);
    for (int c = 0; c < 4; c++) S.epsm_next[c] = tot[A_E11 + c] * inv;
    S.since_ref = 0;
    S.phase = PH_ITER;
  }
}

}  // namespace epfft
