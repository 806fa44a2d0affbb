// Common device types for the epfft CUDA path (sm_103a).
//
// Conventions shared by every kernel of the library:
//   * lattice L x L (L a power of two), pixel x = (x1, x2), linear index
//     x2 * L + x1 (x1 fastest);
//   * strain / stress per pixel: 4 reals (11, 22, 33, 12);
//   * forward DFT kernel exp(-i q.x), q_j = 2 pi m_j / L, which makes the
//     forward difference of Eq. 1 the multiplication by i k_j of Eq. 2.
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace epfft {

template <typename T>
struct C2 {
  T re, im;
};

template <typename T>
__device__ __forceinline__ C2<T> mk(T a, T b) {
  C2<T> r;
  r.re = a;
  r.im = b;
  return r;
}
template <typename T>
__device__ __forceinline__ C2<T> operator+(C2<T> a, C2<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename T>
__device__ __forceinline__ C2<T> operator-(C2<T> a, C2<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename T>
__device__ __forceinline__ C2<T> operator*(C2<T> a, C2<T> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
__device__ __forceinline__ C2<T> operator*(T s, C2<T> a) { return mk(s * a.re, s * a.im); }
template <typename T>
__device__ __forceinline__ C2<T> conj(C2<T> a) { return mk(a.re, -a.im); }
// multiply by -i (forward) or +i (inverse)
template <typename T, bool INV>
__device__ __forceinline__ C2<T> mul_mi(C2<T> a) {
  return INV ? mk(-a.im, a.re) : mk(a.im, -a.re);
}
template <typename T>
__device__ __forceinline__ C2<T> mul_i(C2<T> a) { return mk(-a.im, a.re); }
template <typename T>
__device__ __forceinline__ T norm2(C2<T> a) { return a.re * a.re + a.im * a.im; }

// Green operators of Sec. 2 (values of the ABI's EPFFT_GREEN_*).
enum GreenMode : int32_t {
  GM_EQ3 = 0,  // discrete operator of Eq. 3
  GM_CG1 = 1,  // continuum operator: Eq. 3 with k_j = q_j
  GM_DG1 = 2,  // symmetrized operator G^(1)
  GM_DISP = 3, // not a Green operator: the displacement of Sec. 2 from the
               // strain spectrum (epfft_displacement only; no solve takes it)
};

// Solve phases of the per-solve state machine driven on the device.
enum Phase : int32_t {
  PH_INIT = 0,   // warm start of increment `inc` from the accepted state
  PH_ITER = 1,   // augmented-Lagrangian iterations of increment `inc`
  PH_FINAL = 2,  // write the plastic flags of the last accepted state
  PH_DONE = 3,
  PH_REF = 4,    // defect form: waits for the refresh of its reference (the
                 // passes skip it; the refresh sets PH_ITER)
};

// Per-increment result, written by the device (layout of epfft_record).
struct Record {
  double sig_mean[4];
  double eps_mean[4];
  double eta1, eta2, eta3;
  int32_t iterations, n_plastic, n_clusters, status;
};

// Accumulators of the row pass (per CTA), FP64, in this order.
enum Acc : int {
  A_S11 = 0, A_S22, A_S33, A_S12,  // sum sigma(eps^n)
  A_E11, A_E22, A_E33, A_E12,      // sum of eps of the iterate the pass produces
  A_DIV2,                          // sum |div sigma(eps^n)|^2
  A_COMP,                          // sum (eps^{n+1} - e^{n+1}):(same)
  A_NPL,                           // its plastic pixels (matrix)
  N_ACC
};
constexpr int PART_STRIDE = 12;  // doubles per CTA partial record

// Derived material constants of a solve, formed once on the host in FP64
// (and rounded once to FP32 for the FP32 kernels), so that no kernel thread
// divides or takes square roots to build them.
enum MatConst : int {
  MC_K = 0,       // matrix bulk modulus lambda + 2 mu / 3
  MC_TWO_MU,      // 2 mu
  MC_LAM0,        // lambda0
  MC_TWO_MU0,     // 2 mu0
  MC_YLIM,        // sqrt(2/3) Y
  MC_YLIM2,       // 2/3 Y^2
  MC_INV_3KK0,    // 1 / (3 (K + K0))
  MC_INV_3K0,     // 1 / (3 K0)
  MC_INV_2MUMU0,  // 1 / (2 (mu + mu0))
  MC_INV_2MU0,    // 1 / (2 mu0)
  MC_TRIAL2,      // (mu / (mu + mu0))^2
  MC_MU0,         // mu0
  MC_P_MAT,       // 3 (K - K0): mean part of the polarization of a matrix pixel
  MC_P_VOID,      // -3 K0: the same for a void pixel
  MC_GSC_EL,      // mu / (mu + mu0): 2 mu times the elastic deviator scale of the local step
  MC_3K,          // 3 K
  MC_TSTAR,       // sqrt(2/3) Y (mu + mu0) / mu: |tau'| where the local step turns plastic
  MC_TSTAR2,      // its square
  MC_RY,          // sqrt(2/3) Y / (2 mu0)
  MC_JC,          // mu / ((mu + mu0) 2 mu0)
  N_MC
};

// Device-resident state of one solve of a batch.
struct Solve {
  // material: matrix lambda, mu, Y; reference medium lambda0, mu0
  double lam, mu, Y, lam0, mu0;
  double mcd[N_MC];  // derived constants (MatConst), FP64
  float mcf[N_MC];   // the same rounded to FP32
  double tol_eq, tol_macro;
  int32_t max_iter, n_inc;
  int32_t green;           // Green operator (GreenMode)
  int32_t eq_fixed_point;  // 1: the equilibrium test is eta3, else eta1
  const double* path;  // n_inc * 4 prescribed mean strains (11,22,33,12)
  Record* rec;         // n_inc records
  uint8_t* flags;      // n_inc * L * L plastic flags (may be null)
  const uint8_t* mask; // L * L, 1 = void
  void* eps[2];        // ping-pong local strain, L*L*4 reals
  void* sig[2];        // sigma of the same iterates (the multiplier), L*L*4 reals
  void* spec;          // 3 * L * L/2 complex, tiled column layout
  double* partials;    // n_row_ctas * PART_STRIDE
  // defect-correction form (dcpass.cuh): the FP64 reference state eps_ref,
  // sigma_ref (4 reals per pixel; eps[0] = eps[1] = eref, sig[0] = sig[1] =
  // sref, so that the fields of the final state are read from there), the
  // FP32 differences of the iterates from it (ping-pong, 4 floats per
  // pixel), the FP32 per-pixel data of the reference (base[0]: float4
  // deviator of tau_ref (11, 22, 12) and |tau_ref'|^2 - T*^2; base[1]:
  // float4 e_ref - eps_ref; base[2]: float2 div sigma_ref), the FP64
  // spectrum of the reference transform, per-CTA partial sums of a refresh
  // and the sums of sigma_ref and eps_ref; null / zero otherwise
  void* eref;
  void* sref;
  void* deps[2];
  void* dsig[2];
  void* base[3];
  void* spec64;
  double* refpart;
  double ref_sum[8];
  int32_t zero_mean;   // 1: the column pass puts 0 at q = 0 (not the mean strain)
  int32_t ref_every;   // defect form: iterations between refreshes of the reference
  // mutable state
  int32_t phase, inc, iter, cur;
  int32_t status;
  uint32_t arrive;
  int32_t since_ref;    // defect form: iterations since the last refresh
  int32_t pad1;
  double Eprev[4];
  double sig_prev[4];
  double comp_cur;      // mean fixed-point residual of iterate n (eta3^2 EE)
  double epsm_next[4];  // <eps> of the iterate the last pass produced
  double npl_next;      // its plastic pixels
  int64_t total_iters;  // pixel-iteration accounting: passes that did work
};

// Batch-level control shared by all solves of one launch.
struct BatchCtl {
  uint32_t arrive;          // row-pass CTAs finished in the current step
  int32_t active;           // solves not yet DONE after the last row pass
  int64_t body_iters;       // loop steps executed
  int64_t max_body_iters;   // bound on loop steps (a solve needs at most
                            // n_inc * (max_iter + 2) + 1)
  int32_t timed_out;        // the bound stopped the loop with work left
  int32_t waiting;          // defect form: solves waiting for a refresh (PH_REF)
  int64_t refresh_runs;     // defect form: executions of the loop body's refresh node
  int32_t dc;               // 1: a defect batch (a mixed graph's refresh node covers it)
  int32_t pad;
};

// First failed self-check (builds define EPFFT_CHECKS):
// the access is skipped and its code, index and bound are recorded.
struct CheckRec {
  int32_t code, where;
  int64_t index, bound;
};

}  // namespace epfft

#ifdef EPFFT_CHECKS
static __device__ epfft::CheckRec g_check;
__device__ __forceinline__ bool epfft_chk(bool ok, int code, long long index, long long bound) {
  if (!ok && atomicCAS(&g_check.code, 0, code) == 0) {
    g_check.where = (int32_t)(blockIdx.x * 1024 + threadIdx.x);
    g_check.index = index;
    g_check.bound = bound;
  }
  return ok;
}
#define ECHK(idx, bound, code) epfft_chk((long long)(idx) >= 0 && (long long)(idx) < (long long)(bound), (code), (long long)(idx), (long long)(bound))
#else
#define ECHK(idx, bound, code) true
#endif
