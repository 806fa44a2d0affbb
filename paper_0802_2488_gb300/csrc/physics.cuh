// Pixelwise constitutive law, local step of the augmented Lagrangian and the
// per-frequency discrete Green operator (Willot & Pellegrini, Sec. 2, Eqs. 2-3).
#pragma once
#include "common.cuh"

namespace epfft {

// Material constants of one solve in the working precision, with the
// derived quantities the hot loop needs.
template <typename T>
struct Mat {
  T K, two_mu;      // matrix bulk modulus lambda + 2 mu / 3, 2 mu
  T lam0, two_mu0;  // reference medium C0
  T ylim, ylim2;    // sqrt(2/3) Y and its square (Mises cap on 2 mu |dev eps|)
  T inv_3KK0;       // 1 / (3 (K + K0))
  T inv_3K0;        // 1 / (3 K0)
  T inv_2mumu0;     // 1 / (2 (mu + mu0))
  T inv_2mu0;       // 1 / (2 mu0)
  T trial2;         // (mu / (mu + mu0))^2: |dev| of the elastic trial vs |tau'|
  T p_mat, p_void;  // 3 (K - K0), -3 K0
  T gsc_el;         // mu / (mu + mu0)
  T k3;             // 3 K
};

template <typename T>
__device__ __forceinline__ const T* mat_consts(const Solve& S);
template <>
__device__ __forceinline__ const float* mat_consts<float>(const Solve& S) { return S.mcf; }
template <>
__device__ __forceinline__ const double* mat_consts<double>(const Solve& S) { return S.mcd; }

// Loads the solve's derived constants (formed on the host).
template <typename T>
__device__ __forceinline__ Mat<T> make_mat(const Solve& S) {
  const T* c = mat_consts<T>(S);
  Mat<T> m;
  m.K = c[MC_K];
  m.two_mu = c[MC_TWO_MU];
  m.lam0 = c[MC_LAM0];
  m.two_mu0 = c[MC_TWO_MU0];
  m.ylim = c[MC_YLIM];
  m.ylim2 = c[MC_YLIM2];
  m.inv_3KK0 = c[MC_INV_3KK0];
  m.inv_3K0 = c[MC_INV_3K0];
  m.inv_2mumu0 = c[MC_INV_2MUMU0];
  m.inv_2mu0 = c[MC_INV_2MU0];
  m.trial2 = c[MC_TRIAL2];
  m.p_mat = c[MC_P_MAT];
  m.p_void = c[MC_P_VOID];
  m.gsc_el = c[MC_GSC_EL];
  m.k3 = c[MC_3K];
  return m;
}

// 1/sqrt(x) for x > 0 in normal FP32 range.  FP32: the hardware estimate.
// FP64: the FP32 estimate refined by two Newton-Raphson steps
// y <- y (3/2 - x y^2 / 2), each of which squares the relative error
// (2e-7 -> 1e-13 -> below FP64 rounding), so that the kernel uses FP64 FMAs
// only.
template <typename T>
__device__ __forceinline__ T rsq(T x);
template <>
__device__ __forceinline__ float rsq<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsq<double>(double x) {
  double y = (double)rsqrtf((float)x);
  const double h = 0.5 * x;
  y = y * fma(-h * y, y, 1.5);
  y = y * fma(-h * y, y, 1.5);
  return y;
}

// 1/x for x > 0 in normal FP32 range.  FP32: the fast reciprocal (within
// 2 ulp; the one use, the determinant of the 2x2 acoustic tensor, is at
// least mu0 (lambda0 + 2 mu0) |k|^4 > 0).  FP64: the FP32 reciprocal
// refined by two Newton-Raphson steps r <- r + r (1 - x r).
template <typename T>
__device__ __forceinline__ T rcp(T x);
template <>
__device__ __forceinline__ float rcp<float>(float x) { return __fdividef(1.0f, x); }
template <>
__device__ __forceinline__ double rcp<double>(double x) {
  double r = (double)__frcp_rn((float)x);
  r = fma(r, fma(-x, r, 1.0), r);
  r = fma(r, fma(-x, r, 1.0), r);
  return r;
}

// sigma(eps): void -> 0; matrix -> K tr(eps) I + g dev(eps) with g = 2 mu on
// the elastic branch and g = sqrt(2/3) Y / |dev| once 2 mu |dev| exceeds
// sqrt(2/3) Y (Mises stress capped at Y, deformation theory).  The deviator
// is the 3D one (with eps33).  Returns true on the plastic branch.
template <typename T>
__device__ __forceinline__ bool sigma(const T e[4], bool is_void, const Mat<T>& m, T s[4]) {
  if (is_void) {
    s[0] = s[1] = s[2] = s[3] = T(0);
    return false;
  }
  const T tr = e[0] + e[1] + e[2];
  const T mth = tr * T(1.0 / 3.0);
  const T d0 = e[0] - mth, d1 = e[1] - mth, d2 = e[2] - mth, d3 = e[3];
  const T nd2 = d0 * d0 + d1 * d1 + d2 * d2 + T(2) * d3 * d3;
  const bool pl = m.two_mu * m.two_mu * nd2 > m.ylim2;
  const T g = pl ? m.ylim * rsq(nd2) : m.two_mu;
  const T p = m.K * tr;
  s[0] = p + g * d0;
  s[1] = p + g * d1;
  s[2] = p + g * d2;
  s[3] = g * d3;
  return pl;
}

// Plastic-branch test of sigma alone (for the per-increment plastic flags).
template <typename T>
__device__ __forceinline__ bool is_plastic(const T e[4], bool is_void, const Mat<T>& m) {
  if (is_void) return false;
  const T tr = e[0] + e[1] + e[2];
  const T mth = tr * T(1.0 / 3.0);
  const T d0 = e[0] - mth, d1 = e[1] - mth, d2 = e[2] - mth, d3 = e[3];
  const T nd2 = d0 * d0 + d1 * d1 + d2 * d2 + T(2) * d3 * d3;
  return m.two_mu * m.two_mu * nd2 > m.ylim2;
}

// C0:a, the isotropic reference stiffness (lambda0, mu0).
template <typename T>
__device__ __forceinline__ void c0_apply(const T a[4], const Mat<T>& m, T out[4]) {
  const T l = m.lam0 * (a[0] + a[1] + a[2]);
  out[0] = l + m.two_mu0 * a[0];
  out[1] = l + m.two_mu0 * a[1];
  out[2] = l + m.two_mu0 * a[2];
  out[3] = m.two_mu0 * a[3];
}

// Local step of the augmented Lagrangian: eps solving
//   sigma(eps) + C0:eps = tau,
// split into its mean part (3 (K + K0) eps_m = tau_m, voids 3 K0 eps_m = tau_m)
// and a deviator parallel to tau' = tau - tau_m I:
//   elastic  dev = tau' / (2 (mu + mu0)),
//   plastic  dev = tau' (1 - sqrt(2/3) Y / |tau'|) / (2 mu0),
//   void     dev = tau' / (2 mu0).
// The elastic branch holds while 2 mu |dev| <= sqrt(2/3) Y, i.e.
// (mu / (mu + mu0))^2 |tau'|^2 <= 2/3 Y^2.  Returns true on the plastic branch.
template <typename T>
__device__ __forceinline__ bool local_solve(const T t[4], bool is_void, const Mat<T>& m, T e[4]) {
  const T tm = (t[0] + t[1] + t[2]) * T(1.0 / 3.0);
  const T d0 = t[0] - tm, d1 = t[1] - tm, d2 = t[2] - tm, d3 = t[3];
  T em, sc;
  bool pl = false;
  if (is_void) {
    em = tm * m.inv_3K0;
    sc = m.inv_2mu0;
  } else {
    em = tm * m.inv_3KK0;
    const T nt2 = d0 * d0 + d1 * d1 + d2 * d2 + T(2) * d3 * d3;
    pl = m.trial2 * nt2 > m.ylim2;
    sc = pl ? (T(1) - m.ylim * rsq(nt2)) * m.inv_2mu0 : m.inv_2mumu0;
  }
  e[0] = d0 * sc + em;
  e[1] = d1 * sc + em;
  e[2] = d2 * sc + em;
  e[3] = d3 * sc;
  return pl;
}

// The local step (local_solve) together with the stress of its solution and
// the next polarization p = sigma(eps) - C0:eps, from the step's own
// quantities: with tau' the deviator of tau, eps = sc tau' + em I and
//   sigma(eps) = 3 K em I + gsc tau',   gsc = 2 mu sc (elastic),
//                                       sqrt(2/3) Y / |tau'| (plastic), 0 (void),
// so p = (3 K - 3 K0) em I + (gsc - 2 mu0 sc) tau' (K = 0 for a void).  This
// is sigma of the step's solution on the branch the step chose, without a
// second evaluation of the law (it is also the multiplier update of the
// augmented Lagrangian: lambda + C0:(e - eps) = tau - C0:eps).  Returns true
// on the plastic branch; s holds (11, 22, 33, 12), p the in-plane (11, 22, 12).
template <typename T>
__device__ __forceinline__ bool local_solve_p(const T t[4], bool is_void, const Mat<T>& m, T e[4], T s[4], T p[3]) {
  const T tm = (t[0] + t[1] + t[2]) * T(1.0 / 3.0);
  const T d0 = t[0] - tm, d1 = t[1] - tm, d2 = t[2] - tm, d3 = t[3];
  T em, sc, gsc, pa, sk;
  bool pl = false;
  if (is_void) {
    em = tm * m.inv_3K0;
    sc = m.inv_2mu0;
    gsc = T(0);
    pa = m.p_void;
    sk = T(0);
  } else {
    em = tm * m.inv_3KK0;
    const T nt2 = d0 * d0 + d1 * d1 + d2 * d2 + T(2) * d3 * d3;
    pl = m.trial2 * nt2 > m.ylim2;
    if (pl) {
      const T ri = m.ylim * rsq(nt2);  // sqrt(2/3) Y / |tau'|
      sc = (T(1) - ri) * m.inv_2mu0;
      gsc = ri;
    } else {
      sc = m.inv_2mumu0;
      gsc = m.gsc_el;
    }
    pa = m.p_mat;
    sk = m.k3;
  }
  e[0] = d0 * sc + em;
  e[1] = d1 * sc + em;
  e[2] = d2 * sc + em;
  e[3] = d3 * sc;
  const T sm = sk * em;
  s[0] = gsc * d0 + sm;
  s[1] = gsc * d1 + sm;
  s[2] = gsc * d2 + sm;
  s[3] = gsc * d3;
  const T pb = gsc - m.two_mu0 * sc;
  const T pm = pa * em;
  p[0] = pb * d0 + pm;
  p[1] = pb * d1 + pm;
  p[2] = pb * d3;
  return pl;
}

// Discrete Green operator of Eq. 3 applied at one frequency q != 0 to the
// polarization spectrum (p11, p22, p12), in place, times `scale`.
// With the acoustic tensor N_ab = k*_c C0_acdb k_d (Hermitian 2x2),
// w_a = k*_b p_ab and v = N^{-1} w, Eq. 3 contracts to
//   e_ab = -(k_a v_b + k_b v_a) / 2.
// For the isotropic C0, N11 = (lam0+mu0)|k1|^2 + mu0|k|^2,
// N22 = (lam0+mu0)|k2|^2 + mu0|k|^2, N12 = lam0 k1* k2 + mu0 k1 k2*, and
// det N = mu0 (lam0 + 2 mu0) |k|^4 + 4 lam0 mu0 (Im k1* k2)^2 (a sum of
// non-negative terms, evaluated without cancellation).
template <typename T>
__device__ __forceinline__ void green_apply(C2<T> k1, C2<T> k2, T lam0, T mu0, T scale,
                                            C2<T>& p11, C2<T>& p22, C2<T>& p12) {
  const T a1 = norm2(k1), a2 = norm2(k2), K2 = a1 + a2;
  const T lm = lam0 + mu0;
  const T N11 = lm * a1 + mu0 * K2, N22 = lm * a2 + mu0 * K2;
  const C2<T> c = conj(k1) * k2;
  const C2<T> N12 = mk(lm * c.re, (lam0 - mu0) * c.im);
  const T det = mu0 * (lam0 + T(2) * mu0) * K2 * K2 + T(4) * lam0 * mu0 * c.im * c.im;
  const T idet = scale * rcp(det);
  const C2<T> w1 = conj(k1) * p11 + conj(k2) * p12;
  const C2<T> w2 = conj(k1) * p12 + conj(k2) * p22;
  const C2<T> v1 = idet * (N22 * w1 - N12 * w2);
  const C2<T> v2 = idet * (N11 * w2 - conj(N12) * w1);
  p11 = T(-1) * (k1 * v1);
  p22 = T(-1) * (k2 * v2);
  p12 = T(-0.5) * (k1 * v2 + k2 * v1);
}

// Displacement of Sec. 2 at frequency (m1, m2) != 0 from the strain
// spectrum (e11, e22, e12) in (p11, p22, p12): with k^2 = k1^2 + k2^2,
//   u1 = -(i / k^2) { k1 [e11 - e22] + 2 k2 e12 },
//   u2 =  (i / k^2) { k2 [e11 - e22] - 2 k1 e12 },
// returned in (p11, p22) times `scale`, p12 = 0.  Where k^2 vanishes
// (m = (L/4, 3L/4) and (3L/4, L/4) when 4 divides L) the same relation
// e_ab = (i/2)(k_a u_b + k_b u_a) is solved with |k|^2 instead:
// w_b = k*_a e_ab, s = -i (k*.w) / |k|^2, u_b = (-2 i w_b - k_b s) / |k|^2.
template <typename T>
__device__ __forceinline__ void disp_apply(C2<T> k1, C2<T> k2, int L, int m1, int m2, T scale, C2<T>& p11,
                                           C2<T>& p22, C2<T>& p12) {
  const bool zk = (L % 4 == 0) && ((m1 == L / 4 && m2 == 3 * L / 4) || (m1 == 3 * L / 4 && m2 == L / 4));
  C2<T> u1, u2;
  if (!zk) {
    const C2<T> kk = k1 * k1 + k2 * k2;
    const T r = scale * rcp(norm2(kk));  // scale / |k^2|^2
    const C2<T> d = p11 - p22;
    const C2<T> n1 = k1 * d + T(2) * (k2 * p12), n2 = k2 * d - T(2) * (k1 * p12);
    // -i n1 / kk = -i n1 conj(kk) / |kk|^2, i n2 / kk likewise
    const C2<T> a1 = n1 * conj(kk), a2 = n2 * conj(kk);
    u1 = mk(r * a1.im, -r * a1.re);
    u2 = mk(-r * a2.im, r * a2.re);
  } else {
    const T nk = norm2(k1) + norm2(k2), ri = rcp(nk);
    const C2<T> w1 = conj(k1) * p11 + conj(k2) * p12, w2 = conj(k1) * p12 + conj(k2) * p22;
    const C2<T> kw = conj(k1) * w1 + conj(k2) * w2;
    const C2<T> sd = mk(ri * kw.im, -ri * kw.re);  // -i (k*.w) / |k|^2
    const C2<T> t1 = k1 * sd, t2 = k2 * sd;
    // (-2 i w_b - k_b s) / |k|^2, times scale
    const T sc = scale * ri;
    u1 = mk(sc * (T(2) * w1.im - t1.re), sc * (T(-2) * w1.re - t1.im));
    u2 = mk(sc * (T(2) * w2.im - t2.re), sc * (T(-2) * w2.re - t2.im));
  }
  p11 = u1;
  p22 = u2;
  p12 = mk(T(0), T(0));
}

// The Green operator `mode` of Sec. 2 at frequency (m1, m2) applied to
// (p11, p22, p12) in place, times `scale`.  ktab: k(m) of Eq. 2; qtab: the
// continuum momenta (q~(m), 0) (tables.cuh).
//   GM_EQ3: Eq. 3.
//   GM_CG1: Eq. 3 with k_j = q~_j, averaged over q~_j = +-pi at a Nyquist
//           index (the operator stays even on the grid).
//   GM_DG1: { G(q1,q2) + G(-q1,-q2) + (-1)^(i+j+k+l) [G(-q1,q2) + G(q1,-q2)] } / 4;
//           the sign factor is D G D with D = diag(1, 1, -1) on (11, 22, 12).
template <typename T>
__device__ __forceinline__ void green_op(int mode, const C2<T>* __restrict__ ktab, const C2<T>* __restrict__ qtab,
                                         int L, int m1, int m2, T lam0, T mu0, T scale, C2<T>& p11, C2<T>& p22,
                                         C2<T>& p12) {
  if (mode == GM_EQ3) {
    green_apply(ktab[m1], ktab[m2], lam0, mu0, scale, p11, p22, p12);
    return;
  }
  if (mode == GM_DISP) {
    disp_apply(ktab[m1], ktab[m2], L, m1, m2, scale, p11, p22, p12);
    return;
  }
  const C2<T> a11 = p11, a22 = p22, a12 = p12;
  if (mode == GM_CG1) {
    const bool y1 = 2 * m1 == L, y2 = 2 * m2 == L;
    if (!y1 && !y2) {
      green_apply(qtab[m1], qtab[m2], lam0, mu0, scale, p11, p22, p12);
      return;
    }
    C2<T> s11 = mk(T(0), T(0)), s22 = s11, s12 = s11;
    int cnt = 0;
    for (int s1 = 0; s1 <= (int)y1; s1++)
      for (int s2 = 0; s2 <= (int)y2; s2++) {
        C2<T> k1 = qtab[m1], k2 = qtab[m2];
        if (s1) k1.re = -k1.re;
        if (s2) k2.re = -k2.re;
        C2<T> b11 = a11, b22 = a22, b12 = a12;
        green_apply(k1, k2, lam0, mu0, scale, b11, b22, b12);
        s11 = s11 + b11;
        s22 = s22 + b22;
        s12 = s12 + b12;
        cnt++;
      }
    const T w = T(1) / T(cnt);
    p11 = w * s11;
    p22 = w * s22;
    p12 = w * s12;
    return;
  }
  // GM_DG1
  const int n1 = (L - m1) & (L - 1), n2 = (L - m2) & (L - 1);  // indices of -q1, -q2
  C2<T> b11 = a11, b22 = a22, b12 = a12;
  green_apply(ktab[m1], ktab[m2], lam0, mu0, scale, b11, b22, b12);
  C2<T> s11 = b11, s22 = b22, s12 = b12;
  b11 = a11, b22 = a22, b12 = a12;
  green_apply(ktab[n1], ktab[n2], lam0, mu0, scale, b11, b22, b12);
  s11 = s11 + b11, s22 = s22 + b22, s12 = s12 + b12;
  b11 = a11, b22 = a22, b12 = T(-1) * a12;
  green_apply(ktab[n1], ktab[m2], lam0, mu0, scale, b11, b22, b12);
  s11 = s11 + b11, s22 = s22 + b22, s12 = s12 - b12;
  b11 = a11, b22 = a22, b12 = T(-1) * a12;
  green_apply(ktab[m1], ktab[n2], lam0, mu0, scale, b11, b22, b12);
  s11 = s11 + b11, s22 = s22 + b22, s12 = s12 - b12;
  p11 = T(0.25) * s11;
  p22 = T(0.25) * s22;
  p12 = T(0.25) * s12;
}

}  // namespace epfft
