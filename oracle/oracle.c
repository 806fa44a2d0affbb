/*
 * oracle.c -- plain, slow, FP64 CPU reference for the augmented-Lagrangian
 * FFT iteration with the discrete Green operator of
 *   F. Willot, Y.-P. Pellegrini, "Fast Fourier Transform computations and
 *   build-up of plastic deformation in 2D, elastic-perfectly plastic,
 *   pixelwise disordered porous media" (arXiv:0802.2488).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the ground truth that the CUDA
 * path is compared against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product path never
 * calls it and shares no code, header, table or constant with it.
 *
 * Conventions (all fixed by the paper, Sec. 2):
 *   - L x L periodic lattice, pixel x = (x1, x2), linear index x2*L + x1
 *     (x1 is the fast index).
 *   - Strain / stress tensors are stored as 4 doubles per pixel in the
 *     order (11, 22, 33, 12); 13 = 23 = 0 (generalized plane strain, Sec. 2
 *     after Eq. 3: q3 = 0, in-plane indices only for the Green operator).
 *   - Forward DFT  f^(q) = sum_x f(x) exp(-i q.x),  q_j = 2 pi m_j / L,
 *     inverse with 1/L^2.  This is the sign for which the forward
 *     difference of Eq. 1 has the symbol i k_j of Eq. 2:
 *     u(x + e_j) - u(x)  <->  (exp(i q_j) - 1) u^ = i k_j u^.
 *
 * Functions and the passages they follow:
 *   orc_splitmix64, orc_mask,
 *   orc_void_threshold        : i.i.d. void pixels at concentration f
 *                               (Sec. 2, "randomly chosen as voids, in
 *                               concentration f"); the random numbers are
 *                               the published SplitMix64 stream
 *                               (Steele, Lea, Flood, OOPSLA 2014).
 *   orc_fft2                  : textbook radix-2 Cooley-Tukey FFT.
 *   orc_green                 : Eq. 2 (symbol k_j) and Eq. 3 (G_ijkl and the
 *                               acoustic tensor N), N inverted numerically.
 *   orc_green_mode            : the operators of Sec. 2 built from Eq. 3:
 *                               Eq. 3 itself, the same at mirrored momenta
 *                               (the four operators of DG2), the continuum
 *                               operator CG1 (Eq. 3 with k_j = q_j), and the
 *                               symmetrized DG1 operator (equation after
 *                               Eq. 3); orc_green_apply applies one of them
 *                               to a spectrum (Eqs. 2-3).
 *   orc_avg5                  : the 5-point local average of CG2 (Sec. 2).
 *   orc_displacement          : the displacement field of a strain field (Sec. 2).
 *   orc_sigma, orc_sigma_field: elastic-perfectly plastic Mises law under
 *                               deformation theory (Sec. 2, Sec. 3: plastic
 *                               zone where sigma_eq = Y, voids sigma = 0),
 *                               per pixel and over a field.
 *   orc_local_solve,
 *   orc_local_field           : pixelwise step of the augmented Lagrangian
 *                               (Sec. 1, ref. MICH00), per pixel and over a
 *                               field.
 *   orc_al_step               : one augmented-Lagrangian / Uzawa iteration.
 *   orc_stats                 : the convergence indicators of Sec. 2
 *                               ("Convergence issues"), backward-difference
 *                               divergence of Eq. 1.
 *   orc_solve                 : strain-controlled loading by increments
 *                               (Sec. 2, end of "Discrete Green functions").
 *   orc_label                 : Hoshen-Kopelman nearest-neighbour clusters
 *                               (Sec. 3), periodic lattice.
 *   orc_void_plastic          : clusters of the void-plastic phase with each
 *                               void-free cluster connected to its nearest
 *                               void (Sec. 3), and the counts behind the
 *                               indicators of Sec. 3.
 *   orc_threads, orc_set_threads : OpenMP threads of the loops (the
 *                               benchmark times the oracle on one host core
 *                               and on all of them).
 */
#include <complex.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* Threads of the OpenMP loops below (the benchmark times the oracle on one
 * host core and on all of them); 1 without OpenMP. */
int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* Material                                                            */
/* ------------------------------------------------------------------ */

typedef struct {
  double lambda, mu; /* Lame moduli of the matrix                        */
  double yield;      /* Mises flow stress Y; INFINITY means purely elastic */
  double lambda0;    /* reference medium C0 of the augmented Lagrangian    */
  double mu0;
  int32_t green;     /* Green operator, ORC_GREEN_* below                  */
  int32_t pad;
} orc_material;

/* Green operators of Sec. 2 */
enum {
  ORC_GREEN_EQ3 = 0,      /* G(q1, q2) of Eq. 3                               */
  ORC_GREEN_CG1 = 1,      /* continuum operator: Eq. 3 with k_j = q_j          */
  ORC_GREEN_DG1 = 2,      /* symmetrized G^(1)                                 */
  ORC_GREEN_EQ3_M1 = 3,   /* (-1)^(i+j+k+l) G(-q1, q2)  (DG2 members)          */
  ORC_GREEN_EQ3_M2 = 4,   /* (-1)^(i+j+k+l) G(q1, -q2)                         */
  ORC_GREEN_EQ3_M12 = 5,  /* G(-q1, -q2)                                       */
};

typedef struct {
  double tol_eq;    /* eta_1 */
  double tol_macro; /* eta_2 */
  int32_t max_iter; /* per increment */
  int32_t eq_test;  /* ORC_EQ_* below */
} orc_control;

/* Equilibrium test of an increment */
enum {
  ORC_EQ_OWN = 0,         /* eta1 for the operators of Eq. 3, eta3 for CG1, DG1 */
  ORC_EQ_FIXED_POINT = 1, /* eta3 for every operator (one criterion for all) */
};

typedef struct {
  double sig_mean[4]; /* <sigma> of the accepted iterate, (11,22,33,12) */
  double eps_mean[4]; /* <eps>                                          */
  double eta1, eta2, eta3;
  int32_t iterations;
  int32_t n_plastic;
  int32_t n_clusters;
  int32_t status; /* 0 converged, 1 max_iter reached, 2 NaN/Inf */
} orc_record;

/* ------------------------------------------------------------------ */
/* Random void pixels                                                  */
/* ------------------------------------------------------------------ */

/* i-th output (i = 0, 1, ...) of the SplitMix64 generator seeded with
 * `seed`: the state advances by the golden gamma 0x9e3779b97f4a7c15 and the
 * output is the 64-bit finaliser of the new state. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1u) * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

/* Pixel x is a void iff the top 53 bits of the x-th SplitMix64 output,
 * read as an integer u in [0, 2^53), satisfy u < floor(f * 2^53).  Each
 * pixel is then a void with probability f, independently (Sec. 2). */
uint64_t orc_void_threshold(double f) {
  if (!(f > 0.0)) return 0;
  if (f >= 1.0) return (uint64_t)1 << 53;
  return (uint64_t)floor(f * 9007199254740992.0); /* f * 2^53 is exact */
}

void orc_mask(int L, double f, uint64_t seed, uint8_t *mask) {
  uint64_t T = orc_void_threshold(f);
  for (int64_t x = 0; x < (int64_t)L * L; x++)
    mask[x] = (uint8_t)((orc_splitmix64(seed, (uint64_t)x) >> 11) < T);
}

/* ------------------------------------------------------------------ */
/* FFT: textbook iterative radix-2 Cooley-Tukey                       */
/* ------------------------------------------------------------------ */

/* In place, n a power of two, elements a[0], a[s], ..., a[(n-1)s].
 * sign = -1: sum_x a(x) exp(-2 pi i k x / n); sign = +1: the same with
 * exp(+...).  No normalisation. */
static void fft1(cplx *a, int n, int s, int sign) {
  for (int i = 1, j = 0; i < n; i++) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      cplx t = a[(int64_t)i * s];
      a[(int64_t)i * s] = a[(int64_t)j * s];
      a[(int64_t)j * s] = t;
    }
  }
  for (int len = 2; len <= n; len <<= 1) {
    int h = len / 2;
    for (int k = 0; k < h; k++) {
      double ang = sign * 2.0 * M_PI * (double)k / (double)len;
      cplx w = cos(ang) + I * sin(ang);
      for (int i = 0; i < n; i += len) {
        cplx u = a[(int64_t)(i + k) * s];
        cplx v = a[(int64_t)(i + k + h) * s] * w;
        a[(int64_t)(i + k) * s] = u + v;
        a[(int64_t)(i + k + h) * s] = u - v;
      }
    }
  }
}

/* 2D transform of an L x L array stored with x1 fastest: first along x1
 * (each row), then along x2 (each column).  Unnormalised. */
void orc_fft2(cplx *a, int L, int sign) {
#pragma omp parallel for schedule(static)
  for (int x2 = 0; x2 < L; x2++) fft1(a + (int64_t)x2 * L, L, 1, sign);
#pragma omp parallel for schedule(static)
  for (int x1 = 0; x1 < L; x1++) fft1(a + x1, L, L, sign);
}

/* ------------------------------------------------------------------ */
/* Discrete Green operator, Eqs. 2-3                                   */
/* ------------------------------------------------------------------ */

/* Eq. 2: k_j = 2 sin(q_j / 2) exp(i q_j / 2), q_j = 2 pi m_j / L. */
static cplx ksym(int m, int L) {
  double q = 2.0 * M_PI * (double)m / (double)L;
  return 2.0 * sin(q / 2.0) * cexp(I * q / 2.0);
}

static double kron(int a, int b) { return a == b ? 1.0 : 0.0; }

/* Isotropic stiffness of Lame moduli (lam, mu):
 * C_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk). */
static double stiff(double lam, double mu, int i, int j, int k, int l) {
  return lam * kron(i, j) * kron(k, l) +
         mu * (kron(i, k) * kron(j, l) + kron(i, l) * kron(j, k));
}

/* G_ijkl of Eq. 3 for given momenta symbols k = (k1, k2) and the reference
 * medium (lam0, mu0), in-plane indices i,j,k,l in {0,1} (= 1,2), stored
 * G[((i*2+j)*2+k)*2+l].  The acoustic tensor N_ij = k*_k C_iklj k_l is
 * built and inverted numerically, as the paper does. */
static void green_of_k(double lam0, double mu0, const cplx k[2], cplx *G) {
  cplx N[2][2];
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++) {
      cplx s = 0.0;
      for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
          s += conj(k[a]) * stiff(lam0, mu0, i, a, b, j) * k[b];
      N[i][j] = s;
    }
  cplx det = N[0][0] * N[1][1] - N[0][1] * N[1][0];
  cplx Ni[2][2] = {{N[1][1] / det, -N[0][1] / det},
                   {-N[1][0] / det, N[0][0] / det}};
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++)
      for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
          G[((i * 2 + j) * 2 + a) * 2 + b] =
              -(Ni[j][b] * k[i] * conj(k[a]) + Ni[i][b] * k[j] * conj(k[a]) +
                Ni[j][a] * k[i] * conj(k[b]) + Ni[i][a] * k[j] * conj(k[b])) /
              4.0;
}

/* G_ijkl(q) of Eq. 3 at q = 2 pi (m1, m2) / L.  At q = 0 the operator is
 * set to zero: the mean strain is imposed separately (it is the
 * prescribed E). */
void orc_green(int L, double lam0, double mu0, int m1, int m2, double *Gout) {
  cplx *G = (cplx *)Gout;
  for (int t = 0; t < 16; t++) G[t] = 0.0;
  if (m1 % L == 0 && m2 % L == 0) return;
  cplx k[2] = {ksym(m1, L), ksym(m2, L)};
  green_of_k(lam0, mu0, k, G);
}

/* Continuum momentum of index m: q = 2 pi m~ / L with m~ = m folded into
 * (-L/2, L/2]. */
static double qcont(int m, int L) {
  int mm = ((m % L) + L) % L;
  if (mm > L / 2) mm -= L;
  return 2.0 * M_PI * (double)mm / (double)L;
}

/* The Green operator `mode` (ORC_GREEN_*) at q = 2 pi (m1, m2) / L:
 *   EQ3, EQ3_M1, EQ3_M2, EQ3_M12: Eq. 3 at (q1, q2), (-q1, q2), (q1, -q2),
 *     (-q1, -q2), the four operators DG2 runs in turn; a single mirror
 *     carries the tensor sign (-1)^(i+j+k+l) of that mirror, as in DG1
 *     (without it the operator would solve the problem with E12 and
 *     sigma12 of the opposite sign);
 *   CG1: Eq. 3 with the continuum symbol k_j = q_j, q_j in (-pi, pi] (its
 *     long-wavelength limit; averaged over q_j = +-pi at Nyquist indices);
 *   DG1: { G(q1,q2) + G(-q1,-q2) + (-1)^(i+j+k+l) [G(-q1,q2) + G(q1,-q2)] } / 4.
 * Zero at q = 0. */
void orc_green_mode(int L, double lam0, double mu0, int mode, int m1, int m2, double *Gout) {
  cplx *G = (cplx *)Gout;
  for (int t = 0; t < 16; t++) G[t] = 0.0;
  if (m1 % L == 0 && m2 % L == 0) return;
  if (mode == ORC_GREEN_EQ3) {
    orc_green(L, lam0, mu0, m1, m2, Gout);
  } else if (mode == ORC_GREEN_EQ3_M1 || mode == ORC_GREEN_EQ3_M2) {
    /* single mirror: the momentum changes sign along one axis and the
     * operator takes the tensor sign of that mirror, (-1)^(i+j+k+l) */
    double Gm[32];
    if (mode == ORC_GREEN_EQ3_M1) orc_green(L, lam0, mu0, -m1, m2, Gm);
    else orc_green(L, lam0, mu0, m1, -m2, Gm);
    const cplx *A = (const cplx *)Gm;
    for (int t = 0; t < 16; t++) {
      const int i = t >> 3, j = (t >> 2) & 1, a = (t >> 1) & 1, b = t & 1;
      G[t] = ((i + j + a + b) % 2 == 0) ? A[t] : -A[t];
    }
  } else if (mode == ORC_GREEN_EQ3_M12) {
    orc_green(L, lam0, mu0, -m1, -m2, Gout);
  } else if (mode == ORC_GREEN_CG1) {
    /* At a Nyquist index (m = L/2) the continuum momentum is +pi or -pi;
     * the operator is the mean over both choices, which keeps it even in q
     * on the grid (so real fields stay real). */
    const int n1 = (((m1 % L) + L) % L) * 2 == L, n2 = (((m2 % L) + L) % L) * 2 == L;
    int cnt = 0;
    for (int s1 = 0; s1 <= n1; s1++)
      for (int s2 = 0; s2 <= n2; s2++) {
        cplx k[2] = {s1 ? -qcont(m1, L) : qcont(m1, L), s2 ? -qcont(m2, L) : qcont(m2, L)};
        cplx Gk[16];
        green_of_k(lam0, mu0, k, Gk);
        for (int t = 0; t < 16; t++) G[t] += Gk[t];
        cnt++;
      }
    for (int t = 0; t < 16; t++) G[t] /= (double)cnt;
  } else if (mode == ORC_GREEN_DG1) {
    double Ga[32], Gb[32], Gc[32], Gd[32];
    orc_green(L, lam0, mu0, m1, m2, Ga);
    orc_green(L, lam0, mu0, -m1, -m2, Gb);
    orc_green(L, lam0, mu0, -m1, m2, Gc);
    orc_green(L, lam0, mu0, m1, -m2, Gd);
    const cplx *A = (const cplx *)Ga, *B = (const cplx *)Gb, *C = (const cplx *)Gc, *D = (const cplx *)Gd;
    for (int i = 0; i < 2; i++)
      for (int j = 0; j < 2; j++)
        for (int a = 0; a < 2; a++)
          for (int b = 0; b < 2; b++) {
            /* indices 1,2 of the paper are i+1 etc.: (-1)^(i+j+a+b+4) */
            const double sgn = ((i + j + a + b) % 2 == 0) ? 1.0 : -1.0;
            const int t = ((i * 2 + j) * 2 + a) * 2 + b;
            G[t] = (A[t] + B[t] + sgn * (C[t] + D[t])) / 4.0;
          }
  }
}

/* e^_ij = sum_kl G_ijkl p^_kl (operator `mode`) at every frequency of an
 * L x L spectrum;
 * p^ and e^ hold the components (11, 22, 12) as three L*L complex planes;
 * p^_21 = p^_12.  At q = 0, e^ = L^2 * E (the prescribed mean strain). */
void orc_green_apply(int L, double lam0, double mu0, int mode, const double *E,
                     const double *phat_in, double *ehat_out) {
  const cplx *ph = (const cplx *)phat_in;
  cplx *eh = (cplx *)ehat_out;
  int64_t n = (int64_t)L * L;
  static const int ci[3][2] = {{0, 0}, {1, 1}, {0, 1}};
#pragma omp parallel for schedule(static)
  for (int m2 = 0; m2 < L; m2++)
    for (int m1 = 0; m1 < L; m1++) {
      int64_t q = (int64_t)m2 * L + m1;
      if (m1 == 0 && m2 == 0) {
        eh[q] = (double)n * E[0];
        eh[n + q] = (double)n * E[1];
        eh[2 * n + q] = (double)n * E[3];
        continue;
      }
      double Gd[32];
      orc_green_mode(L, lam0, mu0, mode, m1, m2, Gd);
      cplx *G = (cplx *)Gd;
      cplx P[2][2];
      P[0][0] = ph[q];
      P[1][1] = ph[n + q];
      P[0][1] = P[1][0] = ph[2 * n + q];
      for (int c = 0; c < 3; c++) {
        int i = ci[c][0], j = ci[c][1];
        cplx s = 0.0;
        for (int a = 0; a < 2; a++)
          for (int b = 0; b < 2; b++) s += G[((i * 2 + j) * 2 + a) * 2 + b] * P[a][b];
        eh[c * n + q] = s;
      }
    }
}

/* ------------------------------------------------------------------ */
/* Constitutive law                                                    */
/* ------------------------------------------------------------------ */

static double bulk(double lam, double mu) { return lam + 2.0 * mu / 3.0; }

/* |a| = (a:a)^(1/2) of a symmetric tensor stored (11,22,33,12). */
static double tnorm(const double a[4]) {
  return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + 2.0 * a[3] * a[3]);
}

/* sigma(eps) of a pixel.  Void: sigma = 0.  Matrix: nonlinear-elastic
 * (deformation theory) law whose Mises stress sigma_eq = (3/2 s:s)^(1/2)
 * never exceeds Y:
 *   sigma = K tr(eps) I + 2 mu dev(eps)                     if 2 mu |dev| <= sqrt(2/3) Y
 *   sigma = K tr(eps) I + sqrt(2/3) Y dev(eps) / |dev|      otherwise (sigma_eq = Y).
 * The deviator is the 3D one (tr/3 with eps33, as in the paper's eps_eq).
 * Returns 1 on the plastic branch. */
int orc_sigma(const double eps[4], int is_void, const orc_material *m,
              double sig[4]) {
  if (is_void) {
    sig[0] = sig[1] = sig[2] = sig[3] = 0.0;
    return 0;
  }
  double K = bulk(m->lambda, m->mu);
  double tr = eps[0] + eps[1] + eps[2];
  double d[4] = {eps[0] - tr / 3.0, eps[1] - tr / 3.0, eps[2] - tr / 3.0, eps[3]};
  double nd = tnorm(d);
  double ylim = sqrt(2.0 / 3.0) * m->yield;
  int plastic = 2.0 * m->mu * nd > ylim;
  double g = plastic ? ylim / nd : 2.0 * m->mu;
  sig[0] = K * tr + g * d[0];
  sig[1] = K * tr + g * d[1];
  sig[2] = K * tr + g * d[2];
  sig[3] = g * d[3];
  return plastic;
}

/* C0:a = lam0 tr(a) I + 2 mu0 a. */
static void c0_apply(const orc_material *m, const double a[4], double out[4]) {
  double tr = a[0] + a[1] + a[2];
  out[0] = m->lambda0 * tr + 2.0 * m->mu0 * a[0];
  out[1] = m->lambda0 * tr + 2.0 * m->mu0 * a[1];
  out[2] = m->lambda0 * tr + 2.0 * m->mu0 * a[2];
  out[3] = 2.0 * m->mu0 * a[3];
}

/* Local step of the augmented Lagrangian: the minimiser eps of
 *   w(eps) - tau:eps + 1/2 eps:C0:eps
 * i.e. the solution of sigma(eps) + C0:eps = tau.  Both sigma and C0 are
 * isotropic, so the equation splits into a mean part
 *   3 (K + K0) eps_m = tau_m,        tau_m = tr(tau)/3
 * and a deviatoric part along tau' = tau - tau_m I:
 *   matrix, elastic:  2 (mu + mu0) dev = tau'
 *   matrix, plastic:  sqrt(2/3) Y dev/|dev| + 2 mu0 dev = tau'
 *                     => dev = (tau' - sqrt(2/3) Y tau'/|tau'|) / (2 mu0)
 *   void:             2 mu0 dev = tau',  3 K0 eps_m = tau_m.
 * The elastic solution is taken when it satisfies the elastic test of
 * sigma, i.e. 2 mu |dev| <= sqrt(2/3) Y.  Returns 1 on the plastic branch. */
int orc_local_solve(const double tau[4], int is_void, const orc_material *m,
                    double eps[4]) {
  double K = bulk(m->lambda, m->mu), K0 = bulk(m->lambda0, m->mu0);
  double tm = (tau[0] + tau[1] + tau[2]) / 3.0;
  double td[4] = {tau[0] - tm, tau[1] - tm, tau[2] - tm, tau[3]};
  double em, dev[4];
  int plastic = 0;
  if (is_void) {
    em = tm / (3.0 * K0);
    for (int c = 0; c < 4; c++) dev[c] = td[c] / (2.0 * m->mu0);
  } else {
    em = tm / (3.0 * (K + K0));
    double ylim = sqrt(2.0 / 3.0) * m->yield;
    for (int c = 0; c < 4; c++) dev[c] = td[c] / (2.0 * (m->mu + m->mu0));
    if (2.0 * m->mu * tnorm(dev) > ylim) {
      plastic = 1;
      double nt = tnorm(td);
      for (int c = 0; c < 4; c++)
        dev[c] = (td[c] - ylim * td[c] / nt) / (2.0 * m->mu0);
    }
  }
  eps[0] = dev[0] + em;
  eps[1] = dev[1] + em;
  eps[2] = dev[2] + em;
  eps[3] = dev[3];
  return plastic;
}

/* ------------------------------------------------------------------ */
/* One augmented-Lagrangian (Uzawa) iteration                          */
/* ------------------------------------------------------------------ */

/* Given the local strain eps^n and the Lagrange multiplier lam^n
 * (both L*L*4, in place), performs
 *   p^n     = lam^n - C0:eps^n                         (polarization, in-plane)
 *   e^{n+1} = E + IDFT( G(q) DFT(p^n) )                (compatible strain, Eqs. 2-3)
 *   eps^{n+1} = argmin_eps w(eps) - (lam^n + C0:e^{n+1}):eps + 1/2 eps:C0:eps
 *   lam^{n+1} = lam^n + C0:(e^{n+1} - eps^{n+1})       (multiplier update)
 * e33 = E33 because the Green operator has no 33 output (q3 = 0).
 * e_out (optional, L*L*4) receives e^{n+1}; plastic_out (optional, L*L)
 * the branch taken by the local step. */
void orc_al_step(int L, const uint8_t *mask, const orc_material *m,
                 const double E[4], double *eps, double *lam, double *e_out,
                 uint8_t *plastic_out) {
  int64_t n = (int64_t)L * L;
  cplx *buf = (cplx *)malloc(sizeof(cplx) * 6 * n);
  cplx *ph = buf, *eh = buf + 3 * n;
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < n; x++) {
    double c0e[4];
    c0_apply(m, eps + 4 * x, c0e);
    ph[x] = lam[4 * x + 0] - c0e[0];
    ph[n + x] = lam[4 * x + 1] - c0e[1];
    ph[2 * n + x] = lam[4 * x + 3] - c0e[3];
  }
  for (int c = 0; c < 3; c++) orc_fft2(ph + c * n, L, -1);
  orc_green_apply(L, m->lambda0, m->mu0, m->green, E, (const double *)ph, (double *)eh);
  for (int c = 0; c < 3; c++) orc_fft2(eh + c * n, L, +1);
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < n; x++) {
    double e[4] = {creal(eh[x]) / (double)n, creal(eh[n + x]) / (double)n, E[2],
                   creal(eh[2 * n + x]) / (double)n};
    double c0e[4], tau[4], enew[4], c0d[4], d[4];
    c0_apply(m, e, c0e);
    for (int c = 0; c < 4; c++) tau[c] = lam[4 * x + c] + c0e[c];
    int pl = orc_local_solve(tau, mask[x], m, enew);
    for (int c = 0; c < 4; c++) d[c] = e[c] - enew[c];
    c0_apply(m, d, c0d);
    for (int c = 0; c < 4; c++) {
      lam[4 * x + c] += c0d[c];
      eps[4 * x + c] = enew[c];
      if (e_out) e_out[4 * x + c] = e[c];
    }
    if (plastic_out) plastic_out[x] = (uint8_t)pl;
  }
  free(buf);
}

/* ------------------------------------------------------------------ */
/* Convergence indicators                                              */
/* ------------------------------------------------------------------ */

/* For the constitutive stress sigma(eps): its mean, the mean strain, the
 * mean squared backward-difference divergence of Eq. 1,
 *   div_i(x) = sum_j [ sigma_ij(x) - sigma_ij(x - e^j) ],  i, j in {1, 2},
 * and the number of matrix pixels on the plastic branch (written to
 * plastic_out when given).  Sums are taken row by row and the row sums
 * added in row order, so the result does not depend on the thread count. */
void orc_stats(int L, const uint8_t *mask, const orc_material *m,
               const double *eps, double sig_mean[4], double eps_mean[4],
               double *div2_mean, int32_t *n_plastic, uint8_t *plastic_out) {
  int64_t n = (int64_t)L * L;
  double *sig = (double *)malloc(sizeof(double) * 4 * n);
  double *rows = (double *)calloc((size_t)L * 10, sizeof(double));
  int32_t *rpl = (int32_t *)calloc((size_t)L, sizeof(int32_t));
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < n; x++) {
    int pl = orc_sigma(eps + 4 * x, mask[x], m, sig + 4 * x);
    if (plastic_out) plastic_out[x] = (uint8_t)pl;
  }
#pragma omp parallel for schedule(static)
  for (int x2 = 0; x2 < L; x2++) {
    double *r = rows + (int64_t)x2 * 10;
    for (int x1 = 0; x1 < L; x1++) {
      int64_t x = (int64_t)x2 * L + x1;
      int64_t xm1 = (int64_t)x2 * L + (x1 + L - 1) % L;    /* x - e^1 */
      int64_t xm2 = (int64_t)((x2 + L - 1) % L) * L + x1;  /* x - e^2 */
      const double *s = sig + 4 * x, *s1 = sig + 4 * xm1, *s2 = sig + 4 * xm2;
      /* sigma_11 -> s[0], sigma_22 -> s[1], sigma_12 = sigma_21 -> s[3] */
      double div1 = (s[0] - s1[0]) + (s[3] - s2[3]);
      double div2 = (s[3] - s1[3]) + (s[1] - s2[1]);
      for (int c = 0; c < 4; c++) {
        r[c] += s[c];
        r[4 + c] += eps[4 * x + c];
      }
      r[8] += div1 * div1 + div2 * div2;
      if (!mask[x]) {
        double tmp[4];
        rpl[x2] += orc_sigma(eps + 4 * x, 0, m, tmp);
      }
    }
  }
  double acc[9] = {0};
  int32_t npl = 0;
  for (int x2 = 0; x2 < L; x2++) {
    for (int c = 0; c < 9; c++) acc[c] += rows[(int64_t)x2 * 10 + c];
    npl += rpl[x2];
  }
  for (int c = 0; c < 4; c++) {
    sig_mean[c] = acc[c] / (double)n;
    eps_mean[c] = acc[4 + c] / (double)n;
  }
  *div2_mean = acc[8] / (double)n;
  *n_plastic = npl;
  free(sig);
  free(rows);
  free(rpl);
}

/* In-plane contraction a:b = a11 b11 + a22 b22 + 2 a12 b12 used by the
 * indicators of Sec. 2 ("<sigma>:<sigma>"). */
static double ip_dot(const double a[4], const double b[4]) {
  return a[0] * b[0] + a[1] * b[1] + 2.0 * a[3] * b[3];
}

/* ------------------------------------------------------------------ */
/* Hoshen-Kopelman clusters (union-find form)                          */
/* ------------------------------------------------------------------ */

static int64_t uf_find(int64_t *parent, int64_t a) {
  while (parent[a] != a) {
    parent[a] = parent[parent[a]];
    a = parent[a];
  }
  return a;
}

/* The smaller root becomes the parent, so every root is the smallest
 * linear index of its cluster. */
static void uf_union(int64_t *parent, int64_t a, int64_t b) {
  a = uf_find(parent, a);
  b = uf_find(parent, b);
  if (a == b) return;
  if (a < b) parent[b] = a;
  else parent[a] = b;
}

/* Clusters of flagged pixels connected by the nearest-neighbour criterion
 * (Sec. 3).  Raster scan joining each flagged pixel to its flagged left
 * and upper neighbours, then (periodic != 0) the wrap-around bonds of the
 * periodic cell.  label[x] = smallest linear index of x's cluster, or -1
 * for unflagged pixels.  Returns the number of clusters. */
int32_t orc_label(int L, const uint8_t *flag, int periodic, int32_t *label) {
  int64_t n = (int64_t)L * L;
  int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t x = 0; x < n; x++) parent[x] = x;
  for (int x2 = 0; x2 < L; x2++)
    for (int x1 = 0; x1 < L; x1++) {
      int64_t x = (int64_t)x2 * L + x1;
      if (!flag[x]) continue;
      if (x1 > 0 && flag[x - 1]) uf_union(parent, x, x - 1);
      if (x2 > 0 && flag[x - L]) uf_union(parent, x, x - L);
    }
  if (periodic) {
    for (int x2 = 0; x2 < L; x2++) {
      int64_t a = (int64_t)x2 * L, b = a + L - 1;
      if (flag[a] && flag[b]) uf_union(parent, a, b);
    }
    for (int x1 = 0; x1 < L; x1++) {
      int64_t a = x1, b = (int64_t)(L - 1) * L + x1;
      if (flag[a] && flag[b]) uf_union(parent, a, b);
    }
  }
  int32_t count = 0;
  for (int64_t x = 0; x < n; x++) {
    if (!flag[x]) {
      label[x] = -1;
      continue;
    }
    int64_t r = uf_find(parent, x);
    label[x] = (int32_t)r;
    if (r == x) count++;
  }
  free(parent);
  return count;
}

/* ------------------------------------------------------------------ */
/* Loading by increments                                               */
/* ------------------------------------------------------------------ */

/* Strain-controlled loading (Sec. 2): the prescribed mean strain takes the
 * values E[4*k .. 4*k+3] (11,22,33,12), k = 0 .. n_inc-1.  The lattice
 * starts unstrained; each increment adds E_k - E_{k-1} to the local strain
 * of the previous converged state (deformation theory is reversible, so
 * the converged state is the whole history), sets the multiplier to
 * sigma(eps), and iterates until
 *   <|div sigma|^2> < eta1^2 <sigma>:<sigma>            and
 *   (<sigma^{n+1}> - <sigma^n>):(same) < eta2^2 <sigma^{n+1}>:<sigma^{n+1}>
 * hold at the same iterate (strict), with sigma = sigma(eps^{n+1}), or
 * max_iter iterations.  eta3 = (<(eps-e):(eps-e)> / E:E)^(1/2) with the
 * full (3D) contraction takes the place of eta1 for CG1 and DG1, and for
 * every operator when ctl->eq_test is ORC_EQ_FIXED_POINT; otherwise it is
 * reported only.
 * Optional outputs: eps_final (L*L*4), plastic_all / labels_all
 * (n_inc*L*L: plastic flag of the accepted iterate, its periodic clusters).
 * Returns 0 when every increment converged, else the first nonzero status. */
int32_t orc_solve(int L, const uint8_t *mask, const orc_material *m,
                  const orc_control *ctl, int n_inc, const double *E,
                  orc_record *rec, double *eps_final, uint8_t *plastic_all,
                  int32_t *labels_all) {
  int64_t n = (int64_t)L * L;
  double *eps = (double *)calloc((size_t)(4 * n), sizeof(double));
  double *lam = (double *)malloc(sizeof(double) * 4 * n);
  double *e = (double *)malloc(sizeof(double) * 4 * n);
  uint8_t *pl = (uint8_t *)malloc((size_t)n);
  int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  double Eprev[4] = {0, 0, 0, 0};
  int32_t ret = 0;
  for (int k = 0; k < n_inc; k++) {
    const double *Ek = E + 4 * k;
    orc_record *r = rec + k;
    memset(r, 0, sizeof(*r));
    for (int64_t x = 0; x < n; x++)
      for (int c = 0; c < 4; c++) eps[4 * x + c] += Ek[c] - Eprev[c];
    memcpy(Eprev, Ek, sizeof(Eprev));
    for (int64_t x = 0; x < n; x++) orc_sigma(eps + 4 * x, mask[x], m, lam + 4 * x);
    double sprev[4], eps_m[4], div2;
    int32_t npl;
    orc_stats(L, mask, m, eps, sprev, eps_m, &div2, &npl, NULL);
    double EE = Ek[0] * Ek[0] + Ek[1] * Ek[1] + Ek[2] * Ek[2] + 2.0 * Ek[3] * Ek[3];
    if (EE == 0.0) EE = 1.0;
    int status = 1;
    int it = 0;
    double s[4], eta1 = 0, eta2 = 0, eta3 = 0;
    while (it < ctl->max_iter) {
      orc_al_step(L, mask, m, Ek, eps, lam, e, NULL);
      it++;
      orc_stats(L, mask, m, eps, s, eps_m, &div2, &npl, NULL);
      double ss = ip_dot(s, s);
      double ds[4] = {s[0] - sprev[0], s[1] - sprev[1], s[2] - sprev[2], s[3] - sprev[3]};
      double dd = ip_dot(ds, ds);
      double c2 = 0.0;
      for (int64_t x = 0; x < n; x++) {
        double a[4];
        for (int c = 0; c < 4; c++) a[c] = eps[4 * x + c] - e[4 * x + c];
        c2 += a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + 2.0 * a[3] * a[3];
      }
      if (ss > 0.0) {
        eta1 = sqrt(div2 / ss);
        eta2 = sqrt(dd / ss);
      } else { /* sigma vanishes on average (e.g. all pixels void) */
        eta1 = div2 == 0.0 ? 0.0 : INFINITY;
        eta2 = dd == 0.0 ? 0.0 : INFINITY;
      }
      eta3 = sqrt(c2 / (double)n / EE);
      memcpy(sprev, s, sizeof(sprev));
      if (!isfinite(eta1) || !isfinite(eta2) || !isfinite(s[0]) ||
          !isfinite(s[1]) || !isfinite(s[3])) {
        status = 2;
        break;
      }
      /* Equilibrium test: eta1 (Sec. 2, divergence of Eq. 1) for the
       * operators of Eq. 3.  The continuum (CG1) and symmetrized (DG1)
       * operators are not the Green operators of Eq. 1, so the divergence
       * of Eq. 1 does not vanish at their solutions; there the augmented
       * Lagrangian's own fixed-point residual eta3 (local strain minus
       * compatible strain) takes its place.  With ORC_EQ_FIXED_POINT every
       * operator stops on eta3, so that iteration counts of the operators
       * are counted against one criterion. */
      const int fixed_point = ctl->eq_test == ORC_EQ_FIXED_POINT || m->green == ORC_GREEN_CG1 ||
                              m->green == ORC_GREEN_DG1;
      const double eq = fixed_point ? eta3 : eta1;
      if (eq < ctl->tol_eq && eta2 < ctl->tol_macro) {
        status = 0;
        break;
      }
    }
    orc_stats(L, mask, m, eps, s, eps_m, &div2, &npl, pl);
    for (int64_t x = 0; x < n; x++) pl[x] = (uint8_t)(pl[x] && !mask[x]);
    memcpy(r->sig_mean, s, sizeof(s));
    memcpy(r->eps_mean, eps_m, sizeof(eps_m));
    r->eta1 = eta1;
    r->eta2 = eta2;
    r->eta3 = eta3;
    r->iterations = it;
    r->n_plastic = npl;
    r->n_clusters = orc_label(L, pl, 1, lab);
    r->status = status;
    if (plastic_all) memcpy(plastic_all + (int64_t)k * n, pl, (size_t)n);
    if (labels_all) memcpy(labels_all + (int64_t)k * n, lab, sizeof(int32_t) * (size_t)n);
    if (status != 0 && ret == 0) ret = status;
    if (status == 2) break;
  }
  if (eps_final) memcpy(eps_final, eps, sizeof(double) * 4 * n);
  free(eps);
  free(lam);
  free(e);
  free(pl);
  free(lab);
  return ret;
}

/* ------------------------------------------------------------------ */
/* Field-wide wrappers (for the test suite)                            */
/* ------------------------------------------------------------------ */

/* sigma(eps) on n pixels (eps, sig: n*4); plastic (optional, n). */
void orc_sigma_field(int64_t n, const double *eps, const uint8_t *mask,
                     const orc_material *m, double *sig, uint8_t *plastic) {
  for (int64_t x = 0; x < n; x++) {
    int pl = orc_sigma(eps + 4 * x, mask[x], m, sig + 4 * x);
    if (plastic) plastic[x] = (uint8_t)pl;
  }
}

/* Local step on n pixels (tau, eps: n*4); plastic (optional, n). */
void orc_local_field(int64_t n, const double *tau, const uint8_t *mask,
                     const orc_material *m, double *eps, uint8_t *plastic) {
  for (int64_t x = 0; x < n; x++) {
    int pl = orc_local_solve(tau + 4 * x, mask[x], m, eps + 4 * x);
    if (plastic) plastic[x] = (uint8_t)pl;
  }
}

/* ------------------------------------------------------------------ */
/* CG2 post-processing                                                 */
/* ------------------------------------------------------------------ */

/* Displacement of Sec. 2 from the in-plane strain: with k^2 = k1^2 + k2^2
 * (the discrete symbols of Eq. 2, squared as complex numbers),
 *   u1(q) = -(i / k^2) { k1 [e11 - e22] + 2 k2 e12 },
 *   u2(q) =  (i / k^2) { k2 [e11 - e22] - 2 k1 e12 },
 * and u(0) = 0 (the mode q = 0 is irrelevant).  k^2 vanishes at
 * q = (pi/2, 3pi/2) and (3pi/2, pi/2) (m = (L/4, 3L/4), (3L/4, L/4) when 4
 * divides L), where the formula is 0/0 for a compatible strain; there u is
 * taken from the same relation e_ab = (i/2)(k_a u_b + k_b u_a) solved with
 * the real |k|^2 = |k1|^2 + |k2|^2: w_b = k*_a e_ab, s = k*.u =
 * -i (k*.w) / |k|^2, u_b = (-2 i w_b - k_b s) / |k|^2.  eps: L*L*4
 * (11, 22, 33, 12) at [x2][x1]; u: L*L*2 (u1, u2). */
void orc_displacement(int L, const double *eps, double *u) {
  int64_t n = (int64_t)L * L;
  cplx *e = (cplx *)malloc(sizeof(cplx) * 5 * n);
  cplx *e11 = e, *e22 = e + n, *e12 = e + 2 * n, *u1 = e + 3 * n, *u2 = e + 4 * n;
  for (int64_t x = 0; x < n; x++) {
    e11[x] = eps[4 * x + 0];
    e22[x] = eps[4 * x + 1];
    e12[x] = eps[4 * x + 3];
  }
  orc_fft2(e11, L, -1);
  orc_fft2(e22, L, -1);
  orc_fft2(e12, L, -1);
  for (int m2 = 0; m2 < L; m2++)
    for (int m1 = 0; m1 < L; m1++) {
      int64_t f = (int64_t)m2 * L + m1;
      if (m1 == 0 && m2 == 0) {
        u1[f] = 0.0;
        u2[f] = 0.0;
        continue;
      }
      cplx k1 = ksym(m1, L), k2 = ksym(m2, L);
      int zero_k2 = (L % 4 == 0) && ((m1 == L / 4 && m2 == 3 * L / 4) || (m1 == 3 * L / 4 && m2 == L / 4));
      if (!zero_k2) {
        cplx kk = k1 * k1 + k2 * k2;
        cplx d = e11[f] - e22[f];
        u1[f] = -I / kk * (k1 * d + 2.0 * k2 * e12[f]);
        u2[f] = I / kk * (k2 * d - 2.0 * k1 * e12[f]);
      } else {
        double nk = creal(k1 * conj(k1) + k2 * conj(k2));
        cplx w1 = conj(k1) * e11[f] + conj(k2) * e12[f];
        cplx w2 = conj(k1) * e12[f] + conj(k2) * e22[f];
        cplx sdot = -I * (conj(k1) * w1 + conj(k2) * w2) / nk;
        u1[f] = (-2.0 * I * w1 - k1 * sdot) / nk;
        u2[f] = (-2.0 * I * w2 - k2 * sdot) / nk;
      }
    }
  orc_fft2(u1, L, +1);
  orc_fft2(u2, L, +1);
  for (int64_t x = 0; x < n; x++) {
    u[2 * x + 0] = creal(u1[x]) / (double)n;
    u[2 * x + 1] = creal(u2[x]) / (double)n;
  }
  free(e);
}

/* The local average of CG2 (Sec. 2): every pixel of a field of 4 reals per
 * pixel receives the mean of its own value and those of its four nearest
 * neighbours (periodic lattice). */
void orc_avg5(int L, const double *in, double *out) {
  for (int x2 = 0; x2 < L; x2++)
    for (int x1 = 0; x1 < L; x1++) {
      const int64_t x = (int64_t)x2 * L + x1;
      const int64_t nb[4] = {(int64_t)x2 * L + (x1 + 1) % L, (int64_t)x2 * L + (x1 + L - 1) % L,
                             (int64_t)((x2 + 1) % L) * L + x1, (int64_t)((x2 + L - 1) % L) * L + x1};
      for (int c = 0; c < 4; c++) {
        double s = in[4 * x + c];
        for (int n = 0; n < 4; n++) s += in[4 * nb[n] + c];
        out[4 * x + c] = s / 5.0;
      }
    }
}

/* ------------------------------------------------------------------ */
/* Void-plastic clusters (Sec. 3)                                      */
/* ------------------------------------------------------------------ */

/* Squared distance between pixel centres on the periodic lattice. */
static int64_t pdist2(int L, int64_t a, int64_t b) {
  int64_t d1 = llabs(a % L - b % L), d2 = llabs(a / L - b / L);
  if (d1 > L - d1) d1 = L - d1;
  if (d2 > L - d2) d2 = L - d2;
  return d1 * d1 + d2 * d2;
}

/* Clusters of the void-plastic phase (voids and plastic pixels) of Sec. 3:
 * nearest-neighbour clusters of the phase (periodic), then every cluster
 * without a void is connected to the nearest void: the void pixel at the
 * smallest distance from any of the cluster's pixels (ties: the smallest
 * linear index of the void pixel), computed here by comparing every pixel
 * of the cluster with every void pixel.  label[x] = smallest linear index
 * of x's final cluster, -1 off the phase.
 * stats[0] = number of final clusters, stats[1] = pixels of the largest,
 * stats[2] = final clusters without a plastic pixel (isolated voids),
 * stats[3] = number of clusters of the voids alone, stats[4] = plastic
 * (non-void) pixels, stats[5] = void pixels.  Returns stats[0]. */
int32_t orc_void_plastic(int L, const uint8_t *mask, const uint8_t *plastic, int32_t *label, int32_t *stats) {
  const int64_t n = (int64_t)L * L;
  uint8_t *vp = (uint8_t *)malloc((size_t)n);
  int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  for (int64_t x = 0; x < n; x++) vp[x] = (uint8_t)(mask[x] || plastic[x]);
  orc_label(L, vp, 1, lab);
  /* clusters (by root) that hold a void */
  uint8_t *has_void = (uint8_t *)calloc((size_t)n, 1);
  for (int64_t x = 0; x < n; x++)
    if (mask[x]) has_void[lab[x]] = 1;
  int64_t nvoid = 0;
  for (int64_t x = 0; x < n; x++) nvoid += mask[x] != 0;
  /* target root of each cluster: itself, or the root of its nearest void */
  int64_t *target = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t x = 0; x < n; x++) target[x] = x;
  if (nvoid > 0) {
    for (int64_t r = 0; r < n; r++) {
      if (!vp[r] || lab[r] != r || has_void[r]) continue;
      int64_t best_d = -1, best_v = -1;
      for (int64_t x = 0; x < n; x++) {
        if (lab[x] != r) continue;
        for (int64_t v = 0; v < n; v++) {
          if (!mask[v]) continue;
          const int64_t d = pdist2(L, x, v);
          if (best_d < 0 || d < best_d || (d == best_d && v < best_v)) {
            best_d = d;
            best_v = v;
          }
        }
      }
      target[r] = lab[best_v];
    }
  }
  /* final label: smallest linear index over the merged clusters */
  int64_t *final_root = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t x = 0; x < n; x++) final_root[x] = n;
  for (int64_t r = 0; r < n; r++) {
    if (!vp[r] || lab[r] != r) continue;
    const int64_t t = target[r];
    if (r < final_root[t]) final_root[t] = r;
  }
  for (int64_t x = 0; x < n; x++) {
    if (!vp[x]) {
      label[x] = -1;
      continue;
    }
    label[x] = (int32_t)final_root[target[lab[x]]];
  }
  int32_t count = 0, largest = 0, isolated = 0;
  int32_t *size = (int32_t *)calloc((size_t)n, sizeof(int32_t));
  uint8_t *has_pl = (uint8_t *)calloc((size_t)n, 1);
  for (int64_t x = 0; x < n; x++) {
    if (label[x] < 0) continue;
    size[label[x]]++;
    if (!mask[x]) has_pl[label[x]] = 1;
  }
  for (int64_t x = 0; x < n; x++) {
    if (size[x] == 0) continue;
    count++;
    if (size[x] > largest) largest = size[x];
    if (!has_pl[x]) isolated++;
  }
  stats[0] = count;
  stats[1] = largest;
  stats[2] = isolated;
  stats[3] = orc_label(L, mask, 1, lab);
  int32_t npl = 0;
  for (int64_t x = 0; x < n; x++) npl += plastic[x] && !mask[x];
  stats[4] = npl;
  stats[5] = (int32_t)nvoid;
  free(vp);
  free(lab);
  free(has_void);
  free(target);
  free(final_root);
  free(size);
  free(has_pl);
  return count;
}
