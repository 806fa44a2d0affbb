/*
 * epfft.h -- C ABI of the GB300 (sm_103a) implementation of the
 * augmented-Lagrangian FFT scheme with the discrete Green operator of
 *
 *   F. Willot, Y.-P. Pellegrini, "Fast Fourier Transform computations and
 *   build-up of plastic deformation in 2D, elastic-perfectly plastic,
 *   pixelwise disordered porous media", arXiv:0802.2488.
 *
 * Problem (Sec. 2): an L x L periodic square lattice of pixels, each either a
 * void (stress-free) or an elastic-perfectly plastic Mises element with
 * flow stress Y under deformation theory, loaded by a prescribed mean
 * strain increased by increments.  Strain is the forward difference of the
 * displacement and equilibrium the backward difference of the stress (Eq. 1);
 * the compatible-strain projection uses the discrete Green operator of
 * Eqs. 2-3 (generalized plane strain, q3 = 0).  The nonlinear problem is
 * solved with the augmented-Lagrangian / Uzawa iteration the paper cites
 * (Sec. 1), and each increment stops on the two indicators of Sec. 2
 * ("Convergence issues"):
 *     <|div sigma|^2>               < eta1^2 <sigma>:<sigma>
 *     |<sigma^{n+1}> - <sigma^n>|^2 < eta2^2 <sigma^{n+1}>:<sigma^{n+1}>
 * with a:b = a11 b11 + a22 b22 + 2 a12 b12.
 *
 * Conventions of every call:
 *   - lattice side L: a power of two, 4 <= L <= 4096;
 *   - pixel x = (x1, x2) at linear index x2 * L + x1 (x1 fastest);
 *   - symmetric tensors are 4 reals per pixel in the order (11, 22, 33, 12);
 *   - forward DFT kernel exp(-i q.x), q_j = 2 pi m_j / L (the sign for which
 *     the forward difference of Eq. 1 has the symbol i k_j of Eq. 2).
 *
 * Errors: every int-returning call returns EPFFT_OK (0) or a code below;
 * epfft_strerror() names it.  Invalid arguments never reach the GPU.  There
 * is no CPU fallback: without a usable CUDA device the calls return
 * EPFFT_ERR_CUDA.  A context is used by one host thread at a time.
 *
 * Calls that compute a part of the method cite the passage that defines it.
 * Contexts, batching, serving, tiling and timing have no counterpart in the
 * paper: they are how this library runs the method on a GPU.
 */
#ifndef EPFFT_H
#define EPFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EPFFT_OK 0
#define EPFFT_PENDING 1             /* not finished yet                          */
#define EPFFT_ERR_ARG (-1)          /* invalid argument (nothing was launched)   */
#define EPFFT_ERR_OOM (-2)          /* device allocation failed                  */
#define EPFFT_ERR_NUMERIC (-3)      /* NaN / Inf in a residual or mean stress    */
#define EPFFT_NOT_CONVERGED (-4)    /* some increment hit max_iter; results kept */
#define EPFFT_ERR_DEVICE_TIMEOUT (-5) /* the device loop exceeded its pass bound */
#define EPFFT_ERR_CUDA (-6)         /* a CUDA runtime call failed                */
#define EPFFT_ERR_UNSUPPORTED (-7)  /* size / precision not built                */
#define EPFFT_ERR_SCRATCH_LIMIT (-8) /* larger than epfft_project_static's scratch */

#define EPFFT_FP64 0 /* FP64 fields, FFTs and reductions                        */
#define EPFFT_FP32 1 /* FP32 fields and FFTs, FP64 reductions and macro values  */
#define EPFFT_FP32_DEFECT 2 /* defect correction: FP32 iterations on the     *
                             * differences of strain and stress from an FP64  *
                             * reference state, which a refresh (FP64 law,    *
                             * FP64 transforms of Eqs. 2-3) moves to the      *
                             * current iterate after each warm start and      *
                             * every epfft_set_defect_refresh iterations; the *
                             * FP32 rounding then scales with the distance    *
                             * from the reference, so the tolerances of the   *
                             * FP64 form (Sec. 2) are reached at FP32 cost.   *
                             * Fields are FP64; tilings 0 and 1.              */

#define EPFFT_GREEN_EQ3 0 /* discrete Green operator of Eq. 3                   */
#define EPFFT_GREEN_CG1 1 /* continuum operator (Sec. 2, CG1): Eq. 3 with the   *
                           * momenta k_j = q_j, q_j in (-pi, pi], averaged over  *
                           * q_j = +-pi at Nyquist indices                       */
#define EPFFT_GREEN_DG1 2 /* symmetrized operator (Sec. 2, DG1): the mean of     *
                           * G(q1,q2), G(-q1,-q2) and the tensor-signed          *
                           * (-1)^(i+j+k+l) G(-q1,q2), G(q1,-q2)                 */

/* Equilibrium test of an increment (epfft_problem.eq_test) */
#define EPFFT_EQ_OWN 0         /* eta1 (divergence of Eq. 1, Sec. 2) with the     *
                                * operators of Eq. 3; eta3 with CG1 and DG1      */
#define EPFFT_EQ_FIXED_POINT 1 /* eta3 with every operator: one criterion, so    *
                                * that iteration counts of the operators can be  *
                                * compared (Sec. 2, DG2 against CG1)             */

typedef struct epfft_ctx epfft_ctx;

/* Device memory hook.  alloc returns a device pointer usable on `stream`
 * (NULL on failure); free releases it.  With both NULL the library uses
 * cudaMallocAsync / cudaFreeAsync on its stream. */
typedef void *(*epfft_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*epfft_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

typedef struct {
  int32_t device;          /* CUDA device ordinal                                */
  int32_t reserved;
  void *stream;            /* cudaStream_t to work on; NULL: the context creates  *
                            * its own non-blocking stream                         */
  epfft_alloc_fn alloc;    /* optional allocator hook (see above)                */
  epfft_free_fn free;
  void *alloc_user;
} epfft_options;

/* One solve (Sec. 2): the lattice, its voids, the matrix and the iteration
 * controls.  Copied at call time; the caller keeps ownership of `mask`. */
typedef struct {
  int32_t L;               /* lattice side (see conventions)                      */
  int32_t precision;       /* EPFFT_FP64 or EPFFT_FP32                            */
  double void_fraction;    /* f in [0, 1]: used when mask == NULL                 */
  uint64_t seed;           /* mask seed: pixel x is void iff the top 53 bits of   *
                            * the x-th output of SplitMix64(seed) are below       *
                            * floor(f 2^53) (i.i.d. Bernoulli(f) voids, Sec. 2)   */
  const uint8_t *mask;     /* optional L*L mask, 1 = void; host or device         */
  int32_t mask_on_device;  /* 1 if `mask` is a device pointer                     */
  int32_t green;           /* EPFFT_GREEN_*; with CG1 and DG1 (not Green          *
                            * operators of Eq. 1) the equilibrium test uses eta3 *
                            * in place of eta1 (fixed-point residual)            */
  double mu, lambda;       /* matrix Lame moduli (> 0, lambda + 2 mu / 3 > 0)     */
  double yield_stress;     /* Mises flow stress Y > 0; +inf = elastic matrix      */
  double mu0, lambda0;     /* reference medium C0 of the augmented Lagrangian     */
  double tol_eq;           /* eta1 >= 0                                           */
  double tol_macro;        /* eta2 >= 0                                           */
  int32_t max_iter;        /* >= 1 iterations per increment                       */
  int32_t eq_test;         /* EPFFT_EQ_*; 0 (EPFFT_EQ_OWN) as before              */
} epfft_problem;

/* Prescribed mean strain per increment, n_inc x (E11, E22, E33, E12), host
 * memory.  The lattice starts unstrained; increment k warm-starts from the
 * accepted state of increment k-1 shifted by E_k - E_{k-1}. */
typedef struct {
  int32_t n_inc;
  int32_t reserved;
  const double *E;
} epfft_path;

/* Result of one increment (the accepted iterate). */
typedef struct {
  double sig_mean[4];      /* <sigma> (11, 22, 33, 12)                            */
  double eps_mean[4];      /* <eps>                                               */
  double eta1;             /* (<|div sigma|^2> / <sigma>:<sigma>)^(1/2)           */
  double eta2;             /* |<sigma^{n}> - <sigma^{n-1}>| / |<sigma^{n}>|       */
  double eta3;             /* (<(eps - e):(eps - e)> / E:E)^(1/2), e compatible   */
  int32_t iterations;      /* iterations of this increment                        */
  int32_t n_plastic;       /* matrix pixels with sigma_eq = Y (Sec. 3)            */
  int32_t n_clusters;      /* 4-connected periodic clusters of plastic pixels     */
  int32_t status;          /* 0 converged, 1 max_iter reached, 2 NaN / Inf        */
} epfft_record;

/* Optional field outputs of a solve; NULL members are skipped. */
typedef struct {
  void *eps;               /* L*L*4 reals of the problem's precision: final state */
  uint8_t *plastic;        /* n_inc*L*L: plastic pixels of each accepted state    */
  int32_t *labels;         /* n_inc*L*L: their clusters, label = smallest linear  *
                            * index of the cluster, -1 off the plastic set        */
  int32_t on_device;       /* 1: the pointers are device pointers; 0: host        */
  int32_t reserved;
} epfft_fields;

/* ---------------------------------------------------------------------- */
/* Context                                                                 */
/* ---------------------------------------------------------------------- */

/* Creates a context on opt->device (opt may be NULL: device 0, own stream,
 * cudaMallocAsync).  *out is NULL on error. */
int epfft_create(epfft_ctx **out, const epfft_options *opt);
/* Releases the context and everything it allocated; waits for its stream. */
void epfft_destroy(epfft_ctx *ctx);
/* Static string naming an error code. */
const char *epfft_strerror(int code);
/* 1 if the library was built for lattice side L in `precision`, else 0. */
int epfft_supported(int32_t L, int32_t precision);

/* Accounting of the last solve-type call on a context (epfft_solve,
 * epfft_solve_batch, epfft_iterate, epfft_serve_step). */
typedef struct {
  int64_t loop_steps;       /* steps of the device-side loop (one column and one *
                             * row pass each)                                     */
  int64_t kernel_launches;  /* kernels the call launched on the device           */
  int64_t iterations;       /* augmented-Lagrangian iterations executed, all      *
                             * solves, including the one per increment that only  *
                             * served to evaluate the accepted iterate            */
} epfft_stats;

/* Fills *out for the last solve-type call (zeros before the first). */
int epfft_last_stats(const epfft_ctx *ctx, epfft_stats *out);

/* ---------------------------------------------------------------------- */
/* Solves (Sec. 2: strain-controlled loading by increments)                */
/* ---------------------------------------------------------------------- */

/* Blocking solve of one problem along `path` (Sec. 2: strain-controlled
 * loading by increments, each iterated with the augmented Lagrangian of
 * Sec. 1 and the Green operator of Eq. 3 until the indicators of Sec. 2,
 * "Convergence issues", meet the tolerances).  records: host array of
 * path->n_inc entries (filled).  fields: optional outputs (may be NULL).
 * Returns EPFFT_OK when every increment converged, EPFFT_NOT_CONVERGED when
 * some increment stopped at max_iter (its record has status 1), or an
 * error.  The device state is released before returning. */
int epfft_solve(epfft_ctx *ctx, const epfft_problem *problem, const epfft_path *path,
                epfft_record *records, const epfft_fields *fields);

/* Blocking solve of n independent problems (each as epfft_solve, Sec. 2)
 * advanced together on the device, one augmented-Lagrangian pass of every
 * unfinished problem per step of a single device-side loop (one CUDA graph
 * launch).  Problems may differ in L and precision: those of one (L,
 * precision) form a group whose passes run on a branch of their own in the
 * loop body, all groups concurrently, and the loop goes on while any
 * problem is unfinished.  A group given the on-chip schedule (tiling 3, by
 * epfft_autotune or epfft_set_tiling) runs instead as one kernel launch, one
 * CTA per problem, on a stream forked from the context's stream, while the
 * graph of the other groups runs.  records[i] is a host array of
 * paths[i].n_inc entries; fields may be NULL or an array of n.  The
 * arithmetic of each problem does not depend on the others in the batch. */
int epfft_solve_batch(epfft_ctx *ctx, int32_t n, const epfft_problem *problems,
                      const epfft_path *paths, epfft_record *const *records,
                      const epfft_fields *fields);

/* Mixed-precision solve (Sec. 2 loading; the FP32 path cannot certify
 * tolerances below its rounding floor, eta1 of a few 1e-6 on a 256^2
 * lattice with voids): each increment iterates first in FP32 until eta1 and
 * eta2 fall below max(tol_switch, tolerance) (or max_iter), then continues
 * in FP64 from that state until the problem's tolerances hold (or
 * max_iter), so that the indicators in `records` are FP64 ones.
 * tol_switch = 0 switches automatically at the FP32 floor: the FP32 stage
 * runs in chunks of 2000 iterations, each continuing from the strain of the
 * last (the state is the strain alone), until a chunk improves
 * max(eta1, eta2) by less than a factor 1.5.  problem->precision must be
 * EPFFT_FP64 (the precision of the result and of `fields`); increment k's
 * FP32 stage starts from the accepted FP64 state of increment k-1 shifted by
 * E_k - E_{k-1} and rounded.  records: n_inc FP64-stage records (host);
 * records_fp32 (optional): n_inc records of the FP32 stages (iterations:
 * all of the stage's).  tol_switch < 0: EPFFT_ERR_ARG.  Returns as
 * epfft_solve, from the FP64 stages. */
int epfft_solve_refined(epfft_ctx *ctx, const epfft_problem *problem, const epfft_path *path, double tol_switch,
                        epfft_record *records, epfft_record *records_fp32, const epfft_fields *fields);
/* The same (Sec. 2 loading) for n problems of one lattice side and one
 * increment count, advanced together in both stages (each problem leaves the FP32 stage on
 * its own switch test); records[i], records_fp32[i] (optional array, entries
 * may be NULL): n_inc records each; fields: NULL or n entries. */
int epfft_solve_refined_batch(epfft_ctx *ctx, int32_t n, const epfft_problem *problems, const epfft_path *paths,
                              double tol_switch, epfft_record *const *records, epfft_record *const *records_fp32,
                              const epfft_fields *fields);

/* DG2 (Sec. 2): four complete solves of the problem with the Eq. 3
 * operator at (q1, q2), (-q1, -q2), (-q1, q2) and (q1, -q2) in turn, and the
 * average of the four converged strain fields.  The operator at mirrored
 * momenta (with the tensor sign of the mirror, as in DG1) is exactly the
 * Eq. 3 scheme on the mirrored lattice under the mirrored load, so the
 * members run as one batch of Eq. 3 solves of the lattice and its mirror
 * images (x1, x2 and both; E12 reversed by a single mirror), each tested by
 * its own scheme's indicators, and their fields are mirrored back before
 * averaging.  problem->green must be EPFFT_GREEN_EQ3.
 * records: n_inc entries: per increment the mean of the four members'
 * <sigma> and <eps> (mirrored back), the largest eta1, eta2, eta3 and status,
 * the summed iterations; n_plastic and n_clusters are -1 except in the last
 * record, where they describe the averaged final field.
 * fields (optional): eps = the averaged final strain (L*L*4 reals);
 * plastic = L*L flags of its plastic matrix pixels; labels = L*L clusters of
 * those (4-connected, periodic).  Return codes as epfft_solve. */
int epfft_solve_dg2(epfft_ctx *ctx, const epfft_problem *problem, const epfft_path *path,
                    epfft_record *records, const epfft_fields *fields);

/* Sec. 3: clusters of the void-plastic phase (voids and plastic pixels,
 * 4-neighbours, periodic) where every cluster without a void is connected
 * to its nearest void pixel (periodic Euclidean distance between pixel
 * centres; ties to the smaller linear index), so that each cluster holds a
 * void.  mask_dev: L*L (1 = void); plastic_dev: n_img images of L*L plastic
 * flags (e.g. the per-increment flags of a solve); labels_dev (optional,
 * n_img*L*L): the final clusters, label = smallest linear index, -1 off
 * the phase.  stats (host, n_img x 6): clusters, pixels of the largest,
 * clusters without a plastic pixel (isolated voids), clusters of the voids
 * alone, plastic pixels, void pixels.  Blocking. */
int epfft_void_plastic(epfft_ctx *ctx, int32_t L, int32_t n_img, const uint8_t *mask_dev,
                       const uint8_t *plastic_dev, int32_t *labels_dev, int32_t *stats);

/* The indicators of Sec. 3 per increment from a solve's records and the
 * epfft_void_plastic stats of its increments (host arrays; load: 0
 * equibiaxial, 1 shear).  out: n_inc x 8 doubles: eps0, sigma0 (in-plane
 * means (11 + 22) / 2, or the 12 components in shear), f_p = plastic /
 * matrix pixels, v_max = largest cluster / L^2, i = isolated void clusters /
 * void clusters, n = clusters / void clusters, r = dn/d eps0 and
 * -d2 sigma0 / d eps0^2 (finite differences: second order inside, first
 * order at the ends). */
int epfft_indicators(int32_t n_inc, const epfft_record *records, const int32_t *stats, int32_t L, int32_t load,
                     double *out);

/* Effective in-plane moduli of the lattice of `problem` (mask or f/seed,
 * matrix and reference moduli; its yield stress and green are replaced by
 * an elastic matrix and kept, respectively), used by Eqs. 5-6:
 * *K_eff = <sigma_m> / <eps_m> under equibiaxial strain (E11 = E22 =
 * strain) and *mu_eff = <sigma_12> / (2 <eps_12>) under shear (E12 =
 * strain), sigma_m and eps_m the in-plane means (11 + 22) / 2; the
 * void-free matrix gives 2 (lambda + mu) and mu.  One batch of two
 * one-increment solves.  Return codes as epfft_solve. */
int epfft_effective_moduli(epfft_ctx *ctx, const epfft_problem *problem, double strain, double *K_eff,
                           double *mu_eff);

/* Eqs. 5 (load 0, pressure) and 6 (load 1, shear): the stress-strain curve
 * rebuilt from the indicators `ind` (n_inc x 8, epfft_indicators) and the
 * counts `stats` (n_inc x 6, epfft_void_plastic) with the modulus K~ (Eq. 5)
 * or mu~ (Eq. 6); the fitting number *alpha minimises the squared
 * difference to sigma0, fit (n_inc) receives the curve.  n_inf is n at the
 * last increment; v_p is the void-plastic volume fraction (voids and
 * plastic pixels), v_p^max that of the largest cluster; the integrals are
 * trapezoids from eps0 = 0 with the integrand there equal to its value at
 * the first increment.  Host arithmetic. */
int epfft_empirical_curve(int32_t n_inc, const double *ind, const int32_t *stats, int32_t L, double modulus,
                          int32_t load, double *alpha, double *fit);

/* Equivalent strain of Fig. 1, out(x) = [(2/3) e'_ij e'_ij]^(1/2) with e'
 * the 3D deviator of eps (11, 22, 33, 12; e'_12 counted twice).  Device
 * pointers: eps L*L*4 reals, out L*L reals of `precision`.  Blocking. */
int epfft_eps_eq(epfft_ctx *ctx, int32_t L, int32_t precision, const void *eps_dev, void *out_dev);

/* Displacement field of Sec. 2 from a strain field: per frequency q != 0,
 * with k^2 = k1^2 + k2^2 (the symbols k_j of Eq. 2 squared as complex
 * numbers),
 *   u1(q) = -(i / k^2) { k1 [eps11 - eps22] + 2 k2 eps12 },
 *   u2(q) =  (i / k^2) { k2 [eps11 - eps22] - 2 k1 eps12 },
 * u(0) = 0 (the mode q = 0 is irrelevant).  k^2 vanishes at
 * q = (pi/2, 3pi/2) and (3pi/2, pi/2) when 4 divides L; there the relation
 * eps_ab = (i/2)(k_a u_b + k_b u_a) it inverts is solved with
 * |k|^2 = |k1|^2 + |k2|^2 instead (the same u for a compatible strain).
 * For a compatible strain (one with a periodic displacement, forward
 * differences of Eq. 1) u is that displacement less its mean.  Device
 * pointers: eps L*L*4 reals (11, 22, 33, 12; 33 unused), u L*L*2 reals
 * (u1, u2) of `precision`, both at [x2][x1].  Blocking. */
int epfft_displacement(epfft_ctx *ctx, int32_t L, int32_t precision, const void *eps_dev, void *u_dev);

/* CG2 post-processing (Sec. 2): eps_out(x) = mean of eps_in at x and its
 * four nearest neighbours (periodic), per component.  Device pointers,
 * L*L*4 reals of `precision` each, distinct buffers; blocking on the
 * context stream. */
int epfft_average5(epfft_ctx *ctx, int32_t L, int32_t precision, const void *eps_in_dev, void *eps_out_dev);


/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of independent solves                      */
/* ---------------------------------------------------------------------- */
/* Requests of any lattice side and precision queue in submission order.
 * Each (L, precision) class advances up to slots_per_class solves together
 * in one device-side loop (the epfft_solve_batch machinery); classes run
 * concurrently on their own streams.  epfft_serve_step admits queued
 * requests into free slots while the device state of the running solves
 * stays within hbm_budget_bytes, runs every class with live solves for at
 * most steps_per_launch loop steps, and harvests the solves that finished
 * (cluster labels, records, optionally the final strain) and releases their
 * device state.  A solve's results do not depend on the solves running
 * beside it.  Results stay with the context until epfft_poll returns them. */
typedef struct {
  int64_t hbm_budget_bytes;  /* device bytes the resident solves may hold    */
  int32_t slots_per_class;   /* solves of one class advanced together         */
  int32_t steps_per_launch;  /* loop steps between admissions and harvests    */
} epfft_serve_options;

/* Starts serving on the context (one server per context). */
int epfft_serve_open(epfft_ctx *ctx, const epfft_serve_options *opt);
/* Stops serving; drops queued and running requests and their results. */
int epfft_serve_close(epfft_ctx *ctx);
/* Fields a served solve keeps for its caller (bits of epfft_submit's want) */
#define EPFFT_WANT_EPS 1     /* final strain (returned by epfft_poll)          */
#define EPFFT_WANT_SIG 2     /* final stress sigma(eps), the multiplier         */
#define EPFFT_WANT_PLASTIC 4 /* plastic flags of every accepted increment      */
#define EPFFT_WANT_LABELS 8  /* their periodic cluster labels (Sec. 3)          */

/* Queues one solve (problem and path copied; a device mask is copied to the
 * host now).  *ticket identifies it.  EPFFT_ERR_OOM if its device state
 * alone exceeds the budget.  want: EPFFT_WANT_* bits (0: records only;
 * other bits: EPFFT_ERR_ARG). */
int epfft_submit(epfft_ctx *ctx, const epfft_problem *problem, const epfft_path *path, int32_t want,
                 int64_t *ticket);
/* One admission / device / harvest round (blocking for the device work).
 * n_running, n_queued (optional): solves on the device, still queued. */
int epfft_serve_step(epfft_ctx *ctx, int32_t *n_running, int32_t *n_queued);
/* EPFFT_PENDING while the request runs or waits; then its final code
 * (EPFFT_OK / EPFFT_NOT_CONVERGED / EPFFT_ERR_NUMERIC) with records
 * (host, n_inc entries), the final strain in eps_host (host, L*L*4 reals of
 * the precision, when requested at submission; may be NULL) and the time
 * from submission to harvest in *latency_s (may be NULL).  The ticket is
 * released once it has returned a final code, unless it keeps fields other
 * than the strain (EPFFT_WANT_SIG, _PLASTIC, _LABELS): such a ticket
 * returns its final code on every poll until epfft_release. */
int epfft_poll(epfft_ctx *ctx, int64_t ticket, epfft_record *records, void *eps_host, double *latency_s);
/* Fields of a finished served solve at increment inc (0 <= inc < n_inc),
 * host buffers the caller owns, NULL to skip: eps_host, sig_host (L*L*4
 * reals of the precision; the final accepted state, so only for
 * inc = n_inc - 1), plastic_host (L*L bytes, 1 = matrix pixel on the
 * plastic branch) and labels_host (L*L int32, clusters of Sec. 3 as in
 * epfft_label).  EPFFT_PENDING while the solve runs or waits; EPFFT_ERR_ARG
 * for an unknown ticket, an increment out of range, or a field not asked
 * for at submission. */
int epfft_ticket_fields(epfft_ctx *ctx, int64_t ticket, int32_t inc, void *eps_host, void *sig_host,
                        uint8_t *plastic_host, int32_t *labels_host);
/* Releases a finished ticket and its fields (EPFFT_PENDING, nothing
 * released, while it runs or waits). */
int epfft_release(epfft_ctx *ctx, int64_t ticket);

/* ---------------------------------------------------------------------- */
/* Steps of the iteration, for parity checks and measurement               */
/* ---------------------------------------------------------------------- */

/* Void mask of Sec. 2 (see epfft_problem.seed) into mask_dev (L*L bytes,
 * device).  stream: cudaStream_t or NULL for the legacy default stream.
 * Asynchronous. */
int epfft_mask(int32_t L, double void_fraction, uint64_t seed, uint8_t *mask_dev, void *stream);

/* n_iter augmented-Lagrangian iterations (Sec. 1; Eqs. 2-3 for the
 * compatible strain) of `problem` (mask from the
 * problem) at fixed mean strain E[4], starting from the local strain
 * eps_dev (device, L*L*4 reals of the problem's precision; the multiplier
 * starts at sigma(eps)), which is overwritten with the n_iter-th iterate.
 * out receives the indicators of that iterate (tolerances are ignored).
 * Blocking. */
int epfft_iterate(epfft_ctx *ctx, const epfft_problem *problem, const double E[4],
                  void *eps_dev, int32_t n_iter, epfft_record *out);

/* Compatible strain of a polarization (Eqs. 2-3):
 *   e = E + IDFT( G(q) DFT(p) ),  G(0) = 0,
 * p_dev: 3 planes of L*L reals (p11, p22, p12), e_dev the same for
 * (e11, e22, e12); reals of `precision`; device memory.  Blocking. */
int epfft_project(epfft_ctx *ctx, int32_t L, int32_t precision, double lambda0, double mu0,
                  const double E[4], const void *p_dev, void *e_dev);

/* The same projection as epfft_project for callers that cannot allocate
 * device memory: code running where cudaMalloc is not available or not
 * allowed (inside another framework's memory budget, in a process whose
 * allocator is owned by someone else, or while the caller must not trigger
 * an allocation that could synchronise the device).  The paper has no
 * counterpart; this is a convenience of the library.
 *
 * All working memory is one static device array of the library (1.62 MB:
 * the spectrum, the tables of every side up to 256 in both precisions and a
 * solve record), so lattice sides above 256 are rejected with
 * EPFFT_ERR_SCRATCH_LIMIT.  p_dev / e_dev and the layout are those of
 * epfft_project; the work is queued on `stream` (cudaStream_t of the current
 * device, NULL for the legacy default stream).
 *
 * Set-up: the first call on a device (made with that device current) loads
 * the library's device code onto it, which is when the driver places the
 * array there (it then stays until the process exits); it looks up the
 * array's device address, uploads the tables with a blocking copy and
 * raises the kernels' shared-memory limits.  Make that first call outside
 * any stream capture and outside any region where a driver allocation or a
 * synchronisation is not allowed.  Every later call allocates nothing (no
 * cudaMalloc, cudaFree or allocating library routine), copies nothing from
 * the host and returns without waiting: it only launches kernels on
 * `stream`, the first of which writes the mean strain and the solve record
 * from the call's arguments.
 *
 * Every call on a device uses the same array and leaves the last call's
 * data in it; calls whose work overlaps on the GPU (other streams, other
 * host threads) race on it and must be serialised by the caller. */
int epfft_project_static(int32_t L, int32_t precision, double lambda0, double mu0, const double E[4],
                         const void *p_dev, void *e_dev, void *stream);

/* Nearest-neighbour clusters of the flagged pixels of n_img images
 * (Sec. 3, Hoshen-Kopelman connectivity), periodic when `periodic` != 0.
 * flags_dev: n_img*L*L bytes; labels_dev: n_img*L*L int32 (smallest linear
 * index of the cluster, -1 off the flags); counts (host, n_img, optional):
 * clusters per image.  Blocking. */
int epfft_label(epfft_ctx *ctx, int32_t L, int32_t n_img, const uint8_t *flags_dev,
                int32_t periodic, int32_t *labels_dev, int32_t *counts);

/* Mean device time of the two fused passes of one iteration, measured with
 * CUDA events around n_iter launch pairs of each on the context stream, for
 * a batch of n_batch copies of `problem` (one launch covers the batch),
 * from the uniform state eps = E (iterations never stop early).
 * col_ms: forward column FFT + Green operator + inverse column FFT;
 * row_ms: inverse row FFT + local step + residual partials + forward row FFT.
 * With the on-chip schedule (tiling 3) there are no separate passes: col_ms
 * is 0 and row_ms the time per iteration of one launch running n_iter
 * iterations of the batch.  Blocking. */
int epfft_time_passes(epfft_ctx *ctx, const epfft_problem *problem, int32_t n_batch, const double E[4],
                      int32_t n_iter, float *col_ms, float *row_ms);

/* FP64 arithmetic peak of the context's device, measured: eight 256-thread
 * CTAs per SM, each thread running 8 independent chains of 4096 dependent
 * FP64 FMAs, timed with CUDA events on the context stream (best of five
 * launches after a warm-up).  *tflops = 2 x FMAs / time; *n_sm (optional)
 * the device's SM count; *ms (optional) the best launch time.  The clocks
 * are left as they are.  A measurement aid, with no counterpart in the
 * paper: the denominator of the FP64 passes' roofline.  Blocking. */
int epfft_fp64_peak(epfft_ctx *ctx, double *tflops, int32_t *n_sm, float *ms);

/* ---------------------------------------------------------------------- */
/* Tiling (FFT tile shapes and CTA sizes per lattice side)                 */
/* ---------------------------------------------------------------------- */
/* Up to EPFFT_N_TILINGS tilings are compiled per lattice side and
 * precision: 0 and 1 are two tile shapes of the shared-memory passes (rows
 * per row-pass CTA, tile width of the spectrum layout = columns per
 * column-pass CTA, threads); 2 is the register-staged row and column passes
 * (FP32, sides 256 .. 4096 only), whose spectrum is stored in the row
 * transform's digit-reversed column order; 3 is the on-chip schedule (FP32,
 * sides 16 .. 64 only): one CTA runs a whole solve, every increment and
 * iteration, with the spectrum in shared memory (the fixed-step entry points,
 * projections and serving use tiling 0 instead).  epfft_supported_tiling
 * tells which exist.  epfft_autotune times every compiled one on this device
 * (CUDA events, a batch of n_batch synthetic f = 0.2 lattices) and makes the
 * fastest the context's tiling for (L, precision) and for batches of that
 * class: launches that cover at least 2^21 pixels (L^2 x batch) form one
 * class, smaller ones the other, since small launches favour more and
 * smaller CTAs and large ones fewer and larger.  *chosen receives the
 * choice and ms_per_iteration[EPFFT_N_TILINGS] (optional) the timings (0 for
 * a tiling that is not compiled).  Later solves, batches, projections (class
 * of one solve) and serving classes (class of their slot count) of that size
 * use it.  Blocking. */
#define EPFFT_N_TILINGS 4
int epfft_autotune(epfft_ctx *ctx, int32_t L, int32_t precision, int32_t n_batch, int32_t *chosen,
                   float *ms_per_iteration);
/* 1 if tiling `variant` is compiled for (L, precision), else 0. */
int epfft_supported_tiling(int32_t L, int32_t precision, int32_t variant);
/* Sets the tiling of (L, precision) on the context, for both batch
 * classes; EPFFT_ERR_UNSUPPORTED if it is not compiled for that size. */
int epfft_set_tiling(epfft_ctx *ctx, int32_t L, int32_t precision, int32_t variant);

/* Defect-correction form (EPFFT_FP32_DEFECT): iterations of a solve between
 * two refreshes of its FP64 reference (default 256), for solves set up after
 * the call.  A refresh costs about one FP64 transform pair of the lattice
 * and runs inside the device loop (a conditional node after the row pass),
 * for each solve on its own schedule, so a solve's arithmetic does not
 * depend on the other solves of a batch.  EPFFT_ERR_ARG if steps < 1. */
int epfft_set_defect_refresh(epfft_ctx *ctx, int32_t steps);

#ifdef __cplusplus
}
#endif
#endif /* EPFFT_H */
