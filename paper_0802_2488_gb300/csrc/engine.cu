// Host side of the epfft C ABI: argument checks, device state of a batch of
// solves, the device-driven loop (a CUDA graph whose while node repeats
// one column pass and one row pass until every solve is done), cluster
// labelling and copy-out.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <chrono>
#include <deque>
#include <map>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/epfft.h"
#include "aux_kernels.cuh"
#include "launch.cuh"
#include "post_kernels.cuh"
#include "tables.cuh"

using namespace epfft;

namespace {
struct Server;
}

struct epfft_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;  // work stream
  cudaStream_t cap = nullptr;     // stream used only to capture graph bodies
  std::vector<cudaStream_t> aux;  // fork streams of captures with parallel branches
  cudaStream_t side = nullptr;    // on-chip groups of a call that also runs a graph
  // page-locked copies of the self-check records of the instantiation units
  // and the records' device addresses (serving reads them on its stream)
  CheckRec* h_checks = nullptr;
  void* check_addr[8] = {};
  bool own_stream = false;
  epfft_alloc_fn alloc = nullptr;
  epfft_free_fn freef = nullptr;
  void* user = nullptr;
  // (L, precision) -> device table (layout of tables.cuh), its size in bytes
  // and the offset of k(m) in it (complex units)
  struct Table {
    void* dev;
    size_t bytes;
    int koff;
  };
  std::map<std::pair<int, int>, Table> tables;
  std::map<std::tuple<int, int, int>, bool> prepared;  // (L, precision, tiling variant)
  // tuned tiling per (L, precision, batch class): class 1 when a launch
  // covers at least 2^21 pixels (enough CTAs to fill the GPU), else 0
  std::map<std::tuple<int, int, int>, int> variant;
  epfft_stats last{};
  Server* server = nullptr;
  // defect-correction form: iterations of a solve between refreshes of its
  // reference
  int defect_refresh = 256;
};

namespace {

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return EPFFT_ERR_CUDA; \
  } while (0)

void* dev_alloc(epfft_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (c->alloc) return c->alloc(bytes, c->stream, c->user);
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(epfft_ctx* c, void* p, size_t bytes) {
  if (!p) return;
  if (bytes == 0) bytes = 256;
  if (c->freef) c->freef(p, bytes, c->stream, c->user);
  else cudaFreeAsync(p, c->stream);
}

// RAII list of device blocks of one call.
struct Arena {
  epfft_ctx* c;
  std::vector<std::pair<void*, size_t>> blocks;
  explicit Arena(epfft_ctx* c_) : c(c_) {}
  void* get(size_t bytes) {
    void* p = dev_alloc(c, bytes);
    if (p) blocks.push_back({p, bytes});
    return p;
  }
  ~Arena() {
    cudaStreamSynchronize(c->stream);
    for (auto& b : blocks) dev_free(c, b.first, b.second);
    cudaStreamSynchronize(c->stream);
  }
};

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

bool supported(int L, int prec) {
  PassShape sh;
  if (!is_pow2(L) || L < 4) return false;
  if (prec == EPFFT_FP32) return pass_shape<float>(L, 0, &sh);
  if (prec == EPFFT_FP64) return pass_shape<double>(L, 0, &sh);
  // the defect form: FP32 passes, FP64 refresh
  if (prec == EPFFT_FP32_DEFECT) return pass_shape<float>(L, 0, &sh) && pass_shape<double>(L, 0, &sh);
  return false;
}

// Tile shapes of the loop's passes (the defect form runs the FP32 tilings 0
// and 1).
int shape(int L, int prec, int var, PassShape* sh) {
  bool ok;
  if (var == ONCHIP_VARIANT) ok = prec == EPFFT_FP32 && onchip_supported(L) && pass_shape<float>(L, 0, sh);
  else if (prec == EPFFT_FP32_DEFECT) ok = var < N_DEF_VARIANTS && pass_shape<float>(L, var, sh);
  else ok = prec == EPFFT_FP32 ? pass_shape<float>(L, var, sh) : pass_shape<double>(L, var, sh);
  return ok ? EPFFT_OK : EPFFT_ERR_UNSUPPORTED;
}

// Bytes of one real of the state (strain, stress, fields a caller reads).
size_t real_size(int prec) { return prec == EPFFT_FP32 ? 4 : 8; }
// Bytes of one real of the loop's spectrum and transform tables.
size_t spec_real_size(int prec) { return prec == EPFFT_FP64 ? 8 : 4; }
// Precision of the loop's transform tables.
int table_prec(int prec) { return prec == EPFFT_FP64 ? EPFFT_FP64 : EPFFT_FP32; }

// Device tables of (L, precision) (layout of tables.cuh: twist octant,
// stage twiddles of both tilings' plans, Fourier symbols of Eq. 2
// k(m) = 2 sin(q/2) exp(i q/2)), built once per context in long double and
// rounded once to the working precision.  The device block comes from the
// context's allocator on its stream; the upload is ordered on that stream
// and waited for before the host copy goes away.
int get_tables(epfft_ctx* c, int L, int prec, void** tw, void** ktab) {
  auto key = std::make_pair(L, prec);
  auto it = c->tables.find(key);
  if (it == c->tables.end()) {
    std::vector<float> hf;
    std::vector<double> hd;
    const int koff = prec == EPFFT_FP32 ? host_tables<float>(L, hf) : host_tables<double>(L, hd);
    if (koff < 0) return EPFFT_ERR_ARG;
    const size_t bytes = prec == EPFFT_FP32 ? hf.size() * sizeof(float) : hd.size() * sizeof(double);
    void* d = dev_alloc(c, bytes);
    if (!d) return EPFFT_ERR_OOM;
    const void* src = prec == EPFFT_FP32 ? (const void*)hf.data() : (const void*)hd.data();
    if (cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      cudaGetLastError();
      dev_free(c, d, bytes);
      return EPFFT_ERR_CUDA;
    }
    it = c->tables.emplace(key, epfft_ctx::Table{d, bytes, koff}).first;
  }
  *tw = it->second.dev;
  *ktab = (char*)it->second.dev + (size_t)2 * it->second.koff * real_size(prec);
  return EPFFT_OK;
}

// First recorded self-check failure of any instantiation unit.
cudaError_t read_check_all(CheckRec* out) {
  CheckRec r[8];
  cudaError_t e;
  if ((e = read_check_v<float, 0>(&r[0])) != cudaSuccess) return e;
  if ((e = read_check_v<float, 1>(&r[1])) != cudaSuccess) return e;
  if ((e = read_check_v<double, 0>(&r[2])) != cudaSuccess) return e;
  if ((e = read_check_v<double, 1>(&r[3])) != cudaSuccess) return e;
  if ((e = read_check_v<float, 2>(&r[4])) != cudaSuccess) return e;
  if ((e = read_check_def_v<0>(&r[5])) != cudaSuccess) return e;
  if ((e = read_check_def_v<1>(&r[6])) != cudaSuccess) return e;
  if ((e = read_check_onchip(&r[7])) != cudaSuccess) return e;
  *out = CheckRec{};
  for (auto& x : r)
    if (x.code) {
      *out = x;
      break;
    }
  return cudaSuccess;
}

// Enqueues on stream s the copies of every unit's self-check record into the
// context's page-locked buffer (read them once s is synchronised); the
// buffer and the records' addresses are set up on first use.
cudaError_t enqueue_check_reads(epfft_ctx* c, cudaStream_t s) {
  if (!c->h_checks) {
    cudaError_t e;
    void* a[8] = {};
    if ((e = check_record_v<float, 0>(&a[0])) != cudaSuccess) return e;
    if ((e = check_record_v<float, 1>(&a[1])) != cudaSuccess) return e;
    if ((e = check_record_v<double, 0>(&a[2])) != cudaSuccess) return e;
    if ((e = check_record_v<double, 1>(&a[3])) != cudaSuccess) return e;
    if ((e = check_record_v<float, 2>(&a[4])) != cudaSuccess) return e;
    if ((e = check_record_def_v<0>(&a[5])) != cudaSuccess) return e;
    if ((e = check_record_def_v<1>(&a[6])) != cudaSuccess) return e;
    if ((e = check_record_onchip(&a[7])) != cudaSuccess) return e;
    CheckRec* h = nullptr;
    if ((e = cudaMallocHost((void**)&h, sizeof(CheckRec) * 8)) != cudaSuccess) return e;
    for (int i = 0; i < 8; i++) {
      c->check_addr[i] = a[i];
      h[i] = CheckRec{};
    }
    c->h_checks = h;
  }
  for (int i = 0; i < 8; i++) {
    if (!c->check_addr[i]) continue;
    cudaError_t e = cudaMemcpyAsync(&c->h_checks[i], c->check_addr[i], sizeof(CheckRec), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Raises the shared-memory limits of the kernels of one tiling (once).
int ensure_prepared(epfft_ctx* c, int L, int prec, int var) {
  auto key = std::make_tuple(L, prec, var);
  if (!c->prepared[key]) {
    if (var == ONCHIP_VARIANT) {
      CK(prepare_onchip(L));
    } else if (prec == EPFFT_FP32_DEFECT) {
      // the FP32 column passes and the defect kernels of tiling var
      CK(prepare<float>(L, var));
      CK(prepare_def(L, var));
    } else {
      CK(prec == EPFFT_FP32 ? prepare<float>(L, var) : prepare<double>(L, var));
    }
    c->prepared[key] = true;
  }
  return EPFFT_OK;
}

// Tiling used for (L, precision): the autotuned one, else variant 0.
int batch_class(int L, int nb) { return (int64_t)L * L * nb >= ((int64_t)1 << 21) ? 1 : 0; }

int variant_for(epfft_ctx* c, int L, int prec, int nb);

// The tuned tiling where the two passes run (projections, serving, the
// fixed-step loops): the on-chip schedule maps to tiling 0.
int pass_variant(epfft_ctx* c, int L, int prec, int nb) {
  const int v = variant_for(c, L, prec, nb);
  return v == ONCHIP_VARIANT ? 0 : v;
}

int variant_for(epfft_ctx* c, int L, int prec, int nb) {
  auto it = c->variant.find(std::make_tuple(L, prec, batch_class(L, nb)));
  return it == c->variant.end() ? 0 : it->second;
}

uint64_t void_threshold(double f) {
  if (!(f > 0.0)) return 0;
  if (f >= 1.0) return (uint64_t)1 << 53;
  return (uint64_t)std::floor(f * 9007199254740992.0);
}

int check_problem(const epfft_problem* p) {
  if (!p) return EPFFT_ERR_ARG;
  if (!is_pow2(p->L) || p->L < 4 || p->L > 4096) return EPFFT_ERR_ARG;
  if (p->precision != EPFFT_FP32 && p->precision != EPFFT_FP64 && p->precision != EPFFT_FP32_DEFECT)
    return EPFFT_ERR_ARG;
  if (p->green != EPFFT_GREEN_EQ3 && p->green != EPFFT_GREEN_CG1 && p->green != EPFFT_GREEN_DG1) return EPFFT_ERR_ARG;
  if (!supported(p->L, p->precision)) return EPFFT_ERR_UNSUPPORTED;
  if (!p->mask && !(p->void_fraction >= 0.0 && p->void_fraction <= 1.0)) return EPFFT_ERR_ARG;
  if (!(p->mu > 0.0) || !(p->mu0 > 0.0) || !std::isfinite(p->mu) || !std::isfinite(p->mu0)) return EPFFT_ERR_ARG;
  if (!(p->lambda + 2.0 * p->mu / 3.0 > 0.0) || !(p->lambda0 + 2.0 * p->mu0 / 3.0 > 0.0)) return EPFFT_ERR_ARG;
  if (!(p->lambda0 >= 0.0) || !std::isfinite(p->lambda0) || !std::isfinite(p->lambda)) return EPFFT_ERR_ARG;
  if (!(p->yield_stress > 0.0)) return EPFFT_ERR_ARG;
  if (!(p->tol_eq >= 0.0) || !(p->tol_macro >= 0.0)) return EPFFT_ERR_ARG;
  if (p->max_iter < 1) return EPFFT_ERR_ARG;
  if (p->eq_test != EPFFT_EQ_OWN && p->eq_test != EPFFT_EQ_FIXED_POINT) return EPFFT_ERR_ARG;
  return EPFFT_OK;
}

// Derived material constants of a solve (see MatConst), FP64 and FP32.
void fill_consts(Solve& S) {
  const double K = S.lam + 2.0 * S.mu / 3.0, K0 = S.lam0 + 2.0 * S.mu0 / 3.0;
  const double yl = std::sqrt(2.0 / 3.0) * S.Y;
  const double r = S.mu / (S.mu + S.mu0);
  double* c = S.mcd;
  c[MC_K] = K;
  c[MC_TWO_MU] = 2.0 * S.mu;
  c[MC_LAM0] = S.lam0;
  c[MC_TWO_MU0] = 2.0 * S.mu0;
  c[MC_YLIM] = yl;
  c[MC_YLIM2] = std::isinf(yl) ? yl : yl * yl;
  c[MC_INV_3KK0] = 1.0 / (3.0 * (K + K0));
  c[MC_INV_3K0] = 1.0 / (3.0 * K0);
  c[MC_INV_2MUMU0] = 1.0 / (2.0 * (S.mu + S.mu0));
  c[MC_INV_2MU0] = 1.0 / (2.0 * S.mu0);
  c[MC_TRIAL2] = r * r;
  c[MC_MU0] = S.mu0;
  c[MC_P_MAT] = 3.0 * (K - K0);
  c[MC_P_VOID] = -3.0 * K0;
  c[MC_GSC_EL] = S.mu / (S.mu + S.mu0);
  c[MC_3K] = 3.0 * K;
  c[MC_TSTAR] = yl * (S.mu + S.mu0) / S.mu;
  c[MC_TSTAR2] = std::isinf(yl) ? yl : c[MC_TSTAR] * c[MC_TSTAR];
  c[MC_RY] = yl / (2.0 * S.mu0);
  c[MC_JC] = S.mu / ((S.mu + S.mu0) * 2.0 * S.mu0);
  for (int i = 0; i < N_MC; i++) S.mcf[i] = (float)c[i];
}

// Device state of one batch.
struct Batch {
  int L = 0, prec = 0, nb = 0, var = -1;  // var < 0: the context's tuned tiling
  int general = 0;                        // some solve uses an operator other than Eq. 3
  PassShape sh{};
  void* tw = nullptr;
  void* ktab = nullptr;
  Solve* d_solves = nullptr;
  BatchCtl* d_ctl = nullptr;
  int64_t max_body = 0;  // bound on the loop steps of the batch
  // defect form: FP64 tables and tiling of the refresh, the shadow solves its
  // FP64 column pass reads (spectrum = the FP64 one), refreshes launched
  void* tw64 = nullptr;
  void* ktab64 = nullptr;
  int var64 = 0;
  Solve* d_shadow = nullptr;
  std::vector<Solve> h_shadow;  // serving: host copy of the shadow slots
  int64_t refreshes = 0;  // refreshes launched from the host (fixed-step loops)
  std::vector<Solve> h_solves;
  std::vector<int32_t> n_inc;
};

// The two passes of one loop step of a batch, in its precision.
cudaError_t col_of(Batch& B, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond) {
  if (B.prec == EPFFT_FP64) return launch_col<double>(B.L, B.var, B.nb, s, B.d_solves, B.tw, B.ktab, h, use_cond, B.general);
  return launch_col<float>(B.L, B.var, B.nb, s, B.d_solves, B.tw, B.ktab, h, use_cond, B.general);
}
// hr / use_hr: the condition of the refresh node that follows the row pass
// of a defect batch in a loop body.
cudaError_t row_of(Batch& B, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond,
                   cudaGraphConditionalHandle hr = 0, int use_hr = 0) {
  if (B.prec == EPFFT_FP64) return launch_row<double>(B.L, B.var, B.nb, s, B.d_solves, B.d_ctl, B.tw, h, use_cond);
  if (B.prec == EPFFT_FP32_DEFECT)
    return launch_row_def(B.L, B.var, B.nb, s, B.d_solves, B.d_ctl, B.tw, h, use_cond, hr, use_hr);
  return launch_row<float>(B.L, B.var, B.nb, s, B.d_solves, B.d_ctl, B.tw, h, use_cond);
}

int launch_body(epfft_ctx* c, Batch& B, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond) {
  CK(col_of(B, s, h, use_cond));
  CK(row_of(B, s, h, use_cond));
  (void)c;
  return EPFFT_OK;
}

// Refresh of the defect form's reference (dcpass.cuh) for every solve of
// the batch that waits for it (PH_REF: after a warm start, or ref_every
// iterations after its last refresh; the kernels skip the others): the
// latest iterate becomes the reference; FP64 row transform of its
// polarization, FP64 column pass on the shadow solves, FP64 inverse row
// transform into the reference data, the reference sums.  No-op for other
// precisions.
int refresh_defect(Batch& B, cudaStream_t s) {
  if (B.prec != EPFFT_FP32_DEFECT) return EPFFT_OK;
  CK(launch_ref_forward(B.L, B.var64, B.nb, s, B.d_solves, B.d_shadow, B.tw64));
  CK(launch_col<double>(B.L, B.var64, B.nb, s, B.d_shadow, B.tw64, B.ktab64, 0, 0, B.general));
  CK(launch_ref_inverse(B.L, B.var64, B.nb, s, B.d_solves, B.tw64));
  CK(launch_ref_sums(B.L, B.var64, B.nb, s, B.d_solves));
  return EPFFT_OK;
}

// Bytes of device state one solve holds while it runs.
size_t solve_footprint(int L, int prec, int row_ctas, int n_inc) {
  const size_t LL = (size_t)L * L, rs = real_size(prec);
  auto r = [](size_t b) { return (b + 511) & ~(size_t)511; };
  // the defect form: one FP64 reference state, four FP32 difference fields,
  // the reference data, the FP64 spectrum and the refresh records
  const size_t states = prec == EPFFT_FP32_DEFECT
                            ? r(4 * LL * 8) * 2 + r(4 * LL * 4) * 6 + r(2 * LL * 4) + r(3 * LL * 8) +
                                  r(sizeof(double) * PART_STRIDE * (size_t)L)
                            : r(4 * LL * rs) * 4;
  return states + r(3 * LL * spec_real_size(prec)) +
         r(sizeof(double) * PART_STRIDE * (size_t)row_ctas) + r(LL) + r(LL * (size_t)n_inc) +
         r(sizeof(double) * 4 * (size_t)n_inc) + r(sizeof(Record) * (size_t)n_inc);
}

// Allocates (through `get`) and initialises the device state of one solve on
// stream s: buffers, path, mask, starting strain (eps0: device pointer or
// null for an unstrained lattice).  Fills the host record S.
template <typename Get>
int init_solve(Get&& get, const PassShape& sh, int L, int prec, const epfft_problem& p, const double* path,
               int n_inc, const void* eps0, cudaStream_t s, Solve& S) {
  const size_t LL = (size_t)L * L, rs = real_size(prec);
  std::memset(&S, 0, sizeof(S));
  S.lam = p.lambda;
  S.mu = p.mu;
  S.Y = p.yield_stress;
  S.lam0 = p.lambda0;
  S.mu0 = p.mu0;
  S.tol_eq = p.tol_eq;
  S.tol_macro = p.tol_macro;
  S.max_iter = p.max_iter;
  S.n_inc = n_inc;
  S.green = p.green;
  S.eq_fixed_point = p.eq_test == EPFFT_EQ_FIXED_POINT || p.green == EPFFT_GREEN_CG1 || p.green == EPFFT_GREEN_DG1;
  fill_consts(S);
  const bool dc = prec == EPFFT_FP32_DEFECT;
  // the defect form keeps one FP64 reference state (eps_ref, sigma_ref) and
  // the FP32 differences from it; the others two ping-pong states
  void* eps0d = get(4 * LL * rs);
  void* eps1d = dc ? eps0d : get(4 * LL * rs);
  void* sig0d = get(4 * LL * rs);
  void* sig1d = dc ? sig0d : get(4 * LL * rs);
  void* spec = get(3 * LL * spec_real_size(prec));
  double* part = (double*)get(sizeof(double) * PART_STRIDE * (size_t)sh.row_ctas);
  uint8_t* mask = (uint8_t*)get(LL);
  uint8_t* flags = (uint8_t*)get(LL * (size_t)n_inc);
  double* dpath = (double*)get(sizeof(double) * 4 * (size_t)n_inc);
  Record* rec = (Record*)get(sizeof(Record) * (size_t)n_inc);
  if (!eps0d || !eps1d || !sig0d || !sig1d || !spec || !part || !mask || !flags || !dpath || !rec)
    return EPFFT_ERR_OOM;
  S.eps[0] = eps0d;
  S.eps[1] = eps1d;
  S.sig[0] = sig0d;
  S.sig[1] = sig1d;
  S.spec = spec;
  S.partials = part;
  S.mask = mask;
  S.flags = flags;
  S.path = dpath;
  S.rec = rec;
  S.phase = PH_INIT;
  if (dc) {
    S.eref = eps0d;
    S.sref = sig0d;
    for (int k = 0; k < 2; k++) {
      S.deps[k] = get(4 * LL * 4);
      S.dsig[k] = get(4 * LL * 4);
      if (!S.deps[k] || !S.dsig[k]) return EPFFT_ERR_OOM;
      CK(cudaMemsetAsync(S.deps[k], 0, 4 * LL * 4, s));
      CK(cudaMemsetAsync(S.dsig[k], 0, 4 * LL * 4, s));
    }
    S.base[0] = get(4 * LL * 4);
    S.base[1] = get(4 * LL * 4);
    S.base[2] = get(2 * LL * 4);
    S.spec64 = get(3 * LL * 8);
    // one record per row CTA of the refresh (at most L)
    S.refpart = (double*)get(sizeof(double) * PART_STRIDE * (size_t)L);
    if (!S.base[0] || !S.base[1] || !S.base[2] || !S.spec64 || !S.refpart) return EPFFT_ERR_OOM;
    S.zero_mean = 1;
  }
  CK(cudaMemcpyAsync(dpath, path, sizeof(double) * 4 * (size_t)n_inc, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(rec, 0, sizeof(Record) * (size_t)n_inc, s));
  if (p.mask) {
    CK(cudaMemcpyAsync(mask, p.mask, LL, p.mask_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  } else {
    CK(launch_mask(mask, (int64_t)LL, p.seed, void_threshold(p.void_fraction), s));
  }
  if (eps0) {
    CK(cudaMemcpyAsync(eps0d, eps0, 4 * LL * rs, cudaMemcpyDeviceToDevice, s));
    for (int k = 0; k < 4; k++) S.Eprev[k] = path[k];
  } else {
    CK(cudaMemsetAsync(eps0d, 0, 4 * LL * rs, s));
  }
  return EPFFT_OK;
}

// Builds the device state of n problems.  eps0 (optional, device) gives the
// starting local strain of every solve (then the first increment starts
// from it unshifted); otherwise the lattice starts unstrained.
// onchip: the on-chip schedule may be used (the device-driven solves; the
// fixed-step loops run the two passes).
int setup_batch(epfft_ctx* c, Arena& A, Batch& B, int n, const epfft_problem* probs,
                const epfft_path* paths, const void* const* eps0, bool onchip = true) {
  B.L = probs[0].L;
  B.prec = probs[0].precision;
  B.nb = n;
  for (int i = 0; i < n; i++) B.general |= probs[i].green != EPFFT_GREEN_EQ3;
  if (B.var < 0) B.var = onchip ? variant_for(c, B.L, B.prec, n) : pass_variant(c, B.L, B.prec, n);
  int rc = shape(B.L, B.prec, B.var, &B.sh);
  if (rc) return rc;
  rc = get_tables(c, B.L, table_prec(B.prec), &B.tw, &B.ktab);
  if (!rc) rc = ensure_prepared(c, B.L, B.prec, B.var);
  if (!rc && B.prec == EPFFT_FP32_DEFECT) {
    // the refresh: FP64 tables, FP64 column pass and FP64 row halves of the
    // FP64 tiling tuned for this batch class
    B.var64 = variant_for(c, B.L, EPFFT_FP64, n);
    rc = get_tables(c, B.L, EPFFT_FP64, &B.tw64, &B.ktab64);
    if (!rc) rc = ensure_prepared(c, B.L, EPFFT_FP64, B.var64);
    if (!rc) rc = ensure_prepared(c, B.L, EPFFT_FP32_DEFECT, B.var64);
  }
  if (rc) return rc;
  B.h_solves.resize(n);
  B.n_inc.resize(n);
  int64_t max_body = 0;
  for (int i = 0; i < n; i++) {
    const epfft_problem& p = probs[i];
    B.n_inc[i] = paths[i].n_inc;
    rc = init_solve([&](size_t b) { return A.get(b); }, B.sh, B.L, B.prec, p, paths[i].E, paths[i].n_inc,
                    eps0 ? eps0[i] : nullptr, c->stream, B.h_solves[i]);
    if (rc) return rc;
    B.h_solves[i].ref_every = c->defect_refresh;
    const int64_t need = (int64_t)paths[i].n_inc * ((int64_t)p.max_iter + 2) + 1;
    if (need > max_body) max_body = need;
  }
  B.d_solves = (Solve*)A.get(sizeof(Solve) * (size_t)n);
  B.d_ctl = (BatchCtl*)A.get(sizeof(BatchCtl));
  if (!B.d_solves || !B.d_ctl) return EPFFT_ERR_OOM;
  CK(cudaMemcpyAsync(B.d_solves, B.h_solves.data(), sizeof(Solve) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
  if (B.prec == EPFFT_FP32_DEFECT) {
    // shadow solves of the refresh's FP64 column pass: the FP64 spectrum
    // and 0 at q = 0 (ref_forward mirrors phase, increment and buffer)
    std::vector<Solve> sh = B.h_solves;
    for (auto& z : sh) {
      z.spec = z.spec64;
      z.zero_mean = 1;
    }
    B.d_shadow = (Solve*)A.get(sizeof(Solve) * (size_t)n);
    if (!B.d_shadow) return EPFFT_ERR_OOM;
    CK(cudaMemcpyAsync(B.d_shadow, sh.data(), sizeof(Solve) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
    // the host copy leaves this scope: wait for the upload
    CK(cudaStreamSynchronize(c->stream));
  }
  BatchCtl bc;
  std::memset(&bc, 0, sizeof(bc));
  bc.active = n;
  bc.max_body_iters = max_body + 8;
  bc.dc = B.prec == EPFFT_FP32_DEFECT;
  B.max_body = bc.max_body_iters;
  CK(cudaMemcpyAsync(B.d_ctl, &bc, sizeof(bc), cudaMemcpyHostToDevice, c->stream));
  return EPFFT_OK;
}

// Appends to `body` (after its one leaf node) a conditional IF node on hr
// whose graph runs the refresh of every defect batch of Bs (refresh_defect).
int add_refresh_node(epfft_ctx* c, cudaGraph_t body, cudaGraphConditionalHandle hr, std::vector<Batch*>& Bs) {
  size_t n = 0;
  if (cudaGraphGetNodes(body, nullptr, &n) != cudaSuccess || n == 0) return EPFFT_ERR_CUDA;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(body, nodes.data(), &n) != cudaSuccess) return EPFFT_ERR_CUDA;
  cudaGraphNode_t leaf = nullptr;
  int leaves = 0;
  for (auto nd : nodes) {
    size_t k = 0;
    if (cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &k) != cudaSuccess) return EPFFT_ERR_CUDA;
    if (k == 0) {
      leaf = nd;
      leaves++;
    }
  }
  if (leaves != 1) return EPFFT_ERR_CUDA;
  cudaGraphNodeParams ip = {cudaGraphNodeTypeConditional};
  ip.conditional.handle = hr;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, body, &leaf, nullptr, 1, &ip) != cudaSuccess) return EPFFT_ERR_CUDA;
  cudaGraph_t rb = ip.conditional.phGraph_out[0];
  if (cudaStreamBeginCaptureToGraph(c->cap, rb, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return EPFFT_ERR_CUDA;
  int lrc = EPFFT_OK;
  for (Batch* b : Bs)
    if (!lrc && b->prec == EPFFT_FP32_DEFECT) lrc = refresh_defect(*b, c->cap);
  cudaGraph_t captured = nullptr;
  cudaError_t ec = cudaStreamEndCapture(c->cap, &captured);
  return (lrc != EPFFT_OK || ec != cudaSuccess) ? EPFFT_ERR_CUDA : EPFFT_OK;
}

// One CUDA graph whose while node repeats [column pass, row pass] over the
// batch; the row pass's last CTA sets the loop condition.  The executable
// graph can be launched again (the loop state lives in BatchCtl).
int build_loop_graph(epfft_ctx* c, Batch& B, cudaGraph_t* graph_out, cudaGraphExec_t* exec_out) {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int rc = EPFFT_OK;
  cudaGraphConditionalHandle h;
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cudaGraphNode_t node;
  cudaGraph_t body;
  if (cudaGraphCreate(&graph, 0) != cudaSuccess) return EPFFT_ERR_CUDA;
  do {
    if (cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
      rc = EPFFT_ERR_CUDA;
      break;
    }
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp) != cudaSuccess) {
      rc = EPFFT_ERR_CUDA;
      break;
    }
    body = cp.conditional.phGraph_out[0];
    const bool dc = B.prec == EPFFT_FP32_DEFECT;
    cudaGraphConditionalHandle hr = 0;
    if (dc && cudaGraphConditionalHandleCreate(&hr, graph, 0, 0) != cudaSuccess) {
      rc = EPFFT_ERR_CUDA;
      break;
    }
    if (cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
        cudaSuccess) {
      rc = EPFFT_ERR_CUDA;
      break;
    }
    int lrc = col_of(B, c->cap, h, 1) == cudaSuccess ? EPFFT_OK : EPFFT_ERR_CUDA;
    if (!lrc && row_of(B, c->cap, h, 1, hr, dc ? 1 : 0) != cudaSuccess) lrc = EPFFT_ERR_CUDA;
    cudaGraph_t captured = nullptr;
    cudaError_t ec = cudaStreamEndCapture(c->cap, &captured);
    if (lrc != EPFFT_OK || ec != cudaSuccess) {
      rc = EPFFT_ERR_CUDA;
      break;
    }
    // the defect form: after the row pass, the refresh of the solves that
    // wait for it, when the row pass set its condition
    if (dc) {
      std::vector<Batch*> one{&B};
      if (add_refresh_node(c, body, hr, one) != EPFFT_OK) {
        rc = EPFFT_ERR_CUDA;
        break;
      }
    }
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      rc = EPFFT_ERR_CUDA;
      break;
    }
  } while (0);
  if (rc != EPFFT_OK) {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc;
  }
  *graph_out = graph;
  *exec_out = exec;
  return EPFFT_OK;
}

// Runs the device-side loop of a batch to completion (one graph launch).
int run_graph(epfft_ctx* c, Batch& B) {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int rc = build_loop_graph(c, B, &graph, &exec);
  if (rc) return rc;
  if (cudaGraphLaunch(exec, c->stream) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) {
    rc = EPFFT_ERR_CUDA;
    cudaGetLastError();
  }
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  return rc;
}

// Loop condition of a graph over several batches (sizes, precisions): go on
// while some batch has a solve that is not done and steps left.  One thread.
// With defect batches (use_hr), the condition hr of the refresh node that
// follows: some defect solve waits for its refresh.
__global__ void loop_decide_kernel(BatchCtl* const* ctl, int n, cudaGraphConditionalHandle h,
                                   cudaGraphConditionalHandle hr, int use_hr) {
  bool go = false, wait = false;
  for (int g = 0; g < n; g++) {
    const volatile BatchCtl* b = ctl[g];
    if (b->active > 0 && b->body_iters < b->max_body_iters) go = true;
    wait |= b->dc && b->waiting > 0;
  }
  cudaGraphSetConditional(h, go ? 1u : 0u);
  if (use_hr) {
    cudaGraphSetConditional(hr, wait ? 1u : 0u);
    // the refresh node refreshes every defect batch of the graph
    if (wait)
      for (int g = 0; g < n; g++)
        if (ctl[g]->dc) ctl[g]->refresh_runs += 1;
  }
}

// One CUDA graph that advances several batches of different lattice sides or
// precisions together: a conditional while node whose body runs each
// batch's [column pass, row pass] on a branch of its own (the branches run
// concurrently), then, after they join, a one-thread kernel that sets the
// loop condition from every batch's control block.  The passes of this graph
// leave the condition alone (use_cond = 0).  dctl: device array of the
// batches' control blocks.  The executable graph can be launched again.
int build_mixed_graph(epfft_ctx* c, std::vector<Batch*>& Bs, BatchCtl** dctl, cudaGraph_t* graph_out,
                      cudaGraphExec_t* exec_out) {
  const int G = (int)Bs.size();
  while ((int)c->aux.size() < G) {
    cudaStream_t a;
    CK(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
    c->aux.push_back(a);
  }
  std::vector<cudaEvent_t> ev(G + 1, nullptr);
  for (auto& e : ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool dc = false;
  for (Batch* b : Bs) dc |= b->prec == EPFFT_FP32_DEFECT;
  int rc = EPFFT_OK;
  do {
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) {
      rc = EPFFT_ERR_CUDA;
      break;
    }
    cudaGraphConditionalHandle h, hr = 0;
    if (cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess ||
        (dc && cudaGraphConditionalHandleCreate(&hr, graph, 0, 0) != cudaSuccess)) {
      rc = EPFFT_ERR_CUDA;
      break;
    }
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp) != cudaSuccess) {
      rc = EPFFT_ERR_CUDA;
      break;
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
        cudaSuccess) {
      rc = EPFFT_ERR_CUDA;
      break;
    }
    int lrc = cudaEventRecord(ev[G], c->cap) == cudaSuccess ? EPFFT_OK : EPFFT_ERR_CUDA;
    for (int g = 0; g < G && !lrc; g++) {
      if (cudaStreamWaitEvent(c->aux[g], ev[G], 0) != cudaSuccess) lrc = EPFFT_ERR_CUDA;
      if (!lrc) lrc = launch_body(c, *Bs[g], c->aux[g], h, 0);
      if (!lrc && cudaEventRecord(ev[g], c->aux[g]) != cudaSuccess) lrc = EPFFT_ERR_CUDA;
      if (!lrc && cudaStreamWaitEvent(c->cap, ev[g], 0) != cudaSuccess) lrc = EPFFT_ERR_CUDA;
    }
    if (!lrc) {
      loop_decide_kernel<<<1, 1, 0, c->cap>>>(dctl, G, h, hr, dc ? 1 : 0);
      if (cudaGetLastError() != cudaSuccess) lrc = EPFFT_ERR_CUDA;
    }
    cudaGraph_t captured = nullptr;
    cudaError_t ec = cudaStreamEndCapture(c->cap, &captured);
    if (lrc != EPFFT_OK || ec != cudaSuccess) {
      rc = EPFFT_ERR_CUDA;
      break;
    }
    // defect batches: the refresh node after the loop-condition kernel
    if (dc && add_refresh_node(c, body, hr, Bs) != EPFFT_OK) {
      rc = EPFFT_ERR_CUDA;
      break;
    }
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      rc = EPFFT_ERR_CUDA;
      break;
    }
  } while (0);
  for (auto& e : ev) cudaEventDestroy(e);
  if (rc != EPFFT_OK) {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc;
  }
  *graph_out = graph;
  *exec_out = exec;
  return EPFFT_OK;
}

// Runs several batches to completion in one launch of a mixed graph.
int run_mixed_graph(epfft_ctx* c, Arena& A, std::vector<Batch*>& Bs) {
  const int G = (int)Bs.size();
  BatchCtl** dctl = (BatchCtl**)A.get(sizeof(BatchCtl*) * (size_t)G);
  if (!dctl) return EPFFT_ERR_OOM;
  std::vector<BatchCtl*> h(G);
  for (int g = 0; g < G; g++) h[g] = Bs[g]->d_ctl;
  CK(cudaMemcpyAsync(dctl, h.data(), sizeof(BatchCtl*) * (size_t)G, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int rc = build_mixed_graph(c, Bs, dctl, &graph, &exec);
  if (rc) return rc;
  if (cudaGraphLaunch(exec, c->stream) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) {
    rc = EPFFT_ERR_CUDA;
    cudaGetLastError();
  }
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  return rc;
}

// The same loop for a known number of steps, launched from the host with no
// graph and no synchronisation: steps beyond a solve's DONE phase are
// no-ops (the passes skip DONE solves), so `steps` only has to cover the
// longest solve.  Used where the step count is fixed in advance (a fixed
// number of iterations), so the passes are ordinary stream launches.
int run_host_loop(epfft_ctx* c, Batch& B, int64_t steps) {
  for (int64_t k = 0; k < steps; k++) {
    cudaError_t e = col_of(B, c->stream, 0, 0);
    if (e == cudaSuccess) e = row_of(B, c->stream, 0, 0);
    if (e != cudaSuccess) return EPFFT_ERR_CUDA;
    // the defect form: the refresh of the solves that wait for it
    if (B.prec == EPFFT_FP32_DEFECT) {
      if (refresh_defect(B, c->stream)) return EPFFT_ERR_CUDA;
      B.refreshes += 1;
    }
  }
  CK(cudaStreamSynchronize(c->stream));
  return EPFFT_OK;
}

// Diagnostic loop (EPFFT_SYNC_CHECK=1 in the environment): the same passes
// launched from the host one by one, each followed by a synchronisation
// and an error check that names the pass, phase and step that failed.
int run_checked(epfft_ctx* c, Batch& B) {
  BatchCtl bc;
  std::vector<Solve> hs(B.nb);
  for (int64_t step = 0;; step++) {
    CK(cudaMemcpy(hs.data(), B.d_solves, sizeof(Solve) * B.nb, cudaMemcpyDeviceToHost));
    cudaError_t e = cudaSuccess;
    bool wait = false;
    for (const Solve& z : hs) wait |= z.phase == PH_REF;
    if (wait) {
      if (refresh_defect(B, c->stream)) e = cudaErrorUnknown;
      B.refreshes += 1;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      fprintf(stderr, "epfft check: refresh failed at step %lld (phase %d inc %d iter %d): %s\n",
              (long long)step, hs[0].phase, hs[0].inc, hs[0].iter, cudaGetErrorString(e));
      return EPFFT_ERR_CUDA;
    }
    e = col_of(B, c->stream, 0, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      fprintf(stderr, "epfft check: column pass failed at step %lld (phase %d inc %d iter %d): %s\n",
              (long long)step, hs[0].phase, hs[0].inc, hs[0].iter, cudaGetErrorString(e));
      return EPFFT_ERR_CUDA;
    }
    e = row_of(B, c->stream, 0, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      fprintf(stderr, "epfft check: row pass failed at step %lld (phase %d inc %d iter %d): %s\n",
              (long long)step, hs[0].phase, hs[0].inc, hs[0].iter, cudaGetErrorString(e));
      return EPFFT_ERR_CUDA;
    }
    CheckRec cr;
    CK(read_check_all(&cr));
    if (cr.code)
      fprintf(stderr, "epfft check: step %lld phase %d: self-check %d failed: index %lld bound %lld at %d\n",
              (long long)step, hs[0].phase, cr.code, (long long)cr.index, (long long)cr.bound, cr.where);
    CK(cudaMemcpy(&bc, B.d_ctl, sizeof(bc), cudaMemcpyDeviceToHost));
    if (bc.active == 0) return EPFFT_OK;
    if (bc.body_iters >= bc.max_body_iters) {
      bc.timed_out = 1;
      CK(cudaMemcpy(B.d_ctl, &bc, sizeof(bc), cudaMemcpyHostToDevice));
      return EPFFT_OK;
    }
  }
}

// Labels the per-increment plastic flags of every solve and fills
// n_clusters.  lab_out[i] (may be null): where solve i's labels go (n_inc *
// L * L int32, host or device as `kind` says).  The labels of a solve are
// written to one of two reused device buffers on the work stream and copied
// out on the copy stream `cs` while the next solve is labelled; events keep
// a buffer from being labelled into again before its copy is done.  The
// cluster counts of all solves come back in one copy.
int label_batch(epfft_ctx* c, Arena& A, Batch& B, std::vector<std::vector<Record>>& recs,
                const std::vector<int32_t*>& lab_out, const std::vector<cudaMemcpyKind>& kind, cudaStream_t cs) {
  const size_t LL = (size_t)B.L * B.L;
  int32_t* err = (int32_t*)A.get(sizeof(int32_t));
  if (!err) return EPFFT_ERR_OOM;
  CK(cudaMemsetAsync(err, 0, sizeof(int32_t), c->stream));
  size_t tot = 0, maxn = 0;
  bool out = false;
  for (int i = 0; i < B.nb; i++) {
    tot += (size_t)B.n_inc[i];
    maxn = std::max(maxn, (size_t)B.n_inc[i]);
    out |= lab_out[i] != nullptr;
  }
  int32_t* counts = (int32_t*)A.get(sizeof(int32_t) * tot);
  int32_t* lab[2] = {(int32_t*)A.get(sizeof(int32_t) * LL * maxn), nullptr};
  lab[1] = out ? (int32_t*)A.get(sizeof(int32_t) * LL * maxn) : lab[0];
  if (!counts || !lab[0] || !lab[1]) return EPFFT_ERR_OOM;
  struct Events {
    cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
    ~Events() {
      for (cudaEvent_t x : e)
        if (x) cudaEventDestroy(x);
    }
  } ev;  // [0, 1]: labels of buffer 0 / 1 written; [2, 3]: buffer 0 / 1 copied out
  if (out)
    for (cudaEvent_t& x : ev.e) CK(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
  size_t off = 0;
  for (int i = 0; i < B.nb; i++) {
    const size_t n = (size_t)B.n_inc[i];
    const int h = i & 1;
    // the copy of this buffer's previous solve is done before it is reused
    if (out && i >= 2) CK(cudaStreamWaitEvent(c->stream, ev.e[2 + h], 0));
    CK(launch_label(B.h_solves[i].flags, lab[h], (int64_t)n, B.L, 1, counts + off, err, c->stream));
    if (getenv("EPFFT_SYNC_CHECK")) {
      cudaError_t e = cudaStreamSynchronize(c->stream);
      if (e != cudaSuccess) {
        fprintf(stderr, "epfft check: labelling failed for solve %d: %s\n", i, cudaGetErrorString(e));
        return EPFFT_ERR_CUDA;
      }
    }
    if (out) {
      CK(cudaEventRecord(ev.e[h], c->stream));
      CK(cudaStreamWaitEvent(cs, ev.e[h], 0));
      if (lab_out[i]) CK(cudaMemcpyAsync(lab_out[i], lab[h], sizeof(int32_t) * LL * n, kind[i], cs));
      CK(cudaEventRecord(ev.e[2 + h], cs));
    }
    off += n;
  }
  std::vector<int32_t> hc(tot);
  CK(cudaMemcpyAsync(hc.data(), counts, sizeof(int32_t) * tot, cudaMemcpyDeviceToHost, c->stream));
  int32_t herr = 0;
  CK(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (out) CK(cudaStreamSynchronize(cs));
  off = 0;
  for (int i = 0; i < B.nb; i++) {
    for (size_t k = 0; k < (size_t)B.n_inc[i]; k++) recs[i][k].n_clusters = hc[off + k];
    off += (size_t)B.n_inc[i];
  }
  return herr ? EPFFT_ERR_DEVICE_TIMEOUT : EPFFT_OK;
}

// The final strain and the per-increment plastic flags of solve i, on
// stream s (the labels are copied out by the labelling).
int copy_out(Batch& B, const Solve& S, int i, const epfft_fields* f, cudaStream_t s) {
  if (!f) return EPFFT_OK;
  const size_t LL = (size_t)B.L * B.L, rs = real_size(B.prec);
  const size_t n = (size_t)B.n_inc[i];
  const cudaMemcpyKind k = f->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (f->eps) CK(cudaMemcpyAsync(f->eps, S.eps[S.cur], 4 * LL * rs, k, s));
  if (f->plastic) CK(cudaMemcpyAsync(f->plastic, S.flags, LL * n, k, s));
  return EPFFT_OK;
}

// Solves n problems in one device-driven loop.  Problems of one lattice side
// and precision form a batch; several batches (mixed sides or precisions)
// advance together in one mixed graph (build_mixed_graph).  eps0 / eps_out /
// iter_rec / host_steps (epfft_iterate, the mixed-precision solve) take one
// batch only.
int solve_impl(epfft_ctx* c, int32_t n, const epfft_problem* probs, const epfft_path* paths,
               epfft_record* const* records, const epfft_fields* fields, const void* const* eps0,
               void* const* eps_out, epfft_record* iter_rec, int64_t host_steps = 0) {
  if (!c || n < 1 || !probs || !paths) return EPFFT_ERR_ARG;
  std::vector<std::pair<int, int>> keys;      // (L, precision) of each batch, in order of first appearance
  std::vector<std::vector<int>> members;      // problem indices of each batch
  std::vector<int> where(n), slot(n);         // batch and position within it of each problem
  for (int i = 0; i < n; i++) {
    int rc = check_problem(&probs[i]);
    if (rc) return rc;
    if (paths[i].n_inc < 1 || !paths[i].E) return EPFFT_ERR_ARG;
    for (int k = 0; k < 4 * paths[i].n_inc; k++)
      if (!std::isfinite(paths[i].E[k])) return EPFFT_ERR_ARG;
    if (records && !records[i]) return EPFFT_ERR_ARG;
    const auto key = std::make_pair((int)probs[i].L, (int)probs[i].precision);
    int g = 0;
    while (g < (int)keys.size() && keys[g] != key) g++;
    if (g == (int)keys.size()) {
      keys.push_back(key);
      members.emplace_back();
    }
    where[i] = g;
    slot[i] = (int)members[g].size();
    members[g].push_back(i);
  }
  const int G = (int)keys.size();
  if (G > 1 && (eps0 || eps_out || iter_rec || host_steps > 0)) return EPFFT_ERR_ARG;
  if (cudaSetDevice(c->device) != cudaSuccess) return EPFFT_ERR_CUDA;
  Arena A(c);
  std::vector<Batch> Bs(G);
  std::vector<Batch*> Bp(G);
  for (int g = 0; g < G; g++) {
    std::vector<epfft_problem> pg;
    std::vector<epfft_path> qg;
    for (int i : members[g]) {
      pg.push_back(probs[i]);
      qg.push_back(paths[i]);
    }
    const char* chk0 = getenv("EPFFT_SYNC_CHECK");
    const bool onchip = host_steps == 0 && !(chk0 && chk0[0] == '1');
    int rc = setup_batch(c, A, Bs[g], (int)pg.size(), pg.data(), qg.data(), eps0, onchip);
    if (rc) return rc;
    Bp[g] = &Bs[g];
  }
  const char* chk = getenv("EPFFT_SYNC_CHECK");
  int rc = EPFFT_OK;
  if (chk && chk[0] == '1') {
    for (int g = 0; g < G && !rc; g++) rc = run_checked(c, Bs[g]);
  } else if (host_steps > 0) {
    rc = run_host_loop(c, Bs[0], host_steps);
  } else {
    // on-chip groups: one launch each; the others: one graph over them.
    // When both kinds are present, the on-chip launches go to a side stream
    // forked from the work stream, so that they run while the graph does.
    std::vector<Batch*> stream_groups, onchip_groups;
    for (int g = 0; g < G; g++) (Bs[g].var == ONCHIP_VARIANT ? onchip_groups : stream_groups).push_back(&Bs[g]);
    cudaStream_t ocs = c->stream;
    if (!onchip_groups.empty() && !stream_groups.empty()) {
      cudaEvent_t fork = nullptr;
      if (!c->side && cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess) c->side = nullptr;
      if (c->side && cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess) {
        if (cudaEventRecord(fork, c->stream) == cudaSuccess && cudaStreamWaitEvent(c->side, fork, 0) == cudaSuccess)
          ocs = c->side;
        cudaEventDestroy(fork);
      }
      cudaGetLastError();
    }
    for (Batch* b : onchip_groups)
      if (!rc && launch_onchip(b->L, b->nb, ocs, b->d_solves, b->d_ctl, b->tw, b->ktab) != cudaSuccess)
        rc = EPFFT_ERR_CUDA;
    if (!rc && stream_groups.size() == 1) rc = run_graph(c, *stream_groups[0]);
    else if (!rc && stream_groups.size() > 1) rc = run_mixed_graph(c, A, stream_groups);
    // the side stream's work ends before anything is read back or freed
    if (ocs != c->stream && cudaStreamSynchronize(ocs) != cudaSuccess && !rc) rc = EPFFT_ERR_CUDA;
    if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = EPFFT_ERR_CUDA;
  }
  if (rc) return rc;
  // read back the solve states, the control blocks and the records
  std::vector<BatchCtl> bc(G);
  for (int g = 0; g < G; g++) {
    CK(cudaMemcpyAsync(Bs[g].h_solves.data(), Bs[g].d_solves, sizeof(Solve) * (size_t)Bs[g].nb,
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&bc[g], Bs[g].d_ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  std::vector<std::vector<std::vector<Record>>> recs(G);
  for (int g = 0; g < G; g++) {
    recs[g].resize(Bs[g].nb);
    for (int j = 0; j < Bs[g].nb; j++) {
      recs[g][j].resize(Bs[g].n_inc[j]);
      CK(cudaMemcpyAsync(recs[g][j].data(), Bs[g].h_solves[j].rec, sizeof(Record) * (size_t)Bs[g].n_inc[j],
                         cudaMemcpyDeviceToHost, c->stream));
    }
  }
  CK(cudaStreamSynchronize(c->stream));
  {
    CheckRec cr;
    CK(read_check_all(&cr));
    if (cr.code) {
      fprintf(stderr, "epfft: device self-check %d failed (index %lld, bound %lld, at %d)\n", cr.code,
              (long long)cr.index, (long long)cr.bound, cr.where);
      return EPFFT_ERR_CUDA;
    }
  }
  {
    int64_t its = 0, steps = 0, k = 0;
    int streaming = 0;
    for (int g = 0; g < G; g++) {
      for (int j = 0; j < Bs[g].nb; j++) its += Bs[g].h_solves[j].total_iters;
      if (Bs[g].var == ONCHIP_VARIANT) {
        k += 1;  // one on-chip launch runs the whole batch
        for (int j = 0; j < Bs[g].nb; j++) steps = std::max<int64_t>(steps, Bs[g].h_solves[j].total_iters);
        continue;
      }
      streaming++;
      steps = std::max<int64_t>(steps, bc[g].body_iters);
      // per step a column and a row pass of every batch
      k += 2 * bc[g].body_iters;
    }
    if (streaming > 1) k += steps;  // the loop-condition kernel of the mixed graph
    // the defect form's refreshes: from the host, and the loop body's node
    for (int g = 0; g < G; g++) k += 4 * (Bs[g].refreshes + bc[g].refresh_runs);
    // per solve the mask kernel (when generated) and the four labelling kernels
    for (int i = 0; i < n; i++) k += (probs[i].mask ? 0 : 1) + 4;
    c->last.loop_steps = steps;
    c->last.kernel_launches = k;
    c->last.iterations = its;
  }
  for (int g = 0; g < G; g++)
    if (bc[g].timed_out) return EPFFT_ERR_DEVICE_TIMEOUT;
  // The fields go out on a copy stream while the work stream labels: first
  // the final strains and the plastic flags, then each solve's labels as
  // soon as they are written.  The copy stream's work ends before the call
  // returns (and before the arena's buffers go back), on every path.
  cudaStream_t cs = c->stream;
  if (fields) {
    if (!c->side && cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess) {
      c->side = nullptr;
      cudaGetLastError();
    }
    if (c->side) cs = c->side;
  }
  struct SyncOnExit {
    cudaStream_t s;
    ~SyncOnExit() {
      if (s) cudaStreamSynchronize(s);
    }
  } copies_done{cs != c->stream ? cs : nullptr};
  if (fields)
    for (int i = 0; i < n; i++) {
      Batch& B = Bs[where[i]];
      rc = copy_out(B, B.h_solves[slot[i]], slot[i], &fields[i], cs);
      if (rc) return rc;
    }
  for (int g = 0; g < G; g++) {
    // the caller's label buffers of the batch's solves (labels are copied
    // out by the labelling itself; copy_out does the other fields)
    std::vector<int32_t*> lab_out(Bs[g].nb, nullptr);
    std::vector<cudaMemcpyKind> kind(Bs[g].nb, cudaMemcpyDeviceToHost);
    if (fields)
      for (int j = 0; j < Bs[g].nb; j++) {
        const epfft_fields& f = fields[members[g][j]];
        lab_out[j] = (int32_t*)f.labels;
        kind[j] = f.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
      }
    rc = label_batch(c, A, Bs[g], recs[g], lab_out, kind, cs);
    if (rc) return rc;
  }
  int status = EPFFT_OK;
  for (int i = 0; i < n; i++) {
    Batch& B = Bs[where[i]];
    const int j = slot[i];
    const std::vector<Record>& R = recs[where[i]][j];
    const Solve& S = B.h_solves[j];
    if (S.phase != PH_DONE && S.status == 0) return EPFFT_ERR_DEVICE_TIMEOUT;
    if (records) std::memcpy(records[i], R.data(), sizeof(Record) * (size_t)B.n_inc[j]);
    if (eps_out && eps_out[i])
      CK(cudaMemcpyAsync(eps_out[i], S.eps[S.cur], 4 * (size_t)B.L * B.L * real_size(B.prec),
                         cudaMemcpyDeviceToDevice, c->stream));
    if (iter_rec) std::memcpy(&iter_rec[i], &R[B.n_inc[j] - 1], sizeof(Record));
    for (int k = 0; k < B.n_inc[j]; k++) {
      if (R[k].status == 2) status = EPFFT_ERR_NUMERIC;
      else if (R[k].status == 1 && status == EPFFT_OK) status = EPFFT_NOT_CONVERGED;
    }
  }
  CK(cudaStreamSynchronize(c->stream));
  if (cs != c->stream) CK(cudaStreamSynchronize(cs));
  return status;
}

// Mean CUDA-event time of the column and row passes over n_iter launch
// pairs for n_batch copies of p, tiling `var` (< 0: the tuned one).
int time_passes_impl(epfft_ctx* ctx, epfft_problem p, int n_batch, const double E[4], int n_iter, int var,
                     float* col_ms, float* row_ms) {
  if (cudaSetDevice(ctx->device) != cudaSuccess) return EPFFT_ERR_CUDA;
  p.tol_eq = 0.0;
  p.tol_macro = 0.0;
  p.max_iter = 1 << 30;
  if (var < 0) var = variant_for(ctx, p.L, p.precision, n_batch);
  if (var == ONCHIP_VARIANT) {
    // the on-chip schedule has no separate passes: one launch runs n_iter
    // iterations of the batch (with the warm start and the final flags);
    // row_ms is its time per iteration, col_ms 0
    p.max_iter = n_iter;
    std::vector<epfft_problem> ps(n_batch, p);
    std::vector<epfft_path> paths(n_batch, epfft_path{1, 0, E});
    Arena A(ctx);
    Batch B;
    B.var = var;
    int rc = setup_batch(ctx, A, B, n_batch, ps.data(), paths.data(), nullptr);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, ctx->stream));
    CK(launch_onchip(B.L, B.nb, ctx->stream, B.d_solves, B.d_ctl, B.tw, B.ktab));
    CK(cudaEventRecord(e1, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *col_ms = 0.f;
    *row_ms = ms / (float)n_iter;
    return EPFFT_OK;
  }
  std::vector<epfft_problem> ps(n_batch, p);
  std::vector<epfft_path> paths(n_batch, epfft_path{1, 0, E});
  Arena A(ctx);
  Batch B;
  B.var = var;
  int rc = setup_batch(ctx, A, B, n_batch, ps.data(), paths.data(), nullptr);
  if (rc) return rc;
  const int nb = n_batch;
  // first row pass: warm start (eps = E, spectrum of its polarization); the
  // defect form then refreshes its reference
  CK(row_of(B, ctx->stream, 0, 0));
  if (refresh_defect(B, ctx->stream)) return EPFFT_ERR_CUDA;
  std::vector<cudaEvent_t> ev(3 * (size_t)n_iter);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  for (int it = 0; it < n_iter; it++) {
    CK(cudaEventRecord(ev[3 * it], ctx->stream));
    CK(col_of(B, ctx->stream, 0, 0));
    CK(cudaEventRecord(ev[3 * it + 1], ctx->stream));
    CK(row_of(B, ctx->stream, 0, 0));
    CK(cudaEventRecord(ev[3 * it + 2], ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  double tc = 0, tr = 0;
  for (int it = 0; it < n_iter; it++) {
    float a = 0, b = 0;
    CK(cudaEventElapsedTime(&a, ev[3 * it], ev[3 * it + 1]));
    CK(cudaEventElapsedTime(&b, ev[3 * it + 1], ev[3 * it + 2]));
    tc += a;
    tr += b;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  *col_ms = (float)(tc / n_iter);
  *row_ms = (float)(tr / n_iter);
  return EPFFT_OK;
}

// ---------------------------------------------------------------------------
// Serving: continuous batching of solves of any size
// ---------------------------------------------------------------------------
// Requests queue in submission order.  Each (L, precision) class owns a slot
// table on the device (capacity fixed when the class is first used), its
// own stream and an executable loop graph over the whole table.  A step
// admits queued requests into free slots while the HBM budget allows, runs
// every class with live slots for a bounded number of loop steps (the
// classes run concurrently on their streams), then harvests the solves that
// finished: their clusters are labelled, their records (and optionally the
// final strain) copied to the host, and their device state released.  Empty
// and finished slots are DONE, so the kernels skip them; a solve's
// arithmetic does not depend on which slot it occupies or on its neighbours.

struct ServeSlot {
  bool used = false;
  int64_t ticket = 0;
  size_t bytes = 0;
  std::vector<std::pair<void*, size_t>> blocks;
};

struct ServeClass {
  int L = 0, prec = 0, cap = 0;
  Batch B;  // L, prec, nb = cap, shape, tables, device slot table and control
  std::vector<ServeSlot> slots;
};

struct Ticket {
  int state = 0;  // 0 queued, 1 running, 2 finished
  epfft_problem prob{};
  std::vector<double> path;
  std::vector<uint8_t> mask;  // caller mask copied at submission (empty: generated)
  int32_t want = 0;                  // EPFFT_WANT_* bits given at submission
  std::vector<Record> rec;
  std::vector<unsigned char> eps;    // final strain (EPFFT_WANT_EPS)
  std::vector<unsigned char> sig;    // final stress (EPFFT_WANT_SIG)
  std::vector<uint8_t> flags;        // n_inc * L * L plastic flags (EPFFT_WANT_PLASTIC)
  std::vector<int32_t> labels;       // n_inc * L * L cluster labels (EPFFT_WANT_LABELS)
  int status = 0;
  size_t bytes = 0;
  double t_submit = 0, t_done = 0;
};

struct Server {
  size_t budget = 0, used = 0;
  int steps = 64;
  int cap = 16;
  int64_t next = 1;
  std::deque<int64_t> queue;
  std::map<int64_t, Ticket> tickets;
  // (L, 2 * precision + general) -> class
  std::map<std::pair<int, int>, ServeClass*> classes;
  // one mixed graph over every class (build_mixed_graph), rebuilt when a
  // class is added; dctl: device array of the classes' control blocks
  std::vector<ServeClass*> order;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  BatchCtl** dctl = nullptr;
  size_t dctl_bytes = 0;
  bool dirty = true;
};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

void free_class(epfft_ctx* c, ServeClass* k) {
  cudaStreamSynchronize(c->stream);
  for (auto& sl : k->slots)
    for (auto& b : sl.blocks) dev_free(c, b.first, b.second);
  if (k->B.d_solves) dev_free(c, k->B.d_solves, sizeof(Solve) * (size_t)k->cap);
  if (k->B.d_ctl) dev_free(c, k->B.d_ctl, sizeof(BatchCtl));
  if (k->B.d_shadow) dev_free(c, k->B.d_shadow, sizeof(Solve) * (size_t)k->cap);
  cudaStreamSynchronize(c->stream);
  delete k;
}

void free_mixed(epfft_ctx* c, Server& S) {
  cudaStreamSynchronize(c->stream);
  if (S.exec) cudaGraphExecDestroy(S.exec);
  if (S.graph) cudaGraphDestroy(S.graph);
  if (S.dctl) dev_free(c, S.dctl, S.dctl_bytes);
  S.exec = nullptr;
  S.graph = nullptr;
  S.dctl = nullptr;
  S.dctl_bytes = 0;
  cudaStreamSynchronize(c->stream);
}

// (Re)builds the mixed graph over every class of the server.
int build_serve_graph(epfft_ctx* c, Server& S) {
  free_mixed(c, S);
  S.order.clear();
  std::vector<Batch*> Bp;
  std::vector<BatchCtl*> h;
  for (auto& kv : S.classes) {
    S.order.push_back(kv.second);
    Bp.push_back(&kv.second->B);
    h.push_back(kv.second->B.d_ctl);
  }
  S.dctl_bytes = sizeof(BatchCtl*) * h.size();
  S.dctl = (BatchCtl**)dev_alloc(c, S.dctl_bytes);
  if (!S.dctl) return EPFFT_ERR_OOM;
  CK(cudaMemcpyAsync(S.dctl, h.data(), S.dctl_bytes, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  int rc = build_mixed_graph(c, Bp, S.dctl, &S.graph, &S.exec);
  if (!rc) S.dirty = false;
  return rc;
}

int get_class(epfft_ctx* c, Server& S, int L, int prec, int general, ServeClass** out) {
  auto key = std::make_pair(L, 2 * prec + general);
  auto it = S.classes.find(key);
  if (it != S.classes.end()) {
    *out = it->second;
    return EPFFT_OK;
  }
  ServeClass* k = new ServeClass();
  k->L = L;
  k->prec = prec;
  k->cap = S.cap;
  k->slots.resize(S.cap);
  Batch& B = k->B;
  B.L = L;
  B.prec = prec;
  B.nb = S.cap;
  B.general = general;
  B.var = pass_variant(c, L, prec, S.cap);
  int rc = shape(L, prec, B.var, &B.sh);
  if (!rc) rc = get_tables(c, L, table_prec(prec), &B.tw, &B.ktab);
  if (!rc) rc = ensure_prepared(c, L, prec, B.var);
  if (!rc && prec == EPFFT_FP32_DEFECT) {
    // the refresh between serving steps (FP64 tables, column pass, row halves)
    B.var64 = variant_for(c, L, EPFFT_FP64, S.cap);
    rc = get_tables(c, L, EPFFT_FP64, &B.tw64, &B.ktab64);
    if (!rc) rc = ensure_prepared(c, L, EPFFT_FP64, B.var64);
    if (!rc) rc = ensure_prepared(c, L, EPFFT_FP32_DEFECT, B.var64);
  }
  if (!rc) {
    B.d_solves = (Solve*)dev_alloc(c, sizeof(Solve) * (size_t)S.cap);
    B.d_ctl = (BatchCtl*)dev_alloc(c, sizeof(BatchCtl));
    if (!B.d_solves || !B.d_ctl) rc = EPFFT_ERR_OOM;
    if (!rc && prec == EPFFT_FP32_DEFECT) {
      B.d_shadow = (Solve*)dev_alloc(c, sizeof(Solve) * (size_t)S.cap);
      if (!B.d_shadow) rc = EPFFT_ERR_OOM;
    }
  }
  if (!rc) {
    B.h_solves.assign(S.cap, Solve{});
    for (auto& x : B.h_solves) {
      std::memset(&x, 0, sizeof(x));
      x.phase = PH_DONE;
    }
    B.n_inc.assign(S.cap, 0);
    if (cudaMemcpyAsync(B.d_solves, B.h_solves.data(), sizeof(Solve) * (size_t)S.cap, cudaMemcpyHostToDevice,
                        c->stream) != cudaSuccess)
      rc = EPFFT_ERR_CUDA;
    if (!rc && B.d_shadow) {
      B.h_shadow = B.h_solves;
      if (cudaMemcpyAsync(B.d_shadow, B.h_shadow.data(), sizeof(Solve) * (size_t)S.cap, cudaMemcpyHostToDevice,
                          c->stream) != cudaSuccess)
        rc = EPFFT_ERR_CUDA;
    }
    if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = EPFFT_ERR_CUDA;
  }
  if (rc) {
    free_class(c, k);
    return rc;
  }
  S.classes[key] = k;
  S.dirty = true;  // the mixed graph covers every class
  *out = k;
  return EPFFT_OK;
}

// Admits queued requests in submission order into free slots while the
// budget allows; a request that does not fit yet stays queued (later ones
// may still be admitted).
int serve_admit(epfft_ctx* c, Server& S) {
  for (auto qi = S.queue.begin(); qi != S.queue.end();) {
    Ticket& t = S.tickets[*qi];
    if (S.used + t.bytes > S.budget) {
      ++qi;
      continue;
    }
    ServeClass* k = nullptr;
    int rc = get_class(c, S, t.prob.L, t.prob.precision, t.prob.green != EPFFT_GREEN_EQ3, &k);
    if (rc) return rc;
    int slot = -1;
    for (int i = 0; i < k->cap; i++)
      if (!k->slots[i].used) {
        slot = i;
        break;
      }
    if (slot < 0) {
      ++qi;
      continue;
    }
    ServeSlot& sl = k->slots[slot];
    sl.blocks.clear();
    epfft_problem p = t.prob;
    p.mask = t.mask.empty() ? nullptr : t.mask.data();
    p.mask_on_device = 0;
    if (!p.mask) c->last.kernel_launches += 1;  // the mask kernel
    Solve hs;
    rc = init_solve(
        [&](size_t b) {
          void* q = dev_alloc(c, b);
          if (q) sl.blocks.push_back({q, b});
          return q;
        },
        k->B.sh, k->L, k->prec, p, t.path.data(), (int)(t.path.size() / 4), nullptr, c->stream, hs);
    if (rc) {
      for (auto& b : sl.blocks) dev_free(c, b.first, b.second);
      sl.blocks.clear();
      return rc;
    }
    hs.ref_every = c->defect_refresh;
    k->B.h_solves[slot] = hs;
    k->B.n_inc[slot] = (int)(t.path.size() / 4);
    CK(cudaMemcpyAsync(k->B.d_solves + slot, &k->B.h_solves[slot], sizeof(Solve), cudaMemcpyHostToDevice,
                       c->stream));
    if (k->B.d_shadow) {
      // the slot's shadow for the refresh's FP64 column pass
      Solve z = hs;
      z.spec = hs.spec64;
      z.zero_mean = 1;
      k->B.h_shadow[slot] = z;
      CK(cudaMemcpyAsync(k->B.d_shadow + slot, &k->B.h_shadow[slot], sizeof(Solve), cudaMemcpyHostToDevice,
                         c->stream));
    }
    sl.used = true;
    sl.ticket = *qi;
    sl.bytes = t.bytes;
    S.used += t.bytes;
    t.state = 1;
    qi = S.queue.erase(qi);
  }
  return EPFFT_OK;
}

// Harvests the finished solves of a class (after its stream is idle).
int serve_harvest(epfft_ctx* c, Server& S, ServeClass* k) {
  Batch& B = k->B;
  std::vector<Solve> hs(k->cap);
  CK(cudaMemcpyAsync(hs.data(), B.d_solves, sizeof(Solve) * (size_t)k->cap, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const size_t LL = (size_t)k->L * k->L, rs = real_size(k->prec);
  for (int i = 0; i < k->cap; i++) {
    ServeSlot& sl = k->slots[i];
    if (!sl.used || hs[i].phase != PH_DONE) continue;
    Ticket& t = S.tickets[sl.ticket];
    const int n = B.n_inc[i];
    t.rec.resize(n);
    CK(cudaMemcpyAsync(t.rec.data(), hs[i].rec, sizeof(Record) * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    if (t.want & EPFFT_WANT_EPS) {
      t.eps.resize(4 * LL * rs);
      CK(cudaMemcpyAsync(t.eps.data(), hs[i].eps[hs[i].cur], 4 * LL * rs, cudaMemcpyDeviceToHost, c->stream));
    }
    if (t.want & EPFFT_WANT_SIG) {  // sigma of the accepted iterate (the resident multiplier)
      t.sig.resize(4 * LL * rs);
      CK(cudaMemcpyAsync(t.sig.data(), hs[i].sig[hs[i].cur], 4 * LL * rs, cudaMemcpyDeviceToHost, c->stream));
    }
    if (t.want & EPFFT_WANT_PLASTIC) {
      t.flags.resize(LL * (size_t)n);
      CK(cudaMemcpyAsync(t.flags.data(), hs[i].flags, LL * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    }
    // clusters of every accepted increment
    int32_t* lab = (int32_t*)dev_alloc(c, sizeof(int32_t) * LL * (size_t)n);
    int32_t* cnt = (int32_t*)dev_alloc(c, sizeof(int32_t) * ((size_t)n + 1));
    if (!lab || !cnt) return EPFFT_ERR_OOM;
    CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ((size_t)n + 1), c->stream));
    CK(launch_label(hs[i].flags, lab, n, k->L, 1, cnt, cnt + n, c->stream));
    std::vector<int32_t> hc(n + 1);
    CK(cudaMemcpyAsync(hc.data(), cnt, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToHost, c->stream));
    if (t.want & EPFFT_WANT_LABELS) {
      t.labels.resize(LL * (size_t)n);
      CK(cudaMemcpyAsync(t.labels.data(), lab, sizeof(int32_t) * LL * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    dev_free(c, lab, sizeof(int32_t) * LL * (size_t)n);
    dev_free(c, cnt, sizeof(int32_t) * ((size_t)n + 1));
    int st = EPFFT_OK;
    for (int q = 0; q < n; q++) {
      t.rec[q].n_clusters = hc[q];
      if (t.rec[q].status == 2) st = EPFFT_ERR_NUMERIC;
      else if (t.rec[q].status == 1 && st == EPFFT_OK) st = EPFFT_NOT_CONVERGED;
    }
    if (hs[i].status == 2) st = EPFFT_ERR_NUMERIC;
    t.status = st;
    t.state = 2;
    t.t_done = now_s();
    for (auto& b : sl.blocks) dev_free(c, b.first, b.second);
    CK(cudaStreamSynchronize(c->stream));
    sl.blocks.clear();
    sl.used = false;
    S.used -= sl.bytes;
    sl.bytes = 0;
    // the slot is empty again (DONE state, zero pointers)
    std::memset(&B.h_solves[i], 0, sizeof(Solve));
    B.h_solves[i].phase = PH_DONE;
    CK(cudaMemcpyAsync(B.d_solves + i, &B.h_solves[i], sizeof(Solve), cudaMemcpyHostToDevice, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return EPFFT_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int epfft_create(epfft_ctx** out, const epfft_options* opt) {
  if (!out) return EPFFT_ERR_ARG;
  *out = nullptr;
  static_assert(sizeof(epfft_record) == sizeof(Record), "record layout");
  static_assert(EPFFT_N_TILINGS == N_VARIANTS, "tilings of the ABI");
  epfft_ctx* c = new epfft_ctx();
  if (opt) {
    c->device = opt->device;
    c->alloc = opt->alloc;
    c->freef = opt->free;
    c->user = opt->alloc_user;
    if ((c->alloc == nullptr) != (c->freef == nullptr)) {
      delete c;
      return EPFFT_ERR_ARG;
    }
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || c->device < 0 || c->device >= ndev) {
    cudaGetLastError();
    delete c;
    return EPFFT_ERR_CUDA;
  }
  if (cudaSetDevice(c->device) != cudaSuccess) {
    delete c;
    return EPFFT_ERR_CUDA;
  }
  if (opt && opt->stream) {
    c->stream = (cudaStream_t)opt->stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return EPFFT_ERR_CUDA;
    }
    c->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return EPFFT_ERR_CUDA;
  }
  *out = c;
  return EPFFT_OK;
}

void epfft_destroy(epfft_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->server) epfft_serve_close(c);
  cudaStreamSynchronize(c->stream);
  for (auto& t : c->tables) dev_free(c, t.second.dev, t.second.bytes);
  cudaStreamSynchronize(c->stream);
  cudaStreamDestroy(c->cap);
  for (cudaStream_t a : c->aux) cudaStreamDestroy(a);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->h_checks) cudaFreeHost(c->h_checks);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* epfft_strerror(int code) {
  switch (code) {
    case EPFFT_OK: return "ok";
    case EPFFT_PENDING: return "pending";
    case EPFFT_ERR_ARG: return "invalid argument";
    case EPFFT_ERR_OOM: return "device allocation failed";
    case EPFFT_ERR_NUMERIC: return "non-finite residual or mean stress";
    case EPFFT_NOT_CONVERGED: return "an increment reached max_iter before the tolerances";
    case EPFFT_ERR_DEVICE_TIMEOUT: return "device loop exceeded its bound";
    case EPFFT_ERR_CUDA: return "CUDA runtime error";
    case EPFFT_ERR_UNSUPPORTED: return "lattice size / precision not built";
    case EPFFT_ERR_SCRATCH_LIMIT: return "lattice side above 256: larger than the static scratch of epfft_project_static";
    default: return "unknown error";
  }
}

int epfft_supported(int32_t L, int32_t precision) { return supported(L, precision) ? 1 : 0; }

int epfft_last_stats(const epfft_ctx* ctx, epfft_stats* out) {
  if (!ctx || !out) return EPFFT_ERR_ARG;
  *out = ctx->last;
  return EPFFT_OK;
}

int epfft_solve(epfft_ctx* ctx, const epfft_problem* problem, const epfft_path* path, epfft_record* records,
                const epfft_fields* fields) {
  if (!problem || !path || !records) return EPFFT_ERR_ARG;
  epfft_record* const recs[1] = {records};
  return solve_impl(ctx, 1, problem, path, recs, fields, nullptr, nullptr, nullptr);
}

int epfft_solve_batch(epfft_ctx* ctx, int32_t n, const epfft_problem* problems, const epfft_path* paths,
                      epfft_record* const* records, const epfft_fields* fields) {
  if (!records) return EPFFT_ERR_ARG;
  return solve_impl(ctx, n, problems, paths, records, fields, nullptr, nullptr, nullptr);
}

int epfft_solve_dg2(epfft_ctx* ctx, const epfft_problem* problem, const epfft_path* path, epfft_record* records,
                    const epfft_fields* fields) {
  if (!ctx || !problem || !path || !records) return EPFFT_ERR_ARG;
  int rc = check_problem(problem);
  if (rc) return rc;
  if (problem->green != EPFFT_GREEN_EQ3) return EPFFT_ERR_ARG;
  if (path->n_inc < 1 || !path->E) return EPFFT_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return EPFFT_ERR_CUDA;
  const int L = problem->L, prec = problem->precision, n_inc = path->n_inc;
  const size_t LL = (size_t)L * L, rs = real_size(prec);
  Arena A(ctx);
  // the lattice and its three mirror images (members: none, x1 and x2, x1, x2)
  static const int kAxes[4] = {0, 3, 1, 2};
  uint8_t* masks = (uint8_t*)A.get(4 * LL);
  void* eps = A.get(5 * 4 * LL * rs);  // four members' final fields, then their average
  uint8_t* flags = (uint8_t*)A.get(LL);
  int32_t* lab = (int32_t*)A.get(sizeof(int32_t) * LL);
  int32_t* dcount = (int32_t*)A.get(2 * sizeof(int32_t));
  if (!masks || !eps || !flags || !lab || !dcount) return EPFFT_ERR_OOM;
  if (problem->mask) {
    CK(cudaMemcpyAsync(masks, problem->mask, LL,
                       problem->mask_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  } else {
    CK(launch_mask(masks, (int64_t)LL, problem->seed, void_threshold(problem->void_fraction), ctx->stream));
  }
  for (int m = 1; m < 4; m++) CK(launch_mirror_mask(masks, masks + m * LL, L, kAxes[m], ctx->stream));
  epfft_problem probs[4];
  epfft_path paths[4];
  std::vector<double> E[4];
  epfft_record* recp[4];
  std::vector<epfft_record> recs[4];
  void* outs[4];
  for (int m = 0; m < 4; m++) {
    probs[m] = *problem;
    probs[m].mask = masks + m * LL;
    probs[m].mask_on_device = 1;
    E[m].assign(path->E, path->E + 4 * (size_t)n_inc);
    if (kAxes[m] == 1 || kAxes[m] == 2)  // a single mirror reverses E12
      for (int k = 0; k < n_inc; k++) E[m][4 * k + 3] = -E[m][4 * k + 3];
    paths[m] = epfft_path{n_inc, 0, E[m].data()};
    recs[m].resize(n_inc);
    recp[m] = recs[m].data();
    outs[m] = (char*)eps + m * 4 * LL * rs;
  }
  const int status = solve_impl(ctx, 4, probs, paths, recp, nullptr, nullptr, outs, nullptr);
  if (status != EPFFT_OK && status != EPFFT_NOT_CONVERGED) return status;
  void* avg = (char*)eps + 4 * 4 * LL * rs;
  Solve S;
  std::memset(&S, 0, sizeof(S));
  S.lam = problem->lambda;
  S.mu = problem->mu;
  S.Y = problem->yield_stress;
  S.lam0 = problem->lambda0;
  S.mu0 = problem->mu0;
  fill_consts(S);
  if (prec == EPFFT_FP32) {
    CK(launch_dg2_average<float>((const float*)outs[0], (const float*)outs[1], (const float*)outs[2],
                                 (const float*)outs[3], (float*)avg, L, ctx->stream));
    CK(launch_plastic_flags<float>((const float*)avg, masks, flags, L, S.mcf[MC_TWO_MU], S.mcf[MC_YLIM2],
                                   ctx->stream));
  } else {
    CK(launch_dg2_average<double>((const double*)outs[0], (const double*)outs[1], (const double*)outs[2],
                                  (const double*)outs[3], (double*)avg, L, ctx->stream));
    CK(launch_plastic_flags<double>((const double*)avg, masks, flags, L, S.mcd[MC_TWO_MU], S.mcd[MC_YLIM2],
                                    ctx->stream));
  }
  CK(cudaMemsetAsync(dcount, 0, 2 * sizeof(int32_t), ctx->stream));
  CK(launch_label(flags, lab, 1, L, 1, dcount, dcount + 1, ctx->stream));
  int32_t hc[2] = {0, 0};
  CK(cudaMemcpyAsync(hc, dcount, sizeof(hc), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (hc[1]) return EPFFT_ERR_DEVICE_TIMEOUT;
  // per increment: macro values of the four (mirrored back) averaged, the
  // largest indicators and status, the summed iterations; the plastic set
  // and clusters are those of the averaged final field (last record only)
  for (int k = 0; k < n_inc; k++) {
    epfft_record r = recs[0][k];
    for (int c = 0; c < 4; c++) {
      double s = 0.0, e = 0.0;
      for (int m = 0; m < 4; m++) {
        const double sg = (c == 3 && (kAxes[m] == 1 || kAxes[m] == 2)) ? -1.0 : 1.0;
        s += sg * recs[m][k].sig_mean[c];
        e += sg * recs[m][k].eps_mean[c];
      }
      r.sig_mean[c] = 0.25 * s;
      r.eps_mean[c] = 0.25 * e;
    }
    r.iterations = 0;
    for (int m = 0; m < 4; m++) {
      r.eta1 = std::max(r.eta1, recs[m][k].eta1);
      r.eta2 = std::max(r.eta2, recs[m][k].eta2);
      r.eta3 = std::max(r.eta3, recs[m][k].eta3);
      r.status = std::max(r.status, recs[m][k].status);
      r.iterations += recs[m][k].iterations;
    }
    r.n_plastic = -1;
    r.n_clusters = -1;
    records[k] = r;
  }
  if (fields) {
    const cudaMemcpyKind kd = fields->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (fields->eps) CK(cudaMemcpyAsync(fields->eps, avg, 4 * LL * rs, kd, ctx->stream));
    if (fields->plastic) CK(cudaMemcpyAsync(fields->plastic, flags, LL, kd, ctx->stream));
    if (fields->labels) CK(cudaMemcpyAsync(fields->labels, lab, sizeof(int32_t) * LL, kd, ctx->stream));
  }
  std::vector<uint8_t> hf(LL);
  CK(cudaMemcpyAsync(hf.data(), flags, LL, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  int32_t npl = 0;
  for (size_t i = 0; i < LL; i++) npl += hf[i];
  records[n_inc - 1].n_plastic = npl;
  records[n_inc - 1].n_clusters = hc[0];
  ctx->last.kernel_launches += 3 + (problem->mask ? 0 : 1) + 2 + 4;
  return status;
}

int epfft_void_plastic(epfft_ctx* ctx, int32_t L, int32_t n_img, const uint8_t* mask_dev, const uint8_t* plastic_dev,
                       int32_t* labels_dev, int32_t* stats) {
  if (!ctx || !is_pow2(L) || L < 2 || L > 4096 || n_img < 1 || !mask_dev || !plastic_dev || !stats)
    return EPFFT_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return EPFFT_ERR_CUDA;
  const size_t LL = (size_t)L * L;
  Arena A(ctx);
  uint8_t* vp = (uint8_t*)A.get(LL);
  int32_t* lab = (int32_t*)A.get(sizeof(int32_t) * LL);
  int32_t* out = labels_dev ? nullptr : (int32_t*)A.get(sizeof(int32_t) * LL);
  void* scratch = A.get(22 * LL);
  int32_t* dcnt = (int32_t*)A.get(8 * sizeof(int32_t));
  if (!vp || !lab || (!labels_dev && !out) || !scratch || !dcnt) return EPFFT_ERR_OOM;
  // the voids alone: their clusters and pixels (once)
  CK(cudaMemsetAsync(dcnt, 0, 8 * sizeof(int32_t), ctx->stream));
  CK(launch_label(mask_dev, lab, 1, L, 1, dcnt + 3, dcnt + 7, ctx->stream));
  CK(launch_count(mask_dev, (int64_t)LL, dcnt + 5, ctx->stream));
  int32_t hv[8];
  CK(cudaMemcpyAsync(hv, dcnt, sizeof(hv), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (hv[7]) return EPFFT_ERR_DEVICE_TIMEOUT;
  for (int k = 0; k < n_img; k++) {
    const uint8_t* pl = plastic_dev + (size_t)k * LL;
    int32_t* o = labels_dev ? labels_dev + (size_t)k * LL : out;
    CK(cudaMemsetAsync(dcnt, 0, 8 * sizeof(int32_t), ctx->stream));
    CK(launch_vp_flags(mask_dev, pl, vp, L, ctx->stream));
    CK(launch_label(vp, lab, 1, L, 1, dcnt + 6, dcnt + 7, ctx->stream));
    CK(launch_vp_attach(mask_dev, vp, lab, o, L, scratch, dcnt, hv[5] > 0, ctx->stream));
    CK(launch_count(pl, (int64_t)LL, dcnt + 4, ctx->stream));
    int32_t h[8];
    CK(cudaMemcpyAsync(h, dcnt, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (h[7]) return EPFFT_ERR_DEVICE_TIMEOUT;
    int32_t* st = stats + 6 * (size_t)k;
    st[0] = h[0];
    st[1] = h[1];
    st[2] = h[2];
    st[3] = hv[3];
    st[4] = h[4];
    st[5] = hv[5];
  }
  return EPFFT_OK;
}

int epfft_indicators(int32_t n_inc, const epfft_record* records, const int32_t* stats, int32_t L, int32_t load,
                     double* out) {
  if (n_inc < 1 || !records || !stats || !out || L < 1 || (load != 0 && load != 1)) return EPFFT_ERR_ARG;
  std::vector<double> e0(n_inc), s0(n_inc), nn(n_inc);
  const double npx = (double)L * (double)L;
  for (int k = 0; k < n_inc; k++) {
    const epfft_record& r = records[k];
    const int32_t* st = stats + 6 * (size_t)k;
    e0[k] = load == 0 ? 0.5 * (r.eps_mean[0] + r.eps_mean[1]) : r.eps_mean[3];
    s0[k] = load == 0 ? 0.5 * (r.sig_mean[0] + r.sig_mean[1]) : r.sig_mean[3];
    nn[k] = (double)st[0] / (double)st[3];
    double* o = out + 8 * (size_t)k;
    o[0] = e0[k];
    o[1] = s0[k];
    o[2] = (double)st[4] / (npx - (double)st[5]);
    o[3] = (double)st[1] / npx;
    o[4] = (double)st[2] / (double)st[3];
    o[5] = nn[k];
  }
  // first derivative on the (possibly uneven) grid: second order inside,
  // first order one-sided at the ends
  auto grad = [&](const std::vector<double>& f, std::vector<double>& g) {
    g.assign(n_inc, 0.0);
    if (n_inc < 2) return;
    g[0] = (f[1] - f[0]) / (e0[1] - e0[0]);
    g[n_inc - 1] = (f[n_inc - 1] - f[n_inc - 2]) / (e0[n_inc - 1] - e0[n_inc - 2]);
    for (int k = 1; k + 1 < n_inc; k++) {
      const double h0 = e0[k] - e0[k - 1], h1 = e0[k + 1] - e0[k];
      g[k] = (h0 * h0 * f[k + 1] - h1 * h1 * f[k - 1] + (h1 * h1 - h0 * h0) * f[k]) / (h0 * h1 * (h0 + h1));
    }
  };
  std::vector<double> r, ds, dds;
  grad(nn, r);
  grad(s0, ds);
  grad(ds, dds);
  for (int k = 0; k < n_inc; k++) {
    out[8 * (size_t)k + 6] = r[k];
    out[8 * (size_t)k + 7] = -dds[k];
  }
  return EPFFT_OK;
}

int epfft_effective_moduli(epfft_ctx* ctx, const epfft_problem* problem, double strain, double* K_eff,
                           double* mu_eff) {
  if (!ctx || !problem || !K_eff || !mu_eff || !(std::fabs(strain) > 0.0) || !std::isfinite(strain))
    return EPFFT_ERR_ARG;
  // the same lattice with the elastic matrix, under equibiaxial strain and
  // under shear, as one batch of two one-increment solves
  epfft_problem p[2] = {*problem, *problem};
  for (auto& q : p) q.yield_stress = INFINITY;
  const double Ea[4] = {strain, strain, 0.0, 0.0}, Eb[4] = {0.0, 0.0, 0.0, strain};
  const epfft_path paths[2] = {{1, 0, Ea}, {1, 0, Eb}};
  epfft_record ra, rb;
  epfft_record* recs[2] = {&ra, &rb};
  const int rc = solve_impl(ctx, 2, p, paths, recs, nullptr, nullptr, nullptr, nullptr);
  if (rc != EPFFT_OK && rc != EPFFT_NOT_CONVERGED) return rc;
  *K_eff = (ra.sig_mean[0] + ra.sig_mean[1]) / (ra.eps_mean[0] + ra.eps_mean[1]);
  *mu_eff = rb.sig_mean[3] / (2.0 * rb.eps_mean[3]);
  return rc;
}

int epfft_empirical_curve(int32_t n_inc, const double* ind, const int32_t* stats, int32_t L, double modulus,
                          int32_t load, double* alpha, double* fit) {
  if (n_inc < 1 || !ind || !stats || !alpha || !fit || L < 1 || (load != 0 && load != 1)) return EPFFT_ERR_ARG;
  const double npx = (double)L * (double)L;
  const double ninf = ind[8 * (size_t)(n_inc - 1) + 5];
  std::vector<double> g1(n_inc), g2(n_inc), I1(n_inc), I2(n_inc);
  for (int k = 0; k < n_inc; k++) {
    const double* r = ind + 8 * (size_t)k;
    const int32_t* st = stats + 6 * (size_t)k;
    g1[k] = ninf != 1.0 ? (r[5] - ninf) / (1.0 - ninf) : 0.0;
    g2[k] = ((double)st[4] + (double)st[5]) / npx - r[3];  // v_p - v_p^max
  }
  // trapezoids from eps0 = 0, where the integrand is taken at the first increment
  auto cumint = [&](const std::vector<double>& g, std::vector<double>& I) {
    double acc = 0.0, x0 = 0.0, y0 = g[0];
    for (int k = 0; k < n_inc; k++) {
      const double x = ind[8 * (size_t)k];
      acc += 0.5 * (y0 + g[k]) * (x - x0);
      I[k] = acc;
      x0 = x;
      y0 = g[k];
    }
  };
  cumint(g1, I1);
  std::vector<double> A(n_inc), Bv(n_inc);
  if (load == 0) {
    cumint(g2, I2);
    for (int k = 0; k < n_inc; k++) {
      A[k] = modulus * I1[k];
      Bv[k] = modulus * I2[k];
    }
  } else {
    for (int k = 0; k < n_inc; k++) {
      A[k] = 2.0 * modulus * I1[k];
      Bv[k] = ind[8 * (size_t)k + 2];  // f_p
    }
  }
  double num = 0.0, den = 0.0;
  for (int k = 0; k < n_inc; k++) {
    num += (ind[8 * (size_t)k + 1] - A[k]) * Bv[k];
    den += Bv[k] * Bv[k];
  }
  *alpha = den > 0.0 ? num / den : 0.0;
  for (int k = 0; k < n_inc; k++) fit[k] = A[k] + *alpha * Bv[k];
  return EPFFT_OK;
}

int epfft_eps_eq(epfft_ctx* ctx, int32_t L, int32_t precision, const void* eps_dev, void* out_dev) {
  if (!ctx || !eps_dev || !out_dev || !is_pow2(L) || (precision != EPFFT_FP32 && precision != EPFFT_FP64))
    return EPFFT_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return EPFFT_ERR_CUDA;
  if (precision == EPFFT_FP32) CK(launch_eps_eq<float>((const float*)eps_dev, (float*)out_dev, L, ctx->stream));
  else CK(launch_eps_eq<double>((const double*)eps_dev, (double*)out_dev, L, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return EPFFT_OK;
}

int epfft_average5(epfft_ctx* ctx, int32_t L, int32_t precision, const void* eps_in_dev, void* eps_out_dev) {
  if (!ctx || !eps_in_dev || !eps_out_dev || eps_in_dev == eps_out_dev) return EPFFT_ERR_ARG;
  if (!is_pow2(L) || L < 4 || (precision != EPFFT_FP32 && precision != EPFFT_FP64)) return EPFFT_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return EPFFT_ERR_CUDA;
  if (precision == EPFFT_FP32) CK(launch_avg5<float>((const float*)eps_in_dev, (float*)eps_out_dev, L, ctx->stream));
  else CK(launch_avg5<double>((const double*)eps_in_dev, (double*)eps_out_dev, L, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return EPFFT_OK;
}

int epfft_mask(int32_t L, double void_fraction, uint64_t seed, uint8_t* mask_dev, void* stream) {
  if (!is_pow2(L) || L < 4 || L > 4096 || !mask_dev) return EPFFT_ERR_ARG;
  if (!(void_fraction >= 0.0 && void_fraction <= 1.0)) return EPFFT_ERR_ARG;
  if (launch_mask(mask_dev, (int64_t)L * L, seed, void_threshold(void_fraction), (cudaStream_t)stream) !=
      cudaSuccess)
    return EPFFT_ERR_CUDA;
  return EPFFT_OK;
}

int epfft_solve_refined_batch(epfft_ctx* ctx, int32_t n, const epfft_problem* problems, const epfft_path* paths,
                              double tol_switch, epfft_record* const* records, epfft_record* const* records_fp32,
                              const epfft_fields* fields) {
  if (!ctx || n < 1 || !problems || !paths || !records) return EPFFT_ERR_ARG;
  if (!(tol_switch >= 0.0)) return EPFFT_ERR_ARG;  // 0: automatic switch
  const int L = problems[0].L, n_inc = paths[0].n_inc;
  for (int i = 0; i < n; i++) {
    int rc = check_problem(&problems[i]);
    if (rc) return rc;
    if (problems[i].precision != EPFFT_FP64 || problems[i].L != L) return EPFFT_ERR_ARG;
    if (paths[i].n_inc != n_inc || n_inc < 1 || !paths[i].E || !records[i]) return EPFFT_ERR_ARG;
    for (int k = 0; k < 4 * n_inc; k++)
      if (!std::isfinite(paths[i].E[k])) return EPFFT_ERR_ARG;
  }
  if (!supported(L, EPFFT_FP32)) return EPFFT_ERR_UNSUPPORTED;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return EPFFT_ERR_CUDA;
  const size_t LL = (size_t)L * L;
  Arena A(ctx);
  std::vector<float*> e32(n);
  std::vector<double*> e64(n);
  std::vector<epfft_problem> p64(problems, problems + n), p32(n);
  for (int i = 0; i < n; i++) {
    e32[i] = (float*)A.get(4 * LL * sizeof(float));
    e64[i] = (double*)A.get(4 * LL * sizeof(double));
    if (!e32[i] || !e64[i]) return EPFFT_ERR_OOM;
    if (!problems[i].mask) {  // both stages see the same voids
      uint8_t* m = (uint8_t*)A.get(LL);
      if (!m) return EPFFT_ERR_OOM;
      CK(launch_mask(m, (int64_t)LL, problems[i].seed, void_threshold(problems[i].void_fraction), ctx->stream));
      p64[i].mask = m;
      p64[i].mask_on_device = 1;
    }
    p32[i] = p64[i];
    p32[i].precision = EPFFT_FP32;
    p32[i].tol_eq = std::max(tol_switch, problems[i].tol_eq);
    p32[i].tol_macro = std::max(tol_switch, problems[i].tol_macro);
  }
  // automatic switch: FP32 chunks of kChunk iterations, each continuing from
  // the strain the previous one left (the state is the strain alone: the
  // multiplier is sigma(eps)); a problem leaves the FP32 stage when a chunk
  // improves its max(eta1, eta2) by less than kGain, its tolerances hold, or
  // it reaches max_iter
  constexpr int kChunk = 2000;
  constexpr double kGain = 1.5;
  const double zero[4] = {0.0, 0.0, 0.0, 0.0};
  int status = EPFFT_OK;
  std::vector<epfft_path> pk(n);
  std::vector<epfft_record> r32(n);
  std::vector<int32_t> total(n);
  std::vector<double> prev(n);
  std::vector<epfft_fields> fk(fields ? n : 0);
  for (int k = 0; k < n_inc; k++) {
    // FP32 stage: the accepted FP64 state of increment k - 1 shifted by
    // E_k - E_{k-1} and rounded (increment 0 starts from the unstrained
    // lattice, shifted by E_0 inside the solve)
    for (int i = 0; i < n; i++) {
      const double* Ek = paths[i].E + 4 * k;
      pk[i] = {1, 0, Ek};
      total[i] = 0;
      prev[i] = INFINITY;
      if (k > 0) {
        const double* Ep = paths[i].E + 4 * (k - 1);
        const double dE[4] = {Ek[0] - Ep[0], Ek[1] - Ep[1], Ek[2] - Ep[2], Ek[3] - Ep[3]};
        CK((launch_shift_convert<double, float>(e64[i], e32[i], L, dE, ctx->stream)));
      }
    }
    std::vector<int> act(n);
    for (int i = 0; i < n; i++) act[i] = i;
    for (bool first = true; !act.empty(); first = false) {
      std::vector<epfft_problem> pa;
      std::vector<epfft_path> pth;
      std::vector<epfft_record*> rp;
      std::vector<const void*> in;
      std::vector<void*> out;
      for (int i : act) {
        pa.push_back(p32[i]);
        pa.back().max_iter = tol_switch > 0.0 ? problems[i].max_iter : std::min(kChunk, problems[i].max_iter - total[i]);
        pth.push_back(pk[i]);
        rp.push_back(&r32[i]);
        in.push_back((k == 0 && first) ? nullptr : e32[i]);
        out.push_back(e32[i]);
      }
      int rc = solve_impl(ctx, (int32_t)act.size(), pa.data(), pth.data(), rp.data(), nullptr, in.data(), out.data(),
                          nullptr);
      if (rc != EPFFT_OK && rc != EPFFT_NOT_CONVERGED) return rc;
      std::vector<int> next;
      for (int i : act) {
        total[i] += r32[i].iterations;
        const double eta = std::max(r32[i].eta1, r32[i].eta2);
        if (tol_switch == 0.0 && r32[i].status != 0 && eta * kGain < prev[i] && total[i] < problems[i].max_iter)
          next.push_back(i);
        prev[i] = eta;
      }
      act.swap(next);
    }
    for (int i = 0; i < n; i++) {
      r32[i].iterations = total[i];
      if (records_fp32 && records_fp32[i]) records_fp32[i][k] = r32[i];
      CK((launch_shift_convert<float, double>(e32[i], e64[i], L, zero, ctx->stream)));
      if (fields) {
        fk[i] = fields[i];
        fk[i].eps = k == n_inc - 1 ? fields[i].eps : nullptr;
        fk[i].plastic = fields[i].plastic ? fields[i].plastic + LL * (size_t)k : nullptr;
        fk[i].labels = fields[i].labels ? fields[i].labels + LL * (size_t)k : nullptr;
      }
    }
    // FP64 stage of every problem from its FP32 result, to its tolerances
    std::vector<epfft_record*> rp64(n);
    std::vector<const void*> in64(n);
    std::vector<void*> out64(n);
    for (int i = 0; i < n; i++) {
      rp64[i] = records[i] + k;
      in64[i] = e64[i];
      out64[i] = e64[i];
    }
    int rc = solve_impl(ctx, n, p64.data(), pk.data(), rp64.data(), fields ? fk.data() : nullptr, in64.data(),
                        out64.data(), nullptr);
    if (rc == EPFFT_ERR_NUMERIC) return rc;
    if (rc == EPFFT_NOT_CONVERGED) status = EPFFT_NOT_CONVERGED;
    else if (rc != EPFFT_OK) return rc;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return status;
}

int epfft_solve_refined(epfft_ctx* ctx, const epfft_problem* problem, const epfft_path* path, double tol_switch,
                        epfft_record* records, epfft_record* records_fp32, const epfft_fields* fields) {
  if (!ctx || !problem || !path || !records) return EPFFT_ERR_ARG;
  epfft_record* r[1] = {records};
  epfft_record* r32[1] = {records_fp32};
  return epfft_solve_refined_batch(ctx, 1, problem, path, tol_switch, r, records_fp32 ? r32 : nullptr, fields);
}

int epfft_iterate(epfft_ctx* ctx, const epfft_problem* problem, const double E[4], void* eps_dev, int32_t n_iter,
                  epfft_record* out) {
  if (!ctx || !problem || !E || !eps_dev || n_iter < 1 || !out) return EPFFT_ERR_ARG;
  epfft_problem p = *problem;
  p.tol_eq = 0.0;
  p.tol_macro = 0.0;
  p.max_iter = n_iter;
  epfft_path path = {1, 0, E};
  const void* e0[1] = {eps_dev};
  void* e1[1] = {eps_dev};
  // a fixed step count: warm start, n_iter + 1 iterates (the last one
  // finalizes iterate n_iter), the final flags; the passes are launched from
  // the host rather than from a graph loop
  int rc = solve_impl(ctx, 1, &p, &path, nullptr, nullptr, e0, e1, out, (int64_t)n_iter + 3);
  return rc == EPFFT_NOT_CONVERGED ? EPFFT_OK : rc;
}

int epfft_project(epfft_ctx* ctx, int32_t L, int32_t precision, double lambda0, double mu0, const double E[4],
                  const void* p_dev, void* e_dev) {
  if (!ctx || !E || !p_dev || !e_dev) return EPFFT_ERR_ARG;
  if (!is_pow2(L) || L < 4 || (precision != EPFFT_FP32 && precision != EPFFT_FP64)) return EPFFT_ERR_ARG;
  if (!supported(L, precision)) return EPFFT_ERR_UNSUPPORTED;
  if (!(mu0 > 0.0) || !(lambda0 + 2.0 * mu0 / 3.0 > 0.0)) return EPFFT_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return EPFFT_ERR_CUDA;
  Arena A(ctx);
  void *tw, *ktab;
  const int var = pass_variant(ctx, L, precision, 1);
  int rc = get_tables(ctx, L, precision, &tw, &ktab);
  if (!rc) rc = ensure_prepared(ctx, L, precision, var);
  if (rc) return rc;
  const size_t LL = (size_t)L * L, rs = real_size(precision);
  void* spec = A.get(3 * LL * rs);
  double* dpath = (double*)A.get(4 * sizeof(double));
  Solve* ds = (Solve*)A.get(sizeof(Solve));
  if (!spec || !dpath || !ds) return EPFFT_ERR_OOM;
  Solve S;
  std::memset(&S, 0, sizeof(S));
  S.lam0 = lambda0;
  S.mu0 = mu0;
  S.path = dpath;
  S.spec = spec;
  S.phase = PH_ITER;
  CK(cudaMemcpyAsync(dpath, E, 4 * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ds, &S, sizeof(S), cudaMemcpyHostToDevice, ctx->stream));
  if (precision == EPFFT_FP32) {
    CK(launch_row_forward<float>(L, var, ctx->stream, p_dev, spec, tw));
    CK(launch_col<float>(L, var, 1, ctx->stream, ds, tw, ktab, 0, 0));
    CK(launch_row_inverse<float>(L, var, ctx->stream, spec, e_dev, tw));
  } else {
    CK(launch_row_forward<double>(L, var, ctx->stream, p_dev, spec, tw));
    CK(launch_col<double>(L, var, 1, ctx->stream, ds, tw, ktab, 0, 0));
    CK(launch_row_inverse<double>(L, var, ctx->stream, spec, e_dev, tw));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return EPFFT_OK;
}

int epfft_displacement(epfft_ctx* ctx, int32_t L, int32_t precision, const void* eps_dev, void* u_dev) {
  if (!ctx || !eps_dev || !u_dev) return EPFFT_ERR_ARG;
  if (!is_pow2(L) || L < 4 || (precision != EPFFT_FP32 && precision != EPFFT_FP64)) return EPFFT_ERR_ARG;
  if (!supported(L, precision)) return EPFFT_ERR_UNSUPPORTED;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return EPFFT_ERR_CUDA;
  Arena A(ctx);
  void *tw, *ktab;
  const int var = pass_variant(ctx, L, precision, 1);
  int rc = get_tables(ctx, L, precision, &tw, &ktab);
  if (!rc) rc = ensure_prepared(ctx, L, precision, var);
  if (rc) return rc;
  const size_t LL = (size_t)L * L, rs = real_size(precision);
  void* planes = A.get(3 * LL * rs);
  void* spec = A.get(3 * LL * rs);
  double* dpath = (double*)A.get(4 * sizeof(double));
  Solve* ds = (Solve*)A.get(sizeof(Solve));
  if (!planes || !spec || !dpath || !ds) return EPFFT_ERR_OOM;
  // the column pass in its general form with the displacement operator;
  // the zero path makes the q = 0 mode zero
  Solve S;
  std::memset(&S, 0, sizeof(S));
  S.lam0 = 1.0;
  S.mu0 = 1.0;
  S.green = GM_DISP;
  S.path = dpath;
  S.spec = spec;
  S.phase = PH_ITER;
  CK(cudaMemsetAsync(dpath, 0, 4 * sizeof(double), ctx->stream));
  CK(cudaMemcpyAsync(ds, &S, sizeof(S), cudaMemcpyHostToDevice, ctx->stream));
  if (precision == EPFFT_FP32) {
    CK(launch_strain_planes<float>((const float*)eps_dev, (float*)planes, L, ctx->stream));
    CK(launch_row_forward<float>(L, var, ctx->stream, planes, spec, tw));
    CK(launch_col<float>(L, var, 1, ctx->stream, ds, tw, ktab, 0, 0, 1));
    CK(launch_row_inverse<float>(L, var, ctx->stream, spec, planes, tw));
    CK(launch_disp_pairs<float>((const float*)planes, (float*)u_dev, L, ctx->stream));
  } else {
    CK(launch_strain_planes<double>((const double*)eps_dev, (double*)planes, L, ctx->stream));
    CK(launch_row_forward<double>(L, var, ctx->stream, planes, spec, tw));
    CK(launch_col<double>(L, var, 1, ctx->stream, ds, tw, ktab, 0, 0, 1));
    CK(launch_row_inverse<double>(L, var, ctx->stream, spec, planes, tw));
    CK(launch_disp_pairs<double>((const double*)planes, (double*)u_dev, L, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return EPFFT_OK;
}

int epfft_label(epfft_ctx* ctx, int32_t L, int32_t n_img, const uint8_t* flags_dev, int32_t periodic,
                int32_t* labels_dev, int32_t* counts) {
  if (!ctx || !is_pow2(L) || L < 2 || L > 4096 || n_img < 1 || !flags_dev || !labels_dev) return EPFFT_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return EPFFT_ERR_CUDA;
  Arena A(ctx);
  int32_t* dc = (int32_t*)A.get(sizeof(int32_t) * (size_t)n_img);
  int32_t* err = (int32_t*)A.get(sizeof(int32_t));
  if (!dc || !err) return EPFFT_ERR_OOM;
  CK(cudaMemsetAsync(err, 0, sizeof(int32_t), ctx->stream));
  CK(launch_label(flags_dev, labels_dev, n_img, L, periodic ? 1 : 0, dc, err, ctx->stream));
  int32_t herr = 0;
  if (counts) CK(cudaMemcpyAsync(counts, dc, sizeof(int32_t) * (size_t)n_img, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return herr ? EPFFT_ERR_DEVICE_TIMEOUT : EPFFT_OK;
}

int epfft_serve_open(epfft_ctx* ctx, const epfft_serve_options* opt) {
  if (!ctx || !opt || opt->hbm_budget_bytes <= 0 || opt->slots_per_class < 1 || opt->steps_per_launch < 1)
    return EPFFT_ERR_ARG;
  if (ctx->server) return EPFFT_ERR_ARG;
  Server* S = new Server();
  S->budget = (size_t)opt->hbm_budget_bytes;
  S->cap = opt->slots_per_class;
  S->steps = opt->steps_per_launch;
  ctx->server = S;
  return EPFFT_OK;
}

int epfft_serve_close(epfft_ctx* ctx) {
  if (!ctx || !ctx->server) return EPFFT_ERR_ARG;
  cudaSetDevice(ctx->device);
  free_mixed(ctx, *ctx->server);
  for (auto& kv : ctx->server->classes) free_class(ctx, kv.second);
  delete ctx->server;
  ctx->server = nullptr;
  return EPFFT_OK;
}

int epfft_submit(epfft_ctx* ctx, const epfft_problem* problem, const epfft_path* path, int32_t want,
                 int64_t* ticket) {
  if (!ctx || !ctx->server || !problem || !path || !ticket) return EPFFT_ERR_ARG;
  if (want & ~(EPFFT_WANT_EPS | EPFFT_WANT_SIG | EPFFT_WANT_PLASTIC | EPFFT_WANT_LABELS)) return EPFFT_ERR_ARG;
  int rc = check_problem(problem);
  if (rc) return rc;
  if (path->n_inc < 1 || !path->E) return EPFFT_ERR_ARG;
  for (int k = 0; k < 4 * path->n_inc; k++)
    if (!std::isfinite(path->E[k])) return EPFFT_ERR_ARG;
  Server& S = *ctx->server;
  PassShape sh;
  rc = shape(problem->L, problem->precision, pass_variant(ctx, problem->L, problem->precision, S.cap), &sh);
  if (rc) return rc;
  Ticket t;
  t.prob = *problem;
  t.path.assign(path->E, path->E + 4 * (size_t)path->n_inc);
  t.want = want;
  t.bytes = solve_footprint(problem->L, problem->precision, sh.row_ctas, path->n_inc);
  if (t.bytes > S.budget) return EPFFT_ERR_OOM;
  const size_t LL = (size_t)problem->L * problem->L;
  if (problem->mask) {
    t.mask.resize(LL);
    if (problem->mask_on_device) {
      if (cudaSetDevice(ctx->device) != cudaSuccess ||
          cudaMemcpy(t.mask.data(), problem->mask, LL, cudaMemcpyDeviceToHost) != cudaSuccess)
        return EPFFT_ERR_CUDA;
    } else {
      std::memcpy(t.mask.data(), problem->mask, LL);
    }
  }
  t.t_submit = now_s();
  const int64_t id = S.next++;
  S.tickets.emplace(id, std::move(t));
  S.queue.push_back(id);
  *ticket = id;
  return EPFFT_OK;
}

int epfft_serve_step(epfft_ctx* ctx, int32_t* n_running, int32_t* n_queued) {
  if (!ctx || !ctx->server) return EPFFT_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return EPFFT_ERR_CUDA;
  Server& S = *ctx->server;
  ctx->last = epfft_stats{};
  int rc = serve_admit(ctx, S);
  if (rc) return rc;
  // every class with live slots advances at most S.steps loop steps, all
  // classes in one launch of the mixed graph
  std::vector<ServeClass*> live;
  bool checks_read = false;
  for (auto& kv : S.classes) {
    int used = 0;
    for (auto& sl : kv.second->slots) used += sl.used;
    if (used) live.push_back(kv.second);
  }
  if (!live.empty()) {
    if (S.dirty || !S.exec) {
      rc = build_serve_graph(ctx, S);
      if (rc) return rc;
    }
    std::vector<BatchCtl> bcs(S.order.size());
    for (size_t i = 0; i < S.order.size(); i++) {
      ServeClass* k = S.order[i];
      int used = 0;
      for (auto& sl : k->slots) used += sl.used;
      std::memset(&bcs[i], 0, sizeof(BatchCtl));
      bcs[i].active = used;
      bcs[i].max_body_iters = S.steps;
      bcs[i].dc = k->prec == EPFFT_FP32_DEFECT;
      CK(cudaMemcpyAsync(k->B.d_ctl, &bcs[i], sizeof(BatchCtl), cudaMemcpyHostToDevice, ctx->stream));
    }
    CK(cudaGraphLaunch(S.exec, ctx->stream));
    for (size_t i = 0; i < S.order.size(); i++)
      CK(cudaMemcpyAsync(&bcs[i], S.order[i]->B.d_ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, ctx->stream));
    // the self-check records, behind the step's kernels on the same stream
    CK(enqueue_check_reads(ctx, ctx->stream));
    checks_read = true;
    CK(cudaStreamSynchronize(ctx->stream));
    int64_t steps = 0;
    for (size_t i = 0; i < S.order.size(); i++) steps = std::max<int64_t>(steps, bcs[i].body_iters);
    ctx->last.loop_steps = steps;
    // a column and a row pass of every class, and the loop-condition kernel, per step
    ctx->last.kernel_launches += (2 * (int64_t)S.order.size() + 1) * steps;
    // the defect classes' refresh node
    for (size_t i = 0; i < S.order.size(); i++) ctx->last.kernel_launches += 4 * bcs[i].refresh_runs;
  }
  {
    // the records read with the step (a fired check is cleared by the
    // synchronous read), or read now when no class ran
    CheckRec cr{};
    if (checks_read) {
      for (int i = 0; i < 8 && !cr.code; i++)
        if (ctx->h_checks[i].code) cr = ctx->h_checks[i];
      if (cr.code) {
        CheckRec clr;
        CK(read_check_all(&clr));
      }
    } else {
      CK(read_check_all(&cr));
    }
    if (cr.code) {
      fprintf(stderr, "epfft: device self-check %d failed (index %lld, bound %lld, at %d)\n", cr.code,
              (long long)cr.index, (long long)cr.bound, cr.where);
      return EPFFT_ERR_CUDA;
    }
  }
  for (ServeClass* k : live) {
    int64_t before = 0, after = 0;
    for (auto& sl : k->slots) before += sl.used;
    rc = serve_harvest(ctx, S, k);
    if (rc) return rc;
    for (auto& sl : k->slots) after += sl.used;
    ctx->last.kernel_launches += 4 * (before - after);  // labelling of each harvested solve
  }
  int running = 0;
  for (auto& kv : S.classes)
    for (auto& sl : kv.second->slots) running += sl.used;
  if (n_running) *n_running = running;
  if (n_queued) *n_queued = (int32_t)S.queue.size();
  return EPFFT_OK;
}

int epfft_poll(epfft_ctx* ctx, int64_t ticket, epfft_record* records, void* eps_host, double* latency_s) {
  if (!ctx || !ctx->server) return EPFFT_ERR_ARG;
  Server& S = *ctx->server;
  auto it = S.tickets.find(ticket);
  if (it == S.tickets.end()) return EPFFT_ERR_ARG;
  Ticket& t = it->second;
  if (t.state != 2) return EPFFT_PENDING;
  if (records) std::memcpy(records, t.rec.data(), sizeof(Record) * t.rec.size());
  if (eps_host && !t.eps.empty()) std::memcpy(eps_host, t.eps.data(), t.eps.size());
  if (latency_s) *latency_s = t.t_done - t.t_submit;
  const int st = t.status;
  // a ticket holding fields beyond the strain stays for epfft_ticket_fields
  // until epfft_release
  if (!(t.want & ~EPFFT_WANT_EPS)) S.tickets.erase(it);
  return st;
}

int epfft_ticket_fields(epfft_ctx* ctx, int64_t ticket, int32_t inc, void* eps_host, void* sig_host,
                        uint8_t* plastic_host, int32_t* labels_host) {
  if (!ctx || !ctx->server) return EPFFT_ERR_ARG;
  Server& S = *ctx->server;
  auto it = S.tickets.find(ticket);
  if (it == S.tickets.end()) return EPFFT_ERR_ARG;
  const Ticket& t = it->second;
  if (t.state != 2) return EPFFT_PENDING;
  const int n = (int)t.rec.size();
  if (inc < 0 || inc >= n) return EPFFT_ERR_ARG;
  // the strain and stress are those of the final accepted state only
  if ((eps_host || sig_host) && inc != n - 1) return EPFFT_ERR_ARG;
  if ((eps_host && t.eps.empty()) || (sig_host && t.sig.empty()) || (plastic_host && t.flags.empty()) ||
      (labels_host && t.labels.empty()))
    return EPFFT_ERR_ARG;
  const size_t LL = (size_t)t.prob.L * t.prob.L;
  if (eps_host) std::memcpy(eps_host, t.eps.data(), t.eps.size());
  if (sig_host) std::memcpy(sig_host, t.sig.data(), t.sig.size());
  if (plastic_host) std::memcpy(plastic_host, t.flags.data() + LL * (size_t)inc, LL);
  if (labels_host) std::memcpy(labels_host, t.labels.data() + LL * (size_t)inc, sizeof(int32_t) * LL);
  return EPFFT_OK;
}

int epfft_release(epfft_ctx* ctx, int64_t ticket) {
  if (!ctx || !ctx->server) return EPFFT_ERR_ARG;
  Server& S = *ctx->server;
  auto it = S.tickets.find(ticket);
  if (it == S.tickets.end()) return EPFFT_ERR_ARG;
  if (it->second.state != 2) return EPFFT_PENDING;
  S.tickets.erase(it);
  return EPFFT_OK;
}

int epfft_time_passes(epfft_ctx* ctx, const epfft_problem* problem, int32_t n_batch, const double E[4],
                      int32_t n_iter, float* col_ms, float* row_ms) {
  if (!ctx || !problem || !E || n_iter < 1 || n_batch < 1 || !col_ms || !row_ms) return EPFFT_ERR_ARG;
  int rc = check_problem(problem);
  if (rc) return rc;
  return time_passes_impl(ctx, *problem, n_batch, E, n_iter, -1, col_ms, row_ms);
}

int epfft_fp64_peak(epfft_ctx* ctx, double* tflops, int32_t* n_sm, float* ms) {
  if (!ctx || !tflops) return EPFFT_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return EPFFT_ERR_CUDA;
  int nsm = 0;
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
  Arena A(ctx);
  double* sink = (double*)A.get(sizeof(double));
  if (!sink) return EPFFT_ERR_OOM;
  // eight 256-thread CTAs per SM (64 warps): enough independent FMAs in
  // flight to cover the FP64 pipe's latency
  const int blocks = 8 * nsm, n = 4096;
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  float best = 0.f;
  for (int rep = 0; rep < 6; rep++) {  // the first launch is a warm-up
    CK(cudaEventRecord(a, ctx->stream));
    CK(launch_fp64_fma(blocks, n, sink, ctx->stream));
    CK(cudaEventRecord(b, ctx->stream));
    CK(cudaEventSynchronize(b));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, a, b));
    if (rep > 0 && (best == 0.f || t < best)) best = t;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  const double flops = 2.0 * FMA_CHAINS * (double)n * FMA_THREADS * blocks;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (n_sm) *n_sm = nsm;
  if (ms) *ms = best;
  return EPFFT_OK;
}

int epfft_autotune(epfft_ctx* ctx, int32_t L, int32_t precision, int32_t n_batch, int32_t* chosen,
                   float* ms_per_iteration) {
  if (!ctx || n_batch < 1) return EPFFT_ERR_ARG;
  if (!is_pow2(L) || L < 4 || (precision != EPFFT_FP32 && precision != EPFFT_FP64 && precision != EPFFT_FP32_DEFECT))
    return EPFFT_ERR_ARG;
  if (!supported(L, precision)) return EPFFT_ERR_UNSUPPORTED;
  // a synthetic lattice of the kind the solver serves: f = 0.2 voids, the
  // default matrix, shear at 1.5x the void-free yield strain
  epfft_problem p;
  std::memset(&p, 0, sizeof(p));
  p.L = L;
  p.precision = precision;
  p.void_fraction = 0.2;
  p.seed = 7;
  p.green = EPFFT_GREEN_EQ3;
  p.mu = p.mu0 = 1.0;
  p.lambda = p.lambda0 = 1.5;
  p.yield_stress = 1.0;
  p.max_iter = 1;
  const double E[4] = {0.0, 0.0, 0.0, 1.5 / (2.0 * std::sqrt(3.0))};
  const int64_t px = (int64_t)L * L * n_batch;
  const int n_iter = px >= ((int64_t)1 << 24) ? 10 : 30;
  int best = -1;
  float tbest = 0.f;
  for (int v = 0; v < N_VARIANTS; v++) {
    if (ms_per_iteration) ms_per_iteration[v] = 0.f;
    PassShape sh;
    if (shape(L, precision, v, &sh) != EPFFT_OK) continue;  // not compiled for this size
    float c = 0.f, r = 0.f;
    // warm-up, then the timed launches
    int rc = time_passes_impl(ctx, p, n_batch, E, 3, v, &c, &r);
    if (!rc) rc = time_passes_impl(ctx, p, n_batch, E, n_iter, v, &c, &r);
    if (rc) return rc;
    if (ms_per_iteration) ms_per_iteration[v] = c + r;
    if (best < 0 || c + r < tbest) {
      tbest = c + r;
      best = v;
    }
  }
  ctx->variant[std::make_tuple((int)L, (int)precision, batch_class(L, n_batch))] = best;
  if (chosen) *chosen = best;
  return EPFFT_OK;
}

int epfft_supported_tiling(int32_t L, int32_t precision, int32_t variant) {
  if (variant < 0 || variant >= N_VARIANTS || !supported(L, precision)) return 0;
  PassShape sh;
  return shape(L, precision, variant, &sh) == EPFFT_OK ? 1 : 0;
}

int epfft_set_tiling(epfft_ctx* ctx, int32_t L, int32_t precision, int32_t variant) {
  if (!ctx || variant < 0 || variant >= N_VARIANTS) return EPFFT_ERR_ARG;
  if (!is_pow2(L) || L < 4 || (precision != EPFFT_FP32 && precision != EPFFT_FP64 && precision != EPFFT_FP32_DEFECT))
    return EPFFT_ERR_ARG;
  if (!supported(L, precision)) return EPFFT_ERR_UNSUPPORTED;
  if (!epfft_supported_tiling(L, precision, variant)) return EPFFT_ERR_UNSUPPORTED;
  for (int k = 0; k < 2; k++) ctx->variant[std::make_tuple((int)L, (int)precision, k)] = variant;
  return EPFFT_OK;
}

int epfft_set_defect_refresh(epfft_ctx* ctx, int32_t steps) {
  if (!ctx || steps < 1) return EPFFT_ERR_ARG;
  ctx->defect_refresh = steps;
  return EPFFT_OK;
}

}  // extern "C"
