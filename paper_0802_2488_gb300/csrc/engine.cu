// Host side of the epfft C ABI: argument checks, device state of a batch of
// solves, the device-driven loop (a CUDA graph whose while node repeats
// one column pass and one row pass until every solve is done), cluster
// labelling and copy-out.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

#include "../../include/epfft.h"
#include "aux_kernels.cuh"
#include "launch.cuh"

using namespace epfft;

struct epfft_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;  // work stream
  cudaStream_t cap = nullptr;     // stream used only to capture graph bodies
  bool own_stream = false;
  epfft_alloc_fn alloc = nullptr;
  epfft_free_fn freef = nullptr;
  void* user = nullptr;
  // (L, precision) -> device table: tw[L] then ktab[L] (complex of precision)
  std::map<std::pair<int, int>, void*> tables;
  std::map<std::pair<int, int>, bool> prepared;
  epfft_stats last{};
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
  if (prec == EPFFT_FP32) return pass_shape<float>(L, &sh);
  if (prec == EPFFT_FP64) return pass_shape<double>(L, &sh);
  return false;
}

int shape(int L, int prec, PassShape* sh) {
  bool ok = prec == EPFFT_FP32 ? pass_shape<float>(L, sh) : pass_shape<double>(L, sh);
  return ok ? EPFFT_OK : EPFFT_ERR_UNSUPPORTED;
}

size_t real_size(int prec) { return prec == EPFFT_FP32 ? 4 : 8; }

// Twiddles exp(-2 pi i k / L) and Fourier symbols of Eq. 2,
// k(m) = 2 sin(q/2) exp(i q/2) = (sin q, 2 sin^2(q/2)), q = 2 pi m / L, both
// evaluated in long double and rounded once to the working precision.
template <typename T>
void fill_tables(int L, std::vector<T>& h) {
  h.assign((size_t)4 * L, T(0));
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < L; k++) {
    const long double a = 2.0L * pi * (long double)k / (long double)L;
    const long double hs = sinl(pi * (long double)k / (long double)L);
    h[2 * k] = (T)cosl(a);
    h[2 * k + 1] = (T)(-sinl(a));
    h[2 * L + 2 * k] = (T)sinl(a);
    h[2 * L + 2 * k + 1] = (T)(2.0L * hs * hs);
  }
}

int get_tables(epfft_ctx* c, int L, int prec, void** tw, void** ktab) {
  auto key = std::make_pair(L, prec);
  auto it = c->tables.find(key);
  if (it == c->tables.end()) {
    const size_t bytes = (size_t)4 * L * real_size(prec);
    void* d = nullptr;
    if (cudaMalloc(&d, bytes) != cudaSuccess) {
      cudaGetLastError();
      return EPFFT_ERR_OOM;
    }
    if (prec == EPFFT_FP32) {
      std::vector<float> h;
      fill_tables<float>(L, h);
      CK(cudaMemcpy(d, h.data(), bytes, cudaMemcpyHostToDevice));
    } else {
      std::vector<double> h;
      fill_tables<double>(L, h);
      CK(cudaMemcpy(d, h.data(), bytes, cudaMemcpyHostToDevice));
    }
    it = c->tables.emplace(key, d).first;
  }
  if (!c->prepared[key]) {
    CK(prec == EPFFT_FP32 ? prepare<float>(L) : prepare<double>(L));
    c->prepared[key] = true;
  }
  *tw = it->second;
  *ktab = (char*)it->second + (size_t)2 * L * real_size(prec);
  return EPFFT_OK;
}

uint64_t void_threshold(double f) {
  if (!(f > 0.0)) return 0;
  if (f >= 1.0) return (uint64_t)1 << 53;
  return (uint64_t)std::floor(f * 9007199254740992.0);
}

int check_problem(const epfft_problem* p) {
  if (!p) return EPFFT_ERR_ARG;
  if (!is_pow2(p->L) || p->L < 4 || p->L > 4096) return EPFFT_ERR_ARG;
  if (p->precision != EPFFT_FP32 && p->precision != EPFFT_FP64) return EPFFT_ERR_ARG;
  if (p->green != EPFFT_GREEN_EQ3) return EPFFT_ERR_ARG;
  if (!supported(p->L, p->precision)) return EPFFT_ERR_UNSUPPORTED;
  if (!p->mask && !(p->void_fraction >= 0.0 && p->void_fraction <= 1.0)) return EPFFT_ERR_ARG;
  if (!(p->mu > 0.0) || !(p->mu0 > 0.0) || !std::isfinite(p->mu) || !std::isfinite(p->mu0)) return EPFFT_ERR_ARG;
  if (!(p->lambda + 2.0 * p->mu / 3.0 > 0.0) || !(p->lambda0 + 2.0 * p->mu0 / 3.0 > 0.0)) return EPFFT_ERR_ARG;
  if (!(p->lambda0 >= 0.0) || !std::isfinite(p->lambda0) || !std::isfinite(p->lambda)) return EPFFT_ERR_ARG;
  if (!(p->yield_stress > 0.0)) return EPFFT_ERR_ARG;
  if (!(p->tol_eq >= 0.0) || !(p->tol_macro >= 0.0)) return EPFFT_ERR_ARG;
  if (p->max_iter < 1) return EPFFT_ERR_ARG;
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
  for (int i = 0; i < N_MC; i++) S.mcf[i] = (float)c[i];
}

// Device state of one batch.
struct Batch {
  int L = 0, prec = 0, nb = 0;
  PassShape sh{};
  void* tw = nullptr;
  void* ktab = nullptr;
  Solve* d_solves = nullptr;
  BatchCtl* d_ctl = nullptr;
  std::vector<Solve> h_solves;
  std::vector<int32_t> n_inc;
  std::vector<int32_t*> d_labels;  // per solve, n_inc * L * L (allocated on demand)
};

int launch_body(epfft_ctx* c, Batch& B, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond) {
  if (B.prec == EPFFT_FP32) {
    CK(launch_col<float>(B.L, B.nb, s, B.d_solves, B.tw, B.ktab, h, use_cond));
    CK(launch_row<float>(B.L, B.nb, s, B.d_solves, B.d_ctl, B.tw, h, use_cond));
  } else {
    CK(launch_col<double>(B.L, B.nb, s, B.d_solves, B.tw, B.ktab, h, use_cond));
    CK(launch_row<double>(B.L, B.nb, s, B.d_solves, B.d_ctl, B.tw, h, use_cond));
  }
  (void)c;
  return EPFFT_OK;
}

// Builds the device state of n problems.  eps0 (optional, device) gives the
// starting local strain of every solve (then the first increment starts
// from it unshifted); otherwise the lattice starts unstrained.
int setup_batch(epfft_ctx* c, Arena& A, Batch& B, int n, const epfft_problem* probs,
                const epfft_path* paths, const void* const* eps0) {
  B.L = probs[0].L;
  B.prec = probs[0].precision;
  B.nb = n;
  int rc = shape(B.L, B.prec, &B.sh);
  if (rc) return rc;
  rc = get_tables(c, B.L, B.prec, &B.tw, &B.ktab);
  if (rc) return rc;
  const int L = B.L;
  const size_t LL = (size_t)L * L, rs = real_size(B.prec);
  B.h_solves.resize(n);
  B.n_inc.resize(n);
  int64_t max_body = 0;
  for (int i = 0; i < n; i++) {
    const epfft_problem& p = probs[i];
    const epfft_path& path = paths[i];
    Solve& S = B.h_solves[i];
    std::memset(&S, 0, sizeof(S));
    S.lam = p.lambda;
    S.mu = p.mu;
    S.Y = p.yield_stress;
    S.lam0 = p.lambda0;
    S.mu0 = p.mu0;
    S.tol_eq = p.tol_eq;
    S.tol_macro = p.tol_macro;
    S.max_iter = p.max_iter;
    S.n_inc = path.n_inc;
    fill_consts(S);
    B.n_inc[i] = path.n_inc;
    void* eps0d = A.get(4 * LL * rs);
    void* eps1d = A.get(4 * LL * rs);
    void* spec = A.get(3 * LL * rs);
    double* part = (double*)A.get(sizeof(double) * PART_STRIDE * (size_t)B.sh.row_ctas);
    uint8_t* mask = (uint8_t*)A.get(LL);
    uint8_t* flags = (uint8_t*)A.get(LL * (size_t)path.n_inc);
    double* dpath = (double*)A.get(sizeof(double) * 4 * (size_t)path.n_inc);
    Record* rec = (Record*)A.get(sizeof(Record) * (size_t)path.n_inc);
    if (!eps0d || !eps1d || !spec || !part || !mask || !flags || !dpath || !rec) return EPFFT_ERR_OOM;
    S.eps[0] = eps0d;
    S.eps[1] = eps1d;
    S.spec = spec;
    S.partials = part;
    S.mask = mask;
    S.flags = flags;
    S.path = dpath;
    S.rec = rec;
    S.phase = PH_INIT;
    CK(cudaMemcpyAsync(dpath, path.E, sizeof(double) * 4 * (size_t)path.n_inc, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(rec, 0, sizeof(Record) * (size_t)path.n_inc, c->stream));
    if (p.mask) {
      CK(cudaMemcpyAsync(mask, p.mask, LL, p.mask_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         c->stream));
    } else {
      CK(launch_mask(mask, (int64_t)LL, p.seed, void_threshold(p.void_fraction), c->stream));
    }
    if (eps0 && eps0[i]) {
      CK(cudaMemcpyAsync(eps0d, eps0[i], 4 * LL * rs, cudaMemcpyDeviceToDevice, c->stream));
      for (int k = 0; k < 4; k++) S.Eprev[k] = path.E[k];
    } else {
      CK(cudaMemsetAsync(eps0d, 0, 4 * LL * rs, c->stream));
    }
    const int64_t need = (int64_t)path.n_inc * ((int64_t)p.max_iter + 2) + 1;
    if (need > max_body) max_body = need;
  }
  B.d_solves = (Solve*)A.get(sizeof(Solve) * (size_t)n);
  B.d_ctl = (BatchCtl*)A.get(sizeof(BatchCtl));
  if (!B.d_solves || !B.d_ctl) return EPFFT_ERR_OOM;
  CK(cudaMemcpyAsync(B.d_solves, B.h_solves.data(), sizeof(Solve) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
  BatchCtl bc;
  std::memset(&bc, 0, sizeof(bc));
  bc.active = n;
  bc.max_body_iters = max_body + 8;
  CK(cudaMemcpyAsync(B.d_ctl, &bc, sizeof(bc), cudaMemcpyHostToDevice, c->stream));
  return EPFFT_OK;
}

// Runs the device-side loop to completion: one graph launch whose while
// node repeats [column pass, row pass]; the row pass's last CTA sets the
// loop condition.
int run_graph(epfft_ctx* c, Batch& B) {
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
    if (cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
        cudaSuccess) {
      rc = EPFFT_ERR_CUDA;
      break;
    }
    int lrc = launch_body(c, B, c->cap, h, 1);
    cudaGraph_t captured = nullptr;
    cudaError_t ec = cudaStreamEndCapture(c->cap, &captured);
    if (lrc != EPFFT_OK || ec != cudaSuccess) {
      rc = EPFFT_ERR_CUDA;
      break;
    }
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      rc = EPFFT_ERR_CUDA;
      break;
    }
    if (cudaGraphLaunch(exec, c->stream) != cudaSuccess) {
      rc = EPFFT_ERR_CUDA;
      break;
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) rc = EPFFT_ERR_CUDA;
  } while (0);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (rc != EPFFT_OK) cudaGetLastError();
  return rc;
}

// Diagnostic loop (EPFFT_SYNC_CHECK=1 in the environment): the same passes
// launched from the host one by one, each followed by a synchronisation
// and an error check that names the pass, phase and step that failed.
int run_checked(epfft_ctx* c, Batch& B) {
  BatchCtl bc;
  std::vector<Solve> hs(B.nb);
  for (int64_t step = 0;; step++) {
    CK(cudaMemcpy(hs.data(), B.d_solves, sizeof(Solve) * B.nb, cudaMemcpyDeviceToHost));
    cudaError_t e;
    if (B.prec == EPFFT_FP32) e = launch_col<float>(B.L, B.nb, c->stream, B.d_solves, B.tw, B.ktab, 0, 0);
    else e = launch_col<double>(B.L, B.nb, c->stream, B.d_solves, B.tw, B.ktab, 0, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      fprintf(stderr, "epfft check: column pass failed at step %lld (phase %d inc %d iter %d): %s\n",
              (long long)step, hs[0].phase, hs[0].inc, hs[0].iter, cudaGetErrorString(e));
      return EPFFT_ERR_CUDA;
    }
    if (B.prec == EPFFT_FP32) e = launch_row<float>(B.L, B.nb, c->stream, B.d_solves, B.d_ctl, B.tw, 0, 0);
    else e = launch_row<double>(B.L, B.nb, c->stream, B.d_solves, B.d_ctl, B.tw, 0, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      fprintf(stderr, "epfft check: row pass failed at step %lld (phase %d inc %d iter %d): %s\n",
              (long long)step, hs[0].phase, hs[0].inc, hs[0].iter, cudaGetErrorString(e));
      return EPFFT_ERR_CUDA;
    }
    CheckRec cr;
    CK(B.prec == EPFFT_FP32 ? read_check<float>(&cr) : read_check<double>(&cr));
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

// Labels the per-increment plastic flags of every solve; fills n_clusters.
int label_batch(epfft_ctx* c, Arena& A, Batch& B, std::vector<std::vector<Record>>& recs, bool keep_labels) {
  const size_t LL = (size_t)B.L * B.L;
  int32_t* err = (int32_t*)A.get(sizeof(int32_t));
  if (!err) return EPFFT_ERR_OOM;
  CK(cudaMemsetAsync(err, 0, sizeof(int32_t), c->stream));
  B.d_labels.assign(B.nb, nullptr);
  int32_t* tmp = nullptr;
  size_t tmp_bytes = 0;
  for (int i = 0; i < B.nb; i++) {
    const size_t n = (size_t)B.n_inc[i];
    int32_t* lab;
    if (keep_labels) {
      lab = (int32_t*)A.get(sizeof(int32_t) * LL * n);
    } else {
      if (tmp_bytes < sizeof(int32_t) * LL * n) {
        tmp_bytes = sizeof(int32_t) * LL * n;
        tmp = (int32_t*)A.get(tmp_bytes);
      }
      lab = tmp;
    }
    int32_t* counts = (int32_t*)A.get(sizeof(int32_t) * n);
    if (!lab || !counts) return EPFFT_ERR_OOM;
    CK(launch_label(B.h_solves[i].flags, lab, (int64_t)n, B.L, 1, counts, err, c->stream));
    if (getenv("EPFFT_SYNC_CHECK")) {
      cudaError_t e = cudaStreamSynchronize(c->stream);
      if (e != cudaSuccess) {
        fprintf(stderr, "epfft check: labelling failed for solve %d: %s\n", i, cudaGetErrorString(e));
        return EPFFT_ERR_CUDA;
      }
    }
    std::vector<int32_t> hc(n);
    CK(cudaMemcpyAsync(hc.data(), counts, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (size_t k = 0; k < n; k++) recs[i][k].n_clusters = hc[k];
    B.d_labels[i] = keep_labels ? lab : nullptr;
  }
  int32_t herr = 0;
  CK(cudaMemcpy(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost));
  return herr ? EPFFT_ERR_DEVICE_TIMEOUT : EPFFT_OK;
}

int copy_out(epfft_ctx* c, Batch& B, Solve& S, int i, const epfft_fields* f) {
  if (!f) return EPFFT_OK;
  const size_t LL = (size_t)B.L * B.L, rs = real_size(B.prec);
  const size_t n = (size_t)B.n_inc[i];
  const cudaMemcpyKind k = f->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (f->eps) CK(cudaMemcpyAsync(f->eps, S.eps[S.cur], 4 * LL * rs, k, c->stream));
  if (f->plastic) CK(cudaMemcpyAsync(f->plastic, S.flags, LL * n, k, c->stream));
  if (f->labels && B.d_labels[i]) CK(cudaMemcpyAsync(f->labels, B.d_labels[i], sizeof(int32_t) * LL * n, k, c->stream));
  return EPFFT_OK;
}

int solve_impl(epfft_ctx* c, int32_t n, const epfft_problem* probs, const epfft_path* paths,
               epfft_record* const* records, const epfft_fields* fields, const void* const* eps0,
               void* const* eps_out, epfft_record* iter_rec) {
  if (!c || n < 1 || !probs || !paths) return EPFFT_ERR_ARG;
  for (int i = 0; i < n; i++) {
    int rc = check_problem(&probs[i]);
    if (rc) return rc;
    if (probs[i].L != probs[0].L || probs[i].precision != probs[0].precision) return EPFFT_ERR_ARG;
    if (paths[i].n_inc < 1 || !paths[i].E) return EPFFT_ERR_ARG;
    for (int k = 0; k < 4 * paths[i].n_inc; k++)
      if (!std::isfinite(paths[i].E[k])) return EPFFT_ERR_ARG;
    if (records && !records[i]) return EPFFT_ERR_ARG;
  }
  if (cudaSetDevice(c->device) != cudaSuccess) return EPFFT_ERR_CUDA;
  Arena A(c);
  Batch B;
  int rc = setup_batch(c, A, B, n, probs, paths, eps0);
  if (rc) return rc;
  const char* chk = getenv("EPFFT_SYNC_CHECK");
  rc = (chk && chk[0] == '1') ? run_checked(c, B) : run_graph(c, B);
  if (rc) return rc;
  // read back the solve states and records
  CK(cudaMemcpyAsync(B.h_solves.data(), B.d_solves, sizeof(Solve) * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
  BatchCtl bc;
  CK(cudaMemcpyAsync(&bc, B.d_ctl, sizeof(bc), cudaMemcpyDeviceToHost, c->stream));
  std::vector<std::vector<Record>> recs(n);
  for (int i = 0; i < n; i++) {
    recs[i].resize(B.n_inc[i]);
    // rec pointer is constant; copy after the state read (same stream order)
  }
  CK(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < n; i++)
    CK(cudaMemcpyAsync(recs[i].data(), B.h_solves[i].rec, sizeof(Record) * (size_t)B.n_inc[i],
                       cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  {
    CheckRec cr;
    CK(B.prec == EPFFT_FP32 ? read_check<float>(&cr) : read_check<double>(&cr));
    if (cr.code) {
      fprintf(stderr, "epfft: device self-check %d failed (index %lld, bound %lld, at %d)\n", cr.code,
              (long long)cr.index, (long long)cr.bound, cr.where);
      return EPFFT_ERR_CUDA;
    }
  }
  {
    int64_t its = 0;
    for (int i = 0; i < n; i++) its += B.h_solves[i].total_iters;
    c->last.loop_steps = bc.body_iters;
    // per step a column and a row pass; per solve the mask kernel (when
    // generated) and the four labelling kernels
    int64_t k = 2 * bc.body_iters;
    for (int i = 0; i < n; i++) k += (probs[i].mask ? 0 : 1) + 4;
    c->last.kernel_launches = k;
    c->last.iterations = its;
  }
  if (bc.timed_out) return EPFFT_ERR_DEVICE_TIMEOUT;
  bool keep_labels = false;
  if (fields)
    for (int i = 0; i < n; i++) keep_labels |= fields[i].labels != nullptr;
  rc = label_batch(c, A, B, recs, keep_labels);
  if (rc) return rc;
  int status = EPFFT_OK;
  for (int i = 0; i < n; i++) {
    const Solve& S = B.h_solves[i];
    if (S.phase != PH_DONE && S.status == 0) return EPFFT_ERR_DEVICE_TIMEOUT;
    if (records) std::memcpy(records[i], recs[i].data(), sizeof(Record) * (size_t)B.n_inc[i]);
    if (fields) {
      rc = copy_out(c, B, B.h_solves[i], i, &fields[i]);
      if (rc) return rc;
    }
    if (eps_out && eps_out[i])
      CK(cudaMemcpyAsync(eps_out[i], S.eps[S.cur], 4 * (size_t)B.L * B.L * real_size(B.prec),
                         cudaMemcpyDeviceToDevice, c->stream));
    if (iter_rec) std::memcpy(&iter_rec[i], &recs[i][B.n_inc[i] - 1], sizeof(Record));
    for (int k = 0; k < B.n_inc[i]; k++) {
      if (recs[i][k].status == 2) status = EPFFT_ERR_NUMERIC;
      else if (recs[i][k].status == 1 && status == EPFFT_OK) status = EPFFT_NOT_CONVERGED;
    }
  }
  CK(cudaStreamSynchronize(c->stream));
  return status;
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
  cudaStreamSynchronize(c->stream);
  for (auto& t : c->tables) cudaFree(t.second);
  cudaStreamDestroy(c->cap);
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

int epfft_mask(int32_t L, double void_fraction, uint64_t seed, uint8_t* mask_dev, void* stream) {
  if (!is_pow2(L) || L < 4 || L > 4096 || !mask_dev) return EPFFT_ERR_ARG;
  if (!(void_fraction >= 0.0 && void_fraction <= 1.0)) return EPFFT_ERR_ARG;
  if (launch_mask(mask_dev, (int64_t)L * L, seed, void_threshold(void_fraction), (cudaStream_t)stream) !=
      cudaSuccess)
    return EPFFT_ERR_CUDA;
  return EPFFT_OK;
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
  int rc = solve_impl(ctx, 1, &p, &path, nullptr, nullptr, e0, e1, out);
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
  int rc = get_tables(ctx, L, precision, &tw, &ktab);
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
    CK(launch_row_forward<float>(L, ctx->stream, p_dev, spec, tw));
    CK(launch_col<float>(L, 1, ctx->stream, ds, tw, ktab, 0, 0));
    CK(launch_row_inverse<float>(L, ctx->stream, spec, e_dev, tw));
  } else {
    CK(launch_row_forward<double>(L, ctx->stream, p_dev, spec, tw));
    CK(launch_col<double>(L, 1, ctx->stream, ds, tw, ktab, 0, 0));
    CK(launch_row_inverse<double>(L, ctx->stream, spec, e_dev, tw));
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

int epfft_time_passes(epfft_ctx* ctx, const epfft_problem* problem, int32_t n_batch, const double E[4],
                      int32_t n_iter, float* col_ms, float* row_ms) {
  if (!ctx || !problem || !E || n_iter < 1 || n_batch < 1 || !col_ms || !row_ms) return EPFFT_ERR_ARG;
  int rc = check_problem(problem);
  if (rc) return rc;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return EPFFT_ERR_CUDA;
  epfft_problem p = *problem;
  p.tol_eq = 0.0;
  p.tol_macro = 0.0;
  p.max_iter = 1 << 30;
  std::vector<epfft_problem> ps(n_batch, p);
  std::vector<epfft_path> paths(n_batch, epfft_path{1, 0, E});
  Arena A(ctx);
  Batch B;
  rc = setup_batch(ctx, A, B, n_batch, ps.data(), paths.data(), nullptr);
  if (rc) return rc;
  const int nb = n_batch;
  // first row pass: warm start (eps = E, spectrum of its polarization)
  if (B.prec == EPFFT_FP32) CK(launch_row<float>(B.L, nb, ctx->stream, B.d_solves, B.d_ctl, B.tw, 0, 0));
  else CK(launch_row<double>(B.L, nb, ctx->stream, B.d_solves, B.d_ctl, B.tw, 0, 0));
  std::vector<cudaEvent_t> ev(3 * (size_t)n_iter);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  for (int it = 0; it < n_iter; it++) {
    CK(cudaEventRecord(ev[3 * it], ctx->stream));
    if (B.prec == EPFFT_FP32) CK(launch_col<float>(B.L, nb, ctx->stream, B.d_solves, B.tw, B.ktab, 0, 0));
    else CK(launch_col<double>(B.L, nb, ctx->stream, B.d_solves, B.tw, B.ktab, 0, 0));
    CK(cudaEventRecord(ev[3 * it + 1], ctx->stream));
    if (B.prec == EPFFT_FP32) CK(launch_row<float>(B.L, nb, ctx->stream, B.d_solves, B.d_ctl, B.tw, 0, 0));
    else CK(launch_row<double>(B.L, nb, ctx->stream, B.d_solves, B.d_ctl, B.tw, 0, 0));
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

}  // extern "C"
