// epfft_project_static: the compatible-strain projection for callers that
// cannot allocate device memory.
//
// Its working memory (the half spectrum, the twiddle and Fourier-symbol
// tables of every side up to kMaxL, the solve record read by the column pass
// and the prescribed mean strain) lives in one file-scope device array of
// fixed size, so the call needs no cudaMalloc, cudaFree or allocating library
// routine.  The array belongs to the library's device code: the first call on
// a device loads that code onto the device (which places the array there)
// and the array stays until the process exits.
//
// Set-up, once per device on the first call (with that device current):
// the array's device address is looked up, the tables of every side and
// precision are uploaded into it (a blocking copy) and the kernels' shared
// memory limits are raised.  After that a call only launches kernels: a
// one-thread kernel writes the solve record and the mean strain from its
// by-value arguments, then the three transform passes run.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/epfft.h"
#include "launch.cuh"
#include "tables.cuh"

using namespace epfft;

namespace {

constexpr int kMaxL = 256;  // largest lattice side the static scratch holds
constexpr int kLogMin = 2, kLogMax = 8;  // sides 4 .. 256
constexpr size_t kSpecBytes = (size_t)3 * kMaxL * (kMaxL / 2) * 16;  // 3 components, FP64 complex

template <typename T, int L>
constexpr size_t tab_bytes() {
  return ((size_t)Tables<T, L>::TOTAL * sizeof(C2<T>) + 255) / 256 * 256;
}
template <typename T>
constexpr size_t tab_bytes_all() {
  return tab_bytes<T, 4>() + tab_bytes<T, 8>() + tab_bytes<T, 16>() + tab_bytes<T, 32>() + tab_bytes<T, 64>() +
         tab_bytes<T, 128>() + tab_bytes<T, 256>();
}
// the tables of every side up to kMaxL in both precisions, one after another
constexpr size_t kTabBytes = tab_bytes_all<float>() + tab_bytes_all<double>();
constexpr size_t kSolveBytes = 768;
constexpr size_t kPathBytes = 256;
constexpr size_t kScratchBytes = kSpecBytes + kTabBytes + kSolveBytes + kPathBytes;
static_assert(sizeof(Solve) <= kSolveBytes, "solve record must fit its slot");
static_assert(kSpecBytes % 256 == 0 && kTabBytes % 256 == 0, "slots stay 256-byte aligned");

constexpr int kMaxDevices = 64;
struct DeviceSetup {
  bool done = false;
  char* base = nullptr;  // device address of g_scratch on this device
};
std::mutex g_mu;
DeviceSetup g_dev[kMaxDevices];
// byte offset of the tables of (log2 L, precision 0 = FP32 / 1 = FP64) in the
// table region, and of k(m) within them (complex units); the same on every
// device
size_t g_tab_off[kLogMax + 1][2];
int g_koff[kLogMax + 1][2];

}  // namespace

// kScratchBytes (1.62 MB) of device memory, shared by every call on a device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

namespace {

// Writes the solve record the column pass reads (reference medium, mean
// strain, spectrum) and the mean strain E.  One thread.
__global__ void static_init_kernel(Solve* S, double* path, void* spec, double lam0, double mu0, double E0,
                                   double E1, double E2, double E3) {
  Solve s{};
  s.lam0 = lam0;
  s.mu0 = mu0;
  s.path = path;
  s.spec = spec;
  s.phase = PH_ITER;
  *S = s;
  path[0] = E0;
  path[1] = E1;
  path[2] = E2;
  path[3] = E3;
}

template <typename T>
int upload_tables(int prec_i, std::vector<unsigned char>& host) {
  size_t off = prec_i == 0 ? 0 : tab_bytes_all<float>();
  for (int lg = kLogMin; lg <= kLogMax; lg++) {
    const int L = 1 << lg;
    std::vector<T> h;
    const int koff = host_tables<T>(L, h);
    if (koff < 0) return EPFFT_ERR_UNSUPPORTED;
    const size_t bytes = h.size() * sizeof(T);
    if (off + bytes > kTabBytes) return EPFFT_ERR_CUDA;
    std::memcpy(host.data() + off, h.data(), bytes);
    g_tab_off[lg][prec_i] = off;
    g_koff[lg][prec_i] = koff;
    off += (bytes + 255) / 256 * 256;
    if (prepare<T>(L, 0) != cudaSuccess) return EPFFT_ERR_CUDA;
  }
  return EPFFT_OK;
}

// Set-up of the current device (once): the array's device address, the
// tables and the kernels' shared-memory limits.  The array's name in host
// code is only a stand-in; its address comes from cudaGetSymbolAddress,
// with the device current.
int setup_device(char** base) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return EPFFT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceSetup& D = g_dev[dev];
  if (!D.done) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return EPFFT_ERR_CUDA;
    }
    char* tab = (char*)p + kSpecBytes;
    std::vector<unsigned char> host(kTabBytes, 0);
    int rc = upload_tables<float>(0, host);
    if (!rc) rc = upload_tables<double>(1, host);
    if (rc) return rc;
    if (cudaMemcpy(tab, host.data(), kTabBytes, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      return EPFFT_ERR_CUDA;
    }
    D.base = (char*)p;
    D.done = true;
  }
  *base = D.base;
  return EPFFT_OK;
}

template <typename T>
int project_static(int L, double lambda0, double mu0, const double E[4], const void* p, void* e, cudaStream_t s) {
  PassShape sh;
  if (!pass_shape<T>(L, 0, &sh)) return EPFFT_ERR_UNSUPPORTED;
  char* base = nullptr;
  int rc = setup_device(&base);
  if (rc) return rc;
  int lg = 0;
  while ((1 << lg) < L) lg++;
  const int pi = sizeof(T) == 4 ? 0 : 1;
  char* spec = base;
  char* tab = base + kSpecBytes + g_tab_off[lg][pi];
  Solve* solve = (Solve*)(base + kSpecBytes + kTabBytes);
  double* path = (double*)(base + kSpecBytes + kTabBytes + kSolveBytes);
  static_init_kernel<<<1, 1, 0, s>>>(solve, path, spec, lambda0, mu0, E[0], E[1], E[2], E[3]);
  if (cudaGetLastError() != cudaSuccess) return EPFFT_ERR_CUDA;
  const void* tw = tab;
  const void* ktab = tab + sizeof(T) * 2 * (size_t)g_koff[lg][pi];
  if (launch_row_forward<T>(L, 0, s, p, spec, tw) != cudaSuccess) return EPFFT_ERR_CUDA;
  if (launch_col<T>(L, 0, 1, s, solve, tw, ktab, 0, 0) != cudaSuccess) return EPFFT_ERR_CUDA;
  if (launch_row_inverse<T>(L, 0, s, spec, e, tw) != cudaSuccess) return EPFFT_ERR_CUDA;
  return EPFFT_OK;
}

}  // namespace

extern "C" int epfft_project_static(int32_t L, int32_t precision, double lambda0, double mu0, const double E[4],
                                    const void* p_dev, void* e_dev, void* stream) {
  if (!E || !p_dev || !e_dev) return EPFFT_ERR_ARG;
  if (L < 4 || (L & (L - 1)) != 0) return EPFFT_ERR_ARG;
  if (precision != EPFFT_FP32 && precision != EPFFT_FP64) return EPFFT_ERR_ARG;
  if (L > kMaxL) return EPFFT_ERR_SCRATCH_LIMIT;
  if (!(mu0 > 0.0) || !(lambda0 + 2.0 * mu0 / 3.0 > 0.0)) return EPFFT_ERR_ARG;
  for (int k = 0; k < 4; k++)
    if (!std::isfinite(E[k])) return EPFFT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  return precision == EPFFT_FP32 ? project_static<float>(L, lambda0, mu0, E, p_dev, e_dev, s)
                                 : project_static<double>(L, lambda0, mu0, E, p_dev, e_dev, s);
}
