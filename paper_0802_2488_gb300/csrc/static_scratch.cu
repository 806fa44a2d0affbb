// epfft_project_static: the compatible-strain projection for callers that
// cannot allocate device memory.
//
// Its working memory (the half spectrum, the twiddle and Fourier-symbol
// tables, the solve record read by the column pass and the prescribed mean
// strain) lives in one file-scope device array of fixed size, so the call
// needs no cudaMalloc, cudaFree or allocating library routine.  The array is
// part of the library image: every GPU that loads the library holds it
// until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/epfft.h"
#include "launch.cuh"
#include "tables.cuh"

using namespace epfft;

namespace {

constexpr int kMaxL = 256;  // largest lattice side the static scratch holds
constexpr size_t kSpecBytes = (size_t)3 * kMaxL * (kMaxL / 2) * 16;  // 3 components, FP64 complex
// device tables of the largest side in FP64 (the largest of all sides and types)
constexpr size_t kTabBytes = ((size_t)Tables<double, kMaxL>::TOTAL * 16 + 255) / 256 * 256;
constexpr size_t kSolveBytes = 512;
constexpr size_t kPathBytes = 256;
constexpr size_t kScratchBytes = kSpecBytes + kTabBytes + kSolveBytes + kPathBytes;
static_assert(sizeof(Solve) <= kSolveBytes, "solve record must fit its slot");
static_assert(kSpecBytes % 256 == 0 && kTabBytes % 256 == 0, "slots stay 256-byte aligned");
static_assert(Tables<double, 128>::TOTAL <= Tables<double, kMaxL>::TOTAL &&
                  Tables<float, kMaxL>::TOTAL <= Tables<double, kMaxL>::TOTAL,
              "the table slot holds every side up to kMaxL");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices];  // device address of g_scratch, per device (set up on first use)

}  // namespace

// 1.59 MB (kScratchBytes) of device memory, shared by every call on a device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

namespace {

// Device address of the scratch array on the current device.  The array's
// name in host code is only a stand-in; the address comes from
// cudaGetSymbolAddress, once per device, with that device current.
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return EPFFT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return EPFFT_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return EPFFT_OK;
}

template <typename T>
int project_static(int L, double lambda0, double mu0, const double E[4], const void* p, void* e, cudaStream_t s) {
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  char* spec = (char*)base;
  char* tab = spec + kSpecBytes;
  char* solve = tab + kTabBytes;
  char* path = solve + kSolveBytes;
  std::vector<T> h;  // host copy of the device tables of L
  const int koff = host_tables<T>(L, h);
  if (koff < 0 || h.size() * sizeof(T) > kTabBytes) return EPFFT_ERR_ARG;
  Solve S;
  std::memset(&S, 0, sizeof(S));
  S.lam0 = lambda0;
  S.mu0 = mu0;
  S.path = (const double*)path;
  S.spec = spec;
  S.phase = PH_ITER;
  if (prepare<T>(L, 0) != cudaSuccess) return EPFFT_ERR_CUDA;
  if (cudaMemcpyAsync(tab, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return EPFFT_ERR_CUDA;
  if (cudaMemcpyAsync(path, E, 4 * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess) return EPFFT_ERR_CUDA;
  if (cudaMemcpyAsync(solve, &S, sizeof(S), cudaMemcpyHostToDevice, s) != cudaSuccess) return EPFFT_ERR_CUDA;
  const void* tw = tab;
  const void* ktab = tab + sizeof(T) * 2 * koff;
  if (launch_row_forward<T>(L, 0, s, p, spec, tw) != cudaSuccess) return EPFFT_ERR_CUDA;
  if (launch_col<T>(L, 0, 1, s, (Solve*)solve, tw, ktab, 0, 0) != cudaSuccess) return EPFFT_ERR_CUDA;
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
