// Instantiation of the on-chip schedule (onchip.cuh) for its lattice sides.
#include "launch.cuh"
#include "onchip.cuh"

namespace epfft {

#define EPFFT_ONCHIP_FOR_L(X) X(16) X(32) X(64)

bool onchip_supported(int L) {
  switch (L) {
#define X(n) case n: return true;
    EPFFT_ONCHIP_FOR_L(X)
#undef X
    default: return false;
  }
}

cudaError_t prepare_onchip(int L) {
  switch (L) {
#define X(n) \
  case n: return cudaFuncSetAttribute(solve_onchip<n>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OnChip<n>::SMEM);
    EPFFT_ONCHIP_FOR_L(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_onchip(int L, int nb, cudaStream_t s, Solve* solves, BatchCtl* bc, const void* tw,
                          const void* ktab) {
  switch (L) {
#define X(n)                                                                                       \
  case n:                                                                                          \
    solve_onchip<n><<<nb, OnChip<n>::NT, OnChip<n>::SMEM, s>>>(                                    \
        solves, bc, reinterpret_cast<const C2<float>*>(tw), reinterpret_cast<const C2<float>*>(ktab)); \
    return cudaGetLastError();
    EPFFT_ONCHIP_FOR_L(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t check_record_onchip(void** out) {
#ifdef EPFFT_CHECKS
  return cudaGetSymbolAddress(out, g_check);
#else
  *out = nullptr;
  return cudaSuccess;
#endif
}

cudaError_t read_check_onchip(CheckRec* out) {
#ifdef EPFFT_CHECKS
  cudaError_t e = cudaMemcpyFromSymbol(out, g_check, sizeof(CheckRec));
  if (e != cudaSuccess || out->code == 0) return e;  // a clear record needs no clearing
  CheckRec z = {};
  return cudaMemcpyToSymbol(g_check, &z, sizeof(CheckRec));
#else
  *out = CheckRec{};
  return cudaSuccess;
#endif
}

}  // namespace epfft
