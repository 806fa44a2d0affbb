// Instantiation of the defect-correction kernels (dcpass.cuh) for one
// tiling variant EPFFT_VAR over the supported lattice sides: the row pass
// on the FP32 differences, and the FP64 steps of a refresh.
#pragma once
#include "dcpass.cuh"
#include "launch.cuh"

namespace epfft {

// every side of the FP32 and FP64 builds (the refresh runs FP64 transforms)
#define EPFFT_DEF_FOR_L(X) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)

template <int L>
static cudaError_t prepare_def_L() {
  constexpr int V = EPFFT_VAR;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(row_pass_dc<L, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Cfg<float, L, V>::ROW_SMEM)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(dc_ref_forward<L, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Cfg<double, L, V>::ROW_SMEM)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(dc_ref_inverse<L, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Cfg<double, L, V>::ROW_SMEM);
}

template <>
cudaError_t prepare_def_v<EPFFT_VAR>(int L) {
  switch (L) {
#define X(n) case n: return prepare_def_L<n>();
    EPFFT_DEF_FOR_L(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_row_def_v<EPFFT_VAR>(int L, int nb, cudaStream_t s, Solve* solves, BatchCtl* bc, const void* tw,
                                       cudaGraphConditionalHandle cond, int use_cond,
                                       cudaGraphConditionalHandle rcond, int use_rcond) {
  switch (L) {
#define X(n)                                                                                             \
  case n: {                                                                                              \
    using C = Cfg<float, n, EPFFT_VAR>;                                                                  \
    row_pass_dc<n, EPFFT_VAR><<<dim3(n / C::RR, nb), C::NT_ROW, C::ROW_SMEM, s>>>(                      \
        solves, nb, bc, reinterpret_cast<const C2<float>*>(tw), cond, use_cond, rcond, use_rcond);       \
    return cudaGetLastError();                                                                           \
  }
    EPFFT_DEF_FOR_L(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_ref_forward_v<EPFFT_VAR>(int L, int nb, cudaStream_t s, Solve* solves, Solve* shadow,
                                           const void* tw64) {
  switch (L) {
#define X(n)                                                                                             \
  case n: {                                                                                              \
    using C = Cfg<double, n, EPFFT_VAR>;                                                                 \
    dc_ref_forward<n, EPFFT_VAR><<<dim3(n / C::RR, nb), C::NT_ROW, C::ROW_SMEM, s>>>(                   \
        solves, shadow, reinterpret_cast<const C2<double>*>(tw64));                                      \
    return cudaGetLastError();                                                                           \
  }
    EPFFT_DEF_FOR_L(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_ref_inverse_v<EPFFT_VAR>(int L, int nb, cudaStream_t s, Solve* solves, const void* tw64) {
  switch (L) {
#define X(n)                                                                                             \
  case n: {                                                                                              \
    using C = Cfg<double, n, EPFFT_VAR>;                                                                 \
    dc_ref_inverse<n, EPFFT_VAR><<<dim3(n / C::RR, nb), C::NT_ROW, C::ROW_SMEM, s>>>(                   \
        solves, reinterpret_cast<const C2<double>*>(tw64));                                              \
    return cudaGetLastError();                                                                           \
  }
    EPFFT_DEF_FOR_L(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_ref_sums_v<EPFFT_VAR>(int L, int nb, cudaStream_t s, Solve* solves) {
  switch (L) {
#define X(n)                                                  \
  case n: {                                                   \
    dc_ref_sums<n, EPFFT_VAR, 128><<<nb, 128, 0, s>>>(solves); \
    return cudaGetLastError();                                \
  }
    EPFFT_DEF_FOR_L(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t check_record_def_v<EPFFT_VAR>(void** out) {
#ifdef EPFFT_CHECKS
  return cudaGetSymbolAddress(out, g_check);
#else
  *out = nullptr;
  return cudaSuccess;
#endif
}

template <>
cudaError_t read_check_def_v<EPFFT_VAR>(CheckRec* out) {
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
