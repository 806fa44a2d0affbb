// Instantiation of the launch table for one real type EPFFT_REAL and one
// tiling variant EPFFT_VAR over the supported lattice sides.
#pragma once
#include <type_traits>

#include "colrs.cuh"
#include "launch.cuh"
#include "passes.cuh"

namespace epfft {

#define EPFFT_FOR_L(X) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) EPFFT_L4096(X)

template <typename T, int L>
static bool shape_of(PassShape* o) {
  using C = Cfg<T, L, EPFFT_VAR>;
  o->rows_per_cta = C::RR;
  o->tile_w = C::W;
  o->row_ctas = L / C::RR;
  o->col_ctas = (L / 2) / C::W;
  o->nt_row = C::NT_ROW;
  o->nt_col = C::NT_COL;
  o->row_smem = C::ROW_SMEM;
  o->col_smem = C::COL_SMEM;
  return true;
}

// The column pass of tiling 0 for FP32 lattices of side >= 128 is the
// register-staged kernel (colrs.cuh), which puts several columns in a CTA;
// tiling 1 (many small CTAs, for launches of few pixels) keeps col_pass, as
// do FP64 and smaller sides.
template <typename T, int L>
constexpr bool kRegisterStaged = std::is_same<T, float>::value && L >= 128 && EPFFT_VAR == 0;

// Column-pass CTAs resident on the GPU at once, per lattice side (index
// log2 L), measured at preparation: a CTA prefetches the slab of the CTA
// that many places after it in launch order.
static int g_col_succ[16];

template <typename T, int L>
static cudaError_t prepare_L() {
  using C = Cfg<T, L, EPFFT_VAR>;
  constexpr int V = EPFFT_VAR;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(row_pass<T, L, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::ROW_SMEM)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(col_pass<T, L, V, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::COL_SMEM)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(col_pass<T, L, V, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::COL_SMEM)) != cudaSuccess) return e;
  if constexpr (kRegisterStaged<T, L>) {
    using RC = RsCfg<L, C::W>;
    if ((e = cudaFuncSetAttribute(col_pass_rs<L, C::W, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RC::SMEM)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(col_pass_rs<L, C::W, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RC::SMEM)) != cudaSuccess) return e;
  }
  {
    int dev = 0, nsm = 0, occ = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, col_pass<T, L, V, false>, C::NT_COL, C::COL_SMEM)) != cudaSuccess)
      return e;
    g_col_succ[ilog2c(L)] = nsm * occ;
  }
  if ((e = cudaFuncSetAttribute(row_forward<T, L, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::ROW_SMEM)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(row_inverse<T, L, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::ROW_SMEM);
}

template <>
bool pass_shape_v<EPFFT_REAL, EPFFT_VAR>(int L, PassShape* out) {
  switch (L) {
#define X(n) case n: return shape_of<EPFFT_REAL, n>(out);
    EPFFT_FOR_L(X)
#undef X
    default: return false;
  }
}

template <>
cudaError_t prepare_v<EPFFT_REAL, EPFFT_VAR>(int L) {
  switch (L) {
#define X(n) case n: return prepare_L<EPFFT_REAL, n>();
    EPFFT_FOR_L(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_row_v<EPFFT_REAL, EPFFT_VAR>(int L, int nb, cudaStream_t s, Solve* solves, BatchCtl* bc, const void* tw,
                                   cudaGraphConditionalHandle cond, int use_cond) {
  switch (L) {
#define X(n)                                                                                         \
  case n: {                                                                                          \
    using C = Cfg<EPFFT_REAL, n, EPFFT_VAR>;                                                                    \
    row_pass<EPFFT_REAL, n, EPFFT_VAR><<<dim3(n / C::RR, nb), C::NT_ROW, C::ROW_SMEM, s>>>(                     \
        solves, nb, bc, reinterpret_cast<const C2<EPFFT_REAL>*>(tw), cond, use_cond);                \
    return cudaGetLastError();                                                                       \
  }
    EPFFT_FOR_L(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int L>
static cudaError_t launch_col_L(int nb, cudaStream_t s, Solve* solves, const void* tw, const void* ktab,
                                cudaGraphConditionalHandle cond, int use_cond, int general) {
  using C = Cfg<T, L, EPFFT_VAR>;
  const C2<T>* tw_ = reinterpret_cast<const C2<T>*>(tw);
  const C2<T>* k_ = reinterpret_cast<const C2<T>*>(ktab);
  if constexpr (kRegisterStaged<T, L>) {
    using RC = RsCfg<L, C::W>;
    const dim3 grid((L / 2) / RC::CPC, nb);
    const C2<float>* tws = tw_ + Tables<float, L>::RSOFF;
    if (general)
      col_pass_rs<L, C::W, true, false><<<grid, RC::NT, RC::SMEM, s>>>(solves, k_, tws, cond, use_cond);
    else
      col_pass_rs<L, C::W, false, false><<<grid, RC::NT, RC::SMEM, s>>>(solves, k_, tws, cond, use_cond);
  } else {
    const dim3 grid((L / 2) / C::W, nb);
    if (general)
      col_pass<T, L, EPFFT_VAR, true><<<grid, C::NT_COL, C::COL_SMEM, s>>>(solves, tw_, k_, cond, use_cond, g_col_succ[ilog2c(L)]);
    else
      col_pass<T, L, EPFFT_VAR, false><<<grid, C::NT_COL, C::COL_SMEM, s>>>(solves, tw_, k_, cond, use_cond, g_col_succ[ilog2c(L)]);
  }
  return cudaGetLastError();
}

template <>
cudaError_t launch_col_v<EPFFT_REAL, EPFFT_VAR>(int L, int nb, cudaStream_t s, Solve* solves, const void* tw, const void* ktab,
                                   cudaGraphConditionalHandle cond, int use_cond, int general) {
  switch (L) {
#define X(n) case n: return launch_col_L<EPFFT_REAL, n>(nb, s, solves, tw, ktab, cond, use_cond, general);
    EPFFT_FOR_L(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_row_forward_v<EPFFT_REAL, EPFFT_VAR>(int L, cudaStream_t s, const void* p, void* spec, const void* tw) {
  switch (L) {
#define X(n)                                                                                         \
  case n: {                                                                                          \
    using C = Cfg<EPFFT_REAL, n, EPFFT_VAR>;                                                                    \
    row_forward<EPFFT_REAL, n, EPFFT_VAR><<<n / C::RR, C::NT_ROW, C::ROW_SMEM, s>>>(                            \
        reinterpret_cast<const EPFFT_REAL*>(p), reinterpret_cast<C2<EPFFT_REAL>*>(spec),             \
        reinterpret_cast<const C2<EPFFT_REAL>*>(tw));                                                \
    return cudaGetLastError();                                                                       \
  }
    EPFFT_FOR_L(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_row_inverse_v<EPFFT_REAL, EPFFT_VAR>(int L, cudaStream_t s, const void* spec, void* e, const void* tw) {
  switch (L) {
#define X(n)                                                                                         \
  case n: {                                                                                          \
    using C = Cfg<EPFFT_REAL, n, EPFFT_VAR>;                                                                    \
    row_inverse<EPFFT_REAL, n, EPFFT_VAR><<<n / C::RR, C::NT_ROW, C::ROW_SMEM, s>>>(                            \
        reinterpret_cast<const C2<EPFFT_REAL>*>(spec), reinterpret_cast<EPFFT_REAL*>(e),             \
        reinterpret_cast<const C2<EPFFT_REAL>*>(tw));                                                \
    return cudaGetLastError();                                                                       \
  }
    EPFFT_FOR_L(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t check_record_v<EPFFT_REAL, EPFFT_VAR>(void** out) {
#ifdef EPFFT_CHECKS
  return cudaGetSymbolAddress(out, g_check);
#else
  *out = nullptr;
  return cudaSuccess;
#endif
}

template <>
cudaError_t read_check_v<EPFFT_REAL, EPFFT_VAR>(CheckRec* out) {
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
