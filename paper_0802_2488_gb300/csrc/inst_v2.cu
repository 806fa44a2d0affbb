// Tiling variant 2: the register-staged row pass (rowrs.cuh) with the
// register-staged column pass on its digit-reversed spectrum order
// (colrs.cuh), FP32 lattice sides 256 .. 4096.  FP64 and the other sides
// have no variant 2 (pass_shape returns false; the autotuner skips it).
#include "launch.cuh"
#include "rowrs.cuh"

namespace epfft {

#define EPFFT_V2_FOR_L(X) X(256) X(512) X(1024) X(2048) X(4096)

template <int L>
static bool shape_v2(PassShape* o) {
  using CF = RowRsCfg<L>;
  using RC = RsCfg<L, CF::W>;
  o->rows_per_cta = CF::RR;
  o->tile_w = CF::W;
  o->row_ctas = L / CF::RR;
  o->col_ctas = (L / 2) / RC::CPC;
  o->nt_row = CF::NT;
  o->nt_col = RC::NT;
  o->row_smem = CF::SMEM;
  o->col_smem = RC::SMEM;
  return true;
}

template <int L>
static cudaError_t prepare_v2() {
  using CF = RowRsCfg<L>;
  using RC = RsCfg<L, CF::W>;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(row_pass_rs<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CF::SMEM)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(row_forward_rs<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CF::SMEM)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(row_inverse_rs<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CF::SMEM)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(col_pass_rs<L, CF::W, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RC::SMEM)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(col_pass_rs<L, CF::W, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RC::SMEM);
}

template <int L>
static const C2<float>* row_tables(const void* tw) {
  return reinterpret_cast<const C2<float>*>(tw) + Tables<float, L>::RROFF;
}

template <>
bool pass_shape_v<float, 2>(int L, PassShape* out) {
  switch (L) {
#define X(n) case n: return shape_v2<n>(out);
    EPFFT_V2_FOR_L(X)
#undef X
    default: return false;
  }
}

template <>
cudaError_t prepare_v<float, 2>(int L) {
  switch (L) {
#define X(n) case n: return prepare_v2<n>();
    EPFFT_V2_FOR_L(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_row_v<float, 2>(int L, int nb, cudaStream_t s, Solve* solves, BatchCtl* bc, const void* tw,
                                   cudaGraphConditionalHandle cond, int use_cond) {
  switch (L) {
#define X(n)                                                                                               \
  case n: {                                                                                                \
    using CF = RowRsCfg<n>;                                                                                \
    row_pass_rs<n><<<dim3(n / CF::RR, nb), CF::NT, CF::SMEM, s>>>(solves, nb, bc, row_tables<n>(tw), cond, use_cond); \
    return cudaGetLastError();                                                                             \
  }
    EPFFT_V2_FOR_L(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_col_v<float, 2>(int L, int nb, cudaStream_t s, Solve* solves, const void* tw, const void* ktab,
                                   cudaGraphConditionalHandle cond, int use_cond, int general) {
  switch (L) {
#define X(n)                                                                                               \
  case n: {                                                                                                \
    using CF = RowRsCfg<n>;                                                                                \
    using RC = RsCfg<n, CF::W>;                                                                            \
    const dim3 grid((n / 2) / RC::CPC, nb);                                                                \
    const C2<float>* k_ = reinterpret_cast<const C2<float>*>(ktab);                                        \
    const C2<float>* tws = reinterpret_cast<const C2<float>*>(tw) + Tables<float, n>::RSOFF;               \
    if (general)                                                                                           \
      col_pass_rs<n, CF::W, true, true><<<grid, RC::NT, RC::SMEM, s>>>(solves, k_, tws, cond, use_cond);   \
    else                                                                                                   \
      col_pass_rs<n, CF::W, false, true><<<grid, RC::NT, RC::SMEM, s>>>(solves, k_, tws, cond, use_cond);  \
    return cudaGetLastError();                                                                             \
  }
    EPFFT_V2_FOR_L(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_row_forward_v<float, 2>(int L, cudaStream_t s, const void* p, void* spec, const void* tw) {
  switch (L) {
#define X(n)                                                                                               \
  case n: {                                                                                                \
    using CF = RowRsCfg<n>;                                                                                \
    row_forward_rs<n><<<n / CF::RR, CF::NT, CF::SMEM, s>>>(reinterpret_cast<const float*>(p),              \
                                                           reinterpret_cast<C2<float>*>(spec), row_tables<n>(tw)); \
    return cudaGetLastError();                                                                             \
  }
    EPFFT_V2_FOR_L(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_row_inverse_v<float, 2>(int L, cudaStream_t s, const void* spec, void* e, const void* tw) {
  switch (L) {
#define X(n)                                                                                               \
  case n: {                                                                                                \
    using CF = RowRsCfg<n>;                                                                                \
    row_inverse_rs<n><<<n / CF::RR, CF::NT, CF::SMEM, s>>>(reinterpret_cast<const C2<float>*>(spec),       \
                                                           reinterpret_cast<float*>(e), row_tables<n>(tw)); \
    return cudaGetLastError();                                                                             \
  }
    EPFFT_V2_FOR_L(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t check_record_v<float, 2>(void** out) {
#ifdef EPFFT_CHECKS
  return cudaGetSymbolAddress(out, g_check);
#else
  *out = nullptr;
  return cudaSuccess;
#endif
}

template <>
cudaError_t read_check_v<float, 2>(CheckRec* out) {
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

// no FP64 variant 2
template <>
bool pass_shape_v<double, 2>(int, PassShape*) { return false; }
template <>
cudaError_t prepare_v<double, 2>(int) { return cudaErrorInvalidValue; }
template <>
cudaError_t launch_row_v<double, 2>(int, int, cudaStream_t, Solve*, BatchCtl*, const void*, cudaGraphConditionalHandle, int) {
  return cudaErrorInvalidValue;
}
template <>
cudaError_t launch_col_v<double, 2>(int, int, cudaStream_t, Solve*, const void*, const void*, cudaGraphConditionalHandle,
                                    int, int) {
  return cudaErrorInvalidValue;
}
template <>
cudaError_t launch_row_forward_v<double, 2>(int, cudaStream_t, const void*, void*, const void*) { return cudaErrorInvalidValue; }
template <>
cudaError_t launch_row_inverse_v<double, 2>(int, cudaStream_t, const void*, void*, const void*) { return cudaErrorInvalidValue; }
template <>
cudaError_t read_check_v<double, 2>(CheckRec* out) {
  *out = CheckRec{};
  return cudaSuccess;
}
template <>
cudaError_t check_record_v<double, 2>(void** out) {
  *out = nullptr;
  return cudaSuccess;
}

}  // namespace epfft
