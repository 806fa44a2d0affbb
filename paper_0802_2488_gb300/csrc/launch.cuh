// Launch table of the fused passes.  Each (real type, tiling variant) pair
// is instantiated for every supported lattice side in its own translation
// unit (inst_f32_v0.cu ... inst_f64_v1.cu, inst_v2.cu); the functions below
// dispatch on the variant at run time.  Variants 0 and 1 are two tilings of
// the shared-memory Stockham row pass (passes.cuh): variant 0 (fewer, larger
// CTAs) with the register-staged column pass for FP32 sides >= 128
// (colrs.cuh), variant 1 (many small CTAs, for launches of few pixels) with
// the Stockham column pass; variant 2 is the register-staged row and column
// passes with the digit-reversed spectrum order (rowrs.cuh), FP32 sides
// 256 .. 4096 only.
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace epfft {

// tilings 0-2 of the two passes and the on-chip schedule (3)
constexpr int N_VARIANTS = 4;

struct PassShape {
  int rows_per_cta, tile_w;  // RR, W
  int row_ctas, col_ctas;    // per solve
  int nt_row, nt_col;
  size_t row_smem, col_smem;
};

template <typename T, int V>
bool pass_shape_v(int L, PassShape* out);
template <typename T, int V>
cudaError_t prepare_v(int L);
template <typename T, int V>
cudaError_t launch_row_v(int L, int nb, cudaStream_t s, Solve* solves, BatchCtl* bc, const void* tw,
                         cudaGraphConditionalHandle cond, int use_cond);
// general = 0: every solve of the launch uses the Eq. 3 operator (the
// specialised kernel); 1: each solve's own operator
template <typename T, int V>
cudaError_t launch_col_v(int L, int nb, cudaStream_t s, Solve* solves, const void* tw, const void* ktab,
                         cudaGraphConditionalHandle cond, int use_cond, int general);
template <typename T, int V>
cudaError_t launch_row_forward_v(int L, cudaStream_t s, const void* p, void* spec, const void* tw);
template <typename T, int V>
cudaError_t launch_row_inverse_v(int L, cudaStream_t s, const void* spec, void* e, const void* tw);
// Reads and clears the self-check record of one translation unit (zero
// unless built with EPFFT_CHECKS).
template <typename T, int V>
cudaError_t read_check_v(CheckRec* out);
// Device address of that record (null without EPFFT_CHECKS), for reads
// enqueued on a stream.
template <typename T, int V>
cudaError_t check_record_v(void** out);

// Defect-correction form (dcpass.cuh), tilings 0 and 1: the row pass on the
// FP32 differences (the FP32 tile shapes of tiling V; its column pass is the
// FP32 one), and the FP64 steps of a refresh (the FP64 tile shapes of tiling
// V: forward row half, the FP64 column pass, inverse row half, the sums).
constexpr int N_DEF_VARIANTS = 2;
template <int V>
cudaError_t prepare_def_v(int L);
template <int V>
cudaError_t launch_row_def_v(int L, int nb, cudaStream_t s, Solve* solves, BatchCtl* bc, const void* tw,
                             cudaGraphConditionalHandle cond, int use_cond, cudaGraphConditionalHandle rcond,
                             int use_rcond);
template <int V>
cudaError_t launch_ref_forward_v(int L, int nb, cudaStream_t s, Solve* solves, Solve* shadow, const void* tw64);
template <int V>
cudaError_t launch_ref_inverse_v(int L, int nb, cudaStream_t s, Solve* solves, const void* tw64);
template <int V>
cudaError_t launch_ref_sums_v(int L, int nb, cudaStream_t s, Solve* solves);
template <int V>
cudaError_t read_check_def_v(CheckRec* out);
template <int V>
cudaError_t check_record_def_v(void** out);

template <int D = 0>  // a template, so that the variants may be specialised after it
inline cudaError_t prepare_def(int L, int var) {
  switch (var) {
    case 0: return prepare_def_v<0>(L);
    case 1: return prepare_def_v<1>(L);
    default: return cudaErrorInvalidValue;
  }
}
template <int D = 0>  // a template, so that the variants may be specialised after it
inline cudaError_t launch_row_def(int L, int var, int nb, cudaStream_t s, Solve* solves, BatchCtl* bc,
                                  const void* tw, cudaGraphConditionalHandle cond, int use_cond,
                                  cudaGraphConditionalHandle rcond, int use_rcond) {
  switch (var) {
    case 0: return launch_row_def_v<0>(L, nb, s, solves, bc, tw, cond, use_cond, rcond, use_rcond);
    case 1: return launch_row_def_v<1>(L, nb, s, solves, bc, tw, cond, use_cond, rcond, use_rcond);
    default: return cudaErrorInvalidValue;
  }
}
template <int D = 0>  // a template, so that the variants may be specialised after it
inline cudaError_t launch_ref_forward(int L, int var64, int nb, cudaStream_t s, Solve* solves, Solve* shadow,
                                      const void* tw64) {
  switch (var64) {
    case 0: return launch_ref_forward_v<0>(L, nb, s, solves, shadow, tw64);
    case 1: return launch_ref_forward_v<1>(L, nb, s, solves, shadow, tw64);
    default: return cudaErrorInvalidValue;
  }
}
template <int D = 0>  // a template, so that the variants may be specialised after it
inline cudaError_t launch_ref_inverse(int L, int var64, int nb, cudaStream_t s, Solve* solves, const void* tw64) {
  switch (var64) {
    case 0: return launch_ref_inverse_v<0>(L, nb, s, solves, tw64);
    case 1: return launch_ref_inverse_v<1>(L, nb, s, solves, tw64);
    default: return cudaErrorInvalidValue;
  }
}

template <int D = 0>
inline cudaError_t launch_ref_sums(int L, int var64, int nb, cudaStream_t s, Solve* solves) {
  switch (var64) {
    case 0: return launch_ref_sums_v<0>(L, nb, s, solves);
    case 1: return launch_ref_sums_v<1>(L, nb, s, solves);
    default: return cudaErrorInvalidValue;
  }
}

// On-chip schedule (onchip.cuh, tiling 3): FP32 whole solves, one CTA per
// solve, for the sides onchip_supported accepts.
constexpr int ONCHIP_VARIANT = 3;
bool onchip_supported(int L);
cudaError_t prepare_onchip(int L);
cudaError_t launch_onchip(int L, int nb, cudaStream_t s, Solve* solves, BatchCtl* bc, const void* tw,
                          const void* ktab);
cudaError_t read_check_onchip(CheckRec* out);
cudaError_t check_record_onchip(void** out);

// Returns false when L is not built for T in that variant.
template <typename T>
inline bool pass_shape(int L, int var, PassShape* out) {
  switch (var) {
    case 0: return pass_shape_v<T, 0>(L, out);
    case 1: return pass_shape_v<T, 1>(L, out);
    case 2: return pass_shape_v<T, 2>(L, out);
    default: return false;
  }
}
// Raises the dynamic shared-memory limit of the kernels for L (call before
// any launch or capture).
template <typename T>
inline cudaError_t prepare(int L, int var) {
  switch (var) {
    case 0: return prepare_v<T, 0>(L);
    case 1: return prepare_v<T, 1>(L);
    case 2: return prepare_v<T, 2>(L);
    default: return cudaErrorInvalidValue;
  }
}
template <typename T>
inline cudaError_t launch_row(int L, int var, int nb, cudaStream_t s, Solve* solves, BatchCtl* bc, const void* tw,
                              cudaGraphConditionalHandle cond, int use_cond) {
  switch (var) {
    case 0: return launch_row_v<T, 0>(L, nb, s, solves, bc, tw, cond, use_cond);
    case 1: return launch_row_v<T, 1>(L, nb, s, solves, bc, tw, cond, use_cond);
    case 2: return launch_row_v<T, 2>(L, nb, s, solves, bc, tw, cond, use_cond);
    default: return cudaErrorInvalidValue;
  }
}
template <typename T>
inline cudaError_t launch_col(int L, int var, int nb, cudaStream_t s, Solve* solves, const void* tw,
                              const void* ktab, cudaGraphConditionalHandle cond, int use_cond, int general = 0) {
  switch (var) {
    case 0: return launch_col_v<T, 0>(L, nb, s, solves, tw, ktab, cond, use_cond, general);
    case 1: return launch_col_v<T, 1>(L, nb, s, solves, tw, ktab, cond, use_cond, general);
    case 2: return launch_col_v<T, 2>(L, nb, s, solves, tw, ktab, cond, use_cond, general);
    default: return cudaErrorInvalidValue;
  }
}
template <typename T>
inline cudaError_t launch_row_forward(int L, int var, cudaStream_t s, const void* p, void* spec, const void* tw) {
  switch (var) {
    case 0: return launch_row_forward_v<T, 0>(L, s, p, spec, tw);
    case 1: return launch_row_forward_v<T, 1>(L, s, p, spec, tw);
    case 2: return launch_row_forward_v<T, 2>(L, s, p, spec, tw);
    default: return cudaErrorInvalidValue;
  }
}
template <typename T>
inline cudaError_t launch_row_inverse(int L, int var, cudaStream_t s, const void* spec, void* e, const void* tw) {
  switch (var) {
    case 0: return launch_row_inverse_v<T, 0>(L, s, spec, e, tw);
    case 1: return launch_row_inverse_v<T, 1>(L, s, spec, e, tw);
    case 2: return launch_row_inverse_v<T, 2>(L, s, spec, e, tw);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace epfft
