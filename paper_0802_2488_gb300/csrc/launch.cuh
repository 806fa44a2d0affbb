// Per-precision launch table of the fused passes (instantiated for every
// supported lattice side in inst_f32.cu / inst_f64.cu).
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace epfft {

struct PassShape {
  int rows_per_cta, tile_w;  // RR, W
  int row_ctas, col_ctas;    // per solve
  int nt_row, nt_col;
  size_t row_smem, col_smem;
};

// Returns false when L is not built for T.
template <typename T>
bool pass_shape(int L, PassShape* out);
// Raises the dynamic shared-memory limit of the kernels for L (call before
// any launch or capture).
template <typename T>
cudaError_t prepare(int L);
template <typename T>
cudaError_t launch_row(int L, int nb, cudaStream_t s, Solve* solves, BatchCtl* bc, const void* tw,
                       cudaGraphConditionalHandle cond, int use_cond);
template <typename T>
cudaError_t launch_col(int L, int nb, cudaStream_t s, Solve* solves, const void* tw, const void* ktab,
                       cudaGraphConditionalHandle cond, int use_cond);
template <typename T>
cudaError_t launch_row_forward(int L, cudaStream_t s, const void* p, void* spec, const void* tw);
// Reads and clears the self-check record (zero unless built with EPFFT_CHECKS).
template <typename T>
cudaError_t read_check(CheckRec* out);
template <typename T>
cudaError_t launch_row_inverse(int L, cudaStream_t s, const void* spec, void* e, const void* tw);

}  // namespace epfft
