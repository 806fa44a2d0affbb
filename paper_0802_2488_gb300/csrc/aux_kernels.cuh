// Launchers of the mask and labelling kernels (aux_kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace epfft {
cudaError_t launch_mask(uint8_t* mask, int64_t n, uint64_t seed, uint64_t thr, cudaStream_t s);
// n_img images of L*L flags -> labels (smallest linear index of the cluster,
// -1 off the flags) and counts_dev[n_img]; *err_dev set if a bound tripped.
cudaError_t launch_label(const uint8_t* flags, int32_t* lab, int64_t n_img, int L, int periodic,
                         int32_t* counts_dev, int32_t* err_dev, cudaStream_t s);
}  // namespace epfft
