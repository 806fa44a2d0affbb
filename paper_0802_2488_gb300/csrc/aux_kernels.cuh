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
// FP64 FMA throughput probe: `blocks` CTAs of 256 threads, each thread runs
// FMA_CHAINS independent chains of n dependent FMAs (2 flops each).
constexpr int FMA_CHAINS = 8, FMA_THREADS = 256;
cudaError_t launch_fp64_fma(int blocks, int n, double* sink, cudaStream_t s);
}  // namespace epfft
