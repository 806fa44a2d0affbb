// Launchers of the kernels around the solves (post_kernels.cu): the mirrored
// problems and the average of DG2, plastic flags of a strain field, and the
// 5-point average of CG2 (Sec. 2).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace epfft {
// out(x) = in(mirror(x)) for an L x L u8 image; axes: bit 0 mirrors x1
// (x1 -> -x1 mod L), bit 1 mirrors x2.
cudaError_t launch_mirror_mask(const uint8_t* in, uint8_t* out, int L, int axes, cudaStream_t s);
// DG2 average of four final strain fields (4 reals per pixel), members in
// the order of the mirrors (none, x1 and x2, x1, x2): out(x) is the mean of
// the members read at the mirror image of x, eps12 negated for a single
// mirror.  T = float or double.
template <typename T>
cudaError_t launch_dg2_average(const T* e0, const T* e1, const T* e2, const T* e3, T* out, int L, cudaStream_t s);
// flags(x) = 1 where a matrix pixel of the strain field is on the plastic
// branch of the Mises law (4 mu^2 |dev eps|^2 > 2/3 Y^2), else 0.
template <typename T>
cudaError_t launch_plastic_flags(const T* eps, const uint8_t* mask, uint8_t* flags, int L, T two_mu, T ylim2,
                                 cudaStream_t s);
// CG2: out(x) = (in(x) + in of the four nearest neighbours) / 5, periodic.
template <typename T>
cudaError_t launch_avg5(const T* in, T* out, int L, cudaStream_t s);
}  // namespace epfft
