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
// Sec. 3 void-plastic clusters of one L x L image (all device buffers):
// vp = mask | plastic, then, given lab = the clusters of vp (launch_label),
// every cluster without a void joins the cluster of its nearest void pixel
// (periodic Euclidean distance, ties to the smaller linear index) and
// `out` receives the final labels (smallest linear index, -1 off the
// phase).  stats_dev[0..2]: final clusters, pixels of the largest, clusters
// without a plastic pixel.  scratch: 18 bytes per pixel.
cudaError_t launch_vp_flags(const uint8_t* mask, const uint8_t* plastic, uint8_t* vp, int L, cudaStream_t s);
cudaError_t launch_vp_attach(const uint8_t* mask, const uint8_t* vp, const int32_t* lab, int32_t* out, int L,
                             void* scratch, int32_t* stats_dev, int has_voids, cudaStream_t s);
// out(x) = [(2/3) e'_ij e'_ij]^(1/2) of a strain field (Fig. 1), e' the 3D
// deviator of (11, 22, 33, 12), e'_12 counted twice.
template <typename T>
cudaError_t launch_eps_eq(const T* eps, T* out, int L, cudaStream_t s);
// (L, L, 4) strain -> planes (e11, e22, e12); planes (u1, u2, .) -> (L, L, 2).
template <typename T>
cudaError_t launch_strain_planes(const T* eps, T* planes, int L, cudaStream_t s);
template <typename T>
cudaError_t launch_disp_pairs(const T* planes, T* u, int L, cudaStream_t s);
// out = in + dE on every pixel of an (L, L, 4) strain field, converted
// between precisions (double -> float or float -> double).
template <typename TI, typename TO>
cudaError_t launch_shift_convert(const TI* in, TO* out, int L, const double dE[4], cudaStream_t s);
// *count_dev += number of nonzero bytes of a[0 .. n)
cudaError_t launch_count(const uint8_t* a, int64_t n, int32_t* count_dev, cudaStream_t s);
}  // namespace epfft
