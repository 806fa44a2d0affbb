// Kernels around the solves: mirrored problems and the average of DG2,
// plastic flags of a strain field, the 5-point average of CG2 (Sec. 2).
// Each kernel is a grid-stride loop over pixels; all accesses are checked
// against the image size by the loop bound.
#include "physics.cuh"
#include "post_kernels.cuh"

namespace epfft {
namespace {

int grid_of(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (int)(g < 152 * 16 ? (g < 1 ? 1 : g) : 152 * 16);
}

__device__ __forceinline__ int64_t mirror_index(int64_t i, int L, int axes) {
  int x1 = (int)(i % L), x2 = (int)(i / L);
  if (axes & 1) x1 = (L - x1) & (L - 1);
  if (axes & 2) x2 = (L - x2) & (L - 1);
  return (int64_t)x2 * L + x1;
}

__global__ void mirror_mask_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, int L, int axes) {
  const int64_t n = (int64_t)L * L;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[mirror_index(i, L, axes)];
}

template <typename T>
__global__ void dg2_average_kernel(const T* __restrict__ e0, const T* __restrict__ e1, const T* __restrict__ e2,
                                   const T* __restrict__ e3, T* __restrict__ out, int L) {
  const int64_t n = (int64_t)L * L;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = 4 * i, b = 4 * mirror_index(i, L, 3), c = 4 * mirror_index(i, L, 1),
                  d = 4 * mirror_index(i, L, 2);
    for (int k = 0; k < 3; k++) out[a + k] = (((e0[a + k] + e1[b + k]) + e2[c + k]) + e3[d + k]) * T(0.25);
    out[a + 3] = (((e0[a + 3] + e1[b + 3]) - e2[c + 3]) - e3[d + 3]) * T(0.25);
  }
}

template <typename T>
__global__ void plastic_kernel(const T* __restrict__ eps, const uint8_t* __restrict__ mask, uint8_t* __restrict__ fl,
                               int64_t n, T two_mu, T ylim2) {
  Mat<T> m;
  m.two_mu = two_mu;
  m.ylim2 = ylim2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T e[4] = {eps[4 * i], eps[4 * i + 1], eps[4 * i + 2], eps[4 * i + 3]};
    fl[i] = is_plastic(e, mask[i] != 0, m) ? 1 : 0;
  }
}

template <typename T>
__global__ void avg5_kernel(const T* __restrict__ in, T* __restrict__ out, int L) {
  const int64_t n = (int64_t)L * L;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int x1 = (int)(i % L), x2 = (int)(i / L);
    const int64_t r = (int64_t)x2 * L + ((x1 + 1) & (L - 1)), l = (int64_t)x2 * L + ((x1 + L - 1) & (L - 1));
    const int64_t u = (int64_t)((x2 + 1) & (L - 1)) * L + x1, d = (int64_t)((x2 + L - 1) & (L - 1)) * L + x1;
    for (int k = 0; k < 4; k++)
      out[4 * i + k] = ((((in[4 * i + k] + in[4 * r + k]) + in[4 * l + k]) + in[4 * u + k]) + in[4 * d + k]) / T(5);
  }
}

}  // namespace

cudaError_t launch_mirror_mask(const uint8_t* in, uint8_t* out, int L, int axes, cudaStream_t s) {
  mirror_mask_kernel<<<grid_of((int64_t)L * L), 256, 0, s>>>(in, out, L, axes);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dg2_average(const T* e0, const T* e1, const T* e2, const T* e3, T* out, int L, cudaStream_t s) {
  dg2_average_kernel<T><<<grid_of((int64_t)L * L), 256, 0, s>>>(e0, e1, e2, e3, out, L);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_plastic_flags(const T* eps, const uint8_t* mask, uint8_t* flags, int L, T two_mu, T ylim2,
                                 cudaStream_t s) {
  const int64_t n = (int64_t)L * L;
  plastic_kernel<T><<<grid_of(n), 256, 0, s>>>(eps, mask, flags, n, two_mu, ylim2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_avg5(const T* in, T* out, int L, cudaStream_t s) {
  avg5_kernel<T><<<grid_of((int64_t)L * L), 256, 0, s>>>(in, out, L);
  return cudaGetLastError();
}

template cudaError_t launch_dg2_average<float>(const float*, const float*, const float*, const float*, float*, int,
                                               cudaStream_t);
template cudaError_t launch_dg2_average<double>(const double*, const double*, const double*, const double*, double*,
                                                int, cudaStream_t);
template cudaError_t launch_plastic_flags<float>(const float*, const uint8_t*, uint8_t*, int, float, float,
                                                 cudaStream_t);
template cudaError_t launch_plastic_flags<double>(const double*, const uint8_t*, uint8_t*, int, double, double,
                                                  cudaStream_t);
template cudaError_t launch_avg5<float>(const float*, float*, int, cudaStream_t);
template cudaError_t launch_avg5<double>(const double*, double*, int, cudaStream_t);

}  // namespace epfft
