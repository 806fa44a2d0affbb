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

// --- Sec. 3: void-plastic clusters with nearest-void attachment ----------

__global__ void vp_flags_kernel(const uint8_t* __restrict__ mask, const uint8_t* __restrict__ pl,
                                uint8_t* __restrict__ vp, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    vp[i] = (uint8_t)(mask[i] | pl[i]);
}

// best[] = all ones; final_root[] = n; size[] = 0; has_pl[] = 0
__global__ void vp_init_kernel(unsigned long long* __restrict__ best, int32_t* __restrict__ final_root,
                               int32_t* __restrict__ size, uint8_t* __restrict__ has_pl, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    best[i] = ~0ull;
    final_root[i] = (int32_t)n;
    size[i] = 0;
    has_pl[i] = 0;
  }
}

// has_void[root] = 1 for clusters holding a void
__global__ void vp_mark_kernel(const uint8_t* __restrict__ mask, const int32_t* __restrict__ lab,
                               uint8_t* __restrict__ has_void, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (mask[i] && lab[i] >= 0 && lab[i] < n) has_void[lab[i]] = 1;
}

// Each pixel of a void-free cluster finds its nearest void by Chebyshev
// rings r = 0, 1, ... (periodic), keeping the smallest (d^2, index); ring
// r + 1 holds only pixels with d^2 >= (r + 1)^2, so the search stops once
// that exceeds the best d^2, and at r = L/2 at the latest.  The cluster's
// minimum is the atomic minimum of the packed key d^2 * 2^32 + index.
__global__ void vp_nearest_kernel(const uint8_t* __restrict__ mask, const uint8_t* __restrict__ vp,
                                  const int32_t* __restrict__ lab, const uint8_t* __restrict__ has_void,
                                  unsigned long long* __restrict__ best, int L) {
  const int64_t n = (int64_t)L * L;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!vp[i] || mask[i]) continue;
    const int32_t root = lab[i];
    if (root < 0 || root >= n || has_void[root]) continue;
    const int x1 = (int)(i % L), x2 = (int)(i / L);
    unsigned long long key = ~0ull;
    int64_t bd = -1;
    for (int r = 0; r <= L / 2; r++) {
      if (bd >= 0 && (int64_t)r * r > bd) break;
      for (int dy = -r; dy <= r; dy++) {
        const bool edge_row = dy == -r || dy == r;
        for (int dx = -r; dx <= r; dx += edge_row ? 1 : 2 * r) {
          const int y = (x2 + dy + L) & (L - 1), x = (x1 + dx + L) & (L - 1);
          const int64_t v = (int64_t)y * L + x;
          if (!mask[v]) {
            if (r == 0) break;
            continue;
          }
          const int ady = dy < 0 ? -dy : dy, adx = dx < 0 ? -dx : dx;
          const int64_t d2 = (int64_t)ady * ady + (int64_t)adx * adx;
          const unsigned long long k = ((unsigned long long)d2 << 32) | (unsigned long long)v;
          if (k < key) {
            key = k;
            bd = d2;
          }
          if (r == 0) break;
        }
      }
    }
    if (key != ~0ull) atomicMin(best + root, key);
  }
}

// target[root]: the root itself, or the root of the cluster of its nearest
// void; final_root[target] = smallest root merged into it
__global__ void vp_target_kernel(const uint8_t* __restrict__ vp, const int32_t* __restrict__ lab,
                                 const uint8_t* __restrict__ has_void, const unsigned long long* __restrict__ best,
                                 int32_t* __restrict__ target, int32_t* __restrict__ final_root, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!vp[i] || lab[i] != i) continue;
    int64_t t = i;
    if (!has_void[i] && best[i] != ~0ull) {
      const int64_t v = (int64_t)(best[i] & 0xffffffffull);
      if (v < n && lab[v] >= 0 && lab[v] < n) t = lab[v];
    }
    target[i] = (int32_t)t;
    atomicMin(final_root + t, (int32_t)i);
  }
}

__global__ void vp_relabel_kernel(const uint8_t* __restrict__ mask, const uint8_t* __restrict__ vp,
                                  const int32_t* __restrict__ lab, const int32_t* __restrict__ target,
                                  const int32_t* __restrict__ final_root, int32_t* __restrict__ out,
                                  int32_t* __restrict__ size, uint8_t* __restrict__ has_pl, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!vp[i] || lab[i] < 0 || lab[i] >= n) {
      out[i] = -1;
      continue;
    }
    const int32_t t = target[lab[i]];
    const int32_t f = (t >= 0 && t < n) ? final_root[t] : (int32_t)n;
    out[i] = f < n ? f : -1;
    if (f < n) {
      atomicAdd(size + f, 1);
      if (!mask[i]) has_pl[f] = 1;
    }
  }
}

template <typename T>
__global__ void eps_eq_kernel(const T* __restrict__ eps, T* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T* e = eps + 4 * i;
    const T m = (e[0] + e[1] + e[2]) / T(3);
    const T a = e[0] - m, b = e[1] - m, c = e[2] - m;
    out[i] = sqrt(T(2) / T(3) * (a * a + b * b + c * c + T(2) * e[3] * e[3]));
  }
}

// (L, L, 4) strain -> planes (e11, e22, e12) of L*L each.
template <typename T>
__global__ void strain_planes_kernel(const T* __restrict__ eps, T* __restrict__ planes, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    planes[i] = eps[4 * i + 0];
    planes[n + i] = eps[4 * i + 1];
    planes[2 * n + i] = eps[4 * i + 3];
  }
}

// out = in + dE per pixel (components 11, 22, 33, 12), converted from TI to
// TO (rounded once, after the shift).
template <typename TI, typename TO>
__global__ void shift_convert_kernel(const TI* __restrict__ in, TO* __restrict__ out, int64_t n, double d0,
                                     double d1, double d2, double d3) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    out[4 * i + 0] = (TO)((double)in[4 * i + 0] + d0);
    out[4 * i + 1] = (TO)((double)in[4 * i + 1] + d1);
    out[4 * i + 2] = (TO)((double)in[4 * i + 2] + d2);
    out[4 * i + 3] = (TO)((double)in[4 * i + 3] + d3);
  }
}

// planes (u1, u2, .) of L*L each -> (L, L, 2) pairs.
template <typename T>
__global__ void disp_pairs_kernel(const T* __restrict__ planes, T* __restrict__ u, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    u[2 * i + 0] = planes[i];
    u[2 * i + 1] = planes[n + i];
  }
}

__global__ void count_kernel(const uint8_t* __restrict__ a, int64_t n, int32_t* __restrict__ out) {
  int32_t c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += a[i] != 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

__global__ void vp_stats_kernel(const int32_t* __restrict__ size, const uint8_t* __restrict__ has_pl,
                                int32_t* __restrict__ stats, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (size[i] == 0) continue;
    atomicAdd(stats, 1);
    atomicMax(stats + 1, size[i]);
    if (!has_pl[i]) atomicAdd(stats + 2, 1);
  }
}

}  // namespace

cudaError_t launch_vp_flags(const uint8_t* mask, const uint8_t* plastic, uint8_t* vp, int L, cudaStream_t s) {
  const int64_t n = (int64_t)L * L;
  vp_flags_kernel<<<grid_of(n), 256, 0, s>>>(mask, plastic, vp, n);
  return cudaGetLastError();
}

cudaError_t launch_count(const uint8_t* a, int64_t n, int32_t* count_dev, cudaStream_t s) {
  count_kernel<<<grid_of(n), 256, 0, s>>>(a, n, count_dev);
  return cudaGetLastError();
}

cudaError_t launch_vp_attach(const uint8_t* mask, const uint8_t* vp, const int32_t* lab, int32_t* out, int L,
                             void* scratch, int32_t* stats_dev, int has_voids, cudaStream_t s) {
  const int64_t n = (int64_t)L * L;
  const int g = grid_of(n);
  unsigned long long* best = (unsigned long long*)scratch;                  // 8 n
  int32_t* target = (int32_t*)(best + n);                                   // 4 n
  int32_t* final_root = target + n;                                         // 4 n
  int32_t* size = final_root + n;                                           // 4 n
  uint8_t* has_void = (uint8_t*)(size + n);                                 // n
  uint8_t* has_pl = has_void + n;                                           // n
  cudaError_t e = cudaMemsetAsync(has_void, 0, (size_t)n, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(stats_dev, 0, 3 * sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  vp_init_kernel<<<g, 256, 0, s>>>(best, final_root, size, has_pl, n);
  vp_mark_kernel<<<g, 256, 0, s>>>(mask, lab, has_void, n);
  if (has_voids) vp_nearest_kernel<<<g, 256, 0, s>>>(mask, vp, lab, has_void, best, L);
  vp_target_kernel<<<g, 256, 0, s>>>(vp, lab, has_void, best, target, final_root, n);
  vp_relabel_kernel<<<g, 256, 0, s>>>(mask, vp, lab, target, final_root, out, size, has_pl, n);
  vp_stats_kernel<<<g, 256, 0, s>>>(size, has_pl, stats_dev, n);
  return cudaGetLastError();
}

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
template <typename T>
cudaError_t launch_eps_eq(const T* eps, T* out, int L, cudaStream_t s) {
  const int64_t n = (int64_t)L * L;
  eps_eq_kernel<T><<<grid_of(n), 256, 0, s>>>(eps, out, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_strain_planes(const T* eps, T* planes, int L, cudaStream_t s) {
  const int64_t n = (int64_t)L * L;
  strain_planes_kernel<T><<<grid_of(n), 256, 0, s>>>(eps, planes, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_disp_pairs(const T* planes, T* u, int L, cudaStream_t s) {
  const int64_t n = (int64_t)L * L;
  disp_pairs_kernel<T><<<grid_of(n), 256, 0, s>>>(planes, u, n);
  return cudaGetLastError();
}

template <typename TI, typename TO>
cudaError_t launch_shift_convert(const TI* in, TO* out, int L, const double dE[4], cudaStream_t s) {
  const int64_t n = (int64_t)L * L;
  shift_convert_kernel<TI, TO><<<grid_of(n), 256, 0, s>>>(in, out, n, dE[0], dE[1], dE[2], dE[3]);
  return cudaGetLastError();
}

template cudaError_t launch_shift_convert<double, float>(const double*, float*, int, const double*, cudaStream_t);
template cudaError_t launch_shift_convert<float, double>(const float*, double*, int, const double*, cudaStream_t);
template cudaError_t launch_strain_planes<float>(const float*, float*, int, cudaStream_t);
template cudaError_t launch_strain_planes<double>(const double*, double*, int, cudaStream_t);
template cudaError_t launch_disp_pairs<float>(const float*, float*, int, cudaStream_t);
template cudaError_t launch_disp_pairs<double>(const double*, double*, int, cudaStream_t);
template cudaError_t launch_eps_eq<float>(const float*, float*, int, cudaStream_t);
template cudaError_t launch_eps_eq<double>(const double*, double*, int, cudaStream_t);
template cudaError_t launch_avg5<float>(const float*, float*, int, cudaStream_t);
template cudaError_t launch_avg5<double>(const double*, double*, int, cudaStream_t);

}  // namespace epfft
