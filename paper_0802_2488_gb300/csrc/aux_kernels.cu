// Void mask (Sec. 2) and plastic-cluster labelling (Sec. 3) kernels.
#include "aux_kernels.cuh"

namespace epfft {

// Pixel x is a void iff (SplitMix64 output x of `seed`) >> 11 < thr, where the
// i-th output of SplitMix64 is the 64-bit finaliser of seed + (i+1) gamma,
// gamma = 0x9e3779b97f4a7c15 (Steele, Lea & Flood's generator).
__global__ void mask_kernel(uint8_t* __restrict__ mask, int64_t n, uint64_t seed, uint64_t thr) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + (uint64_t)(i + 1) * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    mask[i] = (uint8_t)((z >> 11) < thr);
  }
}

// --- 4-connected clusters by concurrent union-find ------------------------
// lab[x] is a parent index (<= x) for flagged pixels and -1 otherwise; a
// root is its own parent.  Unions always hang the larger root below the
// smaller one, so each final root is the smallest linear index of its
// cluster, which makes the labels canonical.  Pointer chases are bounded by
// the image size; a chase that exceeds it raises *err and stops.

__device__ __forceinline__ int32_t find_root(const int32_t* lab, int32_t x, int32_t bound, int32_t* err) {
  for (int32_t it = 0; it < bound; it++) {
    const int32_t p = __ldcg(lab + x);
    if (p == x) return x;
    x = p;
  }
  atomicExch(err, 1);
  return x;
}

__device__ __forceinline__ void unite(int32_t* lab, int32_t a, int32_t b, int32_t bound, int32_t* err) {
  for (int32_t it = 0; it < bound; it++) {
    a = find_root(lab, a, bound, err);
    b = find_root(lab, b, bound, err);
    if (a == b) return;
    if (a > b) {
      const int32_t t = a;
      a = b;
      b = t;
    }
    const int32_t old = atomicMin(lab + b, a);
    if (old == b) return;
    b = old;
  }
  atomicExch(err, 1);
}

__global__ void ccl_init(const uint8_t* __restrict__ flags, int32_t* __restrict__ lab, int64_t n_img_px, int L) {
  const int64_t LL = (int64_t)L * L;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_img_px;
       i += (int64_t)gridDim.x * blockDim.x)
    lab[i] = flags[i] ? (int32_t)(i % LL) : -1;
}

__global__ void ccl_merge(const uint8_t* __restrict__ flags, int32_t* lab, int64_t n_img_px, int L,
                          int periodic, int32_t* err) {
  const int64_t LL = (int64_t)L * L;
  const int32_t bound = (int32_t)(LL + 1);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_img_px;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!flags[i]) continue;
    const int64_t img = i / LL;
    const int32_t x = (int32_t)(i - img * LL);
    const int32_t x1 = x % L, x2 = x / L;
    int32_t* l = lab + img * LL;
    const uint8_t* f = flags + img * LL;
    // right and lower neighbours cover every bond once
    if (x1 + 1 < L || periodic) {
      const int32_t y = x2 * L + ((x1 + 1) & (L - 1));
      if (f[y] && y != x) unite(l, x, y, bound, err);
    }
    if (x2 + 1 < L || periodic) {
      const int32_t y = ((x2 + 1) & (L - 1)) * L + x1;
      if (f[y] && y != x) unite(l, x, y, bound, err);
    }
  }
}

__global__ void ccl_flatten(int32_t* lab, int64_t n_img_px, int L, int32_t* counts, int32_t* err) {
  const int64_t LL = (int64_t)L * L;
  const int32_t bound = (int32_t)(LL + 1);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_img_px;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t img = i / LL;
    const int32_t x = (int32_t)(i - img * LL);
    int32_t* l = lab + img * LL;
    if (__ldcg(l + x) < 0) continue;
    const int32_t r = find_root(l, x, bound, err);
    if (r == x) atomicAdd(counts + img, 1);
  }
}

// Labels written after all roots are final (separate launch), so that a
// pixel never reads a half-updated chain.
__global__ void ccl_finish(int32_t* lab, int64_t n_img_px, int L, int32_t* err) {
  const int64_t LL = (int64_t)L * L;
  const int32_t bound = (int32_t)(LL + 1);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_img_px;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t img = i / LL;
    const int32_t x = (int32_t)(i - img * LL);
    int32_t* l = lab + img * LL;
    const int32_t p = __ldcg(l + x);
    if (p < 0 || p == x) continue;
    l[x] = find_root(l, p, bound, err);
  }
}

static int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_mask(uint8_t* mask, int64_t n, uint64_t seed, uint64_t thr, cudaStream_t s) {
  mask_kernel<<<grid_for(n), 256, 0, s>>>(mask, n, seed, thr);
  return cudaGetLastError();
}

cudaError_t launch_label(const uint8_t* flags, int32_t* lab, int64_t n_img, int L, int periodic,
                         int32_t* counts_dev, int32_t* err_dev, cudaStream_t s) {
  const int64_t n = n_img * (int64_t)L * L;
  cudaError_t e = cudaMemsetAsync(counts_dev, 0, sizeof(int32_t) * n_img, s);
  if (e != cudaSuccess) return e;
  const int g = grid_for(n);
  ccl_init<<<g, 256, 0, s>>>(flags, lab, n, L);
  ccl_merge<<<g, 256, 0, s>>>(flags, lab, n, L, periodic, err_dev);
  ccl_flatten<<<g, 256, 0, s>>>(lab, n, L, counts_dev, err_dev);
  ccl_finish<<<g, 256, 0, s>>>(lab, n, L, err_dev);
  return cudaGetLastError();
}

// --- FP64 FMA throughput ---------------------------------------------------
// Every thread advances FMA_CHAINS independent chains x <- x a + b for n
// steps (a slightly below 1, so the values stay bounded); the sum is stored
// only if it equals an impossible value, so the chains cannot be removed.
__global__ void __launch_bounds__(FMA_THREADS) fp64_fma_kernel(int n, double a, double b, double* sink) {
  double x[FMA_CHAINS];
#pragma unroll
  for (int i = 0; i < FMA_CHAINS; i++) x[i] = 1e-3 * threadIdx.x + i;
#pragma unroll 4
  for (int k = 0; k < n; k++)
#pragma unroll
    for (int i = 0; i < FMA_CHAINS; i++) x[i] = fma(x[i], a, b);
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < FMA_CHAINS; i++) s += x[i];
  if (s == -1234.5) *sink = s;
}

cudaError_t launch_fp64_fma(int blocks, int n, double* sink, cudaStream_t s) {
  fp64_fma_kernel<<<blocks, FMA_THREADS, 0, s>>>(n, 0.999999, 1e-6, sink);
  return cudaGetLastError();
}

}  // namespace epfft
