// Observables of the uniform MPS (Sec. 3, Eq. mps2): the site tensors of the
// unit are embedded densely from the kept U / V blocks of the last two
// iterations; the transfer maps that carry environments along the chain run on
// the grouped FP64 GEMM of kernels_f64.cu with block task lists built by the
// host (only the charge-allowed blocks of each site tensor are multiplied).
// This file holds the rest: the embedding, one-CTA reductions (fixed
// summation order, so every result is reproducible), a fused axpby, and the
// initial vectors of the power and subspace iterations.
#include "common.h"

#include <algorithm>

namespace idmrg {

namespace {

constexpr int EMB_ROWS = 16;
constexpr int DOT_THREADS = 1024;

// dst[x][y] = src(x, y) * cs[y] / rs[x]  (rs at or below thr counts as zero,
// the row then vanishes: Eq. wfprediction's zero rule)
__global__ void obs_embed_kernel(const EmbedTask *__restrict__ tasks, const double *__restrict__ scal) {
  const EmbedTask t = tasks[blockIdx.x];
  const int r0 = blockIdx.y * EMB_ROWS;
  if (r0 >= t.rows) return;
  const int r1 = min(t.rows, r0 + EMB_ROWS);
  const int n = (r1 - r0) * t.cols;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int x = r0 + e / t.cols, y = e % t.cols;
    double v = t.trans ? t.src[(int64_t)y * t.src_ld + x] : t.src[(int64_t)x * t.src_ld + y];
    if (t.rs >= 0) {
      const double l = scal[t.rs + x];
      v = (l > t.thr) ? v * (1.0 / l) : 0.0;
    }
    if (t.cs >= 0) v *= scal[t.cs + y];
    t.dst[(int64_t)x * t.dst_ld + y] = v;
  }
}

// *out = (accumulate ? *out : 0) + coef * sum_i x[i] y[i], one CTA
__global__ void __launch_bounds__(DOT_THREADS) obs_dot_kernel(const double *__restrict__ x,
                                                             const double *__restrict__ y, int64_t n, double coef,
                                                             double *out, int accumulate) {
  __shared__ double part[DOT_THREADS / 32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += DOT_THREADS) s = fma(x[i], y[i], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = part[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = (accumulate ? *out : 0.0) + coef * s;
  }
}

// y = a x + b y
// y = a x + b y; a zero coefficient does not read its operand (b = 0
// overwrites y, which may hold anything, including NaN bit patterns left in
// freshly allocated memory)
__global__ void obs_axpby_kernel(const double *x, double *y, int64_t n, double a, double b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ax = a == 0.0 ? 0.0 : a * x[i];
    y[i] = b == 0.0 ? ax : ax + b * y[i];
  }
}

__device__ __forceinline__ uint64_t obs_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// mode 0: value * identity (D x D); mode 1: SplitMix64 numbers uniform in
// [-1, 1) (element e takes output e of the generator seeded with `seed`)
__global__ void obs_fill_kernel(double *x, int D, int mode, double value, uint64_t seed) {
  const int64_t n = (int64_t)D * D;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    if (mode == 0) {
      x[e] = (e / D == e % D) ? value : 0.0;
    } else {
      const uint64_t z = obs_mix64(seed + (uint64_t)(e + 1) * 0x9E3779B97F4A7C15ull);
      x[e] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
  }
}

// keeps the entries of charge difference q[a] - q[b] == delta, zeroes the rest
__global__ void obs_mask_kernel(double *x, int D, const int *__restrict__ q, int delta) {
  const int64_t n = (int64_t)D * D;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    if (q[e / D] - q[e % D] != delta) x[e] = 0.0;
}

int grid_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 8);
}

}  // namespace

cudaError_t launch_obs_embed(const EmbedTask *tasks, int ntasks, int max_rows, const double *scal, cudaStream_t st) {
  if (ntasks > 0 && max_rows > 0) {
    dim3 grid(ntasks, (max_rows + EMB_ROWS - 1) / EMB_ROWS);
    obs_embed_kernel<<<grid, 256, 0, st>>>(tasks, scal);
  }
  return cudaGetLastError();
}

cudaError_t launch_obs_dot(const double *x, const double *y, int64_t n, double coef, double *out, int accumulate,
                           cudaStream_t st) {
  obs_dot_kernel<<<1, DOT_THREADS, 0, st>>>(x, y, n, coef, out, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_obs_axpby(const double *x, double *y, int64_t n, double a, double b, cudaStream_t st) {
  if (n > 0) obs_axpby_kernel<<<grid_for(n), 256, 0, st>>>(x, y, n, a, b);
  return cudaGetLastError();
}

cudaError_t launch_obs_fill(double *x, int D, int mode, double value, uint64_t seed, cudaStream_t st) {
  if (D > 0) obs_fill_kernel<<<grid_for((int64_t)D * D), 256, 0, st>>>(x, D, mode, value, seed);
  return cudaGetLastError();
}

cudaError_t launch_obs_mask(double *x, int D, const int *q, int delta, cudaStream_t st) {
  if (D > 0) obs_mask_kernel<<<grid_for((int64_t)D * D), 256, 0, st>>>(x, D, q, delta);
  return cudaGetLastError();
}

}  // namespace idmrg
