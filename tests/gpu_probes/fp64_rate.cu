// Issue latency and throughput of FP64 FMA, FP32 FMA, a double shuffle and a
// CTA barrier on the GPU it runs on, timed with clock64() (one block per
// measurement, every access in bounds).  The FP64 figures fix the ALU
// roofline of the FP64 kernels: dependent FMAs, FMAs with four independent
// chains per thread at 1..16 warps per CTA, and a warp with a single active
// lane.
#include <cstdio>
#include <cuda_runtime.h>
__global__ void chain(double *out, long long *cyc, int iters, int active, double seed) {
  double a = seed + threadIdx.x, b = 1.0000001, c = 1e-9;
  long long t0 = clock64();
  if ((int)(threadIdx.x & 31) < active) {
    for (int i = 0; i < iters; ++i) {
      a = fma(a, b, c);
      a = fma(a, b, c);
      a = fma(a, b, c);
      a = fma(a, b, c);
    }
  }
  __syncwarp();
  long long t1 = clock64();
  out[blockIdx.x * blockDim.x + threadIdx.x] = a;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}
// 4 independent chains per thread
__global__ void ilp(double *out, long long *cyc, int iters, double seed) {
  double a0 = seed + threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, b = 1.0000001, c = 1e-9;
  long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
  }
  __syncthreads();
  long long t1 = clock64();
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}
__global__ void fchain(float *out, long long *cyc, int iters, float seed) {
  float a = seed + threadIdx.x, b = 1.0000001f, c = 1e-9f;
  long long t0 = clock64();
  for (int i = 0; i < iters; ++i) { a = fmaf(a, b, c); a = fmaf(a, b, c); a = fmaf(a, b, c); a = fmaf(a, b, c); }
  __syncwarp();
  long long t1 = clock64();
  out[blockIdx.x * blockDim.x + threadIdx.x] = a;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}
__global__ void shfl_chain(double *out, long long *cyc, int iters) {
  double a = threadIdx.x;
  long long t0 = clock64();
  for (int i = 0; i < iters; ++i) a += __shfl_xor_sync(0xffffffffu, a, 1 + (i & 15)) * 1e-3;
  long long t1 = clock64();
  out[threadIdx.x] = a;
  if (threadIdx.x == 0) cyc[0] = t1 - t0;
}
__global__ void sync_chain(long long *cyc, int iters) {
  long long t0 = clock64();
  for (int i = 0; i < iters; ++i) __syncthreads();
  long long t1 = clock64();
  if (threadIdx.x == 0) cyc[0] = t1 - t0;
}
int main() {
  double *out; float *fo; long long *cyc, h[64];
  cudaMalloc(&out, 64 * 1024 * sizeof(double)); cudaMalloc(&fo, 64 * 1024 * sizeof(float)); cudaMalloc(&cyc, 64 * sizeof(long long));
  const int it = 1000;
  for (int active : {32, 1}) {
    chain<<<1, 32>>>(out, cyc, it, active, 1.0); cudaMemcpy(h, cyc, 8, cudaMemcpyDeviceToHost);
    printf("dfma dependent chain, 1 warp, %2d active lanes: %.1f cycles/fma\n", active, h[0] / (4.0 * it));
  }
  for (int warps : {1, 2, 4, 8, 16}) {
    ilp<<<1, 32 * warps>>>(out, cyc, it, 1.0); cudaMemcpy(h, cyc, 8, cudaMemcpyDeviceToHost);
    printf("dfma 4 chains/thread, %2d warps in 1 CTA: %.2f cycles per warp-fma issued (SM)\n", warps, h[0] / (4.0 * it * warps));
  }
  fchain<<<1, 32>>>(fo, cyc, it, 1.0f); cudaMemcpy(h, cyc, 8, cudaMemcpyDeviceToHost);
  printf("ffma dependent chain: %.1f cycles/fma\n", h[0] / (4.0 * it));
  shfl_chain<<<1, 32>>>(out, cyc, it); cudaMemcpy(h, cyc, 8, cudaMemcpyDeviceToHost);
  printf("shfl(double)+dfma chain: %.1f cycles/step\n", h[0] / (1.0 * it));
  sync_chain<<<1, 256>>>(cyc, it); cudaMemcpy(h, cyc, 8, cudaMemcpyDeviceToHost);
  printf("__syncthreads 256 thr: %.1f cycles\n", h[0] / (1.0 * it));
  cudaError_t e = cudaDeviceSynchronize();
  printf("status %s\n", cudaGetErrorString(e));
  return e == cudaSuccess ? 0 : 1;
}
