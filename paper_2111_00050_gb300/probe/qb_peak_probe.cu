// Arithmetic throughput probe for the roofline denominators of the qb kernels:
// FP64 FMA, FP32 FMA and 32-bit integer multiply-add rates of the current GPU,
// from 8 independent dependency chains per thread over a grid of 8 CTAs per SM.
// Build and run: python -m paper_2111_00050_gb300.probe
#include <cstdio>
#include <cuda_runtime.h>
template <typename T>
__global__ void fma_chain(T* out, T a, T b, int iters) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
      x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
__global__ void int_chain(unsigned* out, unsigned a, unsigned b, int iters) {
  unsigned x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
      x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
int main() {
  cudaDeviceProp p; cudaGetDeviceProperties(&p, 0);
  int clk = 0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  printf("name %s SMs %d l2 %d smem/SM %zu clock(kHz) %d\n", p.name, p.multiProcessorCount, p.l2CacheSize, p.sharedMemPerMultiprocessor, clk);
  int blocks = p.multiProcessorCount * 8, threads = 256;
  size_t n = (size_t)blocks * threads;
  double* dd; float* df; unsigned* du;
  cudaMalloc(&dd, n * 8); cudaMalloc(&df, n * 4); cudaMalloc(&du, n * 4);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float ms;
  for (int rep = 0; rep < 2; ++rep) {
    int it = 64;
    cudaEventRecord(e0); fma_chain<double><<<blocks, threads>>>(dd, 0.999, 1e-3, it); cudaEventRecord(e1);
    cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    double fmas = (double)n * it * 16 * 8;
    printf("DFMA: %.3f ms  %.3f TFMA/s  %.3f TFLOP/s  per SM per clk(at %d MHz)=%.2f\n", ms, fmas / ms / 1e9, 2 * fmas / ms / 1e9,
           clk / 1000, fmas / (ms * 1e-3) / p.multiProcessorCount / (clk * 1e3));
    it = 4096;
    cudaEventRecord(e0); fma_chain<float><<<blocks, threads>>>(df, 0.999f, 1e-3f, it); cudaEventRecord(e1);
    cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    fmas = (double)n * it * 16 * 8;
    printf("FFMA: %.3f ms  %.3f TFMA/s  per SM per clk=%.2f\n", ms, fmas / ms / 1e9, fmas / (ms * 1e-3) / p.multiProcessorCount / (clk * 1e3));
    cudaEventRecord(e0); int_chain<<<blocks, threads>>>(du, 3u, 7u, it); cudaEventRecord(e1);
    cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    printf("IMAD: %.3f ms  %.3f TIMAD/s  per SM per clk=%.2f\n", ms, fmas / ms / 1e9, fmas / (ms * 1e-3) / p.multiProcessorCount / (clk * 1e3));
  }
  cudaError_t err = cudaGetLastError();
  printf("status %s\n", cudaGetErrorString(err));
  return err == cudaSuccess ? 0 : 1;
}
