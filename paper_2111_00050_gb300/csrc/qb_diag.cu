// Diagnostics and measurement helpers (include/qb_diag.h): the device status
// word of a space, and the FP64 FMA rate of the GPU for the roofline denominator.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/qb_diag.h"
#include "qb_device.cuh"
#include "qb_internal.h"

namespace qb {

// 8 independent chains x = x a + b per thread, `iters` x 16 steps each
__global__ void __launch_bounds__(256) dfma_chain_kernel(double* out, double a, double b, int iters) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

}  // namespace qb

using namespace qb;

extern "C" int qb_space_status(qb_space* space, int set_bits, int* status, void* stream) {
  Space* sp = reinterpret_cast<Space*>(space);
  if (!sp) return fail(QB_EINVAL, "space is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  int* d = reinterpret_cast<int*>(sp->d_scratch);  // the status word heads the scratch area
  int h = 0;
  QB_CUDA(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st));
  QB_CUDA(cudaStreamSynchronize(st));
  if (set_bits) {
    h |= set_bits;
    QB_CUDA(cudaMemcpyAsync(d, &h, sizeof(int), cudaMemcpyHostToDevice, st));
    QB_CUDA(cudaStreamSynchronize(st));
  }
  if (status) *status = h;
  return QB_OK;
}

extern "C" int qb_measure_fp64_fma(int reps, double* tflops, void* stream) {
  if (reps < 1 || !tflops) return fail(QB_EINVAL, "reps must be >= 1 and tflops non-NULL");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  QB_CUDA(cudaGetDevice(&dev));
  QB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256, iters = 128;
  double* out = nullptr;
  QB_CUDA(cudaMalloc(&out, sizeof(double) * (size_t)blocks * threads));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float best = 0.f;
  int rc = QB_OK;
  auto cleanup = [&]() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
  };
  do {
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      rc = fail(QB_ECUDA, "cudaEventCreate failed");
      break;
    }
    dfma_chain_kernel<<<blocks, threads, 0, st>>>(out, 0.999, 1e-3, iters);  // untimed
    for (int r = 0; r < reps && rc == QB_OK; ++r) {
      cudaEventRecord(e0, st);
      dfma_chain_kernel<<<blocks, threads, 0, st>>>(out, 0.999, 1e-3, iters);
      cudaEventRecord(e1, st);
      const cudaError_t e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = fail(QB_ECUDA, std::string("DFMA timing: ") + cudaGetErrorString(cudaGetLastError()));
        break;
      }
      if (r == 0 || ms < best) best = ms;
    }
  } while (false);
  const cudaError_t le = cudaGetLastError();
  if (rc == QB_OK && le != cudaSuccess) rc = fail(QB_ECUDA, std::string("DFMA probe: ") + cudaGetErrorString(le));
  cleanup();
  if (rc) return rc;
  const double fmas = (double)blocks * threads * iters * 16 * 8;
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  return QB_OK;
}
