// Measurement helper (not part of the method): the FP32 FMA rate this GPU
// sustains, the denominator of the resident fine kernel's roofline.  Every
// thread runs 16 independent FMA chains (enough to cover the FMA latency
// with 1,024 threads per SM), two CTAs of 512 threads per SM.
#include <cuda_runtime.h>

#include "mm_internal.h"

namespace {

constexpr int kChains = 16;

__global__ void __launch_bounds__(512) ffma_probe_kernel(float* sink, int iters, int write) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.0f + 1e-7f * (float)(threadIdx.x + k);
  const float m = 0.99999f, c = 1e-6f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = __fmaf_rn(a[k], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (write) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains alive
}

}  // namespace

extern "C" mm_status mm_probe_fp32(double* tflops, void* stream) {
  if (!tflops) return mm_fail(MM_ERR_INVALID, "tflops is NULL");
  int dev = 0, n_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return mm_cuda_fail(e, "probe: device");
  cudaStream_t s = (cudaStream_t)stream;
  const int threads = 512, blocks = 2 * n_sm, iters = 1 << 16;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  ffma_probe_kernel<<<blocks, threads, 0, s>>>(nullptr, iters / 16, 0);  // warm-up
  cudaEventRecord(e0, s);
  ffma_probe_kernel<<<blocks, threads, 0, s>>>(nullptr, iters, 0);
  cudaEventRecord(e1, s);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return mm_cuda_fail(e, "probe: run");
  const double flops = 2.0 * kChains * (double)iters * threads * blocks;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return MM_OK;
}
