// fp64_rate.cu -- the FP64 FMA throughput of the device, measured: the
// denominator of the FP64 push's roofline (that kernel is bound by the FP64
// pipes, whose rate on this part is a small fraction of the FP32 rate).
//
// Each thread runs kChains independent FMA chains (enough to cover the pipe
// latency), the chains' results are stored so that nothing is optimised away,
// and the kernel is timed with CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include "../../include/pic.h"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 2048;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fp64_fma(double b, double c, double* out) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (double)(threadIdx.x + k);
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int pic_fp64_fma_rate(void* cuda_stream, double* tflops) {
  if (!tflops) return PIC_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_fma, kThreads, 0) != cudaSuccess)
    return PIC_ERR_CUDA;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  double* out = nullptr;
  if (cudaMallocAsync((void**)&out, (size_t)blocks * kThreads * sizeof(double), st) != cudaSuccess)
    return PIC_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 0.0f;
  cudaError_t e = cudaSuccess;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first launch warms up
    cudaEventRecord(e0, st);
    k_fp64_fma<<<blocks, kThreads, 0, st>>>(0.999999, 1e-7, out);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && e == cudaSuccess && (best == 0.0f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess || !(best > 0.0f)) return PIC_ERR_CUDA;
  const double flops = 2.0 * kChains * (double)kIters * blocks * kThreads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return PIC_OK;
}
