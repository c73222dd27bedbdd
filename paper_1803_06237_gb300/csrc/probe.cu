// Arithmetic throughput probes: the FP32 and FP64 fused multiply-add rates
// of the current GPU, measured with dependent FMA chains that keep every
// scheduler busy (eight independent chains per thread).  They give the ALU
// roofline against which the operator passes, whose butterflies are FP32
// (complex64) or FP64 (complex128) adds and multiplies, are reported.  The
// paper has no counterpart.
#include <cuda_runtime.h>

#include "vie_internal.cuh"

namespace vie {

constexpr int kChains = 8;

template <typename R>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, R b, R c, R* sink) {
  R a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (R)(threadIdx.x + k) * (R)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
  }
  R t = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) t += a[k];
  if (t == (R)-1.2345e-7) sink[threadIdx.x] = t;   // never true for these inputs; keeps the chains live
}

template <typename R>
static vie_status run_probe(int iters, double* tflops, cudaStream_t s) {
  int dev = 0, sms = 0;
  VIE_CUDA_TRY(cudaGetDevice(&dev));
  VIE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  R* sink = nullptr;
  VIE_CUDA_TRY(cudaMalloc((void**)&sink, 256 * sizeof(R)));
  const dim3 grid(sms * 8), block(256);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // warm-up launch (clocks up), then the timed one
  fma_probe_kernel<R><<<grid, block, 0, s>>>(iters / 4 + 1, (R)0.999999, (R)1e-7, sink);
  cudaEventRecord(e0, s);
  fma_probe_kernel<R><<<grid, block, 0, s>>>(iters, (R)0.999999, (R)1e-7, sink);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) {
    set_error("throughput probe: %s", cudaGetErrorString(e));
    return VIE_ERR_CUDA;
  }
  const double flops = 2.0 * kChains * 16.0 * iters * (double)grid.x * block.x;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return VIE_OK;
}

}  // namespace vie

extern "C" vie_status vie_probe_fma_tflops(int dtype, double* tflops, void* stream) {
  using namespace vie;
  clear_error();
  if (!tflops) { set_error("null argument"); return VIE_ERR_INVALID; }
  if (dtype == VIE_C64) return run_probe<float>(4096, tflops, (cudaStream_t)stream);
  if (dtype == VIE_C128) return run_probe<double>(128, tflops, (cudaStream_t)stream);
  set_error("dtype must be VIE_C64 (FP32 rate) or VIE_C128 (FP64 rate)");
  return VIE_ERR_INVALID;
}
