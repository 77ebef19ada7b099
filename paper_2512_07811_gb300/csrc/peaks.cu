// Arithmetic peaks of the GPU the library runs on, measured with the
// library's own kernels (not in the paper): the rooflines of the float and
// FP64 CUDA-core kernels are quoted against these numbers.
//
// FMA peak: every thread of a full grid (4 CTAs of 256 threads per SM) runs
// eight independent chains a_i <- a_i * b + c of `iters` fused multiply-adds
// each (two flops per FMA); the chains hide the FMA latency, so the grid
// issues FMAs every cycle on every scheduler.  The result is stored so the
// chains cannot be removed.  Timed with CUDA events around the launch, best
// of five launches after one warm-up.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/qtt.h"
#include "engine.h"

namespace {

template <class T>
__global__ void __launch_bounds__(256) fma_chain_kernel(T b, T c, int iters, T* __restrict__ out) {
  T a0 = (T)threadIdx.x, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
  T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, b, c);
    a1 = fma(a1, b, c);
    a2 = fma(a2, b, c);
    a3 = fma(a3, b, c);
    a4 = fma(a4, b, c);
    a5 = fma(a5, b, c);
    a6 = fma(a6, b, c);
    a7 = fma(a7, b, c);
  }
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
}

template <class T>
int fma_peak(qtt_ctx* c, int iters, double* tflops) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms < 1)
    return QTT_ERR_CUDA;
  const int blocks = 4 * sms, threads = 256;
  DBuf out;
  int s = out.alloc(c, (size_t)blocks * threads * sizeof(T));
  if (s) return s;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  // b slightly below 1 and c small keep the chains bounded and normal
  const T b = (T)0.999999, cc = (T)1e-3;
  for (int rep = 0; rep < 6; ++rep) {
    cudaEventRecord(e0, c->stream);
    fma_chain_kernel<T><<<blocks, threads, 0, c->stream>>>(b, cc, iters, out.as<T>());
    cudaEventRecord(e1, c->stream);
    c->launches++;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      s = QTT_ERR_CUDA;
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s) return s;
  if (cudaGetLastError() != cudaSuccess) return QTT_ERR_CUDA;
  const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return QTT_OK;
}

}  // namespace

extern "C" int qtt_measure_peak(qtt_ctx* c, int which, double* tflops) {
  if (!c || !tflops) return QTT_ERR_ARG;
  switch (which) {
    case QTT_PEAK_FP32_FMA: return fma_peak<float>(c, 1 << 16, tflops);
    case QTT_PEAK_FP64_FMA: return fma_peak<double>(c, 1 << 12, tflops);
    default: return QTT_ERR_ARG;
  }
}
