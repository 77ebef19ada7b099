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
//
// Tensor-core peak: one CTA per SM keeps issuing tcgen05.mma (M = 128,
// N = 256, K one 128-byte swizzle atom per four instructions) from operand
// tiles already in shared memory into a 256-column FP32 accumulator in
// tensor memory, kind::tf32 or kind::f16 with BF16 operands; no loads, so
// the number is the tensor pipe's issue rate (2 M N K flops per MMA).  The
// issuing thread commits to an mbarrier at the end; every wait is bounded
// and a timeout is reported as an error, the tensor memory released in any
// case.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/qtt.h"
#include "engine.h"
#include "kernels.h"

#define TRY_ST(e)                  \
  do {                             \
    int _s = (e);                  \
    if (_s != QTT_OK) return _s;   \
  } while (0)

namespace {

constexpr int PK_M = 128, PK_N = 256;
constexpr int PK_A_BYTES = PK_M * 128, PK_B_BYTES = PK_N * 128;   // one 128-byte K atom per row
constexpr uint32_t PK_WAIT_LIMIT = 1u << 26;

__device__ __forceinline__ uint32_t pk_smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// K-major operand, 128-byte swizzle: start >> 4, leading byte offset 16,
// stride byte offset 1024 (eight 128-byte rows), version 1, swizzle mode 2
__device__ __forceinline__ uint64_t pk_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(16 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// instruction descriptors: D F32 (bit 4), A and B formats (bits 7, 10:
// TF32 = 2 for kind::tf32, BF16 = 1 for kind::f16), both K-major, N / 8 at
// bit 17, M / 16 at bit 24
__host__ __device__ constexpr uint32_t pk_idesc(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <int BF16>
__global__ void __launch_bounds__(128, 1) tc_peak_kernel(int iters, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~(uintptr_t)1023);
  __shared__ uint64_t done_bar;
  __shared__ uint32_t tmem_sh;
  const int warp = threadIdx.x >> 5;
  // operand tiles: small nonzero values (their bit patterns are valid TF32
  // and BF16 pairs alike)
  for (int i = threadIdx.x; i < (PK_A_BYTES + PK_B_BYTES) / 4; i += blockDim.x)
    reinterpret_cast<uint32_t*>(smem)[i] = 0x3C003C00u ^ ((uint32_t)(i * 2654435761u) & 0x00FF00FFu);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(pk_smem_u32(&done_bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(pk_smem_u32(&tmem_sh)),
                 "r"(PK_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_sh;
  if (threadIdx.x == 0) {
    const uint32_t a = pk_smem_u32(smem), b = a + PK_A_BYTES;
    const uint32_t idesc = pk_idesc(BF16 ? 1 : 2, PK_M, PK_N);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t da = pk_desc(a + kk * 32), db = pk_desc(b + kk * 32);
        const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
        if (BF16)
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(da), "l"(db), "r"(idesc), "r"(acc));
        else
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(da), "l"(db), "r"(idesc), "r"(acc));
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        pk_smem_u32(&done_bar)));
  }
  __syncwarp();
  // every thread waits (bounded) for the MMAs to finish
  bool ok = false;
  for (uint32_t t = 0; t < PK_WAIT_LIMIT && !ok; ++t) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(pk_smem_u32(&done_bar)), "r"(0)
        : "memory");
    ok = done != 0;
  }
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PK_N));
}

template <int BF16>
int tc_peak(qtt_ctx* c, double* tflops) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms < 1)
    return QTT_ERR_CUDA;
  const int iters = 1 << 14;
  const size_t smem = (size_t)PK_A_BYTES + PK_B_BYTES + 1024;
  if (qtt_allow_max_smem((const void*)tc_peak_kernel<BF16>) != QTT_OK) return QTT_ERR_CUDA;
  DBuf errb;
  int s = errb.alloc(c, sizeof(int));
  if (s) return s;
  cudaMemsetAsync(errb.p, 0, sizeof(int), c->stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, c->stream);
    tc_peak_kernel<BF16><<<sms, 128, smem, c->stream>>>(iters, errb.as<int>());
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
  int h = 0;
  TRY_ST(sync_read(c, &h, errb.p, sizeof(int)));
  if (h) return QTT_ERR_TIMEOUT;
  if (cudaGetLastError() != cudaSuccess) return QTT_ERR_CUDA;
  const double kper = BF16 ? 16.0 : 8.0;
  const double flops = 2.0 * PK_M * PK_N * kper * 4.0 * (double)iters * sms;
  *tflops = flops / (best * 1e-3) / 1e12;
  return QTT_OK;
}

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
    case QTT_PEAK_TF32_MMA: return tc_peak<0>(c, tflops);
    case QTT_PEAK_BF16_MMA: return tc_peak<1>(c, tflops);
    default: return QTT_ERR_ARG;
  }
}
