// Batched complex GEMM over two-level multi-indices (CUDA cores, FP64 / FP32).
//
// Every core contraction of the tensor-train path (absorbing R or U*S into a
// neighbouring core, transfer matrices of inner products, the structured
// sketch contractions of operator-times-train products) is one call of this
// kernel with suitable index strides, so no contraction needs an explicit
// permutation pass.
#include "common.cuh"
#include "kernels.h"

namespace {

template <class R, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
gemm_midx_kernel(GemmDesc g, cplx<R> alpha, cplx<R> beta,
                 const cplx<R>* __restrict__ A, const cplx<R>* __restrict__ B,
                 cplx<R>* __restrict__ C) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int TX = BN / TN;
  __shared__ cplx<R> As[BK][BM + 1];
  __shared__ cplx<R> Bs[BK][BN + 1];

  const int64_t b = blockIdx.z;
  const int64_t m0 = (int64_t)blockIdx.y * BM;
  const int64_t n0 = (int64_t)blockIdx.x * BN;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;

  const int64_t offA = midx_off(g.bA, b), offB = midx_off(g.bB, b), offC = midx_off(g.bC, b);

  cplx<R> acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = cplx<R>(0, 0);

  for (int64_t k0 = 0; k0 < g.K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += NT) {
      int mm = e % BM, kk = e / BM;
      int64_t m = m0 + mm, k = k0 + kk;
      cplx<R> v(0, 0);
      if (m < g.M && k < g.K) {
        v = A[offA + midx_off(g.mA, m) + midx_off(g.kA, k)];
        if (g.conjA) v.im = -v.im;
      }
      As[kk][mm] = v;
    }
    for (int e = tid; e < BN * BK; e += NT) {
      int nn = e % BN, kk = e / BN;
      int64_t n = n0 + nn, k = k0 + kk;
      cplx<R> v(0, 0);
      if (n < g.N && k < g.K) {
        v = B[offB + midx_off(g.kB, k) + midx_off(g.nB, n)];
        if (g.conjB) v.im = -v.im;
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      cplx<R> a[TM], bb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * (BM / TM)];
#pragma unroll
      for (int j = 0; j < TN; ++j) bb[j] = Bs[kk][tx + j * TX];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) cfma(acc[i][j], a[i], bb[j]);
    }
    __syncthreads();
  }
  const bool use_beta = (beta.re != R(0) || beta.im != R(0));
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int64_t m = m0 + ty + i * (BM / TM);
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int64_t n = n0 + tx + j * TX;
      if (n >= g.N) continue;
      int64_t o = offC + midx_off(g.mC, m) + midx_off(g.nC, n);
      cplx<R> v = alpha * acc[i][j];
      if (use_beta) v = v + beta * C[o];
      C[o] = v;
    }
  }
}

}  // namespace

template <class R>
int qtt_gemm(const GemmDesc& g, cplx<R> alpha, cplx<R> beta, const cplx<R>* A,
             const cplx<R>* B, cplx<R>* C, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return QTT_OK;
  if (g.K <= 0) {
    // C = beta * C; scale through the kernel with K = 0 (loop body skipped)
  }
  constexpr int BM = 64, BN = 64, TM = 4, TN = 4;
  constexpr int BK = sizeof(R) == 8 ? 8 : 16;
  dim3 grid((unsigned)((g.N + BN - 1) / BN), (unsigned)((g.M + BM - 1) / BM), (unsigned)g.batch);
  if (grid.y > 65535 || grid.z > 65535) return QTT_ERR_ARG;
  gemm_midx_kernel<R, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, s>>>(g, alpha, beta, A, B, C);
  return cudaGetLastError() == cudaSuccess ? QTT_OK : QTT_ERR_CUDA;
}

template int qtt_gemm<double>(const GemmDesc&, zc, zc, const zc*, const zc*, zc*, cudaStream_t);
template int qtt_gemm<float>(const GemmDesc&, cc, cc, const cc*, const cc*, cc*, cudaStream_t);
